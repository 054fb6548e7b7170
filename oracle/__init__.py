"""FP64 CPU oracle of the coupled BSSN-Valencia spectral right-hand side.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA library: every operator here is written from the paper's
definitions (Methods: grid discretisation, spectral derivative operators,
dealiasing and filtering, primitive recovery, fluxes and sources, Runge-Kutta
integration, BSSN evolution equations) in plain numpy, slow and literal.

Modules
  spectral     nodes, Chebyshev coefficient-route and Fourier DFT derivatives,
               modal filters, quadrature weights
  kerr_schild  Kerr-Schild line element, 3+1 split, extrinsic curvature, BSSN data
  valencia     primitive <-> conserved maps, primitive recovery, fluxes, T^{mu nu},
               geometric sources, 3+1 matter terms
  bssn         BSSN + gauge right-hand side at points
  solver       multi-element grid, full RHS with interface coupling, RK stages,
               post-step filter, CFL time step, diagnostics, initial data
  xcts         approximate XCTS initial data: flat-Laplacian boundary-value problem,
               fixed-point relaxation on psi, the conformally flat slice
  rounding     the oracle's own rounding floor per component (the oracle evaluated
               again with one more rounding after every stage), which sets the parity
               bar of components that are residues of cancelling terms

Parity pins live in tests/test_oracle_*.py; functions without one say
"parity unpinned" in their docstring.
"""
