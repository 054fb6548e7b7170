"""Pins of the oracle's Hamiltonian-constraint diagnostic H = R + (2/3) K^2 - Atilde.Atilde
- 16 pi rho (BSSN form of R + K^2 - K_ij K^ij - 16 pi rho).

* The vacuum Kerr-Schild slice satisfies the constraint: H -> 0 spectrally with resolution.
* A conformally flat slice psi^4 (flat metric) with K = 0 and Atilde = 0 has
  R = -8 psi^-5 lap(psi): with a manufactured psi and no matter, H must converge to that;
  adding the matter lowers H by exactly 16 pi E.  This fixes the normalisation and sign of
  every term.
"""
import numpy as np

from oracle import solver as so
from oracle import xcts
from workloads import config, primitive_profiles


def _vacuum_H(n):
    cfg = config("c1", n_elem=2, n_r=n, n_theta=n, n_phi=4, theta_min=np.pi / 4,
                 theta_max=3 * np.pi / 4)
    g, p, U = so.workload_state(cfg)
    U[so.I_D:] = 0.0
    U[so.I_D] = 1e-20                     # atmosphere: no matter
    H = so.hamiltonian_constraint(U, g, p)
    return np.abs(H[:, 1:-1]).max()       # radial element interiors


def test_vacuum_kerr_schild_satisfies_the_constraint():
    errs = [_vacuum_H(n) for n in (8, 12, 16)]
    assert errs[2] < 1e-5 and errs[0] > 10 * errs[2], errs


def _conformally_flat_state(n):
    """A conformally flat slice psi^4 (flat metric), K = 0, on a theta band (Chebyshev theta,
    smooth there), psi = 1 + M/(2r) + a Gaussian shell with l = 0 and l = 1 parts; no matter.
    Its scalar curvature is R = -8 psi^-5 lap(psi) with the analytic flat Laplacian."""
    cfg = config("c1", n_elem=3, n_r=n, n_theta=n, n_phi=4, theta_min=np.pi / 4,
                 theta_max=3 * np.pi / 4)
    p = so.Params.from_config(cfg)
    g = so.Grid(p)
    R, T, P = g.R, g.T, g.P
    c, r0, w = 0.05, 6.0, 1.5
    f = c * np.exp(-((R - r0) / w) ** 2)
    f1 = -2.0 * (R - r0) / w ** 2 * f
    f2 = (4.0 * (R - r0) ** 2 / w ** 4 - 2.0 / w ** 2) * f
    Y1 = 0.3 * np.sin(T) * np.cos(P) + 0.2 * np.cos(T)
    psi = 1.0 + p.M / (2.0 * R) + f * (1.0 + Y1)
    lap = (f2 + 2.0 * f1 / R) * (1.0 + Y1) - 2.0 * f / R ** 2 * Y1
    prim = primitive_profiles(cfg, g.R, g.T, g.P)
    U = so.initial_state(g, p, prim, bssn=xcts.bssn_data(g, psi))
    return g, p, U, -8.0 * lap / psi ** 5


def test_conformally_flat_curvature_fixes_the_normalisation():
    """With the matter removed H = R, which must converge to -8 psi^-5 lap(psi); with the
    matter put back H drops by exactly 16 pi E (E the Eulerian energy density)."""
    errs = []
    for n in (10, 14, 18):
        g, p, U, R_exact = _conformally_flat_state(n)
        V = U.copy()
        V[so.I_D:] = 0.0
        V[so.I_D] = 1e-20
        H0 = so.hamiltonian_constraint(V, g, p)
        errs.append(np.abs((H0 - R_exact)[:, 1:-1]).max() / np.abs(R_exact).max())
    # spectral convergence (2.5e-2, 8.4e-4, 1.1e-4); a wrong term or factor stays O(1)
    assert errs[2] < 1e-3 and errs[0] > 100 * errs[2] and errs[1] > errs[2], errs
    pr = so.primitives(U, p)
    f = so.unpack_bssn(U)
    gam, _ = so.metric_from_bssn(f)
    T = so.va.stress_energy(pr["rho"], pr["v"], pr["eps"], pr["B"], f["alpha"], f["beta"], gam,
                            p.gamma_eos)
    E = so.va.matter_3p1(T, f["alpha"], f["beta"], gam)[0]
    H1 = so.hamiltonian_constraint(U, g, p, pr)
    np.testing.assert_allclose(H1 - H0, -16.0 * np.pi * E, rtol=1e-10, atol=1e-12 * np.abs(H0).max())


def test_diagnostics_report_H():
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=4)
    g, p, U = so.workload_state(cfg)
    d = so.diagnostics(U, g, p)
    assert d.shape == (6,) and np.isfinite(d).all() and d[4] >= d[5] > 0


def test_weighted_rms_is_a_mean_over_every_node():
    """The RMS of a constant field is its magnitude, a field that is c on one radial element
    and 0 on the other has RMS c sqrt(V_e / V) with V_e the element's quadrature volume, and
    no RMS exceeds the maximum (positive weights) -- with the weights broadcast over phi, a
    sum of w alone would miss the factor N_phi."""
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=16)
    g, p, U = so.workload_state(cfg)
    w = so.quadrature_weights(g)
    assert np.all(w > 0)
    shape = U.shape[1:]
    np.testing.assert_allclose(so.weighted_rms(np.full(shape, -3.0), w), 3.0, rtol=1e-14)
    f = np.zeros(shape)
    f[1] = 2.0
    wf = np.broadcast_to(w, shape)
    np.testing.assert_allclose(so.weighted_rms(f, w), 2.0 * np.sqrt(wf[1].sum() / wf.sum()),
                               rtol=1e-14)
    H = so.hamiltonian_constraint(U, g, p)
    for e in range(2):
        assert so.weighted_rms(H[e], w[e]) <= np.abs(H[e]).max() * (1 + 1e-14)
    d = so.diagnostics(U, g, p)
    np.testing.assert_allclose(d[4], np.abs(H).max(), rtol=1e-14)
    np.testing.assert_allclose(d[5], so.weighted_rms(H, w), rtol=1e-14)
