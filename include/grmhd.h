/*
 * grmhd.h - C ABI of the GB300 coupled BSSN-Valencia spectral right-hand side.
 *
 * The library evolves the unsplit coupled system of the paper (arXiv 2508.18221):
 * the Valencia form of ideal GRMHD ("GRMHD Conservative Form": conserved variables,
 * fluxes, geometric source) together with the BSSN equations, 1+log slicing and the
 * Gamma-driver shift (Methods: "BSSN Evolution Equations", "Gauge Conditions"), on a
 * multi-element mapped Chebyshev (r) x Chebyshev (theta) x Fourier (phi) grid around a
 * Kerr-Schild black hole (Methods: "Grid Discretization", "The Spectral Derivative
 * Operators"), with the paper's modal filter ("Dealiasing and Spectral Filtering"),
 * primitive recovery ("The Primitive Variable Recovery") and Runge-Kutta time
 * integration ("Time Integration", SSP-RK3 by default, the printed RK4 as option).
 *
 * Conventions shared by every call
 *   - Every function returns an int status: GRMHD_OK (0), a negative error code, or a
 *     positive warning (the call did its work; see GRMHD_WPRECISION).
 *     No call aborts, traps or exits the process; after an error the context stays
 *     usable and grmhd_last_error() describes the cause.
 *   - Field arrays use the canonical layout double[nv][E][N_r][N_theta][N_phi] with phi
 *     fastest and radial nodes ascending inside each element (adjacent elements share
 *     their interface radius: that node is stored once per element).
 *   - Variable order (nv = 32): 0-5 gammatilde_{rr,rth,rph,thth,thph,phph}; 6 phi;
 *     7-12 Atilde_ij (same order); 13 K; 14-16 Gammatilde^i; 17 alpha; 18-20 beta^i;
 *     21-23 B^i (Gamma-driver); 24 sqrt(gamma) D; 25-27 sqrt(gamma) S_i (covariant);
 *     28 sqrt(gamma) tau; 29-31 sqrt(gamma) B^i (Eulerian field, contravariant).
 *   - Primitive layout (7 fields): rho, v^r, v^theta, v^phi (Eulerian, contravariant),
 *     eps, p, W.
 *   - A pointer argument is caller-owned; it is read or written only during the call.
 *     `on_device` = 1 means the pointer is CUDA device memory (stream-ordered on the
 *     context's stream), 0 means host memory (the call synchronises before returning).
 *   - All work of a context is issued on the CUDA stream given to grmhd_create
 *     (NULL = legacy default stream).  One GPU; the device current at create time.
 */
#ifndef GRMHD_H
#define GRMHD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GRMHD_OK = 0,
    GRMHD_EINVAL = -1,        /* invalid argument (sizes, ranges, NULL pointers)       */
    GRMHD_ENOMEM = -2,        /* device or host allocation failed                      */
    GRMHD_ECUDA = -3,         /* a CUDA runtime call failed (message in last_error)    */
    GRMHD_ENAN = -4,          /* a non-finite value appeared in the evolved state      */
    GRMHD_ETIMEOUT = -5,      /* a bounded device-side wait gave up                    */
    GRMHD_EUNSUPPORTED = -6,  /* option value not built into this library              */
    /* positive statuses are warnings: the call did its work and its outputs are valid */
    GRMHD_WPRECISION = 1      /* created with precision 2 (TF32 contractions), a mode
                                 whose error exceeds the mixed-precision bar: its state's
                                 relative L2 error reaches O(1) within 100 steps on the
                                 2-element 12 x 12 x 16 workload; precision 1 stays below
                                 the spectral truncation level there                   */
};

enum { GRMHD_NV = 32, GRMHD_NPRIM = 7, GRMHD_NDIAG = 8 };

/* Grid (Methods, "Grid Discretization").  Radial elements [r_e, r_{e+1}] with
 * r_e = r_min (r_max/r_min)^(e/E) (elem_map = 1) or equal widths (elem_map = 0); each
 * element carries n_r Chebyshev-Gauss-Lobatto nodes under an affine map.  theta_basis 0
 * (default): theta uses n_theta Chebyshev-Gauss nodes on [theta_min, theta_max] (no node
 * on a pole).  theta_basis 1: the paper's uniform theta grid with a Fourier derivative
 * ("Pseudo-spectral theta derivative"): theta_k = (k + 1/2) pi / n_theta over the whole
 * sphere (theta_min = 0 and theta_max = pi required; the half-node shift keeps nodes off
 * the axis), every theta derivative and the theta filter acting on the double-Fourier
 * extension of the line over [0, 2 pi), whose values at 2 pi - theta are s u(theta,
 * phi + pi), s = -1 per theta index of a coordinate-basis component and -1 once more for
 * the sqrt(gamma)-weighted Valencia variables.  phi uses n_phi uniform nodes
 * 2 pi l / n_phi.  Limits: 1 <= n_elem, 4 <= n_r <= 64, 4 <= n_theta <= 128,
 * 4 <= n_phi <= 128 and even, 0 < r_min < r_max, 0 <= theta_min < theta_max <= pi. */
typedef struct {
    int n_elem;
    double r_min, r_max;
    int elem_map;
    int n_r, n_theta, n_phi;
    double theta_min, theta_max;
    int theta_basis;
} grmhd_grid;

/* Physics: Kerr-Schild mass M and spin a (|a| < M), Gamma-law index (p = (Gamma-1) rho
 * eps, Methods "Ideal-gas EOS"), floors of rho and eps used by primitive recovery. */
typedef struct {
    double M, a, gamma_eos;
    double rho_atm, eps_atm;
} grmhd_physics;

/* Options.  precision: 0 = FP64 values everywhere; 1 = mixed: derivative contractions
 * as split-BF16 x3 tensor-core products with FP32 results and the BSSN / Valencia
 * algebra in FP32, while the metric determinant and inverse, the conformal factor, the
 * interface penalty, the Runge-Kutta sums, the primitive recovery and the filter stay
 * FP64; 2 = as 1 with TF32 products (at most 128 nodes per direction for 1 and 2).
 * integrator: 0 SSP-RK3, 1 RK4.
 * evolve_metric: 1 evolve BSSN + gauge, 0 keep the metric fixed (RHS of variables
 * 0-23 is zero).  gauge: 0 1+log + Gamma-driver with damping eta, 1 frozen lapse/shift.
 * filter: bits 0/1/2 filter the Valencia variables in r/theta/phi, bits 3/4/5 the BSSN
 * variables in r/theta/phi (default 47: all but theta for BSSN); filt_alpha, filt_p are
 * the exponential-filter constants (paper: 36, 8); dealias23_phi applies the 2/3 rule
 * in phi, dealias23_theta in theta under theta_basis 1 (|k| > 2 n_theta / 3 of the
 * extended line zeroed; default 1; the Chebyshev theta filter has no 2/3 rule).  cfl: Courant factor for dt <= 0.  c2p_maxit, c2p_tol: iteration limit
 * and relative tolerance of the primitive recovery.  c2p_lambda: 0 (default) solves the
 * one-variable master function in mu = 1/(h W) by safeguarded Newton (tolerance: of the
 * step in mu); in (0, 1] it runs the paper's damped iteration instead ("The Primitive
 * Variable Recovery"): from the stored primitives (or, after grmhd_set_state, the dust
 * estimates v^i = gamma^ij S_j / (tau + D), eps = (tau + D)/(D W) - 1), the update
 * v^i += lam gamma^ij dS_j / (rho h W^2), eps += lam dtau / (rho W^2), rho = D / W with
 * lam = c2p_lambda at first and halved while the residual grows, until ||dS|| + |dtau| <
 * c2p_tol D or c2p_maxit updates (the paper: 30-40), then one Newton update of eps.  It
 * converges linearly: after 40 iterations from a cold start eps is within about 1e-9 of
 * the exact root on the 2-element workload (2e-11 in the torus), so the default stays
 * the Newton solve.  contraction: how the FP64
 * spectral contractions (all derivatives at precision 0, the filter at every precision)
 * run: 0 (default) on the FP16 tensor cores with exact base-256 digit slices of the
 * FP64 values (Ozaki splitting; up to 128 nodes per direction; each digit-order sum in an
 * exact accumulator of its own, error about 1e-15 of sum_j |D_ij| max_j |u_j|; above 64
 * Chebyshev nodes the FP64 units take the derivatives), 1 on the FP64 units.  coupling: 0 (default) one
 * unsplit right-hand side over all 32 variables per Runge-Kutta stage; 1 the paper's
 * coupled loop ("Coupled Main Loop"): per step the fluid is advanced by the selected
 * Runge-Kutta scheme on the frozen metric, then BSSN + gauge take one forward-Euler step
 * with the fluid frozen (matter sources from the updated fluid), then the filter.  glm: 1
 * adds GLM divergence cleaning ("GLM Constraint Damping Source") with the scalar psi as
 * variable 32 (state arrays then hold 33 fields, see grmhd_num_vars): d_t psi =
 * alpha (-glm_ch^2 D_i B^i - psi / glm_tau), D_i B^i = d_i(sqrt(gamma) B^i) / sqrt(gamma),
 * and -alpha sqrt(gamma) gamma^ij d_j psi added to the right-hand side of sqrt(gamma) B^i
 * (defaults glm_ch = 1, glm_tau = 1; psi starts at zero, is filtered with the Valencia
 * variables and averaged at duplicated interface nodes). */
typedef struct {
    int precision;
    int integrator;
    int evolve_metric;
    int gauge;
    double eta, cfl;
    int filter;
    double filt_alpha, filt_p;
    int dealias23_phi;
    int c2p_maxit;
    double c2p_tol;
    int contraction;
    int coupling;
    int glm;
    double glm_ch, glm_tau;
    int dealias23_theta;
    double c2p_lambda;
} grmhd_opts;

typedef struct grmhd_ctx grmhd_ctx;
typedef struct grmhd_batch grmhd_batch;

/* Fill the structs with the defaults listed above (M = 1, a = 0.5, Gamma = 4/3,
 * rho_atm = 1e-12, eps_atm = 1e-10, eta = 2, cfl = 0.3, filter = 47, 36, 8,
 * dealias on, c2p_maxit = 60, c2p_tol = 1e-15, c2p_lambda = 0). Any pointer may be NULL. */
int grmhd_defaults(grmhd_grid* grid, grmhd_physics* phys, grmhd_opts* opts);

/* Create a context for one instance of the paper's problem: a Kerr-Schild black hole of
 * mass M and spin a (Methods, "Background Geometry: ADM Split in Kerr-Schild Coordinates"),
 * a Gamma-law gas ("Ideal-gas EOS") and the multi-element Chebyshev x theta x Fourier grid
 * ("Grid Discretization", "The Spectral Derivative Operators").  Validates the parameters
 * (GRMHD_EINVAL), builds the operator matrices on the host, allocates every device buffer
 * (GRMHD_ENOMEM), and binds the CUDA stream `cuda_stream` (a cudaStream_t, or NULL).
 * *out receives the handle, which the caller releases with grmhd_destroy (NULL is a
 * no-op there); on an error *out is left NULL and nothing stays allocated.  With
 * opts.precision = 2 the context is created and the status is GRMHD_WPRECISION. */
int grmhd_create(const grmhd_grid* grid, const grmhd_physics* phys, const grmhd_opts* opts,
                 void* cuda_stream, grmhd_ctx** out);
int grmhd_destroy(grmhd_ctx* ctx);

/* Number of nodes E * n_r * n_theta * n_phi. */
long long grmhd_num_points(const grmhd_ctx* ctx);

/* Evolved variables per node: GRMHD_NV (32), or 33 with GLM cleaning (psi last).  Every
 * state and right-hand-side array of the context holds this many fields of
 * grmhd_num_points doubles; -1 for a NULL context. */
int grmhd_num_vars(const grmhd_ctx* ctx);

/* Node coordinates in canonical point order (3 arrays of num_points doubles: r, theta,
 * phi).  Any of the pointers may be NULL. Host memory. */
int grmhd_coords(const grmhd_ctx* ctx, double* r, double* theta, double* phi);

/* Initial data: exact Kerr-Schild slice converted to BSSN variables (phi = ln(det
 * gamma)/12, gammatilde = e^{-4phi} gamma, K = gamma^ij K_ij, Atilde = e^{-4phi}(K_ij -
 * gamma_ij K/3), Gammatilde^i = gammatilde^jk Gammatilde^i_jk, Gamma-driver B = 0)
 * plus matter given by primitives on the nodes: rho, p, v^r, v^theta, v^phi and the
 * vector potential A_phi (6 arrays of num_points doubles, host memory).  The
 * densitized field is sqrt(gamma) B^r = d_theta A_phi, sqrt(gamma) B^theta =
 * -d_r A_phi, B^phi = 0 with the grid's own derivative operators.  Replaces the state
 * and resets the primitive guess. */
int grmhd_init_prims(grmhd_ctx* ctx, const double* rho, const double* p, const double* vr,
                     const double* vth, const double* vph, const double* A_phi);

/* Copy a full canonical state (grmhd_num_vars * num_points doubles) in / out: the evolved
 * BSSN variables ("BSSN Evolution Equations", "Gauge Conditions", "Gamma-driver shift")
 * and the densitized conserved variables ("Conserved variables U").  set_state also
 * resets the primitive guess (the next primitive recovery starts from a bracket).  A NULL
 * pointer gives GRMHD_EINVAL; a device copy that fails gives GRMHD_ECUDA. */
int grmhd_set_state(grmhd_ctx* ctx, const double* state, int on_device);
int grmhd_get_state(grmhd_ctx* ctx, double* state, int on_device);

/* L(U) of the current state: one right-hand-side evaluation (one Runge-Kutta stage) of
 * the unsplit coupled system (Methods, "Numerical Algorithm and Mathematical Formulation",
 * "The Conserved Fluxes and Geometric Source Terms", "BSSN Evolution Equations", "Gauge
 * Conditions") without the post-step filter, written to rhs_out (grmhd_num_vars *
 * num_points doubles, caller-owned, canonical layout).  The state is unchanged; the
 * primitive guess is updated by the recovery inside.  GRMHD_EINVAL for a NULL rhs_out. */
int grmhd_rhs(grmhd_ctx* ctx, double* rhs_out, int on_device);

/* Primitive recovery (Methods, "The Primitive Variable Recovery") of the current state
 * into prim_out (GRMHD_NPRIM * num_points doubles, caller-owned); *n_failed (may be NULL)
 * receives the number of points where the floor eps_atm was applied or the recovery did
 * not converge (a count, not an error status).  Updates the stored guess.  With
 * opts.c2p_lambda > 0 the recovery is the paper's damped fixed-point iteration instead
 * (see grmhd_opts). */
int grmhd_con2prim(grmhd_ctx* ctx, double* prim_out, int on_device, long long* n_failed);

/* Advance nsteps time steps of size dt (Methods, "Time Integration: The Fourth-Order
 * Runge-Kutta", "The Stability and Complexity", "Dealiasing and Spectral Filtering",
 * "Coupled Main Loop"; dt <= 0: dt from the CFL condition of the current state, computed
 * once per call).  Each step: SSP-RK3 (3 stages) or RK4 (4), then the post-step filter.
 * The nsteps loop is captured in a CUDA graph (rebuilt when nsteps or the dt mode
 * changes).  Returns GRMHD_EINVAL for nsteps < 1, GRMHD_ENAN if the state is non-finite
 * afterwards, GRMHD_ETIMEOUT when a bounded device wait gave up.  *dt_used (may be NULL)
 * receives dt. */
int grmhd_step(grmhd_ctx* ctx, double dt, int nsteps, double* dt_used);

/* dt of the CFL condition for the current state (Methods, "The Stability and
 * Complexity"): cfl * min over nodes of min(dr, r dtheta, r sin(theta) dphi) divided
 * by max over nodes of |beta|_gamma + max(alpha, sqrt(2 alpha)). */
int grmhd_cfl_dt(grmhd_ctx* ctx, double* dt);

/* Diagnostics (out[GRMHD_NDIAG]): 0 rest mass sum w D~, 1 entropy sum w rho s sqrt(gamma)
 * with s = ln(p/rho^Gamma)/(Gamma-1) (Methods, "The Entropy Stability and
 * Convergence", quadrature weights as the cell volume), 2 max |d_i(sqrt(gamma) B^i)|,
 * 3 floor/failed points of the last recovery, 4 dt of the last step, 5 max |H| and 6 the
 * quadrature RMS of the Hamiltonian constraint H = R + (2/3) K^2 - Atilde_ij Atilde^ij -
 * 16 pi rho (rho the Eulerian energy density; the right-hand side's derivatives; FP32
 * algebra in the mixed modes), 7 reserved.  Costs one right-hand-side evaluation. */
int grmhd_diag(grmhd_ctx* ctx, double out[GRMHD_NDIAG]);

/* Kernel launches issued by the last grmhd_step / grmhd_rhs call (per step / per call). */
long long grmhd_launch_count(const grmhd_ctx* ctx);

/* Profiling: time each kernel class of one right-hand-side evaluation and of the filter
 * on the current state, `reps` launches each, with CUDA events on the context's stream.
 * ms_out[0..n-1] (n <= GRMHD_NKT) receives the mean milliseconds per launch of:
 * 0 prep (metric + primitive recovery + fluxes), 1-3 first-derivative contractions
 * r/theta/phi, 4 interface mean of d_r, 5-7 second-derivative contractions r/theta/phi,
 * 8 interface mean of d_rr, 9 rhs (BSSN + Valencia + penalty + RK), 10-12 filter
 * contractions r/theta/phi.  For the contraction classes, flops_out (may be NULL)
 * receives the algorithmic flops of one launch (FP64 modes: 2 N per output node for a
 * dense row, about N for the reflection-split form, counted exactly; mixed modes: the
 * tensor-core MMA flops of the padded tiles and slice products) and bytes_out (may be
 * NULL) the algorithmic HBM bytes (each source element read once, each result written
 * once, accumulated results read too); 0 for the other classes.  The state is left
 * unchanged. */
enum { GRMHD_NKT = 13 };
int grmhd_kernel_times(grmhd_ctx* ctx, int reps, double* ms_out, double* flops_out,
                       double* bytes_out, int n);

/* Independent instances advanced together (the batched workload of many black-hole
 * set-ups; each instance is the problem of grmhd_create, advanced as grmhd_step does,
 * Methods "Numerical Implementation of Coupled GRMHD-Einstein Evolution").  Instances that share n_r, n_theta, n_phi, the theta range, gamma_eos, the
 * floors and every option field form one group; a group is one grid whose radial
 * elements are the instances' elements in order (the right-hand side does not depend
 * on M and a, which enter only through the initial data), with interface coupling and
 * the outer-boundary freeze applied per instance and a per-instance time step.  Each
 * group therefore advances with the launches of a single instance, and all groups of a
 * step are recorded in one CUDA graph.  Instances may differ in spin, mass, element
 * count and radial range inside a group, and in anything across groups.  grids, phys
 * and opts are arrays of n entries.  All instances share the stream given here.
 * n < 1, a NULL array or any instance's parameters outside the ranges grmhd_create
 * accepts give GRMHD_EINVAL before any device work. */
int grmhd_batch_create(int n, const grmhd_grid* grids, const grmhd_physics* phys,
                       const grmhd_opts* opts, void* cuda_stream, grmhd_batch** out);
int grmhd_batch_num_groups(const grmhd_batch* b);
/* nodes of instance i (its canonical arrays have grmhd_batch_num_vars(b, i) * that many
 * doubles) */
long long grmhd_batch_num_points(const grmhd_batch* b, int i);
/* evolved variables of instance i (32, or 33 with GLM cleaning); -1 on a bad index */
int grmhd_batch_num_vars(const grmhd_batch* b, int i);
/* node coordinates of instance i (host arrays of num_points doubles, any may be NULL) */
int grmhd_batch_coords(const grmhd_batch* b, int i, double* r, double* theta, double* phi);
/* initial data of instance i from primitives on its nodes (as grmhd_init_prims) */
int grmhd_batch_init_prims(grmhd_batch* b, int i, const double* rho, const double* p,
                           const double* vr, const double* vth, const double* vph,
                           const double* A_phi);
/* canonical state of instance i in / out (layout and on_device as grmhd_set_state) */
int grmhd_batch_set_state(grmhd_batch* b, int i, const double* state, int on_device);
int grmhd_batch_get_state(grmhd_batch* b, int i, double* state, int on_device);
/* CFL time step of every instance's current state (dt_out: host array of n) */
int grmhd_batch_cfl_dt(grmhd_batch* b, double* dt_out);
/* kernel launches per step issued by the last grmhd_batch_step (all groups) */
long long grmhd_batch_launch_count(const grmhd_batch* b);
/* nsteps steps of every instance, instance i with time step dt[i] > 0 (host array) */
int grmhd_batch_step(grmhd_batch* b, const double* dt, int nsteps);
int grmhd_batch_destroy(grmhd_batch* b);
const char* grmhd_batch_last_error(const grmhd_batch* b);

/* Approximate XCTS initial data (paper: "Initial Data: Approximate XCTS Solution"): solves
 * the conformal Hamiltonian constraint lap psi = -2 pi rho psi^5 (flat conformal metric,
 * A_ij = 0) by the paper's fixed-point relaxation psi_{k+1} = L^-1(-2 pi rho psi_k^5) from
 * the puncture psi = 1 + M / (2 r), with d_r psi = -M / (2 r_min^2) at r_min, psi + r d_r psi
 * = 1 at r_max and C^1 matching at element interfaces, then sets the state to the slice
 * gamma_ij = psi^4 (flat metric), K = 0 (lapse psi^-2, shift zero) carrying the fluid and
 * field of the given primitives (as grmhd_init_prims).  Host arrays of num_points values in
 * the canonical node order; rho is the primitive rest-mass density.  At most `iters`
 * iterations, fewer when max |psi_{k+1} - psi_k| < tol (tol = 0: all).  psi_out (may be NULL)
 * receives psi; changes (iters entries, may be NULL) the change of every iteration; stats
 * (3 entries, may be NULL) the set-up time in ms (the angular operators' real Schur forms
 * on the host and the inversion of the radial systems), the mean time per iteration
 * and the iterations done.  Each phi mode's operator is solved through the real Schur form
 * Q T Q^T of its angular part: in the orthogonal basis Q it is block upper triangular, a back
 * substitution over n_theta radial systems of E n_r unknowns, which the library inverts
 * and solves in its own kernels.  Needs theta_basis = 1 and a single-instance context
 * (GRMHD_EUNSUPPORTED otherwise, or when an angular operator has no real Schur form, or
 * above 12,800 radial nodes); GRMHD_ENAN when the fixed
 * point diverges (too dense a source).  Allocates 2 (N_phi/2 + 1) n_theta (E n_r)^2 doubles
 * of device memory for the call. */
int grmhd_xcts_init(grmhd_ctx* ctx, const double* rho, const double* p, const double* vr,
                    const double* vth, const double* vph, const double* A_phi, int iters, double tol,
                    double* psi_out, double* changes, double* stats);

/* Autotuner of the FP64 digit-slice contractions (a service of the library, outside the
 * paper).  The tensor-core contraction of a class (direction dir 0 r / 1 theta / 2 phi,
 * nodes n along it, kind 0 derivative / 1 filter) runs either with one TMEM accumulator
 * set (two CTAs per SM up to 32 nodes: 7 x 32 columns) or with two (one CTA per SM; the
 * MMAs of the next 128-line tile run while the previous tile's results are converted and
 * stored).  A process-wide table keeps the choice per class: 0 = not tuned
 * (one set), 1 or 2 sets.  At the first context or batch of a process the library reads
 * the table a previous run stored, from the file the environment variable
 * GRMHD_TUNING_FILE names or else fx_tuning.txt next to the library (lines
 * "dir n kind sets"; python -m paper_2508_18221_gb300.autotune writes it).
 * grmhd_tune_contractions times both choices for every class the context uses (nfields
 * fields of its own state per launch, reps launches each, CUDA events on its stream), keeps
 * the faster in the table (two sets only when they are at least 2 % faster: the
 * launch-to-launch spread is about 1 %) and returns the mean ms per launch in ms_out[(dir * 2 + kind) * 2 +
 * sets - 1] (kind 0 derivative, 1 filter; -1 where the choice does not exist) and the choice
 * in choice_out[dir * 2 + kind] (0 where the class runs on the FP64 units); either may be
 * NULL.  It overwrites the context's scratch buffers only.  GRMHD_EINVAL for nfields
 * outside [1, 32] or reps < 1; GRMHD_EUNSUPPORTED on a batch's group context.
 * grmhd_tune_set sets one entry (GRMHD_EINVAL outside the ranges above); grmhd_tune_get
 * returns it (or GRMHD_EINVAL). */
int grmhd_tune_contractions(grmhd_ctx* ctx, int nfields, int reps, double* ms_out, int* choice_out);
int grmhd_tune_set(int dir, int n, int kind, int sets);
int grmhd_tune_get(int dir, int n, int kind);

/* Test hook: apply the first derivative along direction dir (0 r, 1 theta, 2 phi) to
 * `nfields` canonical fields (nfields * num_points doubles) with the library's
 * operators (radial: per element, one-sided at element ends).  Device pointers. */
int grmhd_debug_deriv(grmhd_ctx* ctx, const double* in, double* out, int nfields, int dir);

/* Test hook of the device-side wait limits: one digit-slice contraction whose tiles are
 * withheld, so that every bounded wait of the kernel runs out (about 0.5 s); the CTAs leave,
 * free their tensor memory and flag the failure, and the call returns GRMHD_ETIMEOUT with the
 * context still usable (GRMHD_OK would mean the limit did not act; GRMHD_EUNSUPPORTED
 * without digit-slice operators).  Nothing faults or hangs. */
int grmhd_debug_wait_timeout(grmhd_ctx* ctx);

/* Test hook: the theta derivative (filter = 0) or the theta filter (filter = 1) of
 * `nfields` canonical fields (device pointers, nfields * num_points doubles each), field f
 * taken with parity[f] = +1 or -1 (host array) under theta_basis 1 (ignored under the
 * Chebyshev basis).  GRMHD_EINVAL for other parities or more fields than the context's
 * folding buffers hold (at least 24). */
int grmhd_debug_theta(grmhd_ctx* ctx, const double* in, double* out, int nfields, const int* parity,
                      int filter);

/* Allocation-free CFL time step (the paper has no counterpart: this is a service of the
 * library).  Some callers cannot call cudaMalloc: hosts that own every byte of device
 * memory through their own pool allocator and forbid outside allocations, and
 * latency-bound loops where an allocation (which can synchronise the whole device) is
 * not acceptable.  They cannot create a context either, since grmhd_create allocates.
 * This entry point computes the same dt as grmhd_cfl_dt from a caller-owned canonical
 * state (device pointer, GRMHD_NV * n_points doubles) and the grid's smallest node
 * spacing hmin = min over nodes of min(dr, r dtheta, r sin(theta) dphi), writing dt to
 * the device pointer dt_out, stream-ordered on cuda_stream (NULL = legacy default).
 * It allocates nothing: its reduction scratch is a fixed 512 KiB array in the library's
 * device memory, which every GPU that loads the library holds until the process exits.
 * Limits: n_points <= 16,777,216 (larger inputs return GRMHD_EINVAL before any work);
 * hmin > 0, cfl > 0.  The first call on a device looks up that array's device address
 * (with the device current): make that first call before any stream capture.  The
 * address belongs to the device's context; after a cudaDeviceReset the next call finds
 * a new context and looks the address up again, so the first call after a reset, too,
 * belongs before any stream capture.  All
 * calls share the array and it keeps the last call's contents (every call overwrites
 * what it reads, so nothing needs clearing); calls that overlap on the GPU (several
 * streams, threads or devices' work in flight on the same device at once) race. */
int grmhd_cfl_dt_noalloc(const double* state, long long n_points, double hmin, double cfl,
                         double* dt_out, void* cuda_stream);

const char* grmhd_strerror(int status);
const char* grmhd_last_error(const grmhd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRMHD_H */
