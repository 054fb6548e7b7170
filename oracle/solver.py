"""Multi-element spectral right-hand side, Runge-Kutta stages, post-step filter,
CFL step, diagnostics and initial data.  Test infrastructure only.

Paper: Methods ("Numerical Algorithm and Mathematical Formulation", "Grid
Discretization", "The Spectral Derivative Operators", "Dealiasing and Spectral
Filtering", "Time Integration", "The Stability and Complexity", "The Entropy
Stability and Convergence", "Coupled Main Loop").

Readings (the paper describes a "discontinuous spectral method on mapped
Chebyshev-Fourier grids" without stating the coupling):
* r: E radial elements with log-spaced (or equal) bounds, CGL nodes per element
  (ascending), affine map per element; theta: Chebyshev-Gauss nodes on
  [theta_min, theta_max]; phi: uniform periodic grid with a Fourier derivative;
* unsplit method of lines: one RHS over all 32 variables per stage;
* BSSN (second order in space): at the duplicated interface nodes, the one-sided
  radial first derivatives of both elements are replaced by their mean, and the
  radial second derivative D_r(mean d_r u) is averaged again; mixed second
  derivatives are D_theta / D_phi of the averaged radial derivative;
* Valencia: strong-form interface penalty with the Rusanov flux
  F* = (F_L + F_R)/2 - lambda (U_R - U_L)/2, lambda = max over both sides of
  |beta^r| + alpha sqrt(gamma^rr) (light-cone bound), scaled by
  1/(w_end J) with the Clenshaw-Curtis end weight;
* outer radial node: RHS = 0 (frozen); inner node (inside the horizon): no condition;
* time integrator: SSP-RK3 (Shu-Osher) by default, the paper's RK4 as an option;
* coupling: the unsplit method of lines by default; as an option the paper's coupled
  loop ("Coupled Main Loop", "Main Coupled Evolution Loop"): per step the fluid is
  advanced by the Runge-Kutta scheme on the frozen metric, then BSSN and gauge take one
  forward-Euler step with the fluid frozen, the matter sources computed from the
  updated fluid (first-order Lie splitting; the paper's "half-step" is read as the
  fluid half of the split step, both halves advancing by dt, since a fluid advanced by
  dt/2 per step would fall behind the metric);
* GLM divergence cleaning ("GLM Constraint Damping Source"), option glm = 1: a 33rd
  variable psi with d_t psi = alpha (-c_h^2 D_i B^i - psi / tau), D_i B^i =
  d_i(sqrt(gamma) B^i) / sqrt(gamma) the covariant divergence, and the source
  -alpha sqrt(gamma) gamma^ij d_j psi added to the right-hand side of sqrt(gamma) B^i
  (readings: the paper's flat-space "div B" is the covariant divergence; both terms
  carry the lapse, as every source of the Valencia system does; the field source has
  the sign of Dedner et al. 2002, -grad psi, since the printed +d_i psi makes the psi-B
  subsystem anti-damped instead of a wave equation; c_h = 1, tau = 1 by default, the
  paper states no values).  Radial derivatives of psi and the divergence are averaged
  at interfaces, psi is filtered with the Valencia variables and averaged at duplicated
  nodes after the filter, like the BSSN variables;
* post-step filter: exponential (alpha = 36, p = 8) on the Chebyshev modes in r
  (per element) and theta and on the Fourier modes in phi, plus the 2/3 rule in
  phi; then the BSSN variables of duplicated interface nodes are averaged;
* theta_basis = 1, the paper's own polar discretisation ("Pseudo-spectral theta
  derivative": Fourier on an evenly spaced theta grid): theta_k = (k + 1/2) pi / N_theta
  on the whole of (0, pi), and every theta derivative and theta filter acts on the
  double-Fourier extension of the line over [0, 2 pi), the values at 2 pi - theta being
  s u(theta, phi + pi) with the parity s of the component (-1 per theta index of a
  coordinate-basis component, and -1 once more for a sqrt(gamma)-weighted density, which
  behaves like sin(theta) on the axis); the theta filter uses k_max = N_theta and, with
  dealias23_theta, the 2/3 rule of the extended line.  The derivative of a component with
  parity s has parity -s, so second derivatives are compositions with the parity of
  the inner result.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import spectral as sp
from . import kerr_schild as ks
from . import valencia as va
from . import bssn as bs

NV = 32
SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
# canonical variable slots
I_GT, I_PHI, I_AT, I_K, I_GAM, I_ALPHA, I_BETA, I_BG = 0, 6, 7, 13, 14, 17, 18, 21
I_D, I_S, I_TAU, I_B = 24, 25, 28, 29
I_PSI = 32                      # GLM scalar (glm = 1 only: 33 variables)
N_BSSN = 24
# fields whose first derivatives are taken (all BSSN + gauge except the driver B^i)
DERIV1 = list(range(0, 21))
# fields whose second derivatives are taken: gammatilde_ij, phi, alpha, beta^i
DERIV2 = [0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20]


def theta_parity(nv=NV + 1):
    """Sign of each canonical variable under the double-Fourier extension in theta.

    The extension maps the chart (theta, phi) to (-theta, phi + pi), whose Jacobian is
    diag(1, -1, 1) in (r, theta, phi): a coordinate-basis component changes sign once for
    every theta index it carries.  The evolved Valencia variables are densities
    sqrt(gamma) U, and sqrt(gamma) = r^2 sin(theta) x (a smooth even factor) changes sign
    with sin(theta), so they take one more sign (reading: the extension is chosen to be
    smooth across the axis)."""
    par = np.ones(nv)
    th = lambda *idx: (-1.0) ** sum(1 for i in idx if i == 1)
    for n, (i, j) in enumerate(SYM):
        par[I_GT + n] = th(i, j)
        par[I_AT + n] = th(i, j)
    for i in range(3):
        par[I_GAM + i] = th(i)
        par[I_BETA + i] = th(i)
        par[I_BG + i] = th(i)
        par[I_S + i] = -th(i)
        par[I_B + i] = -th(i)
    par[I_D] = -1.0
    par[I_TAU] = -1.0
    return par


THETA_PAR = theta_parity()
# parity of the theta flux sqrt(gamma) F^theta of each Valencia variable: one more
# theta index than the variable itself
FLUX_T_PAR = -THETA_PAR[I_D:I_D + 8]


def _bc(par):
    """Parity vector broadcast over the four grid axes."""
    return np.asarray(par)[:, None, None, None, None]


@dataclasses.dataclass
class Params:
    M: float = 1.0
    a: float = 0.5
    gamma_eos: float = 4.0 / 3.0
    n_elem: int = 2
    r_min: float = 1.8
    r_max: float = 20.0
    elem_map: int = 1
    n_r: int = 12
    n_theta: int = 12
    n_phi: int = 16
    theta_min: float = 0.0
    theta_max: float = math.pi
    evolve_metric: int = 1
    gauge: int = 0
    eta: float = 2.0
    integrator: int = 0          # 0 SSP-RK3, 1 RK4
    # bits 0/1/2: r/theta/phi filter on the 8 Valencia variables; bits 3/4/5: r/theta/phi
    # on the 24 BSSN + gauge variables.  Default 47: everything except theta on BSSN.
    filter_mask: int = 47
    filt_alpha: float = 36.0
    filt_p: float = 8.0
    dealias23_phi: int = 1
    cfl: float = 0.3
    eps_atm: float = 1e-10       # floor of the specific internal energy
    coupling: int = 0            # 0 unsplit method of lines, 1 the paper's split loop
    evolve_fluid: int = 1        # 0: Valencia right-hand side zero (BSSN half of a split step)
    glm: int = 0                 # 1: GLM divergence cleaning with the scalar psi (variable 32)
    glm_ch: float = 1.0
    glm_tau: float = 1.0
    theta_basis: int = 0         # 0 Chebyshev-Gauss in theta, 1 the paper's Fourier theta
    dealias23_theta: int = 1     # 2/3 rule in the theta filter (theta_basis = 1 only)

    @classmethod
    def from_config(cls, cfg, **kw):
        base = dict(M=cfg.M, a=cfg.a, gamma_eos=cfg.gamma_eos, n_elem=cfg.n_elem,
                    r_min=cfg.r_min, r_max=cfg.r_max, elem_map=cfg.elem_map, n_r=cfg.n_r,
                    n_theta=cfg.n_theta, n_phi=cfg.n_phi, theta_min=cfg.theta_min,
                    theta_max=cfg.theta_max, cfl=cfg.cfl,
                    theta_basis=getattr(cfg, "theta_basis", 0))
        base.update(kw)
        return cls(**base)


class Grid:
    """Node coordinates and per-element affine maps."""

    def __init__(self, p: Params):
        self.p = p
        E = p.n_elem
        if p.elem_map == 1:
            self.bounds = p.r_min * (p.r_max / p.r_min) ** (np.arange(E + 1) / E)
        else:
            self.bounds = p.r_min + (p.r_max - p.r_min) * np.arange(E + 1) / E
        self.bounds[0], self.bounds[-1] = p.r_min, p.r_max
        self.xr = sp.cgl_nodes(p.n_r)
        self.xt = sp.gauss_nodes(p.n_theta)
        a_, b_ = self.bounds[:-1], self.bounds[1:]
        self.r = 0.5 * (a_ + b_)[:, None] + 0.5 * (b_ - a_)[:, None] * self.xr[None, :]
        self.r_scale = 2.0 / (b_ - a_)                       # dx/dr per element
        self.fourier_theta = p.theta_basis == 1
        if self.fourier_theta:
            if abs(p.theta_min) > 1e-12 or abs(p.theta_max - np.pi) > 1e-12:
                raise ValueError("the Fourier theta basis covers the whole of [0, pi]")
            self.theta = sp.uniform_theta_nodes(p.n_theta)
            self.t_scale = 1.0
        else:
            self.theta = (p.theta_min + 0.5 * (p.theta_max - p.theta_min) * (1.0 + self.xt))
            self.t_scale = 2.0 / (p.theta_max - p.theta_min)
        self.phi = sp.fourier_nodes(p.n_phi)
        self.shape = (E, p.n_r, p.n_theta, p.n_phi)
        R = self.r[:, :, None, None]
        T = self.theta[None, None, :, None]
        P = self.phi[None, None, None, :]
        self.R, self.T, self.P = np.broadcast_arrays(R, T, P)

    # derivative operators on arrays whose last four axes are (E, N_r, N_theta, N_phi)
    def d_r(self, u):
        out = np.empty_like(u)
        for e in range(self.p.n_elem):
            out[..., e, :, :, :] = sp.cheb_deriv(u[..., e, :, :, :], self.xr, axis=u.ndim - 4,
                                                 scale=self.r_scale[e])
        return out

    def d_t(self, u, parity=None):
        """theta derivative; parity (scalar or broadcastable to u) is the sign of the
        component under the double-Fourier extension and must be given for the Fourier
        basis (ignored by the Chebyshev basis)."""
        if self.fourier_theta:
            if parity is None:
                raise ValueError("the Fourier theta derivative needs the parity of the field")
            return sp.fourier_theta_deriv(u, u.ndim - 2, u.ndim - 1, parity)
        return sp.cheb_deriv(u, self.xt, axis=u.ndim - 2, scale=self.t_scale)

    def d_p(self, u):
        return sp.fourier_deriv(u, axis=u.ndim - 1)

    def average_interfaces(self, u):
        """Replace both copies of every duplicated interface node by their mean."""
        u = u.copy()
        for e in range(self.p.n_elem - 1):
            m = 0.5 * (u[..., e, -1, :, :] + u[..., e + 1, 0, :, :])
            u[..., e, -1, :, :] = m
            u[..., e + 1, 0, :, :] = m
        return u


# ---------------------------------------------------------------- state <-> tensors
def sym_from(u, base):
    """[..., 3, 3] symmetric tensor from six canonical slots starting at base."""
    t = np.empty(u.shape[1:] + (3, 3))
    for n, (i, j) in enumerate(SYM):
        t[..., i, j] = u[base + n]
        t[..., j, i] = u[base + n]
    return t


def vec_from(u, base):
    return np.stack([u[base], u[base + 1], u[base + 2]], axis=-1)


def unpack_bssn(U):
    return {"gt": sym_from(U, I_GT), "phi": U[I_PHI], "At": sym_from(U, I_AT), "K": U[I_K],
            "Gt": vec_from(U, I_GAM), "alpha": U[I_ALPHA], "beta": vec_from(U, I_BETA),
            "B": vec_from(U, I_BG)}


def metric_from_bssn(f):
    """gamma_ij = e^{4 phi} gammatilde_ij, sqrt(gamma) = sqrt(det gamma_ij)."""
    gam = np.exp(4.0 * f["phi"])[..., None, None] * f["gt"]
    return gam, np.sqrt(ks.det3(gam))


# ------------------------------------------------------------------- right-hand side
def primitives(U, p: Params):
    """Primitive recovery at every node (undensitizing with the current sqrt(gamma))."""
    f = unpack_bssn(U)
    gam, sqg = metric_from_bssn(f)
    D = U[I_D] / sqg
    S_d = vec_from(U, I_S) / sqg[..., None]
    tau = U[I_TAU] / sqg
    B_u = vec_from(U, I_B) / sqg[..., None]
    rho, v_u, eps, pr, W, ok = va.con2prim(D, S_d, tau, B_u, gam, p.gamma_eos, eps_min=p.eps_atm)
    return {"rho": rho, "v": v_u, "eps": eps, "p": pr, "W": W, "ok": ok, "B": B_u}


def _derivs(g: Grid, U):
    """First derivatives of the 21 differentiated BSSN fields, radial ones averaged at
    interfaces; second derivatives of the 11 second-order fields."""
    src = U[DERIV1]
    par1 = _bc(THETA_PAR[DERIV1])
    dr = g.average_interfaces(g.d_r(src))
    dt = g.d_t(src, par1)
    dp = g.d_p(src)
    d1 = np.stack([dr, dt, dp], axis=0)           # [3(d), 21, E, Nr, Nt, Np]
    idx2 = [DERIV1.index(v) for v in DERIV2]
    par2 = _bc(THETA_PAR[DERIV2])
    a_r, a_t, a_p = dr[idx2], dt[idx2], dp[idx2]
    d_rr = g.average_interfaces(g.d_r(a_r))
    d_rt = g.d_t(a_r, par2)
    d_rp = g.d_p(a_r)
    d_tt = g.d_t(a_t, -par2)                      # d_theta u has the opposite parity
    d_tp = g.d_p(a_t)
    d_pp = g.d_p(a_p)
    d2 = np.empty((3, 3) + a_r.shape)
    d2[0, 0], d2[1, 1], d2[2, 2] = d_rr, d_tt, d_pp
    d2[0, 1] = d2[1, 0] = d_rt
    d2[0, 2] = d2[2, 0] = d_rp
    d2[1, 2] = d2[2, 1] = d_tp
    return d1, d2


def _d1_fields(d1):
    """Map the stacked first derivatives to tensor arrays [..., d, ...]."""
    def scal(v):
        return np.moveaxis(d1[:, DERIV1.index(v)], 0, -1)

    def vec(base):
        return np.stack([scal(base), scal(base + 1), scal(base + 2)], axis=-1)

    def sym(base):
        t = np.empty(d1.shape[2:] + (3, 3, 3))
        for n, (i, j) in enumerate(SYM):
            t[..., :, i, j] = scal(base + n)
            t[..., :, j, i] = scal(base + n)
        return t
    return {"gt": sym(I_GT), "phi": scal(I_PHI), "At": sym(I_AT), "K": scal(I_K),
            "Gt": vec(I_GAM), "alpha": scal(I_ALPHA), "beta": vec(I_BETA)}


def _d2_fields(d2):
    def scal(v):
        a = d2[:, :, DERIV2.index(v)]
        return np.moveaxis(np.moveaxis(a, 0, -1), 0, -1)  # [..., d, e]

    def vec(base):
        return np.stack([scal(base), scal(base + 1), scal(base + 2)], axis=-1)

    def sym(base):
        t = np.empty(d2.shape[3:] + (3, 3, 3, 3))
        for n, (i, j) in enumerate(SYM):
            t[..., :, :, i, j] = scal(base + n)
            t[..., :, :, j, i] = scal(base + n)
        return t
    return {"gt": sym(I_GT), "phi": scal(I_PHI), "alpha": scal(I_ALPHA), "beta": vec(I_BETA)}


def cc_end_weight(n):
    """Clenshaw-Curtis end-node weight on [-1, 1] for n CGL nodes."""
    return sp.clenshaw_curtis_weights(n)[0]


def rhs_from_prims(U, prim, g: Grid, p: Params, freeze_outer=True):
    """L(U) given the primitives at every node (the primitive recovery is done by the
    caller, see rhs).  freeze_outer=False skips the outer-boundary freeze (tests)."""
    E = p.n_elem
    f = unpack_bssn(U)
    gam, sqg = metric_from_bssn(f)
    alpha, beta = f["alpha"], f["beta"]
    rho, v, eps, B = prim["rho"], prim["v"], prim["eps"], prim["B"]

    # fluxes (densitized) and stress-energy tensor
    F = va.fluxes(rho, v, eps, B, alpha, beta, gam, p.gamma_eos) * sqg[..., None, None]
    T = va.stress_energy(rho, v, eps, B, alpha, beta, gam, p.gamma_eos)
    rho_adm, S_d, S_dd, S = va.matter_3p1(T, alpha, beta, gam)

    # spectral derivatives
    d1, d2 = _derivs(g, U)
    D1 = _d1_fields(d1)
    D2 = _d2_fields(d2)

    rhs = np.zeros_like(U)
    # ---- Valencia
    Fr = np.moveaxis(F[..., 0, :], -1, 0)
    Ft = np.moveaxis(F[..., 1, :], -1, 0)
    Fp = np.moveaxis(F[..., 2, :], -1, 0)
    div = g.d_r(Fr) + g.d_t(Ft, _bc(FLUX_T_PAR)) + g.d_p(Fp)
    e4 = np.exp(4.0 * f["phi"])
    dgam = e4[..., None, None, None] * (D1["gt"] + 4.0 * np.einsum("...ij,...d->...dij",
                                                                      f["gt"], D1["phi"]))
    Kij = e4[..., None, None] * (f["At"] + f["gt"] * f["K"][..., None, None] / 3.0)
    S_S, S_tau = va.sources_3p1(T, alpha, beta, gam, D1["alpha"], D1["beta"], dgam, Kij)
    asg = alpha * sqg
    rhs[I_D:I_D + 8] = -div
    rhs[I_S:I_S + 3] += np.moveaxis(asg[..., None] * S_S, -1, 0)
    rhs[I_TAU] += asg * S_tau

    # ---- GLM divergence cleaning
    if p.glm:
        psi = U[I_PSI]
        dpsi = np.stack([g.average_interfaces(g.d_r(psi)), g.d_t(psi, THETA_PAR[I_PSI]),
                         g.d_p(psi)], axis=-1)
        divB = g.average_interfaces(g.d_r(U[I_B]) + g.d_t(U[I_B + 1], THETA_PAR[I_B + 1])
                                    + g.d_p(U[I_B + 2]))
        ginv = ks.inv3(gam)
        rhs[I_PSI] = alpha * (-p.glm_ch ** 2 * divB / sqg - psi / p.glm_tau)
        rhs[I_B:I_B + 3] += np.moveaxis(-asg[..., None] * np.einsum("...ij,...j->...i", ginv, dpsi), -1, 0)

    # interface penalty (Rusanov) for the Valencia variables
    if E > 1:
        wend = cc_end_weight(p.n_r)
        ginv = ks.inv3(gam)
        lam = np.abs(beta[..., 0]) + alpha * np.sqrt(ginv[..., 0, 0])
        Ucons = U[I_D:I_D + 8]
        for e in range(E - 1):
            FL, FR = Fr[:, e, -1], Fr[:, e + 1, 0]
            UL, UR = Ucons[:, e, -1], Ucons[:, e + 1, 0]
            lmax = np.maximum(lam[e, -1], lam[e + 1, 0])
            Fs = 0.5 * (FL + FR) - 0.5 * lmax * (UR - UL)
            JL = 1.0 / g.r_scale[e]
            JR = 1.0 / g.r_scale[e + 1]
            rhs[I_D:I_D + 8, e, -1] += (FL - Fs) / (wend * JL)
            rhs[I_D:I_D + 8, e + 1, 0] -= (FR - Fs) / (wend * JR)

    # ---- BSSN + gauge
    if p.evolve_metric:
        matter = {"rho": rho_adm, "S_d": S_d, "S_dd": S_dd, "S": S}
        r = bs.bssn_rhs(f, D1, D2, matter, gauge=p.gauge, eta=p.eta)
        for n, (i, j) in enumerate(SYM):
            rhs[I_GT + n] = r["gt"][..., i, j]
            rhs[I_AT + n] = r["At"][..., i, j]
        rhs[I_PHI] = r["phi"]
        rhs[I_K] = r["K"]
        for i in range(3):
            rhs[I_GAM + i] = r["Gt"][..., i]
            rhs[I_BETA + i] = r["beta"][..., i]
            rhs[I_BG + i] = r["B"][..., i]
        rhs[I_ALPHA] = r["alpha"]

    if not p.evolve_fluid:
        rhs[I_D:] = 0.0
    # frozen outer boundary
    if freeze_outer:
        rhs[:, E - 1, -1] = 0.0
    return rhs


def rhs(U, g: Grid, p: Params, return_prims=False):
    """One right-hand-side evaluation L(U) (one Runge-Kutta stage)."""
    prim = primitives(U, p)
    out = rhs_from_prims(U, prim, g, p)
    return (out, prim) if return_prims else out


# ------------------------------------------------------------------------- filter
def apply_filter(U, g: Grid, p: Params):
    """Post-step modal filter in r (per element), theta, phi on the variable groups
    selected by filter_mask; then average BSSN variables at duplicated interface
    nodes.  The default leaves the BSSN variables unfiltered in theta: in spherical
    Kerr-Schild coordinates they behave like ln(sin theta) and sin^(+-2/3) theta
    near the poles, so their theta modes do not decay and the filter would move
    them by O(10%) (reading of the paper's "filter every mode")."""
    out = U.copy()
    m = p.filter_mask
    for grp, sl in ((0, slice(N_BSSN, U.shape[0])), (3, slice(0, N_BSSN))):
        if m & (1 << grp):
            for e in range(p.n_elem):
                out[sl, e] = sp.cheb_filter(out[sl, e], g.xr, axis=1, alpha=p.filt_alpha,
                                            p=p.filt_p)
        if m & (2 << grp):
            if g.fourier_theta:
                par = _bc(THETA_PAR[sl][:out[sl].shape[0]])
                out[sl] = sp.fourier_theta_filter(out[sl], 3, 4, par, alpha=p.filt_alpha,
                                                  p=p.filt_p, dealias23=bool(p.dealias23_theta))
            else:
                out[sl] = sp.cheb_filter(out[sl], g.xt, axis=3, alpha=p.filt_alpha, p=p.filt_p)
        if m & (4 << grp):
            out[sl] = sp.fourier_filter(out[sl], axis=4, alpha=p.filt_alpha, p=p.filt_p,
                                        dealias23=bool(p.dealias23_phi))
    out[:N_BSSN] = g.average_interfaces(out[:N_BSSN])
    if U.shape[0] > NV:
        out[I_PSI] = g.average_interfaces(out[I_PSI])
    return out


# ---------------------------------------------------------------------- time step
def rk_step(U, dt, g: Grid, p: Params):
    """One time step: SSP-RK3 in Shu-Osher form (or classical RK4), then the filter.
    With coupling = 1 the paper's split loop: the fluid step on the frozen metric, then
    one forward-Euler step of BSSN + gauge with the fluid frozen, then the filter."""
    if p.coupling == 1:
        pf = dataclasses.replace(p, coupling=0, evolve_metric=0, filter_mask=0)
        Uf = rk_step(U, dt, g, pf)
        U3 = Uf
        if p.evolve_metric:
            pb = dataclasses.replace(p, coupling=0, evolve_fluid=0)
            U3 = Uf + dt * rhs(Uf, g, pb)
        return apply_filter(U3, g, p) if p.filter_mask else U3
    if p.integrator == 0:
        U1 = U + dt * rhs(U, g, p)
        U2 = 0.75 * U + 0.25 * (U1 + dt * rhs(U1, g, p))
        U3 = U / 3.0 + 2.0 / 3.0 * (U2 + dt * rhs(U2, g, p))
    else:
        k1 = rhs(U, g, p)
        k2 = rhs(U + 0.5 * dt * k1, g, p)
        k3 = rhs(U + 0.5 * dt * k2, g, p)
        k4 = rhs(U + dt * k3, g, p)
        U3 = U + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return apply_filter(U3, g, p) if p.filter_mask else U3


def cfl_dt(U, g: Grid, p: Params):
    """dt = cfl * min_nodes min(dr, r dtheta, r sin(theta) dphi) / max_nodes lambda,
    lambda = |beta|_gamma + max(alpha, sqrt(2 alpha)) (light cone and 1+log gauge
    speed bound; the paper's c_fast is unstated).  Spacings are the smaller gap to
    a neighbouring node along each direction."""
    f = unpack_bssn(U)
    gam, _ = metric_from_bssn(f)
    alpha, beta = f["alpha"], f["beta"]
    bnorm = np.sqrt(np.einsum("...i,...ij,...j->...", beta, gam, beta))
    lam = bnorm + np.maximum(alpha, np.sqrt(2.0 * alpha))

    def gaps(x):
        d = np.diff(x)
        out = np.empty_like(x)
        out[0], out[-1] = d[0], d[-1]
        out[1:-1] = np.minimum(d[:-1], d[1:])
        return out
    dr = np.stack([gaps(g.r[e]) for e in range(p.n_elem)])[:, :, None, None]
    dth = gaps(g.theta)[None, None, :, None]
    dph = 2.0 * np.pi / p.n_phi
    h = np.minimum(np.minimum(np.broadcast_to(dr, g.shape), g.R * dth), g.R * np.sin(g.T) * dph)
    return p.cfl * h.min() / lam.max()


# ---------------------------------------------------------------------- diagnostics
def quadrature_weights(g: Grid):
    """w_r J_e (Clenshaw-Curtis per element) x w_theta x 2 pi / N_phi, with w_theta the
    Fejer weights / t_scale (Chebyshev theta) or the Fejer weights in x = -cos(theta)
    divided by sin(theta) (Fourier theta; exact for sqrt(gamma)-weighted integrands)."""
    wr = sp.clenshaw_curtis_weights(g.p.n_r)[None, :] / g.r_scale[:, None]
    if g.fourier_theta:
        wt = sp.fourier_theta_weights(g.p.n_theta)
    else:
        wt = sp.fejer_weights(g.p.n_theta) / g.t_scale
    wp = 2.0 * np.pi / g.p.n_phi
    return wr[:, :, None, None] * wt[None, None, :, None] * wp


def diagnostics(U, g: Grid, p: Params):
    """[rest mass, entropy, max |d_i B~^i|, c2p failures, max |H|, quadrature RMS of H] with
    H the Hamiltonian constraint.
    Entropy follows the paper's discrete functional E = sum rho s sqrt(gamma) dV with
    s = ln(p / rho^Gamma)/(Gamma-1) and dV the quadrature weight (reading: the paper's
    "cell volume" on spectral nodes).  The paper prints no values; mass and entropy are
    pinned by closed-form integrals on flat space."""
    w = quadrature_weights(g)
    prim = primitives(U, p)
    f = unpack_bssn(U)
    _, sqg = metric_from_bssn(f)
    mass = np.sum(w * U[I_D])
    s = np.log(prim["p"] / prim["rho"] ** p.gamma_eos) / (p.gamma_eos - 1.0)
    ent = np.sum(w * prim["rho"] * s * sqg)
    divB = g.d_r(U[I_B]) + g.d_t(U[I_B + 1], THETA_PAR[I_B + 1]) + g.d_p(U[I_B + 2])
    H = hamiltonian_constraint(U, g, p, prim)
    return np.array([mass, ent, np.max(np.abs(divB)), float(np.sum(~prim["ok"])),
                     np.max(np.abs(H)), weighted_rms(H, w)])


def weighted_rms(f, w):
    """Quadrature root mean square sqrt(sum w f^2 / sum w) over every node; w may be
    broadcast over phi (quadrature_weights), so its sum is taken at f's full shape."""
    wf = np.broadcast_to(w, f.shape)
    return np.sqrt(np.sum(wf * f * f) / np.sum(wf))


def hamiltonian_constraint(U, g: Grid, p: Params, prim=None):
    """Hamiltonian constraint at every node (the right-hand side's derivatives: radial first
    derivatives interface-averaged, second derivatives as the compositions of the RHS),
    with the Eulerian energy density of the matter."""
    prim = prim if prim is not None else primitives(U, p)
    f = unpack_bssn(U)
    gam, _ = metric_from_bssn(f)
    T = va.stress_energy(prim["rho"], prim["v"], prim["eps"], prim["B"], f["alpha"], f["beta"],
                         gam, p.gamma_eos)
    rho_adm = va.matter_3p1(T, f["alpha"], f["beta"], gam)[0]
    d1, d2 = _derivs(g, U)
    return bs.hamiltonian(f, _d1_fields(d1), _d2_fields(d2), rho_adm)


# ----------------------------------------------------------------- initial data
def initial_state(g: Grid, p: Params, prim, bssn=None):
    """Canonical state from Kerr-Schild BSSN data (or the given BSSN data, e.g. the XCTS
    slice) and primitive profiles.

    prim: dict with rho, p, vr, vth, vph, A_phi on the node grid.  The densitized
    field is B~^r = d_theta A_phi, B~^theta = -d_r A_phi, B~^phi = 0 (so that
    d_i B~^i = 0 for the tensor-product operators), B^i = B~^i / sqrt(gamma)."""
    ksd = bssn if bssn is not None else ks.bssn_data(p.M, p.a, g.R, g.T)
    U = np.zeros((NV + (1 if p.glm else 0),) + g.shape)
    for n, (i, j) in enumerate(SYM):
        U[I_GT + n] = ksd["gt"][..., i, j]
        U[I_AT + n] = ksd["At"][..., i, j]
    U[I_PHI] = ksd["phi"]
    U[I_K] = ksd["K"]
    for i in range(3):
        U[I_GAM + i] = ksd["Gt"][..., i]
        U[I_BETA + i] = ksd["beta"][..., i]
    U[I_ALPHA] = ksd["alpha"]
    f = unpack_bssn(U)
    gam, sqg = metric_from_bssn(f)
    A = prim["A_phi"]
    # A_phi is a covariant phi component: parity +1 under the theta extension
    Bt = np.stack([g.d_t(A, 1.0), -g.d_r(A), np.zeros_like(A)], axis=-1)
    B_u = Bt / sqg[..., None]
    v_u = np.stack([prim["vr"], prim["vth"], prim["vph"]], axis=-1)
    eps = prim["p"] / ((p.gamma_eos - 1.0) * prim["rho"])
    D, S_d, tau, _ = va.prim_to_cons(prim["rho"], v_u, eps, B_u, f["alpha"], f["beta"], gam,
                                     p.gamma_eos)
    U[I_D] = sqg * D
    for i in range(3):
        U[I_S + i] = sqg * S_d[..., i]
        U[I_B + i] = Bt[..., i]
    U[I_TAU] = sqg * tau
    return U


def workload_state(cfg, **kw):
    """Grid, params and initial state for a workload configuration (oracle side)."""
    from workloads import primitive_profiles
    p = Params.from_config(cfg, **kw)
    g = Grid(p)
    prim = primitive_profiles(cfg, g.R, g.T, g.P)
    return g, p, initial_state(g, p, prim)
