"""Valencia GRMHD pieces at points.  Test infrastructure only.

Paper sections: "GRMHD Conservative Form" (conserved variables, fluxes, Lorentz
factor, magnetic four-vector, source term), "The Energy of the Fluid and
Electromagnetic Stress" (T^{mu nu}), "The Primitive Variable Recovery",
"The Conserved Fluxes and Geometric Source Terms".

Readings of the paper (its printed formulas are written for alpha = 1, beta = 0
and are mutually inconsistent for tau):
* conserved variables with h* = 1 + eps + (p + b^2)/rho, p* = p + b^2/2:
  D = rho W, S_j = rho h* W^2 v_j - alpha b^0 b_j,
  tau = rho h* W^2 - p* - alpha^2 (b^0)^2 - D;
* fluxes carry the lapse and shift (script-F^i = alpha F^i with v^i -> v^i - beta^i/alpha),
  evolved form d_t(sqrt(gamma) U) + d_i(sqrt(gamma) script-F^i) = alpha sqrt(gamma) S;
* b^0 = W v_i B^i / alpha, b^i = (B^i + alpha b^0 u^i)/W (as printed).
Arrays: scalars [...], vectors [..., 3], tensors [..., 3, 3] / [..., 4, 4].
"""
from __future__ import annotations

import numpy as np

from .kerr_schild import inv3, det3


def lower(gam, v_u):
    return np.einsum("...ij,...j->...i", gam, v_u)


def metric4_from_adm(alpha, beta_u, gam):
    """g_{mu nu} from the 3+1 split: g_00 = -alpha^2 + beta_k beta^k, g_0i = beta_i, g_ij."""
    beta_d = lower(gam, beta_u)
    g = np.zeros(alpha.shape + (4, 4))
    g[..., 0, 0] = -alpha ** 2 + np.einsum("...i,...i->...", beta_d, beta_u)
    g[..., 0, 1:] = beta_d
    g[..., 1:, 0] = beta_d
    g[..., 1:, 1:] = gam
    return g


def inverse_metric4_from_adm(alpha, beta_u, gam):
    """g^{mu nu}: g^00 = -1/alpha^2, g^0i = beta^i/alpha^2, g^ij = gamma^ij - beta^i beta^j/alpha^2."""
    ginv = inv3(gam)
    a2 = alpha ** 2
    g = np.zeros(alpha.shape + (4, 4))
    g[..., 0, 0] = -1.0 / a2
    g[..., 0, 1:] = beta_u / a2[..., None]
    g[..., 1:, 0] = beta_u / a2[..., None]
    g[..., 1:, 1:] = ginv - np.einsum("...i,...j->...ij", beta_u, beta_u) / a2[..., None, None]
    return g


def lorentz_factor(v_u, gam):
    """W = 1/sqrt(1 - gamma_ij v^i v^j)."""
    return 1.0 / np.sqrt(1.0 - np.einsum("...i,...i->...", lower(gam, v_u), v_u))


def four_vectors(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos):
    """u^mu, b^mu, b_mu, b^2, W, p for the Eulerian velocity v^i and Eulerian field B^i."""
    W = lorentz_factor(v_u, gam)
    p = (gamma_eos - 1.0) * rho * eps
    u = np.zeros(alpha.shape + (4,))
    u[..., 0] = W / alpha
    u[..., 1:] = W[..., None] * (v_u - beta_u / alpha[..., None])
    v_d = lower(gam, v_u)
    b = np.zeros(alpha.shape + (4,))
    b[..., 0] = W * np.einsum("...i,...i->...", v_d, B_u) / alpha
    b[..., 1:] = (B_u + alpha[..., None] * b[..., 0:1] * u[..., 1:]) / W[..., None]
    g4 = metric4_from_adm(alpha, beta_u, gam)
    b_d = np.einsum("...mn,...n->...m", g4, b)
    b2 = np.einsum("...m,...m->...", b, b_d)
    return u, b, b_d, b2, W, p


def prim_to_cons(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos):
    """Undensitized (D, S_j, tau, B^k) from primitives via the four-vector form."""
    u, b, b_d, b2, W, p = four_vectors(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos)
    h_star = 1.0 + eps + (p + b2) / rho
    p_star = p + 0.5 * b2
    v_d = lower(gam, v_u)
    D = rho * W
    S_d = (rho * h_star * W ** 2)[..., None] * v_d - (alpha * b[..., 0])[..., None] * b_d[..., 1:]
    tau = rho * h_star * W ** 2 - p_star - alpha ** 2 * b[..., 0] ** 2 - D
    return D, S_d, tau, B_u.copy()


def prim_to_cons_eulerian(rho, v_u, eps, B_u, gam, gamma_eos):
    """Same map written with Eulerian quantities only (no four-vectors):
    Z = rho h W^2, S_j = (Z + B^2) v_j - (v.B) B_j,
    tau = Z + B^2 - p - (B^2/W^2 + (v.B)^2)/2 - D.  Used to pin prim_to_cons."""
    W = lorentz_factor(v_u, gam)
    p = (gamma_eos - 1.0) * rho * eps
    h = 1.0 + eps + p / rho
    Z = rho * h * W ** 2
    v_d = lower(gam, v_u)
    B_d = lower(gam, B_u)
    B2 = np.einsum("...i,...i->...", B_d, B_u)
    vB = np.einsum("...i,...i->...", v_d, B_u)
    S_d = (Z + B2)[..., None] * v_d - vB[..., None] * B_d
    tau = Z + B2 - p - 0.5 * (B2 / W ** 2 + vB ** 2) - rho * W
    return rho * W, S_d, tau


# ----------------------------------------------------------------- primitive recovery
def _master(mu, D, q, r2, bb, rb2, gamma_eos, eps_min=0.0):
    """One-variable master function in mu = 1/(h W) of Kastaun, Kalinani & Ciolfi
    (PRD 103, 023018, 2021), restated from its definitions; its unique root gives
    the primitives.  Returns f(mu) and the quantities needed afterwards."""
    x = 1.0 / (1.0 + mu * bb)
    rbar2 = r2 * x * x + mu * x * (1.0 + x) * rb2
    qbar = q - 0.5 * bb - 0.5 * mu * mu * x * x * (bb * r2 - rb2)
    v0sq = r2 / (1.0 + r2)
    v2 = np.minimum(mu * mu * rbar2, v0sq)
    W = 1.0 / np.sqrt(1.0 - v2)
    rho = D / W
    eps = W * (qbar - mu * rbar2) + v2 * W * W / (1.0 + W)
    eps_c = np.maximum(eps, eps_min)
    p = (gamma_eos - 1.0) * rho * eps_c
    a_hat = p / (rho * (1.0 + eps_c))
    h = (1.0 + eps_c) * (1.0 + a_hat)
    nu_a = h / W
    nu_b = (1.0 + a_hat) * (1.0 + qbar - mu * rbar2)
    nu = np.maximum(nu_a, nu_b)
    f = mu - 1.0 / (nu + mu * rbar2)
    return f, x, W, rho, eps


def con2prim(D, S_d, tau, B_u, gam, gamma_eos, eps_min=0.0, n_scan=256, n_bisect=200):
    """Exact primitive recovery for the Gamma-law gas: bracket the unique root of the
    master function on mu in (0, 1] (h >= 1) and bisect to rounding.

    The specific internal energy inside the master function is clamped to
    eps >= eps_min (the valid range of the equation of state), so a state whose
    exact inversion would have eps < eps_min still has a unique root; there the
    returned eps is eps_min and ok is False (counted as a floor correction).

    Inputs undensitized.  Returns rho, v^i, eps, p, W, ok (bool array).
    The paper's damped Newton iteration converges to the same root; this routine
    does not use it (a different algorithm for the same unique result)."""
    D = np.asarray(D, dtype=np.float64)
    ginv = inv3(gam)
    S_u = np.einsum("...ij,...j->...i", ginv, S_d)
    q = tau / D
    r2 = np.einsum("...i,...i->...", S_d, S_u) / D ** 2
    B2 = np.einsum("...i,...i->...", lower(gam, B_u), B_u)
    bb = B2 / D
    SB = np.einsum("...i,...i->...", S_d, B_u)
    rb2 = SB ** 2 / D ** 3
    args = (D, q, r2, bb, rb2, gamma_eos, eps_min)
    # scan for the first sign change from negative to non-negative
    mus = np.concatenate([[0.0], np.geomspace(1e-12, 1.0, n_scan)])
    lo = np.zeros(D.shape)
    hi = np.full(D.shape, np.nan)
    prev = mus[0] * np.ones(D.shape)
    found = np.zeros(D.shape, dtype=bool)
    for m in mus[1:]:
        fm = _master(np.full(D.shape, m), *args)[0]
        new = (~found) & (fm >= 0.0)
        lo = np.where(new, prev, lo)
        hi = np.where(new, m, hi)
        found |= new
        prev = np.where(found, prev, m)
    ok = found.copy()
    hi = np.where(found, hi, 1.0)
    for _ in range(n_bisect):
        mid = 0.5 * (lo + hi)
        fm = _master(mid, *args)[0]
        neg = fm < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    mu = 0.5 * (lo + hi)
    f, x, W, rho, eps = _master(mu, *args)
    v_d = (mu * x)[..., None] * (S_d / D[..., None]
                                 + (mu * SB / D ** 2)[..., None] * lower(gam, B_u))
    v_u = np.einsum("...ij,...j->...i", ginv, v_d)
    ok &= eps >= eps_min
    eps = np.maximum(eps, eps_min)
    p = (gamma_eos - 1.0) * rho * eps
    return rho, v_u, eps, p, W, ok


def con2prim_damped_guess(D, S_d, tau, gam, w_max=10.0, eps_min=0.0):
    """Cold start of the damped iteration when no previous primitives exist: the dust
    estimates v^i = gamma^ij S_j / (tau + D) (momentum over energy density, |v| capped at
    the W <= w_max limit), W from v, eps = (tau + D)/(D W) - 1 (floored), rho = D / W.
    (A reading: the paper starts the iteration from given primitives.)"""
    ginv = inv3(gam)
    v_u = np.einsum("...ij,...j->...i", ginv, S_d) / (tau + D)[..., None]
    v2max = 1.0 - 1.0 / w_max ** 2
    v2 = np.einsum("...i,...i->...", lower(gam, v_u), v_u)
    v_u = v_u * np.sqrt(np.minimum(1.0, v2max / np.maximum(v2, 1e-300)))[..., None]
    W = lorentz_factor(v_u, gam)
    eps = np.maximum((tau + D) / (D * W) - 1.0, eps_min)
    return D / W, v_u, eps


def con2prim_damped(D, S_d, tau, B_u, gam, gamma_eos, rho, v_u, eps, lam0=0.5, maxit=40,
                    tol=1e-13, eps_min=0.0, w_max=10.0, max_halvings=30):
    """The paper's primitive recovery ("The Primitive Variable Recovery"), step by step,
    from the primitives (rho, v^i, eps) given as the starting point:

      1. W = (1 - v^2)^(-1/2), p = (Gamma - 1) rho eps, h = 1 + eps + p / rho, and the
         conserved variables these primitives predict (S_i, tau; the map of
         prim_to_cons_eulerian, which carries the metric and the field);
      2. residuals dS_i = S_i - S_i^pred, dtau = tau - tau^pred;
      3. damped update v^i += lam gamma^ij dS_j / (rho h W^2), eps += lam dtau / (rho W^2),
         with lam = 0.5 at first; when the residual of the updated primitives exceeds
         the current one, lam is halved and the update retried (lam stays halved);
      4. rho = D / W of the updated velocity;
      5. stop when ||dS|| + |dtau| < tol D (||dS||^2 = gamma^ij dS_i dS_j);
    at most maxit iterations; a point still above tol then takes one Newton-Raphson update
    of eps on the tau residual at fixed v and rho (d tau^pred / d eps = rho (Gamma W^2 -
    Gamma + 1)).  Readings: the residual is measured relative to D (the paper's tol is
    absolute, for states of density ~1); the indices are raised with the spatial metric
    (the printed update is flat-space); v^2 is capped at W <= w_max and eps floored at
    eps_min after every update.  Inputs undensitized; returns rho, v^i, eps, p, W, ok
    (converged without the final Newton update and without a floor) and the iterations
    taken."""
    ginv = inv3(gam)
    v2max = 1.0 - 1.0 / w_max ** 2

    def clamp(v_u, eps):
        v2 = np.einsum("...i,...i->...", lower(gam, v_u), v_u)
        v_u = v_u * np.sqrt(np.minimum(1.0, v2max / np.maximum(v2, 1e-300)))[..., None]
        return v_u, np.maximum(eps, eps_min)

    def residual(rho, v_u, eps):
        _, Sp, tp = prim_to_cons_eulerian(rho, v_u, eps, B_u, gam, gamma_eos)
        dS = S_d - Sp
        dt = tau - tp
        nrm = np.sqrt(np.maximum(np.einsum("...i,...ij,...j->...", dS, ginv, dS), 0.0)) + np.abs(dt)
        return dS, dt, nrm

    rho = np.array(rho, dtype=np.float64)
    v_u = np.array(v_u, dtype=np.float64)
    eps = np.array(eps, dtype=np.float64)
    v_u, eps = clamp(v_u, eps)
    rho = D / lorentz_factor(v_u, gam)
    lam = np.full(D.shape, float(lam0))
    done = np.zeros(D.shape, dtype=bool)
    iters = np.zeros(D.shape, dtype=np.int64)
    for _ in range(maxit):
        dS, dt, r0 = residual(rho, v_u, eps)
        done |= r0 < tol * D
        if done.all():
            break
        W = lorentz_factor(v_u, gam)
        p = (gamma_eos - 1.0) * rho * eps
        h = 1.0 + eps + p / rho
        dv = np.einsum("...ij,...j->...i", ginv, dS) / (rho * h * W * W)[..., None]
        de = dt / (rho * W * W)
        trial_lam = lam.copy()
        new_v, new_e, new_r = v_u.copy(), eps.copy(), rho.copy()
        pending = ~done
        for _h in range(max_halvings + 1):
            tv, te = clamp(v_u + trial_lam[..., None] * dv, eps + trial_lam * de)
            tr = D / lorentz_factor(tv, gam)
            _, _, r1 = residual(tr, tv, te)
            accept = pending & ((r1 <= r0) | (_h == max_halvings))
            new_v = np.where(accept[..., None], tv, new_v)
            new_e = np.where(accept, te, new_e)
            new_r = np.where(accept, tr, new_r)
            lam = np.where(accept, trial_lam, lam)
            pending &= ~accept
            if not pending.any():
                break
            trial_lam = np.where(pending, 0.5 * trial_lam, trial_lam)
        v_u, eps, rho = new_v, new_e, new_r
        iters += ~done
    dS, dt, r0 = residual(rho, v_u, eps)
    done |= r0 < tol * D
    # the final Newton-Raphson update of eps for the points still above tol
    W = lorentz_factor(v_u, gam)
    dtde = rho * (gamma_eos * W * W - gamma_eos + 1.0)
    eps = np.where(done, eps, eps + dt / dtde)
    ok = done & (eps >= eps_min)
    eps = np.maximum(eps, eps_min)
    p = (gamma_eos - 1.0) * rho * eps
    return rho, v_u, eps, p, W, ok, iters


# ------------------------------------------------------------------ fluxes and T^{mu nu}
def fluxes(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos):
    """script-F^i for the 8 undensitized conserved variables, shape [..., 3(i), 8].

    Order of variables: D, S_r, S_theta, S_phi, tau, B^r, B^theta, B^phi.
    script-F^i_D = D vt^i, script-F^i_{S_j} = S_j vt^i + alpha p* delta^i_j - alpha b_j B^i/W,
    script-F^i_tau = tau vt^i + alpha p* v^i - alpha^2 b^0 B^i/W,
    script-F^i_{B^k} = vt^i B^k - vt^k B^i, with vt^i = alpha v^i - beta^i."""
    u, b, b_d, b2, W, p = four_vectors(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos)
    D, S_d, tau, _ = prim_to_cons(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos)
    p_star = p + 0.5 * b2
    vt = alpha[..., None] * v_u - beta_u
    F = np.zeros(alpha.shape + (3, 8))
    for i in range(3):
        F[..., i, 0] = D * vt[..., i]
        for j in range(3):
            F[..., i, 1 + j] = (S_d[..., j] * vt[..., i] + alpha * p_star * (i == j)
                                - alpha * b_d[..., 1 + j] * B_u[..., i] / W)
        F[..., i, 4] = (tau * vt[..., i] + alpha * p_star * v_u[..., i]
                        - alpha ** 2 * b[..., 0] * B_u[..., i] / W)
        for k in range(3):
            F[..., i, 5 + k] = vt[..., i] * B_u[..., k] - vt[..., k] * B_u[..., i]
    return F


def stress_energy(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos):
    """T^{mu nu} = rho h* u^mu u^nu + p* g^{mu nu} - b^mu b^nu (Methods, stress-energy tensor)."""
    u, b, b_d, b2, W, p = four_vectors(rho, v_u, eps, B_u, alpha, beta_u, gam, gamma_eos)
    rho_h_star = rho * (1.0 + eps) + p + b2
    p_star = p + 0.5 * b2
    ginv4 = inverse_metric4_from_adm(alpha, beta_u, gam)
    return (rho_h_star[..., None, None] * np.einsum("...m,...n->...mn", u, u)
            + p_star[..., None, None] * ginv4 - np.einsum("...m,...n->...mn", b, b))


def matter_3p1(T, alpha, beta_u, gam):
    """rho_ADM = n_mu n_nu T^{mu nu}, S_i = -gamma_{i mu} n_nu T^{mu nu},
    S_ij = gamma_{i mu} gamma_{j nu} T^{mu nu}, S = gamma^ij S_ij, with
    n_mu = (-alpha, 0, 0, 0) and gamma_{i mu} = g_{i mu}."""
    g4 = metric4_from_adm(alpha, beta_u, gam)
    rho_adm = alpha ** 2 * T[..., 0, 0]
    gi = g4[..., 1:, :]  # gamma_{i mu}
    S_d = alpha[..., None] * np.einsum("...im,...m->...i", gi, T[..., :, 0])
    S_dd = np.einsum("...im,...jn,...mn->...ij", gi, gi, T)
    S = np.einsum("...ij,...ij->...", inv3(gam), S_dd)
    return rho_adm, S_d, S_dd, S


def sources_3p1(T, alpha, beta_u, gam, dalpha, dbeta, dgam, Kij):
    """Momentum and energy sources in 3+1 form (no time derivative of the metric):
    S_{S_j} = 1/2 T^{mu nu} d_j g_{mu nu} expanded:
      T^00 (1/2 beta^k beta^l d_j gamma_kl - alpha d_j alpha) + T^0i beta^k d_j gamma_ik
      + T^0_i d_j beta^i + 1/2 T^ik d_j gamma_ik,
    S_tau = T^00 (beta^i beta^j K_ij - beta^i d_i alpha) + T^0i (2 beta^j K_ij - d_i alpha)
      + T^ij K_ij.
    dalpha[..., j], dbeta[..., j, i] = d_j beta^i, dgam[..., j, i, k] = d_j gamma_ik.
    Returns S_S[..., 3], S_tau (the RHS of sqrt(gamma) U receives alpha sqrt(gamma) S)."""
    T00 = T[..., 0, 0]
    T0i = T[..., 0, 1:]
    Tij = T[..., 1:, 1:]
    g4 = metric4_from_adm(alpha, beta_u, gam)
    T0_low = np.einsum("...im,...m->...i", g4[..., 1:, :], T[..., 0, :])  # T^0_i
    S_S = (T00[..., None] * (0.5 * np.einsum("...k,...l,...jkl->...j", beta_u, beta_u, dgam)
                             - alpha[..., None] * dalpha)
           + np.einsum("...i,...k,...jik->...j", T0i, beta_u, dgam)
           + np.einsum("...i,...ji->...j", T0_low, dbeta)
           + 0.5 * np.einsum("...ik,...jik->...j", Tij, dgam))
    S_tau = (T00 * (np.einsum("...i,...j,...ij->...", beta_u, beta_u, Kij)
                    - np.einsum("...i,...i->...", beta_u, dalpha))
             + np.einsum("...i,...i->...", T0i,
                         2.0 * np.einsum("...j,...ij->...i", beta_u, Kij) - dalpha)
             + np.einsum("...ij,...ij->...", Tij, Kij))
    return S_S, S_tau


def sources_christoffel(T, g4, dg4):
    """Sources from the covariant form of the paper's "Source term" with d_t g = 0:
    S_j = T^{mu nu}(d_mu g_{nu j} - Gamma^lambda_{mu nu} g_{lambda j}) and
    S_tau = alpha (T^{mu 0} d_mu ln alpha - T^{mu nu} Gamma^0_{mu nu}).
    dg4[..., m, a, b] = d_m g_{ab} (m = 0 row is zero for a stationary metric).
    Used only to pin sources_3p1 on stationary data."""
    ginv4 = np.linalg.inv(g4)
    low = 0.5 * (np.einsum("...mla->...lma", dg4) + np.einsum("...alm->...lma", dg4)
                 - dg4)
    # low[..., l, m, a] = Gamma_{l m a} = 1/2 (d_m g_la + d_a g_lm - d_l g_ma)
    Gam = np.einsum("...kl,...lma->...kma", ginv4, low)
    S = (np.einsum("...mn,...mnj->...j", T, dg4[..., :, :, 1:])
         - np.einsum("...mn,...lmn,...lj->...j", T, Gam, g4[..., :, 1:]))
    alpha = 1.0 / np.sqrt(-ginv4[..., 0, 0])
    # d_mu ln alpha with alpha = (-g^00)^{-1/2}: d alpha = alpha^3 (d g^00)/2 with
    # d g^{00} = -g^{0a} g^{0b} d g_{ab}
    dg00 = -np.einsum("...a,...b,...mab->...m", ginv4[..., 0, :], ginv4[..., 0, :], dg4)
    dlna = 0.5 * alpha[..., None] ** 2 * dg00
    S_tau = alpha * (np.einsum("...m,...m->...", T[..., :, 0], dlna)
                     - np.einsum("...mn,...mn->...", T, Gam[..., 0, :, :]))
    return S, S_tau
