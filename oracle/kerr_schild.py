"""Kerr-Schild geometry in spherical coordinates (t, r, theta, phi).
Test infrastructure only.

Authority: the explicit line element of the paper (section "The Kerr-Schild
Metric and 3+1 Decomposition", "Metric"), with Sigma = r^2 + a^2 cos^2 theta.
The printed null vector l_mu and eta = diag(-1,1,1,1) do not reproduce that line
element in spherical coordinates, so they are not used (reading of the paper).
Lapse, shift and 3-metric are extracted from g_{mu nu} by the generic 3+1 split;
derivatives in r and theta use the complex-step method (exact to rounding).
"""
from __future__ import annotations

import numpy as np

H_STEP = 1e-30


def det3(m):
    """Determinant of [..., 3, 3] by cofactor expansion along the first row."""
    return (m[..., 0, 0] * (m[..., 1, 1] * m[..., 2, 2] - m[..., 1, 2] * m[..., 2, 1])
            - m[..., 0, 1] * (m[..., 1, 0] * m[..., 2, 2] - m[..., 1, 2] * m[..., 2, 0])
            + m[..., 0, 2] * (m[..., 1, 0] * m[..., 2, 1] - m[..., 1, 1] * m[..., 2, 0]))


def inv3(m):
    """Inverse of [..., 3, 3] as adjugate / determinant."""
    c = np.empty_like(m)
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != j]
            s = [x for x in range(3) if x != i]
            minor = (m[..., r[0], s[0]] * m[..., r[1], s[1]]
                     - m[..., r[0], s[1]] * m[..., r[1], s[0]])
            c[..., i, j] = (-1) ** (i + j) * minor
    return c / det3(m)[..., None, None]


def metric4(M, a, r, th):
    """g_{mu nu} [..., 4, 4] read off the Kerr-Schild line element."""
    r = np.asarray(r)
    th = np.asarray(th)
    sig = r * r + a * a * np.cos(th) ** 2
    s2 = np.sin(th) ** 2
    twoH = 2.0 * M * r / sig
    g = np.zeros(np.broadcast(r, th).shape + (4, 4), dtype=np.result_type(r, th, np.float64))
    g[..., 0, 0] = -(1.0 - twoH)
    g[..., 0, 1] = g[..., 1, 0] = twoH                    # (4Mr/Sigma) dt dr
    g[..., 0, 3] = g[..., 3, 0] = -a * twoH * s2          # -(4 a M r sin^2/Sigma) dt dphi
    g[..., 1, 1] = 1.0 + twoH
    g[..., 1, 3] = g[..., 3, 1] = -a * s2 * (1.0 + twoH)  # -2 a sin^2 (1+2H) dr dphi
    g[..., 2, 2] = sig
    g[..., 3, 3] = s2 * (sig + a * a * s2 * (1.0 + twoH))
    return g


def adm_from_metric4(g):
    """Generic 3+1 split: gamma_ij = g_ij, beta_i = g_0i, beta^i = gamma^ij beta_j,
    alpha^2 = beta_i beta^i - g_00."""
    gam = g[..., 1:, 1:]
    beta_d = g[..., 0, 1:]
    ginv = inv3(gam)
    beta_u = np.einsum("...ij,...j->...i", ginv, beta_d)
    alpha = np.sqrt(np.einsum("...i,...i->...", beta_d, beta_u) - g[..., 0, 0])
    return alpha, beta_u, beta_d, gam


def _cstep(f, M, a, r, th, wrt):
    """Complex-step derivative of f(M, a, r, th) with respect to r (wrt=0) or theta."""
    h = H_STEP
    if wrt == 0:
        return np.imag(f(M, a, r + 1j * h, th + 0j)) / h
    return np.imag(f(M, a, r + 0j, th + 1j * h)) / h


def adm(M, a, r, th):
    """alpha, beta^i, gamma_ij of Kerr-Schild at (r, theta)."""
    alpha, beta_u, _, gam = adm_from_metric4(metric4(M, a, r, th))
    return alpha, beta_u, gam


def _gamma_dd(M, a, r, th):
    return metric4(M, a, r, th)[..., 1:, 1:]


def _beta_d(M, a, r, th):
    return metric4(M, a, r, th)[..., 0, 1:]


def _beta_u(M, a, r, th):
    return adm_from_metric4(metric4(M, a, r, th))[1]


def _alpha(M, a, r, th):
    return adm_from_metric4(metric4(M, a, r, th))[0]


def _spatial_grad(f, M, a, r, th):
    """[..., 3(d), ...] derivative d_d f with d_phi f = 0 (axisymmetry)."""
    dr = _cstep(f, M, a, r, th, 0)
    dth = _cstep(f, M, a, r, th, 1)
    return np.stack([dr, dth, np.zeros_like(dr)], axis=-1 if np.ndim(dr) == np.ndim(r) else 0)


def christoffel3(gam, dgam):
    """Gamma^k_ij = 1/2 gamma^kl (d_i gamma_lj + d_j gamma_li - d_l gamma_ij).

    dgam[..., d, i, j] = d_d gamma_ij."""
    ginv = inv3(gam)
    low = 0.5 * (np.einsum("...ilj->...lij", dgam) + np.einsum("...jli->...lij", dgam)
                 - dgam)  # low[..., l, i, j] = Gamma_{l ij}
    return np.einsum("...kl,...lij->...kij", ginv, low)


def extrinsic_curvature(M, a, r, th):
    """K_ij of the stationary slice: K_ij = (D_i beta_j + D_j beta_i) / (2 alpha),
    D_i beta_j = d_i beta_j - Gamma^k_ij beta_k (from d_t gamma_ij = 0 in the ADM
    evolution equation -2 alpha K_ij + D_i beta_j + D_j beta_i)."""
    alpha, beta_u, beta_d, gam = adm_from_metric4(metric4(M, a, r, th))
    dgam = np.stack([_cstep(_gamma_dd, M, a, r, th, 0), _cstep(_gamma_dd, M, a, r, th, 1),
                     np.zeros(gam.shape)], axis=-3)
    dbd = np.stack([_cstep(_beta_d, M, a, r, th, 0), _cstep(_beta_d, M, a, r, th, 1),
                    np.zeros(beta_d.shape)], axis=-2)  # [..., d, j]
    Gam = christoffel3(gam, dgam)
    Dbeta = dbd - np.einsum("...kij,...k->...ij", Gam, beta_d)
    return (Dbeta + np.swapaxes(Dbeta, -1, -2)) / (2.0 * alpha[..., None, None])


def _conformal_metric(M, a, r, th):
    gam = _gamma_dd(M, a, r, th)
    return gam * det3(gam)[..., None, None] ** (-1.0 / 3.0)


def bssn_data(M, a, r, th):
    """BSSN variables of the Kerr-Schild slice.

    phi = ln(det gamma)/12 (so that det gammatilde = 1; the paper's 1/4 is a
    misprint under gamma = e^{4 phi} gammatilde), gammatilde = e^{-4phi} gamma,
    K = gamma^ij K_ij, Atilde_ij = e^{-4 phi}(K_ij - gamma_ij K/3),
    Gammatilde^i = gammatilde^jk Gammatilde^i_jk, gauge B^i = 0.
    Returns dict of arrays (tensors as [..., 3] / [..., 3, 3])."""
    alpha, beta_u, beta_d, gam = adm_from_metric4(metric4(M, a, r, th))
    detg = det3(gam)
    phi = np.log(detg) / 12.0
    e4 = np.exp(-4.0 * phi)
    gt = gam * e4[..., None, None]
    Kij = extrinsic_curvature(M, a, r, th)
    ginv = inv3(gam)
    K = np.einsum("...ij,...ij->...", ginv, Kij)
    At = (Kij - gam * K[..., None, None] / 3.0) * e4[..., None, None]
    dgt = np.stack([_cstep(_conformal_metric, M, a, r, th, 0),
                    _cstep(_conformal_metric, M, a, r, th, 1), np.zeros(gt.shape)], axis=-3)
    Gt_ijk = christoffel3(gt, dgt)
    gtinv = inv3(gt)
    Gt = np.einsum("...jk,...ijk->...i", gtinv, Gt_ijk)
    return {"gt": gt, "phi": phi, "At": At, "K": K, "Gt": Gt, "alpha": alpha,
            "beta": beta_u, "B": np.zeros_like(beta_u), "gamma": gam, "Kij": Kij}


def horizon_radius(M, a):
    """r_h = M + sqrt(M^2 - a^2) (Results, equatorial embedding section)."""
    return M + np.sqrt(M * M - a * a)
