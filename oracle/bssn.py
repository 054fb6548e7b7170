"""BSSN + gauge right-hand side at points.  Test infrastructure only.

Paper: Methods, "BSSN Evolution Equations", "Gauge Conditions" (1+log slicing,
Gamma-driver shift) and "Stress-Energy Tensor" (matter coupling).

Readings where the printed system is incomplete or misprinted (standard BSSN of
Baumgarte & Shapiro 1998, the paper's cited textbook form):
* phi = ln(det gamma)/12 with gamma_ij = e^{4 phi} gammatilde_ij;
* the Gammatilde equation carries + 12 alpha Atilde^ij d_j phi and the matter term
  -16 pi alpha gammatilde^ij S_j (the printed "8 pi j^i" inside 2 alpha(...));
* Ricci: R_ij = Rtilde_ij + R^phi_ij; Rtilde_ij uses the evolved Gammatilde^k in
  gammatilde_k(i d_j) Gammatilde^k and the computed gammatilde^lm Gammatilde^k_lm
  in Gammatilde^k Gammatilde_(ij)k;
* D_i D_j alpha uses the physical Christoffel symbols;
* Lie derivatives of the weight -2/3 densities as printed (advection + the
  -2/3 divergence terms), plus - Gammatilde^j d_j beta^i + 2/3 Gammatilde^i d_j beta^j
  for Gammatilde^i (evolved Gammatilde in both);
* matter: rho_ADM, S_i, S_ij, S from T^{mu nu} (see valencia.matter_3p1);
* gauge: d_t alpha = -2 alpha K + beta^i d_i alpha, d_t beta^i = 3/4 B^i,
  d_t B^i = d_t Gammatilde^i - eta B^i exactly as printed (no advection);
  gauge=1 freezes alpha, beta, B (stationary gauge).
"""
from __future__ import annotations

import numpy as np

from .kerr_schild import inv3, christoffel3

EIGHT_PI = 8.0 * np.pi


def bssn_rhs(f, d1, d2, matter, gauge=0, eta=2.0):
    """Right-hand side of the 24 BSSN + gauge variables at every point.

    f: dict with gt[...,3,3], phi, At[...,3,3], K, Gt[...,3], alpha, beta[...,3], B[...,3]
    d1: first derivatives, leading derivative index after the point axes:
        gt[...,d,i,j], phi[...,d], At[...,d,i,j], K[...,d], Gt[...,d,i], alpha[...,d],
        beta[...,d,i]
    d2: second derivatives gt[...,d,e,i,j], phi[...,d,e], alpha[...,d,e], beta[...,d,e,i]
    matter: rho, S_d[...,3], S_dd[...,3,3], S
    Returns dict of the same keys as f holding d_t of each variable.
    """
    gt, phi, At, K, Gt = f["gt"], f["phi"], f["At"], f["K"], f["Gt"]
    alpha, beta, B = f["alpha"], f["beta"], f["B"]
    dgt, dphi, dAt, dK, dGt = d1["gt"], d1["phi"], d1["At"], d1["K"], d1["Gt"]
    dalpha, dbeta = d1["alpha"], d1["beta"]
    ddgt, ddphi, ddalpha, ddbeta = d2["gt"], d2["phi"], d2["alpha"], d2["beta"]

    gtinv = inv3(gt)
    e4m = np.exp(-4.0 * phi)
    Chr = christoffel3(gt, dgt)                               # Gammatilde^k_ij [k,i,j]
    divb = np.einsum("...kk->...", dbeta)
    Ric = ricci_bssn(f, d1, d2)

    # physical second covariant derivative of the lapse
    eye = np.eye(3)
    Chr_phys = (Chr + 2.0 * (np.einsum("ki,...j->...kij", eye, dphi)
                             + np.einsum("kj,...i->...kij", eye, dphi)
                             - np.einsum("...ij,...kl,...l->...kij", gt, gtinv, dphi)))
    DDalpha = ddalpha - np.einsum("...kij,...k->...ij", Chr_phys, dalpha)
    trDDalpha = e4m * np.einsum("...ij,...ij->...", gtinv, DDalpha)

    At_uu = np.einsum("...ik,...jl,...kl->...ij", gtinv, gtinv, At)
    At_ud = np.einsum("...kl,...lj->...kj", gtinv, At)         # Atilde^k_j
    AA = np.einsum("...ij,...ij->...", At, At_uu)

    out = {}
    out["gt"] = (-2.0 * alpha[..., None, None] * At
                 + np.einsum("...k,...kij->...ij", beta, dgt)
                 + np.einsum("...ik,...jk->...ij", gt, dbeta)
                 + np.einsum("...jk,...ik->...ij", gt, dbeta)
                 - 2.0 / 3.0 * gt * divb[..., None, None])
    out["phi"] = -alpha * K / 6.0 + np.einsum("...k,...k->...", beta, dphi) + divb / 6.0

    X = -DDalpha + alpha[..., None, None] * (Ric - EIGHT_PI * matter["S_dd"])
    trX = np.einsum("...kl,...kl->...", gtinv, X)
    XTF = X - gt * trX[..., None, None] / 3.0
    out["At"] = (e4m[..., None, None] * XTF
                 + alpha[..., None, None] * (K[..., None, None] * At
                                             - 2.0 * np.einsum("...ik,...kj->...ij", At, At_ud))
                 + np.einsum("...k,...kij->...ij", beta, dAt)
                 + np.einsum("...ik,...jk->...ij", At, dbeta)
                 + np.einsum("...jk,...ik->...ij", At, dbeta)
                 - 2.0 / 3.0 * At * divb[..., None, None])
    out["K"] = (-trDDalpha + alpha * (AA + K * K / 3.0)
                + 4.0 * np.pi * alpha * (matter["rho"] + matter["S"])
                + np.einsum("...k,...k->...", beta, dK))
    out["Gt"] = (np.einsum("...jk,...jki->...i", gtinv, ddbeta)
                 + np.einsum("...ij,...jkk->...i", gtinv, ddbeta) / 3.0
                 + np.einsum("...j,...ji->...i", beta, dGt)
                 - np.einsum("...j,...ji->...i", Gt, dbeta)
                 + 2.0 / 3.0 * Gt * divb[..., None]
                 - 2.0 * np.einsum("...ij,...j->...i", At_uu, dalpha)
                 + 2.0 * alpha[..., None] * (np.einsum("...ijk,...jk->...i", Chr, At_uu)
                                             + 6.0 * np.einsum("...ij,...j->...i", At_uu, dphi)
                                             - 2.0 / 3.0 * np.einsum("...ij,...j->...i",
                                                                     gtinv, dK))
                 - 2.0 * EIGHT_PI * alpha[..., None]
                 * np.einsum("...ij,...j->...i", gtinv, matter["S_d"]))
    if gauge == 0:
        out["alpha"] = -2.0 * alpha * K + np.einsum("...i,...i->...", beta, dalpha)
        out["beta"] = 0.75 * B
        out["B"] = out["Gt"] - eta * B
    else:
        out["alpha"] = np.zeros_like(alpha)
        out["beta"] = np.zeros_like(beta)
        out["B"] = np.zeros_like(B)
    return out


def ricci_bssn(f, d1, d2):
    """Physical Ricci tensor R_ij = Rtilde_ij + R^phi_ij in BSSN variables (evolved
    Gammatilde^k in the derivative term, computed Gammatilde^k in the Gammatilde^k
    Gammatilde_(ij)k term)."""
    gt, Gt = f["gt"], f["Gt"]
    dgt, dphi, dGt = d1["gt"], d1["phi"], d1["Gt"]
    ddgt, ddphi = d2["gt"], d2["phi"]
    gtinv = inv3(gt)
    Chr = christoffel3(gt, dgt)                               # Gammatilde^k_ij [k,i,j]
    Chr_low = np.einsum("...il,...ljk->...ijk", gt, Chr)      # Gammatilde_ijk
    Gt_d = np.einsum("...jk,...ijk->...i", gtinv, Chr)        # computed Gammatilde^i
    # conformal Ricci tensor
    Rt = (-0.5 * np.einsum("...lm,...lmij->...ij", gtinv, ddgt)
          + 0.5 * (np.einsum("...ki,...jk->...ij", gt, dGt)
                   + np.einsum("...kj,...ik->...ij", gt, dGt))
          + 0.5 * (np.einsum("...k,...ijk->...ij", Gt_d, Chr_low)
                   + np.einsum("...k,...jik->...ij", Gt_d, Chr_low))
          + np.einsum("...lm,...kli,...jkm->...ij", gtinv, Chr, Chr_low)
          + np.einsum("...lm,...klj,...ikm->...ij", gtinv, Chr, Chr_low)
          + np.einsum("...lm,...kim,...klj->...ij", gtinv, Chr, Chr_low))
    # conformal-factor part
    DDphi = ddphi - np.einsum("...kij,...k->...ij", Chr, dphi)
    lap_phi = np.einsum("...lm,...lm->...", gtinv, DDphi)
    dphi2 = np.einsum("...lm,...l,...m->...", gtinv, dphi, dphi)
    Rphi = (-2.0 * DDphi - 2.0 * gt * lap_phi[..., None, None]
            + 4.0 * np.einsum("...i,...j->...ij", dphi, dphi)
            - 4.0 * gt * dphi2[..., None, None])
    return Rt + Rphi


def hamiltonian(f, d1, d2, rho):
    """Hamiltonian constraint H = R + K^2 - K_ij K^ij - 16 pi rho in BSSN variables:
    R = e^{-4 phi} gammatilde^ij R_ij, K_ij K^ij = Atilde_ij Atilde^ij + K^2 / 3, so
    H = R + (2/3) K^2 - Atilde_ij Atilde^ij - 16 pi rho (rho the Eulerian energy density)."""
    gtinv = inv3(f["gt"])
    R = np.exp(-4.0 * f["phi"]) * np.einsum("...ij,...ij->...", gtinv, ricci_bssn(f, d1, d2))
    At_uu = np.einsum("...ik,...jl,...kl->...ij", gtinv, gtinv, f["At"])
    AA = np.einsum("...ij,...ij->...", f["At"], At_uu)
    return R + 2.0 / 3.0 * f["K"] ** 2 - AA - 2.0 * EIGHT_PI * rho


def ricci_physical(gam, dgam, ddgam):
    """Physical Ricci tensor from the 3-metric by the textbook formula
    R_ij = d_k Gamma^k_ij - d_j Gamma^k_ik + Gamma^k_kl Gamma^l_ij - Gamma^k_jl Gamma^l_ik.
    Used only by the pins (ADM route)."""
    ginv = inv3(gam)
    Chr = christoffel3(gam, dgam)
    # d_m Gamma^k_ij = d_m(g^kl) Gamma_lij + g^kl d_m Gamma_lij
    dginv = -np.einsum("...ka,...mab,...bl->...mkl", ginv, dgam, ginv)
    low = 0.5 * (np.einsum("...ilj->...lij", dgam) + np.einsum("...jli->...lij", dgam) - dgam)
    dlow = 0.5 * (np.einsum("...milj->...mlij", ddgam) + np.einsum("...mjli->...mlij", ddgam)
                  - ddgam)
    dChr = (np.einsum("...mkl,...lij->...mkij", dginv, low)
            + np.einsum("...kl,...mlij->...mkij", ginv, dlow))
    return (np.einsum("...kkij->...ij", dChr) - np.einsum("...jkik->...ij", dChr)
            + np.einsum("...kkl,...lij->...ij", Chr, Chr)
            - np.einsum("...kjl,...lik->...ij", Chr, Chr))
