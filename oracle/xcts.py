"""Approximate XCTS initial data (paper: "Initial Data: Approximate XCTS Solution" and the
"Initial Data Solver XCTS Approximation" item of its version history).  Test
infrastructure only.

The paper solves the conformal Hamiltonian constraint  lap~ psi = -2 pi rho psi^5  by a
fixed-point relaxation on psi with A_ij = 0 (so the momentum constraint is left aside),
then sets gamma_ij = psi^4 gammatilde_ij and K = 0.

Readings (the paper states none of these):
* gammatilde_ij is the flat metric in spherical coordinates and lap~ its Laplacian,
  d_rr + (2/r) d_r + (d_thth + cot(th) d_th + d_phph / sin^2 th) / r^2 (conformally flat
  data, the usual choice with A = 0 and K = 0);
* rho is the primitive rest-mass density (the paper's symbol throughout);
* the black hole of mass M enters as a puncture: psi = 1 + M/(2r) solves the vacuum
  problem.  Boundary conditions: at r_min, d_r psi = -M/(2 r_min^2) (the puncture's own
  radial derivative: no flux of the matter correction through the inner sphere); at r_max
  the Robin condition d_r(r (psi - 1)) = 0, i.e. psi + r d_r psi = 1 (psi - 1 falls off
  like 1/r);
* radial elements: the Laplacian holds at every node except the element ends; at a shared
  interface the left copy carries continuity of psi, the right copy continuity of d_r psi;
  inside an element every derivative is the element's own (no interface mean);
* the whole sphere with the Fourier theta basis (theta_basis = 1; psi is a scalar, parity
  +1 under the double-Fourier extension), d_thth the composition of two theta
  derivatives;
* fixed point: psi_{k+1} = L^-1(-2 pi rho psi_k^5, boundary data) from
  psi_0 = 1 + M/(2r), a stated number of iterations;
* initial slice: gammatilde_ij = gamma_ij / det(gamma)^(1/3) (det gammatilde = 1, as in
  the evolution), phi = ln(det gamma)/12, Atilde = 0, K = 0, Gammatilde^i from the
  Christoffel symbols of gammatilde; lapse alpha = psi^-2, shift and driver zero (the paper
  gives no gauge for the initial slice).
"""
from __future__ import annotations

import numpy as np

from . import kerr_schild as ks
from . import solver as so


def _unit_fields(g):
    """The identity as n fields on the grid (n = number of nodes)."""
    n = int(np.prod(g.shape))
    return np.eye(n).reshape((n,) + g.shape)


def operator_matrices(g):
    """Dense n x n matrices (rows = output node, flattened (E, N_r, N_theta, N_phi)) of the
    element-local d_r, d_rr and of the flat angular Laplacian's pieces, built by applying
    the oracle's own derivative operators to every unit field."""
    if not g.fourier_theta:
        raise ValueError("the XCTS solve covers the whole sphere: Fourier theta basis only")
    n = int(np.prod(g.shape))
    I = _unit_fields(g)

    def mat(a):
        return a.reshape(n, n).T          # column j = operator applied to unit field j

    dr = g.d_r(I)
    dt = g.d_t(I, 1.0)
    return {"dr": mat(dr), "drr": mat(g.d_r(dr)), "dt": mat(dt), "dtt": mat(g.d_t(dt, -1.0)),
            "dpp": mat(g.d_p(g.d_p(I)))}


def laplacian(g, ops=None):
    """Flat Laplacian in spherical coordinates at every node (n x n)."""
    ops = ops or operator_matrices(g)
    r = g.R.reshape(-1)[:, None]
    th = g.T.reshape(-1)[:, None]
    return (ops["drr"] + 2.0 / r * ops["dr"]
            + (ops["dtt"] + np.cos(th) / np.sin(th) * ops["dt"]
               + ops["dpp"] / np.sin(th) ** 2) / r ** 2)


def system_matrix(g, M, ops=None):
    """The Laplacian with the rows of the element end nodes replaced by the boundary and
    interface conditions; returns (matrix, boundary data vector, mask of PDE rows)."""
    ops = ops or operator_matrices(g)
    A = laplacian(g, ops)
    E, Nr, Nt, Np = g.shape
    idx = np.arange(A.shape[0]).reshape(g.shape)
    bvals = np.zeros(A.shape[0])
    pde = np.ones(A.shape[0], dtype=bool)
    eye = np.eye(A.shape[0])
    r_min, r_max = g.bounds[0], g.bounds[-1]
    for e in range(E):
        first, last = idx[e, 0].reshape(-1), idx[e, Nr - 1].reshape(-1)
        pde[first] = False
        pde[last] = False
        if e == 0:
            A[first] = ops["dr"][first]
            bvals[first] = -M / (2.0 * r_min ** 2)
        else:
            prev_last = idx[e - 1, Nr - 1].reshape(-1)
            A[first] = ops["dr"][first] - ops["dr"][prev_last]
        if e == E - 1:
            A[last] = eye[last] + r_max * ops["dr"][last]
            bvals[last] = 1.0
        else:
            next_first = idx[e + 1, 0].reshape(-1)
            A[last] = eye[last] - eye[next_first]
    return A, bvals, pde


def solve_psi(g, p, rho, iters=20):
    """Fixed-point relaxation: psi_{k+1} solves the boundary-value problem with the source
    -2 pi rho psi_k^5.  Returns psi (grid shape) and the max |psi_{k+1} - psi_k| per
    iteration."""
    A, bvals, pde = system_matrix(g, p.M)
    psi = 1.0 + p.M / (2.0 * g.R)
    rho = np.asarray(rho).reshape(-1)
    changes = []
    for _ in range(iters):
        f = np.where(pde, -2.0 * np.pi * rho * psi.reshape(-1) ** 5, bvals)
        new = np.linalg.solve(A, f).reshape(g.shape)
        changes.append(float(np.abs(new - psi).max()))
        psi = new
    return psi, changes


def _conformal_flat(r, th):
    """gammatilde_ij = flat spherical metric / det^(1/3): (r^4 sin^2 th)^(-1/3) diag(1, r^2, r^2 sin^2 th)."""
    r = np.asarray(r)
    th = np.asarray(th)
    f = (r ** 4 * np.sin(th) ** 2) ** (-1.0 / 3.0)
    g = np.zeros(np.broadcast(r, th).shape + (3, 3), dtype=np.result_type(r, th, np.float64))
    g[..., 0, 0] = f
    g[..., 1, 1] = f * r ** 2
    g[..., 2, 2] = f * r ** 2 * np.sin(th) ** 2
    return g


def bssn_data(g, psi):
    """BSSN variables of the slice gamma_ij = psi^4 (flat spherical metric), K = 0."""
    R, T = g.R, g.T
    gt = _conformal_flat(R, T)
    h = 1e-30
    dgt = np.stack([np.imag(_conformal_flat(R + 1j * h, T + 0j)) / h,
                    np.imag(_conformal_flat(R + 0j, T + 1j * h)) / h,
                    np.zeros(gt.shape)], axis=-3)
    Gt = np.einsum("...jk,...ijk->...i", ks.inv3(gt), ks.christoffel3(gt, dgt))
    gam = psi[..., None, None] ** 4 * np.einsum("...ij,...->...ij", gt,
                                                (R ** 4 * np.sin(T) ** 2) ** (1.0 / 3.0))
    return {"gt": gt, "phi": np.log(ks.det3(gam)) / 12.0, "At": np.zeros(gt.shape),
            "K": np.zeros(R.shape), "Gt": Gt, "alpha": psi ** -2.0,
            "beta": np.zeros(R.shape + (3,)), "B": np.zeros(R.shape + (3,)), "gamma": gam}


def xcts_state(g, p, prim, iters=20):
    """Canonical state on the XCTS slice: psi from the fixed point with the primitive
    density, then the same matter and field construction as the Kerr-Schild initial data."""
    psi, changes = solve_psi(g, p, prim["rho"], iters)
    return so.initial_state(g, p, prim, bssn=bssn_data(g, psi)), psi, changes
