"""Pins of the oracle's approximate XCTS initial data (paper: "Initial Data: Approximate XCTS
Solution").

Checked against things fixed outside the oracle: harmonic polynomials (the flat Laplacian
of x, z, r^2 P_2(cos theta) vanishes, of r^2 it is 6), the vacuum puncture 1 + M/(2r),
a manufactured solution whose density comes from the analytic Laplacian, the contraction
of the fixed point, and closed forms of the conformally flat slice.
"""
import numpy as np
import pytest

from oracle import solver as so
from oracle import xcts
from workloads import config


def _grid(E=2, nr=12, nt=8, nph=8, **kw):
    cfg = config("c1", theta_min=0.0, theta_max=np.pi, theta_basis=1, n_elem=E, n_r=nr,
                 n_theta=nt, n_phi=nph, **kw)
    p = so.Params.from_config(cfg)
    return so.Grid(p), p


def test_laplacian_exact_on_harmonic_polynomials():
    g, p = _grid()
    L = xcts.laplacian(g)
    R, T, P = g.R, g.T, g.P
    cases = [(R * np.cos(T), 0.0), (R * np.sin(T) * np.cos(P), 0.0),
             (R ** 2 * (3 * np.cos(T) ** 2 - 1), 0.0),
             (R ** 2 * np.sin(T) ** 2 * np.cos(2 * P), 0.0), (R ** 2, 6.0)]
    for u, lap in cases:
        res = (L @ u.reshape(-1)).reshape(g.shape) - lap
        assert np.abs(res).max() < 1e-10 * max(1.0, np.abs(u).max())
    # a wrong sign of the cot(theta) term or a missing 2/r term would show here
    u = R * np.cos(T) + R ** 2
    assert np.abs((L @ u.reshape(-1)).reshape(g.shape) - 6.0).max() < 1e-9


def test_vacuum_is_the_puncture():
    errs = []
    for nr in (10, 16, 24):
        g, p = _grid(E=3, nr=nr, nt=6, nph=4)
        psi, ch = xcts.solve_psi(g, p, np.zeros(g.shape), iters=2)
        errs.append(np.abs(psi - (1.0 + p.M / (2.0 * g.R))).max())
        assert ch[1] == 0.0                       # zero source: the first solve is the fixed point
    assert errs[2] < 1e-9 and errs[1] < errs[0] and errs[2] < errs[1], errs


def _manufactured(g, M):
    """psi = 1 + M/(2r) + f(r) Y(theta, phi), f a Gaussian shell away from both boundaries;
    rho = -lap(psi) / (2 pi psi^5) from the analytic Laplacian (Y has l = 0 and l = 1 parts:
    the angular Laplacian of the l = 1 part is -2 / r^2 times it)."""
    R, T, P = g.R, g.T, g.P
    c, r0, w = 0.02, 8.0, 1.2
    f = c * np.exp(-((R - r0) / w) ** 2)
    f1 = -2.0 * (R - r0) / w ** 2 * f
    f2 = (4.0 * (R - r0) ** 2 / w ** 4 - 2.0 / w ** 2) * f
    Y1 = 0.3 * np.sin(T) * np.cos(P) + 0.2 * np.cos(T)
    Y = 1.0 + Y1
    psi = 1.0 + M / (2.0 * R) + f * Y
    lap = (f2 + 2.0 * f1 / R) * Y - 2.0 * f / R ** 2 * Y1
    return psi, -lap / (2.0 * np.pi * psi ** 5)


def test_manufactured_solution_converges():
    errs = []
    for nr in (12, 20, 28):
        g, p = _grid(E=3, nr=nr, nt=6, nph=4)
        psi_ex, rho = _manufactured(g, p.M)
        psi, ch = xcts.solve_psi(g, p, rho, iters=25)
        assert ch[-1] < 1e-11                     # converged to the rounding of the solve
        errs.append(np.abs(psi - psi_ex).max())
    # spectral convergence (8e-4, 4e-5, 2e-7 for this shell, which straddles an interface)
    assert errs[2] < 1e-6 and errs[0] > 10 * errs[1] > 100 * errs[2], errs


def test_fixed_point_contracts():
    """The paper's plain fixed point contracts when 10 pi rho psi^4 is small against the
    Laplacian's smallest eigenvalue: the power-law gas at rho0 = 1e-4 (at 1e-2, the evolution
    workloads' density, it diverges)."""
    from workloads import primitive_profiles
    cfg = config("c1", theta_min=0.0, theta_max=np.pi, theta_basis=1, n_elem=2, n_r=10,
                 n_theta=6, n_phi=4, rho0=1e-4)
    p = so.Params.from_config(cfg)
    g = so.Grid(p)
    prim = primitive_profiles(cfg, g.R, g.T, g.P)
    psi, ch = xcts.solve_psi(g, p, prim["rho"], iters=12)
    # contraction while the change is above the rounding floor of psi ~ 1 (a few 1e-14)
    ch = np.array(ch)
    k = int(np.argmax(ch < 1e-12))
    assert k >= 6, ch
    ratios = ch[2:k] / ch[1:k - 1]
    assert np.all(ratios < 0.1) and ch[-1] < 1e-12, ch
    assert np.all(psi > 1.0 + p.M / (2.0 * g.R) - 1e-12)   # positive density raises psi


def test_conformally_flat_slice_closed_forms():
    g, p = _grid(E=2, nr=6, nt=6, nph=4)
    psi = 1.0 + p.M / (2.0 * g.R) + 0.01 * np.cos(g.T)
    d = xcts.bssn_data(g, psi)
    R, T = g.R, g.T
    np.testing.assert_allclose(np.linalg.det(d["gt"]), 1.0, rtol=1e-13)
    np.testing.assert_allclose(d["phi"], np.log(psi) + np.log(R ** 4 * np.sin(T) ** 2) / 12.0,
                               rtol=1e-13, atol=1e-14)
    # Gammatilde^i = -d_j gammatilde^ij for det gammatilde = 1
    np.testing.assert_allclose(d["Gt"][..., 0], -4.0 / 3.0 * R ** (1 / 3) * np.sin(T) ** (2 / 3),
                               rtol=1e-12)
    np.testing.assert_allclose(d["Gt"][..., 1],
                               -2.0 / 3.0 * R ** (-2 / 3) * np.sin(T) ** (-1 / 3) * np.cos(T),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(d["Gt"][..., 2], 0.0, atol=1e-14)
    np.testing.assert_allclose(d["alpha"], psi ** -2, rtol=1e-15)


def test_chebyshev_theta_refused():
    g = so.Grid(so.Params.from_config(config("c1")))
    with pytest.raises(ValueError):
        xcts.operator_matrices(g)
