"""Pins of the oracle's Fourier theta basis (Methods: "Grid Discretization", "Pseudo-spectral
theta derivative", "Dealiasing and Spectral Filtering") and of its parity table.

The checks compare against things fixed outside the oracle: derivatives of trigonometric
polynomials that are smooth on the sphere, closed-form filter factors of pure modes,
exact integrals, the coordinate transformation of smooth Cartesian tensors (which fixes
the sign of every component under the extension across the pole), the Kerr-Schild
slice's own analytic theta derivatives, and the equatorial symmetry of the whole
right-hand side.
"""
import dataclasses

import numpy as np
import pytest

from oracle import kerr_schild as ks
from oracle import solver as so
from oracle import spectral as sp


def _grid(n_t=16, n_p=12):
    th = sp.uniform_theta_nodes(n_t)
    ph = sp.fourier_nodes(n_p)
    return np.meshgrid(th, ph, indexing="ij")


def _dth(u, parity):
    return sp.fourier_theta_deriv(u, 0, 1, parity)


def test_nodes_uniform_and_pole_free():
    th = sp.uniform_theta_nodes(8)
    np.testing.assert_allclose(np.diff(th), np.pi / 8, rtol=1e-14)
    np.testing.assert_allclose(th[0], np.pi / 16, rtol=1e-15)
    np.testing.assert_allclose(th + th[::-1], np.pi, rtol=1e-15)
    # x = -cos(theta) gives the Chebyshev-Gauss points
    np.testing.assert_allclose(-np.cos(th), sp.gauss_nodes(8), atol=1e-15)


def test_derivative_exact_on_smooth_sphere_functions():
    T, P = _grid()
    # a scalar (parity +1): x/r, z/r and a degree-2 harmonic
    u = np.sin(T) * np.cos(P) + np.cos(T) + np.sin(T) ** 2 * np.cos(2 * P)
    du = np.cos(T) * np.cos(P) - np.sin(T) + 2 * np.sin(T) * np.cos(T) * np.cos(2 * P)
    np.testing.assert_allclose(_dth(u, 1.0), du, atol=1e-13)
    # the theta component of the constant vector x-hat, r V^theta = cos(theta) cos(phi): -1
    v = np.cos(T) * np.cos(P)
    np.testing.assert_allclose(_dth(v, -1.0), -np.sin(T) * np.cos(P), atol=1e-13)
    # a density like sqrt(gamma) = r^2 sin(theta) (1 + cos^2 theta): -1
    w = np.sin(T) * (1 + np.cos(T) ** 2)
    dw = np.cos(T) * (1 + np.cos(T) ** 2) - 2 * np.sin(T) ** 2 * np.cos(T)
    np.testing.assert_allclose(_dth(w, -1.0), dw, atol=1e-13)
    # the wrong sign gives an O(1) error: the extension is not decorative
    assert np.abs(_dth(u, -1.0) - du).max() > 0.1
    assert np.abs(_dth(w, 1.0) - dw).max() > 0.1


def test_second_derivative_is_composition_with_flipped_parity():
    T, P = _grid(20, 8)
    u = np.cos(T) ** 3 + np.sin(T) ** 2 * np.sin(2 * P)
    d2 = -3 * np.cos(T) * (np.cos(T) ** 2 - 2 * np.sin(T) ** 2) + 2 * np.cos(2 * T) * np.sin(2 * P)
    got = _dth(_dth(u, 1.0), -1.0)
    np.testing.assert_allclose(got, d2, atol=1e-12)
    # and the paper's (i k)^2 multiplier on the extended line gives the same values
    direct = np.take(sp.fourier_deriv(sp.parity_extend(u, 0, 1, 1.0), 0, order=2), np.arange(20), 0)
    np.testing.assert_allclose(direct, d2, atol=1e-12)


@pytest.mark.parametrize("parity", [1.0, -1.0])
def test_filter_pure_modes(parity):
    n = 12
    T, P = _grid(n, 4)
    # cos(m theta) is even about the poles (parity +1 for phi-independent data),
    # sin(m theta) odd: both are single Fourier modes of the extended line
    for m in range(0, 2 * n):
        u = np.cos(m * T) if parity > 0 else np.sin(m * T)
        if parity < 0 and m == 0:
            continue
        kk = m if m <= n else 2 * n - m
        sig = np.exp(-36.0 * (kk / n) ** 8)
        if kk > 2 * n / 3:
            sig = 0.0
        got = sp.fourier_theta_filter(u, 0, 1, parity, dealias23=True)
        if m == n:
            # the Nyquist mode of the extended line: cos(n theta) vanishes on the nodes
            # (parity +1), sin(n theta) = +-1 is kept with the Nyquist factor
            continue
        np.testing.assert_allclose(got, sig * u, atol=1e-13)
        nod = sp.fourier_theta_filter(u, 0, 1, parity, dealias23=False)
        np.testing.assert_allclose(nod, np.exp(-36.0 * (kk / n) ** 8) * u, atol=1e-13)


def test_quadrature_exact_for_density_integrands():
    for n in (4, 9, 16):
        w = sp.fourier_theta_weights(n)
        th = sp.uniform_theta_nodes(n)
        for j in range(0, n // 2):
            got = w @ (np.sin(th) * np.cos(th) ** (2 * j))
            np.testing.assert_allclose(got, 2.0 / (2 * j + 1), rtol=1e-13)
        np.testing.assert_allclose(w @ (np.sin(th) * np.cos(th)), 0.0, atol=1e-14)


# ------------------------------------------------------------------ the parity table
def _jac(r, T, P):
    """J[a, i] = d x^a / d q^i, q = (r, theta, phi)."""
    st, ct, sp_, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    J = np.empty((3, 3) + T.shape, dtype=np.result_type(T, 1.0))
    J[0] = [st * cp, r * ct * cp, -r * st * sp_]
    J[1] = [st * sp_, r * ct * sp_, r * st * cp]
    J[2] = [ct, -r * st, np.zeros_like(T)]
    return J


def _jinv(r, T, P):
    """K[i, a] = d q^i / d x^a."""
    st, ct, sp_, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    K = np.empty((3, 3) + T.shape, dtype=np.result_type(T, 1.0))
    K[0] = [st * cp, st * sp_, ct]
    K[1] = [ct * cp / r, ct * sp_ / r, -st / r]
    K[2] = [-sp_ / (r * st), cp / (r * st), np.zeros_like(T)]
    return K


def _check_slot(f, parity):
    """f(theta) smooth on the sphere: the extended derivative with the table's parity is
    exact (complex-step reference), the opposite parity is not."""
    n_t, n_p = 18, 8
    T, P = _grid(n_t, n_p)
    h = 1e-30
    ref = np.imag(f(T + 1j * h, P)) / h
    u = np.real(f(T + 0j, P))
    scale = max(np.abs(ref).max(), np.abs(u).max())
    err = np.abs(_dth(u, parity) - ref).max()
    assert err < 1e-12 * scale, err
    bad = np.abs(_dth(u, -parity) - ref).max()
    assert bad > 1e-3 * scale or scale < 1e-12


def test_parity_table_from_coordinate_transformation():
    """Smooth Cartesian fields mapped to the spherical coordinate basis: every slot of
    the canonical state gets the sign that makes its extension smooth."""
    rng = np.random.default_rng(4)
    S = rng.normal(size=(3, 3))
    S = S + S.T                                   # constant symmetric Cartesian tensor
    V = rng.normal(size=3)                        # constant vector
    r = 2.0
    par = so.THETA_PAR
    # covariant symmetric tensors: gammatilde_ij, Atilde_ij
    for n, (i, j) in enumerate(so.SYM):
        def f(T, P, i=i, j=j):
            J = _jac(r, T, P)
            return sum(J[a, i] * J[b, j] * S[a, b] for a in range(3) for b in range(3))
        _check_slot(f, par[so.I_GT + n])
        _check_slot(f, par[so.I_AT + n])
    for i in range(3):
        # contravariant vectors (Gammatilde^i, beta^i, B^i of the gauge): sin^2 removes
        # the 1/sin(theta) of the phi component without changing its sign
        def fu(T, P, i=i):
            K = _jinv(r, T, P)
            return sum(K[i, a] * V[a] for a in range(3)) * np.sin(T) ** 2
        for base in (so.I_GAM, so.I_BETA, so.I_BG):
            _check_slot(fu, par[base + i])

        # densities sqrt(gamma) S_i (covariant) and sqrt(gamma) B^i (contravariant),
        # sqrt(gamma) = r^2 sin(theta) of flat space
        def fS(T, P, i=i):
            J = _jac(r, T, P)
            return r * r * np.sin(T) * sum(J[a, i] * V[a] for a in range(3))

        def fB(T, P, i=i):
            K = _jinv(r, T, P)
            return r * r * np.sin(T) * sum(K[i, a] * V[a] for a in range(3))
        _check_slot(fS, par[so.I_S + i])
        _check_slot(fB, par[so.I_B + i])

    def fscal(T, P):
        return 1.0 + 0.3 * np.cos(T) + 0.2 * np.sin(T) * np.cos(P)
    for v in (so.I_PHI, so.I_K, so.I_ALPHA, so.I_PSI):
        _check_slot(fscal, par[v])
    for v in (so.I_D, so.I_TAU):
        _check_slot(lambda T, P: r * r * np.sin(T) * fscal(T, P), par[v])
    # fluxes: sqrt(gamma) F^theta carries one more theta index
    np.testing.assert_array_equal(so.FLUX_T_PAR, -par[so.I_D:so.I_D + 8])


def test_kerr_schild_lapse_and_volume_element_are_smooth_with_their_parity():
    """The Kerr-Schild lapse (parity +1) and sqrt(gamma) (parity -1) of the slice:
    extended derivatives converge to the analytic ones."""
    M, a, r = 1.0, 0.9, 3.0
    errs = {}
    for n in (16, 32):
        T, P = _grid(n, 4)
        R = np.full_like(T, r)
        alpha, _, gam = ks.adm(M, a, R + 0j, T + 1e-30j)
        dalpha = np.imag(alpha) / 1e-30
        sqg = np.sqrt(ks.det3(gam)) * np.sign(np.sin(T))
        dsqg = np.imag(sqg) / 1e-30
        errs[n] = (np.abs(_dth(np.real(alpha), so.THETA_PAR[so.I_ALPHA]) - dalpha).max(),
                   np.abs(_dth(np.real(sqg), so.THETA_PAR[so.I_D]) - dsqg).max() / np.abs(dsqg).max())
    assert errs[32][0] < 1e-9 and errs[32][1] < 1e-9, errs
    assert errs[32][0] < errs[16][0] or errs[16][0] < 1e-12


# ------------------------------------------------------------------ the whole solver
def _fourier_case(**kw):
    from workloads import config
    cfg = config("c1", n_elem=2, n_r=8, n_theta=12, n_phi=8, theta_min=0.0, theta_max=np.pi,
                 theta_basis=1, noise_amp=0.0, profile="torus", A0=0.05, **kw)
    return so.workload_state(cfg)


def test_fourier_theta_rhs_equatorial_symmetry():
    """Kerr-Schild plus a torus without noise is symmetric under theta -> pi - theta; the
    right-hand side must be too, each component with the sign (-1)^(theta indices), the
    magnetic field (an axial vector: B = curl A with A_phi even about the equator) with
    one more sign (densities do not change sign here: sin(pi - theta) = sin(theta))."""
    g, p, U = _fourier_case()
    L = so.rhs(U, g, p)
    assert np.all(np.isfinite(L))
    sgn = np.ones(so.NV)
    for n, (i, j) in enumerate(so.SYM):
        sgn[so.I_GT + n] = sgn[so.I_AT + n] = (-1.0) ** ((i == 1) + (j == 1))
    for i in range(3):
        s = -1.0 if i == 1 else 1.0
        sgn[so.I_GAM + i] = sgn[so.I_BETA + i] = sgn[so.I_BG + i] = s
        sgn[so.I_S + i] = s
        sgn[so.I_B + i] = -s
    mirrored = L[:, :, :, ::-1, :] * sgn[:, None, None, None, None]
    # per variable, floored at 1e-6 of the largest right-hand side (components that
    # vanish analytically carry only rounding)
    scale = np.maximum(np.abs(L).max(axis=(1, 2, 3, 4)), 1e-6 * np.abs(L).max())
    err = np.abs(L - mirrored).max(axis=(1, 2, 3, 4)) / scale
    assert err.max() < 1e-9, (int(err.argmax()), float(err.max()))


def test_fourier_theta_step_and_diagnostics():
    g, p, U = _fourier_case()
    dt = so.cfl_dt(U, g, p)
    # the node nearest the pole sets the azimuthal spacing r sin(theta_0) dphi
    assert dt > 0
    U1 = so.rk_step(U, dt, g, p)
    assert np.all(np.isfinite(U1))
    d = so.diagnostics(U, g, p)
    assert np.isfinite(d).all() and d[0] > 0
    # filter with 2/3 rule in theta leaves a band-limited Valencia field unchanged up to
    # the exponential factor of its modes: check on the density of a uniform gas
    p0 = dataclasses.replace(p, filter_mask=2)    # theta filter, Valencia group only
    V = U.copy()
    V[so.I_D] = np.sin(g.T) * 2.0                 # parity -1, single mode k = 1
    F = so.apply_filter(V, g, p0)
    np.testing.assert_allclose(F[so.I_D], V[so.I_D] * np.exp(-36.0 * (1.0 / g.p.n_theta) ** 8),
                               rtol=1e-12)
    with pytest.raises(ValueError):
        g.d_t(U[0])                                # the Fourier basis needs a parity
