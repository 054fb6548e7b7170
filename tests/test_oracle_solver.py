"""Pins of the oracle's assembled right-hand side, interface coupling, Runge-Kutta
stages and initial data.

Paper: Methods ("Numerical Algorithm", "Time Integration", "GRMHD Conservative Form",
"Magnetic Constraint").
"""
import numpy as np
import pytest

from oracle import solver as so
from oracle import valencia as va
from oracle import spectral as sp

from helpers import assert_within


def _dust_state(n, Q, E=2):
    """Geodesic dust falling from rest at infinity onto a Schwarzschild hole in
    Kerr-Schild coordinates (u_t = -1, u^r = -sqrt(2M/r)), rho ~ r^-3/2 so that
    sqrt(-g) rho u^r is constant, plus a monopole field sqrt(gamma) B^r = Q sin(theta).
    This is an exact stationary solution of the Valencia equations on the fixed metric."""
    p = so.Params(a=0.0, n_elem=E, r_min=1.5, r_max=8.0, n_r=n, n_theta=n, n_phi=4,
                  theta_min=np.pi / 4, theta_max=3 * np.pi / 4, gauge=1, evolve_metric=0)
    g = so.Grid(p)
    z = np.zeros(g.shape)
    U = so.initial_state(g, p, dict(rho=np.ones(g.shape), p=np.full(g.shape, 1e-30), vr=z,
                                    vth=z, vph=z, A_phi=z))
    f = so.unpack_bssn(U)
    gam, sqg = so.metric_from_bssn(f)
    s = np.sqrt(2.0 / g.R)
    ut = (1 + s + s * s) / (1 + s)
    al, be = f["alpha"], f["beta"]
    vr = -s / (al * ut) + be[..., 0] / al
    rho = 1e-2 / (g.R ** 2 * s)
    Bt = np.zeros(g.shape + (3,))
    Bt[..., 0] = Q * np.sin(g.T)
    B = Bt / sqg[..., None]
    v = np.stack([vr, z, z], -1)
    D, S, tau, _ = va.prim_to_cons(rho, v, z, B, al, be, gam, p.gamma_eos)
    U[so.I_D] = sqg * D
    for i in range(3):
        U[so.I_S + i] = sqg * S[..., i]
        U[so.I_B + i] = Bt[..., i]
    U[so.I_TAU] = sqg * tau
    prim = dict(rho=rho, v=v, eps=z, p=z, W=al * ut, B=B)
    return g, p, U, prim


@pytest.mark.parametrize("Q", [0.0, 0.3])
def test_dust_accretion_stationary(Q):
    errs = []
    for n in (8, 12, 16, 20):
        g, p, U, prim = _dust_state(n, Q)
        R = so.rhs_from_prims(U, prim, g, p)
        sc = np.abs(U[24:29]).max()
        errs.append(np.abs(R[24:32]).max() / sc)
    assert errs[0] > 1e-6
    assert all(b < a / 5 for a, b in zip(errs[:-1], errs[1:]))
    assert errs[-1] < 1e-10


def test_mass_identity():
    """Clenshaw-Curtis x Fejer x trapezoid quadrature of RHS(D~) over all elements equals
    the boundary flux terms to rounding: the interface penalties telescope (both sides use
    the same F*), so sum w RHS = F^r(r_min) - F^r(r_max) - [F^theta]_{theta ends}, the
    theta term being the interpolating polynomial's end values.  A noisy, non-smooth
    state makes the interface jumps non-zero."""
    from workloads import config
    cfg = config("c1", n_elem=3, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg, evolve_metric=0)
    # break continuity at the interfaces so that the penalty terms are active
    rng = np.random.default_rng(4)
    U[so.I_D:so.I_D + 5, 0, -1] *= 1 + 0.01 * rng.uniform(size=U[so.I_D:so.I_D + 5, 0, -1].shape)
    U[so.I_D:so.I_D + 5, 1, -1] *= 1 - 0.01 * rng.uniform(size=U[so.I_D:so.I_D + 5, 1, -1].shape)
    prim = so.primitives(U, p)
    f = so.unpack_bssn(U)
    gam, sqg = so.metric_from_bssn(f)
    F = va.fluxes(prim["rho"], prim["v"], prim["eps"], prim["B"], f["alpha"], f["beta"], gam,
                  p.gamma_eos) * sqg[..., None, None]
    R = so.rhs_from_prims(U, prim, g, p, freeze_outer=False)
    w = so.quadrature_weights(g)
    wt = sp.fejer_weights(p.n_theta) / g.t_scale
    wp = 2 * np.pi / p.n_phi
    Fr = F[..., 0, 0]
    inner = np.sum(Fr[0, 0] * wt[:, None] * wp)
    outer = np.sum(Fr[-1, -1] * wt[:, None] * wp)
    c = sp.cheb_coeffs(F[..., 1, 0], g.xt, axis=2)
    ends = (sp.cheb_eval(c, np.array([1.0]), axis=2)[:, :, 0]
            - sp.cheb_eval(c, np.array([-1.0]), axis=2)[:, :, 0])
    wr = sp.clenshaw_curtis_weights(p.n_r)[None, :] / g.r_scale[:, None]
    theta_term = np.sum(wr[:, :, None] * ends * wp)
    total = np.sum(w * R[so.I_D])
    assert np.abs(U[so.I_D, 0, -1] - U[so.I_D, 1, 0]).max() > 0
    np.testing.assert_allclose(total, inner - outer - theta_term, rtol=1e-11,
                               atol=1e-13 * np.abs(inner))


def test_divergence_free_initial_field():
    from workloads import config
    cfg = config("c1", n_elem=2, n_r=10, n_theta=10, n_phi=8)
    g, p, U = so.workload_state(cfg)
    div = g.d_r(U[so.I_B]) + g.d_t(U[so.I_B + 1]) + g.d_p(U[so.I_B + 2])
    scale = np.abs(g.d_r(U[so.I_B + 1])).max()
    assert scale > 0
    assert np.abs(div).max() < 1e-12 * scale


@pytest.mark.parametrize("integrator,amp", [
    (0, lambda z: 1 + z + z ** 2 / 2 + z ** 3 / 6),
    (1, lambda z: 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)])
def test_rk_amplification(monkeypatch, integrator, amp):
    """u' = lambda u: SSP-RK3 / RK4 amplification polynomials."""
    lam = -0.7 + 0.3j
    lam_r = np.real(lam)
    monkeypatch.setattr(so, "rhs", lambda U, g, p: lam_r * U)
    p = so.Params(integrator=integrator, filter_mask=0)
    U = np.ones((32, 1, 1, 1, 1))
    dt = 0.4
    out = so.rk_step(U, dt, None, p)
    np.testing.assert_allclose(out, amp(lam_r * dt) * U, rtol=1e-15)


def test_cfl_and_interfaces():
    from workloads import config
    g, p, U = so.workload_state(config("c1"))
    dt = so.cfl_dt(U, g, p)
    assert 0 < dt < 0.1
    p2 = so.Params(**{**p.__dict__, "cfl": 0.15})
    np.testing.assert_allclose(so.cfl_dt(U, g, p2), dt / 2, rtol=1e-14)
    # the filter leaves BSSN interface copies equal
    Uf = so.apply_filter(U, g, p)
    np.testing.assert_array_equal(Uf[:24, 0, -1], Uf[:24, 1, 0])


# ---------------------------------------------------------------- split coupling
# The paper's coupled loop ("Coupled Main Loop"): fluid step on the frozen metric, then a
# forward-Euler BSSN + gauge step with the fluid frozen (first-order Lie splitting).
def _split_setup():
    import dataclasses
    from workloads import config
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg)
    p = dataclasses.replace(p, integrator=1, filter_mask=0)
    return g, p, U


def test_split_step_parts():
    """Valencia part = fixed-metric RK4 step; BSSN part = one Euler step of the BSSN RHS
    evaluated on (updated fluid, old metric); the filter-free step has no other term."""
    import dataclasses
    g, p, U = _split_setup()
    dt = 2e-3
    got = so.rk_step(U, dt, g, dataclasses.replace(p, coupling=1))
    fluid = so.rk_step(U, dt, g, dataclasses.replace(p, evolve_metric=0))
    assert np.array_equal(got[so.I_D:], fluid[so.I_D:])
    assert np.array_equal(fluid[:so.N_BSSN], U[:so.N_BSSN])      # metric frozen in the fluid half
    Lb = so.rhs(fluid, g, dataclasses.replace(p, evolve_fluid=0))
    assert np.all(Lb[so.I_D:] == 0.0)
    assert np.array_equal(got[:so.N_BSSN], fluid[:so.N_BSSN] + dt * Lb[:so.N_BSSN])


def test_split_error_is_second_order():
    """One split step differs from the unsplit RK4 step by O(dt^2) (Lie splitting):
    halving dt divides the difference by ~4."""
    import dataclasses
    g, p, U = _split_setup()
    diffs = []
    for dt in (4e-3, 2e-3, 1e-3):
        a = so.rk_step(U, dt, g, dataclasses.replace(p, coupling=1))
        b = so.rk_step(U, dt, g, p)
        diffs.append(np.max(np.abs(a - b)))
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, (diffs, r1, r2)


@pytest.mark.parametrize("theta_basis", [0, 1])
def test_mass_and_entropy_closed_form(theta_basis):
    """Rest mass and entropy diagnostics on flat space in spherical coordinates
    (sqrt(gamma) = r^2 sin(theta)) against their integrals written out by hand.

    rho = rho0 (1 + r/4), a uniform radial velocity v^r = 0.3 (W = 1/sqrt(1 - 0.09)),
    p = rho^Gamma exp((Gamma - 1) s) with the specific entropy s = s0 + s1 r.  Then
    mass = W int rho dV and entropy = int rho s dV, dV = r^2 sin(theta) dr dtheta dphi;
    both radial integrands are polynomials the Clenshaw-Curtis rule integrates exactly,
    and the theta factor is int sin(theta) dtheta.  A dropped sqrt(gamma), D in place of
    rho in the entropy, a missing 1/(Gamma - 1) in s or wrong per-element weights each
    change one of the two numbers at O(1)."""
    if theta_basis:
        p = so.Params(M=0.0, a=0.0, n_elem=3, r_min=2.0, r_max=6.0, n_r=8, n_theta=16,
                      n_phi=4, theta_basis=1)
    else:
        p = so.Params(M=0.0, a=0.0, n_elem=3, r_min=2.0, r_max=6.0, n_r=8, n_theta=16,
                      n_phi=4, theta_min=0.3, theta_max=2.5)
    g = so.Grid(p)
    rho0, s0, s1, vr, G = 1e-2, 0.7, -0.15, 0.3, p.gamma_eos
    z = np.zeros(g.shape)
    rho = rho0 * (1.0 + g.R / 4.0)
    s = s0 + s1 * g.R
    pr = rho ** G * np.exp((G - 1.0) * s)
    U = so.initial_state(g, p, dict(rho=rho, p=pr, vr=np.full(g.shape, vr), vth=z, vph=z,
                                    A_phi=z))
    _, sqg = so.metric_from_bssn(so.unpack_bssn(U))
    np.testing.assert_allclose(sqg, g.R ** 2 * np.sin(g.T), rtol=1e-13)
    a, b = p.r_min, p.r_max
    th0, th1 = (0.0, np.pi) if theta_basis else (p.theta_min, p.theta_max)
    ang = 2.0 * np.pi * (np.cos(th0) - np.cos(th1))

    def mom(k):                                     # int_a^b r^k dr
        return (b ** (k + 1) - a ** (k + 1)) / (k + 1)
    W = 1.0 / np.sqrt(1.0 - vr * vr)
    mass = W * rho0 * (mom(2) + mom(3) / 4.0) * ang
    ent = rho0 * (s0 * mom(2) + (s0 / 4.0 + s1) * mom(3) + s1 / 4.0 * mom(4)) * ang
    d = so.diagnostics(U, g, p)
    assert d[3] == 0.0
    np.testing.assert_allclose(d[0], mass, rtol=1e-12)
    np.testing.assert_allclose(d[1], ent, rtol=1e-11)
