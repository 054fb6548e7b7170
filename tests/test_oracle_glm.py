"""Oracle pins for GLM divergence cleaning ("GLM Constraint Damping Source"): the psi
equation d_t psi = alpha (-c_h^2 D_i B^i - psi / tau) and the field source
-alpha sqrt(gamma) gamma^ij d_j psi, checked against closed forms on the Kerr-Schild grid
(polynomial profiles in r are differentiated exactly by the spectral operators)."""
import dataclasses

import numpy as np

from oracle import kerr_schild as ks
from oracle import solver as so
from workloads import config


def _setup(**kw):
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg, glm=1, **kw)
    return g, p, U


def _metric(U):
    f = so.unpack_bssn(U)
    gam, sqg = so.metric_from_bssn(f)
    return f["alpha"], gam, sqg


def test_uniform_psi_decays_with_the_rk_polynomial():
    """Frozen metric, no filter, c_h = 0 (psi decoupled from the divergence), uniform
    psi0: one SSP-RK3 step multiplies psi at every (non-frozen) node by
    R(z) = 1 + z + z^2/2 + z^3/6, z = -alpha dt / tau (the lapse varies in space, so grad
    psi and the field source appear during the step, but they do not feed back)."""
    g, p, U = _setup(evolve_metric=0, filter_mask=0)
    p = dataclasses.replace(p, glm_tau=0.7, glm_ch=0.0)
    psi0 = 1e-3
    U[so.I_PSI] = psi0
    dt = 5e-3
    out = so.rk_step(U, dt, g, p)
    alpha, _, _ = _metric(U)
    z = -alpha * dt / p.glm_tau
    ref = psi0 * (1 + z + z * z / 2 + z ** 3 / 6)
    got = out[so.I_PSI]
    interior = np.ones(got.shape, dtype=bool)
    interior[-1, -1] = False                     # frozen outer node
    assert np.max(np.abs(got - ref)[interior]) <= 1e-12 * psi0


def test_divergence_drives_psi():
    """psi = 0, sqrt(gamma) B^r = f(r) cubic, B^theta = B^phi = 0: the psi right-hand side
    is -alpha c_h^2 f'(r) / sqrt(gamma)."""
    g, p, U = _setup()
    p = dataclasses.replace(p, glm_ch=1.3)
    r = g.R
    f = 1e-6 * (0.3 * r ** 3 - 2.0 * r ** 2 + r + 5.0)
    fp = 1e-6 * (0.9 * r ** 2 - 4.0 * r + 1.0)
    U[so.I_B] = f
    U[so.I_B + 1] = 0.0
    U[so.I_B + 2] = 0.0
    U[so.I_PSI] = 0.0
    R = so.rhs(U, g, p)
    alpha, _, sqg = _metric(U)
    ref = -alpha * p.glm_ch ** 2 * fp / sqg
    interior = np.ones(ref.shape, dtype=bool)
    interior[-1, -1] = False
    assert np.max(np.abs(R[so.I_PSI] - ref)[interior]) <= 1e-11 * np.max(np.abs(ref))


def test_psi_gradient_sources_the_field():
    """psi = h(r) quadratic: the field right-hand side changes by
    -alpha sqrt(gamma) gamma^{i r} h'(r), and psi's own right-hand side is -alpha h / tau
    (the initial field is discretely divergence-free)."""
    g, p, U = _setup()
    r = g.R
    h = 1e-4 * (r * r - 3.0 * r + 1.0)
    hp = 1e-4 * (2.0 * r - 3.0)
    U[so.I_PSI] = h
    R1 = so.rhs(U, g, p)
    R0 = so.rhs(U[:so.NV], g, dataclasses.replace(p, glm=0))
    alpha, gam, sqg = _metric(U)
    ginv = ks.inv3(gam)
    interior = np.ones(h.shape, dtype=bool)
    interior[-1, -1] = False
    for i in range(3):
        ref = -alpha * sqg * ginv[..., i, 0] * hp
        diff = R1[so.I_B + i] - R0[so.I_B + i]
        scale = max(np.max(np.abs(ref)), 1e-20)
        assert np.max(np.abs(diff - ref)[interior]) <= 1e-11 * max(scale, np.max(np.abs(R0[so.I_B + i]))), i
    ref_psi = -alpha * h / p.glm_tau
    assert np.max(np.abs(R1[so.I_PSI] - ref_psi)[interior]) <= 1e-11 * np.max(np.abs(ref_psi))
    # every other variable is untouched by psi
    others = [v for v in range(so.NV) if v not in (so.I_B, so.I_B + 1, so.I_B + 2)]
    assert np.array_equal(R1[others], R0[others])
