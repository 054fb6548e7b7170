"""GLM divergence cleaning on the GPU (glm = 1: psi is variable 32) against the oracle:
right-hand side and two SSP-RK3 steps, with psi nonzero and a field perturbed away from
zero divergence so that both GLM terms act."""
import numpy as np
import pytest

from oracle import solver as so
from workloads import config

from oracle import rounding as fpf
import test_gpu_parity as tp
from test_gpu_parity import pkg  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu



def _glm_state(cfg, **kw):
    g, p, U = so.workload_state(cfg, glm=1, **kw)
    U[so.I_PSI] = 1e-4 * np.sin(3.0 * g.T) * np.cos(g.P) * (g.R / g.R.max())
    U[so.I_B] = U[so.I_B] * (1.0 + 0.05 * np.cos(2.0 * g.P))   # d_i (sqrt(gamma) B^i) != 0
    return g, p, U


@pytest.mark.parametrize("contraction", [0, 1])
def test_glm_rhs_parity(pkg, contraction):  # noqa: F811
    cfg = config("c1")
    g, p, U = _glm_state(cfg)
    ctx = tp._ctx(pkg, cfg, glm=1, contraction=contraction)
    assert ctx.nv == 33
    R = tp._gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    assert np.abs(Rref[so.I_PSI]).max() > 0
    tp.assert_parity(R, Rref, f"glm rhs contraction {contraction}", lambda X: so.rhs(X, g, p), U)
    ctx.close()


def test_glm_step_parity(pkg):  # noqa: F811
    import torch
    cfg = config("c1", n_elem=3, n_r=9, n_theta=10, n_phi=8)
    g, p, U = _glm_state(cfg)
    ctx = tp._ctx(pkg, cfg, glm=1)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    dt = 2e-3
    ctx.step(dt, 2)
    got = np.empty(U.size)
    ctx.get_state(got, False)
    two = lambda X: so.rk_step(so.rk_step(X, dt, g, p), dt, g, p)  # noqa: E731
    tp.assert_parity(got.reshape(U.shape), two(U), "glm 2 steps", two, U, trials=2)
    ctx.close()


def test_glm_mixed_rhs(pkg):  # noqa: F811
    """split-BF16 x3 contractions with FP32 algebra: within the mixed bar 2e-6."""
    cfg = config("c1")
    g, p, U = _glm_state(cfg)
    ctx = tp._ctx(pkg, cfg, glm=1, precision=1)
    R = tp._gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    tp.assert_parity(R, Rref, "glm mixed rhs", lambda X: so.rhs(X, g, p), U, tol=2e-6, eps=fpf.EPS32, kappa=1.0)
    ctx.close()
