"""Robustness of the GPU path without faulting the GPU: the device-side wait limits and
checkpoint / resume.

* The digit-slice contraction waits on mbarriers with a time limit (about 0.5 s per wait,
  globaltimer).  grmhd_debug_wait_timeout withholds the kernel's tiles on request, so every
  wait runs out: the call must report GRMHD_ETIMEOUT and the context must keep working
  (the next right-hand side still matches the oracle at the FP64 bar).
* Resume: state written out, the context destroyed, a new one created from the state, the
  stepping continued: the same states as an uninterrupted run.  Not bit for bit: the
  primitive recovery starts each stage's Newton iteration from the previous stage's
  primitives, which a new context does not have, so the roots may differ in the last bits
  (the FP64 bar 1e-11 applies, measured ~1e-15).
"""
import numpy as np
import pytest

from oracle import solver as so
from workloads import config

import test_gpu_parity as tp
from test_gpu_parity import pkg  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def test_wait_limit_reports_timeout_and_context_survives(pkg):  # noqa: F811
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg)
    ctx = tp._ctx(pkg, cfg)
    R0 = tp._gpu_rhs(pkg, ctx, U)
    assert ctx.debug_wait_timeout() == pkg.GRMHD_ETIMEOUT
    assert "timed out" in ctx.lib.grmhd_last_error(ctx.h).decode()
    R1 = tp._gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    fn = lambda X: so.rhs(X, g, p)  # noqa: E731
    tp.assert_parity(R0, Rref, "rhs before the timed-out wait", fn, U)
    tp.assert_parity(R1, Rref, "rhs after the timed-out wait", fn, U)
    ctx.close()
    # a context without digit-slice operators has nothing to stall
    ctx = tp._ctx(pkg, cfg, contraction=1)
    assert ctx.debug_wait_timeout() == pkg.GRMHD_EUNSUPPORTED
    ctx.close()


def test_resume_after_destroy(pkg):  # noqa: F811
    import torch
    cfg = config("c1", n_elem=3, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg)
    dt = 1e-3
    ctx = tp._ctx(pkg, cfg)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    ctx.step(dt, 2)
    ctx.step(dt, 2)
    ref = np.empty(U.size)
    ctx.get_state(ref, False)
    ctx.close()

    ctx = tp._ctx(pkg, cfg)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    ctx.step(dt, 2)
    mid = np.empty(U.size)
    ctx.get_state(mid, False)
    ctx.close()
    ctx = tp._ctx(pkg, cfg)
    ctx.set_state(mid, False)
    ctx.step(dt, 2)
    got = np.empty(U.size)
    ctx.get_state(got, False)
    ctx.close()
    # the resumed run restarts the primitive recovery from a bracket (set_state), so it
    # differs from the uninterrupted run by rounding: the parity bar with the oracle's
    # floor of four steps
    four = lambda X: so.rk_step(so.rk_step(so.rk_step(so.rk_step(X, dt, g, p), dt, g, p), dt, g, p),  # noqa: E731
                                dt, g, p)
    tp.assert_parity(got.reshape(U.shape), ref.reshape(U.shape), "resumed run", four, U, trials=2)


def test_unphysical_states_are_floored_not_trapped(pkg):  # noqa: F811
    """Conserved states with no admissible inversion (tau lowered below the internal
    energy at a few nodes) injected on the host: the primitive recovery floors eps there,
    counts the nodes, agrees with the oracle's floored primitives, and a time step stays
    finite (no trap, no NaN)."""
    import torch
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, p, U = so.workload_state(cfg)
    bad = U.copy()
    rng = np.random.default_rng(3)
    nodes = [tuple(int(rng.integers(0, n)) for n in g.shape) for _ in range(6)]
    prim0 = so.primitives(U, p)
    for nd in nodes:
        D = bad[(so.I_D,) + nd]
        bad[(so.I_TAU,) + nd] -= 2.0 * prim0["eps"][nd] * D + 0.1 * D
    ref = so.primitives(bad, p)
    ctx = tp._ctx(pkg, cfg)
    ctx.set_state(torch.from_numpy(bad.reshape(-1).copy()).cuda(), True)
    out = torch.empty(7 * U[0].size, dtype=torch.float64, device="cuda")
    nf = ctx.con2prim(out, True)
    P = out.cpu().numpy().reshape((7,) + U.shape[1:])
    assert nf == int(np.sum(~ref["ok"])) and nf >= len(set(nodes)) - 1
    assert np.all(np.isfinite(P))
    np.testing.assert_allclose(P[4], ref["eps"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(P[0], ref["rho"], rtol=1e-12)
    ctx.step(1e-4, 1)
    after = np.empty(U.size)
    ctx.get_state(after, False)
    assert np.all(np.isfinite(after))
    ctx.close()
