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
    tp.assert_parity(R0, Rref, "rhs before the timed-out wait", U=U, g=g)
    tp.assert_parity(R1, Rref, "rhs after the timed-out wait", U=U, g=g)
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
    tp.assert_parity(got.reshape(U.shape), ref.reshape(U.shape), "resumed run", tol=1e-11, U=U)
