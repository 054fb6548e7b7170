"""Batched instances (grmhd_batch_*): instances with the same node counts are advanced
as one group, concatenated along r.  Every instance of a batch must evolve exactly as
the same instance alone (the per-node arithmetic is the same), and match the oracle."""
import numpy as np
import pytest

from oracle import solver as so
from workloads import config

from test_gpu_parity import assert_parity, pkg  # noqa: F401

pytestmark = pytest.mark.gpu


def _instances():
    # two shape groups; spins, element counts and radial ranges differ inside a group
    return [config("c1", a=0.3, n_elem=2, r_min=1.9, r_max=12.0, n_r=8, n_theta=8, n_phi=8),
            config("c1", a=0.8, n_elem=3, r_min=1.5, r_max=30.0, n_r=8, n_theta=8, n_phi=8),
            config("c1", a=0.6, n_elem=1, r_min=1.7, r_max=8.0, n_r=9, n_theta=6, n_phi=4),
            config("c1", a=0.1, n_elem=2, r_min=2.0, r_max=20.0, n_r=8, n_theta=8, n_phi=8),
            config("c1", a=0.95, n_elem=2, r_min=1.2, r_max=10.0, n_r=9, n_theta=6, n_phi=4)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_instances(pkg, precision):
    import torch
    cfgs = _instances()
    structs = [pkg.make_structs(c, precision=precision) for c in cfgs]
    batch = pkg.Batch(structs)
    assert batch.num_groups() == 2
    states, dts = [], []
    for i, c in enumerate(cfgs):
        g, p, U = so.workload_state(c)
        assert batch.num_points(i) == U[0].size
        r, t, ph = batch.coords(i)
        np.testing.assert_allclose(r.reshape(g.shape), g.R, rtol=1e-15)
        batch.set_state(i, U.reshape(-1).copy(), False)
        states.append(U)
        dts.append(1e-3 * (1 + 0.1 * i))
    batch.step(dts, 3)
    for i, c in enumerate(cfgs):
        got = np.empty(states[i].size)
        batch.get_state(i, got, False)
        grid, phys, opts = structs[i]
        ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
        ctx.set_state(torch.from_numpy(states[i].reshape(-1).copy()).cuda(), True)
        ctx.step(dts[i], 3)
        ref = np.empty(states[i].size)
        ctx.get_state(ref, False)
        ctx.close()
        np.testing.assert_array_equal(got, ref)
    batch.close()


def test_batch_instance_matches_oracle(pkg):
    cfgs = _instances()
    batch = pkg.Batch([pkg.make_structs(c) for c in cfgs])
    i = 1
    g, p, U = so.workload_state(cfgs[i])
    for k, c in enumerate(cfgs):
        _, _, Uk = so.workload_state(c)
        batch.set_state(k, Uk.reshape(-1).copy(), False)
    dt = 1e-3
    batch.step([dt] * len(cfgs), 2)
    got = np.empty(U.size)
    batch.get_state(i, got, False)
    two = lambda X: so.rk_step(so.rk_step(X, dt, g, p), dt, g, p)  # noqa: E731
    assert_parity(got.reshape(U.shape), two(U), "batch instance 2 steps", two, U, trials=2)
    batch.close()


def test_batch_init_prims(pkg):
    from workloads import primitive_profiles
    cfgs = _instances()
    batch = pkg.Batch([pkg.make_structs(c) for c in cfgs])
    for i, c in enumerate(cfgs):
        r, t, ph = batch.coords(i)
        pr = primitive_profiles(c, r.reshape(c.shape), t.reshape(c.shape), ph.reshape(c.shape))
        batch.init_prims(i, pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    for i, c in enumerate(cfgs):
        g, p, U = so.workload_state(c)
        got = np.empty(U.size)
        batch.get_state(i, got, False)
        got = got.reshape(U.shape)
        for v in range(32):
            sc = np.abs(U[v]).max()
            assert np.abs(got[v] - U[v]).max() <= 1e-12 * max(sc, np.abs(U[:24]).max() if v < 24 else sc)
    batch.close()
