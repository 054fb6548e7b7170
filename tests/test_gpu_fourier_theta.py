"""The paper's Fourier theta basis on the GPU (grid.theta_basis = 1) against the oracle.

The theta contractions fold the phi pairs (l, l + N_phi/2) into half sums and differences,
contract each half with the even or odd operator of the double-Fourier extension and
unfold; the checks compare them with the oracle's explicit extension + DFT derivative
(per field parity, every contraction kind, sizes that take the digit-slice kernel, the
reflection-split kernel and the dense kernel), then the whole right-hand side, two time
steps, the CFL step, the diagnostics and the initial data at the FP64 bar 1e-11 (mixed
precision at its bar 2e-6).
"""
import numpy as np
import pytest

from oracle import solver as so
from oracle import spectral as sp
from workloads import config

from oracle import rounding as fpf
import test_gpu_parity as tp
from test_gpu_parity import pkg  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _fcfg(**kw):
    base = dict(theta_min=0.0, theta_max=np.pi, theta_basis=1)
    base.update(kw)
    return config("c1", **base)


def _state(cfg, **kw):
    return so.workload_state(cfg, **kw)


def _row_abs_sum(n):
    """sum_k |c_k| of the 2n-node periodic derivative row (operator norm bound)."""
    m = np.arange(1, 2 * n)
    return np.sum(np.abs(0.5 / np.tan(m * np.pi / (2 * n))))


def _filter_row_abs_sum(n):
    """sum_k |f_k| of the 2n-node periodic filter row (the filter of a unit impulse)."""
    e0 = np.zeros(2 * n)
    e0[0] = 1.0
    return np.abs(sp.fourier_filter(e0, axis=0, dealias23=True)).sum()


@pytest.mark.parametrize("contraction", [0, 1])
def test_theta_derivative_and_filter_operators(pkg, contraction):  # noqa: F811
    """Random fields of both parities.  Sizes: folded halves with an even number of lines
    (digit-slice kernel) and an odd one (reflection-split / dense kernels), theta orders with
    and without a compiled reflection-split instance, up to 128 nodes.  Bar: 4e-14 of
    sum_j |operator row| max |u|, a few times the worst-case rounding of an FP64 dot
    product of 2 N_theta terms (the oracle's DFT route differs from the matrix route by
    about 5e-15 of that bound)."""
    import torch
    from test_gpu_fx import _report
    rng = np.random.default_rng(21)
    worst = {}
    for nt, nph in ((12, 16), (9, 12), (16, 10), (32, 64), (33, 8), (64, 4), (100, 8), (128, 4)):
        cfg = _fcfg(n_elem=2, n_r=5, n_theta=nt, n_phi=nph)
        g = so.Grid(so.Params.from_config(cfg))
        grid, phys, opts = pkg.make_structs(cfg, contraction=contraction)
        ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
        par = [1, -1, -1, 1]
        u = rng.normal(size=(4,) + g.shape) * 10.0 ** rng.uniform(-3, 3, size=(4, 1, 1, 1, 1))
        src = torch.from_numpy(u.reshape(-1).copy()).cuda()
        dst = torch.empty_like(src)
        for filt in (False, True):
            ctx.debug_theta(src, dst, par, filter=filt)
            got = dst.cpu().numpy().reshape(u.shape)
            for f, s in enumerate(par):
                if filt:
                    ref = sp.fourier_theta_filter(u[f], 2, 3, s, dealias23=True)
                    bound = _filter_row_abs_sum(nt) * np.abs(u[f]).max()
                else:
                    ref = sp.fourier_theta_deriv(u[f], 2, 3, s)
                    bound = _row_abs_sum(nt) * np.abs(u[f]).max()
                err = np.abs(got[f] - ref).max() / bound
                worst[f"{nt}x{nph} {'filter' if filt else 'derivative'}"] = max(
                    worst.get(f"{nt}x{nph} {'filter' if filt else 'derivative'}", 0.0), float(err))
                assert err <= 4e-14, (nt, nph, filt, f, err)
        ctx.close()
    _report(f"fourier_theta_contraction{contraction}", worst)


RHS_CASES = [
    ({}, 1e-11),
    ({"contraction": 1}, 1e-11),
    ({"evolve_metric": 0}, 1e-11),
    ({"precision": 1}, 2e-6),
]


@pytest.mark.parametrize("kw,tol", RHS_CASES)
def test_fourier_theta_rhs_parity(pkg, kw, tol):  # noqa: F811
    cfg = _fcfg(n_elem=2, n_r=10, n_theta=12, n_phi=16)
    okw = {k: v for k, v in kw.items() if k in ("evolve_metric",)}
    g, p, U = _state(cfg, **okw)
    ctx = tp._ctx(pkg, cfg, **kw)
    R = tp._gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    worst, _ = tp.assert_parity(R, Rref, f"fourier theta rhs {kw}", lambda X: so.rhs(X, g, p), U, tol=tol,
                                eps=fpf.EPS32 if kw.get("precision") else fpf.EPS64,
                                kappa=1.0 if kw.get("precision") else fpf.KAPPA)
    if kw.get("precision"):
        assert worst > 1e-12          # the tensor-core path really ran
    ctx.close()


def test_fourier_theta_rhs_parity_ragged(pkg):  # noqa: F811
    """Odd theta order, folded halves of odd width, three elements."""
    cfg = _fcfg(n_elem=3, n_r=7, n_theta=11, n_phi=6)
    g, p, U = _state(cfg)
    ctx = tp._ctx(pkg, cfg)
    R = tp._gpu_rhs(pkg, ctx, U)
    tp.assert_parity(R, so.rhs(U, g, p), "fourier theta rhs ragged", lambda X: so.rhs(X, g, p), U)
    ctx.close()


def test_fourier_theta_glm_rhs_parity(pkg):  # noqa: F811
    cfg = _fcfg(n_elem=2, n_r=8, n_theta=10, n_phi=8)
    g, p, U = _state(cfg, glm=1)
    U[so.I_PSI] = 1e-4 * np.cos(g.T) * np.cos(g.P) * (g.R / g.R.max())
    U[so.I_B] = U[so.I_B] * (1.0 + 0.05 * np.cos(2.0 * g.P))
    ctx = tp._ctx(pkg, cfg, glm=1)
    R = tp._gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    assert np.abs(Rref[so.I_PSI]).max() > 0
    tp.assert_parity(R, Rref, "fourier theta glm rhs", lambda X: so.rhs(X, g, p), U)
    ctx.close()


@pytest.mark.parametrize("filt", [47, 63])
def test_fourier_theta_step_parity(pkg, filt):  # noqa: F811
    """Two SSP-RK3 steps with the post-step filter (63 also filters BSSN in theta)."""
    import torch
    cfg = _fcfg(n_elem=3, n_r=8, n_theta=10, n_phi=8)
    g, p, U = _state(cfg, filter_mask=filt)
    ctx = tp._ctx(pkg, cfg, filter=filt)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    dt = 5e-4
    ctx.step(dt, 2)
    got = np.empty(U.size)
    ctx.get_state(got, False)
    two = lambda X: so.rk_step(so.rk_step(X, dt, g, p), dt, g, p)  # noqa: E731
    tp.assert_parity(got.reshape(U.shape), two(U), f"fourier theta 2 steps filter {filt}", two, U, trials=2)
    ctx.close()


def test_fourier_theta_init_cfl_diag(pkg):  # noqa: F811
    import torch
    from workloads import primitive_profiles
    cfg = _fcfg(n_elem=2, n_r=8, n_theta=12, n_phi=8)
    g, p, U = _state(cfg)
    ctx = tp._ctx(pkg, cfg)
    r, t, ph = ctx.coords()
    np.testing.assert_allclose(t.reshape(g.shape), g.T, rtol=1e-15)
    pr = primitive_profiles(cfg, r.reshape(g.shape), t.reshape(g.shape), ph.reshape(g.shape))
    ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    got = np.empty(U.size)
    ctx.get_state(got, False)
    got = got.reshape(U.shape)
    for v in range(32):
        sc = max(np.abs(U[w]).max() for w in tp.TENSOR_OF[v])
        assert np.abs(got[v] - U[v]).max() <= 1e-12 * sc, v
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    np.testing.assert_allclose(ctx.cfl_dt(), so.cfl_dt(U, g, p), rtol=1e-13)
    dg = ctx.diag()
    ref = so.diagnostics(U, g, p)
    np.testing.assert_allclose(dg[0], ref[0], rtol=1e-13)
    np.testing.assert_allclose(dg[1], ref[1], rtol=1e-12)
    assert ref[4] > 0
    np.testing.assert_allclose(dg[5], ref[4], rtol=1e-9)
    np.testing.assert_allclose(dg[6], ref[5], rtol=1e-9)
    ctx.close()


def test_fourier_theta_invalid_range(pkg):  # noqa: F811
    import torch
    cfg = config("c1", theta_basis=1)          # polar band: not a whole sphere
    grid, phys, opts = pkg.make_structs(cfg)
    with pytest.raises(pkg.GrmhdError, match="-1"):
        pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)


def test_fourier_theta_batch_equals_single_instances(pkg):  # noqa: F811
    """Fourier theta instances in a batch (two shape groups, next to a Chebyshev-theta
    instance, which forms its own group) evolve bit for bit as alone."""
    import torch
    cfgs = [_fcfg(a=0.3, n_elem=2, r_min=1.9, r_max=12.0, n_r=8, n_theta=8, n_phi=8),
            _fcfg(a=0.8, n_elem=3, r_min=1.5, r_max=30.0, n_r=8, n_theta=8, n_phi=8),
            _fcfg(a=0.6, n_elem=1, r_min=1.7, r_max=8.0, n_r=9, n_theta=6, n_phi=4),
            config("c1", a=0.5, n_elem=2, n_r=8, n_theta=8, n_phi=8)]
    structs = [pkg.make_structs(c) for c in cfgs]
    batch = pkg.Batch(structs)
    assert batch.num_groups() == 3
    states, dts = [], []
    for i, c in enumerate(cfgs):
        g, p, U = so.workload_state(c)
        batch.set_state(i, U.reshape(-1).copy(), False)
        states.append(U)
        dts.append(5e-4 * (1 + 0.1 * i))
    batch.step(dts, 2)
    for i in range(len(cfgs)):
        got = np.empty(states[i].size)
        batch.get_state(i, got, False)
        grid, phys, opts = structs[i]
        ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
        ctx.set_state(torch.from_numpy(states[i].reshape(-1).copy()).cuda(), True)
        ctx.step(dts[i], 2)
        ref = np.empty(states[i].size)
        ctx.get_state(ref, False)
        ctx.close()
        np.testing.assert_array_equal(got, ref)
    batch.close()


def test_fourier_theta_glm_mixed_rhs(pkg):  # noqa: F811
    """GLM cleaning with split-BF16 x3 contractions on the Fourier theta basis: the mixed
    bar 2e-6."""
    cfg = _fcfg(n_elem=2, n_r=8, n_theta=10, n_phi=8)
    g, p, U = _state(cfg, glm=1)
    U[so.I_PSI] = 1e-4 * np.cos(g.T) * np.cos(g.P) * (g.R / g.R.max())
    ctx = tp._ctx(pkg, cfg, glm=1, precision=1)
    R = tp._gpu_rhs(pkg, ctx, U)
    tp.assert_parity(R, so.rhs(U, g, p), "fourier theta glm mixed rhs", lambda X: so.rhs(X, g, p), U,
                     tol=2e-6, eps=fpf.EPS32, kappa=1.0)
    ctx.close()


def test_fourier_theta_split_coupling_rk4(pkg):  # noqa: F811
    """The paper's split loop with RK4 on the Fourier theta basis, two steps."""
    import torch
    cfg = _fcfg(n_elem=2, n_r=8, n_theta=10, n_phi=8)
    g, p, U = _state(cfg, integrator=1, coupling=1)
    ctx = tp._ctx(pkg, cfg, integrator=1, coupling=1)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    dt = 5e-4
    ctx.step(dt, 2)
    got = np.empty(U.size)
    ctx.get_state(got, False)
    two = lambda X: so.rk_step(so.rk_step(X, dt, g, p), dt, g, p)  # noqa: E731
    tp.assert_parity(got.reshape(U.shape), two(U), "fourier theta split rk4", two, U, trials=2)
    ctx.close()


@pytest.mark.slow
def test_fourier_theta_rhs_parity_full_size(pkg):  # noqa: F811
    """The benchmarked Fourier theta instance (393,216 nodes) in the benchmark's launch
    configuration: every node of one RHS evaluation against the oracle."""
    cfg = config("c2f")
    g, p, U = _state(cfg)
    ctx = tp._ctx(pkg, cfg)
    R = tp._gpu_rhs(pkg, ctx, U)
    tp.assert_parity(R, so.rhs(U, g, p), "fourier theta rhs c2f full size", lambda X: so.rhs(X, g, p), U,
                     trials=2)
    ctx.close()
