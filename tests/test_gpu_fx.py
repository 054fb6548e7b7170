"""FP64 spectral contractions on the GPU, both kinds: digit-sliced tensor-core products
(contraction = 0) and FP64 units (contraction = 1), against the oracle's derivative
operators (coefficient route, numpy FP64).

An FP64 dot product sum_j D_ij u_j is exact to a few units of 2^-53 of
b_i = sum_j |D_ij| max_j |u_j|; both kinds must stay within 2e-14 b_i of the oracle (the
oracle's own coefficient route and the library's barycentric matrices differ by about
1e-15 b_i).  Lines of very different magnitude (1e-100 .. 1e100) check that every line
is scaled by its own exponent; a NaN must spread over its line only; zero stays zero.
"""
import json
import os

import numpy as np
import pytest

from oracle import solver as so
from workloads import config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_18221_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2508_18221_gb300 import _build
        _build.build()
    pkg.load()
    return pkg


def _setup(pkg, cfg, contraction):
    import torch
    g = so.Grid(so.Params.from_config(cfg))
    grid, phys, opts = pkg.make_structs(cfg, contraction=contraction)
    ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
    return g, ctx


def _abs_ops(g):
    """|D| per direction from the oracle operators applied to unit vectors."""
    E, Nr, Nt, Np = g.shape
    out = []
    for d, (op, n, ax) in enumerate(((g.d_r, Nr, 1), (g.d_t, Nt, 2), (g.d_p, Np, 3))):
        cols = []
        for j in range(n):
            u = np.zeros(g.shape)
            idx = [slice(None)] * 4
            idx[ax] = j
            u[tuple(idx)] = 1.0
            cols.append(op(u))
        out.append(np.abs(np.stack(cols, axis=-1)))   # (..., j) along the last axis
    return out


def _bound(g, absD, u, d):
    """b = sum_j |D_ij| max_j |u_j| on every node for direction d."""
    ax = d + 1
    m = np.max(np.abs(u), axis=ax, keepdims=True)
    return np.sum(absD[d], axis=-1) * m


def _run(pkg, ctx, u, d):
    import torch
    src = torch.from_numpy(u.reshape(-1).copy()).cuda()
    dst = torch.zeros_like(src)
    ctx.debug_deriv(src, dst, 1, d)
    return dst.cpu().numpy().reshape(u.shape)


def _report(name, value):
    """measured errors go to fx_accuracy.json in the folder GRMHD_REPORT_DIR names, when set"""
    out = os.environ.get("GRMHD_REPORT_DIR")
    if not out or not os.path.isdir(out):
        return
    fn = os.path.join(out, "fx_accuracy.json")
    data = json.load(open(fn)) if os.path.exists(fn) else {}
    data[name] = value
    with open(fn, "w") as fh:
        json.dump(data, fh, indent=1)


@pytest.mark.parametrize("contraction", [0, 1])
def test_contraction_accuracy(pkg, contraction):
    cfg = config("c1", n_elem=3, n_r=10, n_theta=9, n_phi=8)
    g, ctx = _setup(pkg, cfg, contraction)
    absD = _abs_ops(g)
    rng = np.random.default_rng(11)
    ops = (g.d_r, g.d_t, g.d_p)
    worst = []
    for d in range(3):
        # values spanning 12 decades inside every line, line magnitudes 1e-100 .. 1e100
        u = rng.normal(size=g.shape) * 10.0 ** rng.uniform(-6, 6, size=g.shape)
        line_shape = list(g.shape)
        line_shape[d + 1] = 1
        u = u * 10.0 ** rng.integers(-100, 100, size=line_shape)
        got = _run(pkg, ctx, u, d)
        ref = ops[d](u)
        b = _bound(g, absD, u, d)
        err = np.abs(got - ref) / b
        assert np.all(np.isfinite(got))
        worst.append(float(err.max()))
        assert err.max() <= 2e-14, (d, float(err.max()))
    _report(f"accuracy_contraction{contraction}", worst)
    ctx.close()


@pytest.mark.parametrize("contraction", [0, 1])
def test_contraction_nan_and_zero(pkg, contraction):
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, ctx = _setup(pkg, cfg, contraction)
    rng = np.random.default_rng(5)
    for d in range(3):
        u = rng.normal(size=g.shape)
        u[1, 3, 4, 5] = np.nan
        got = _run(pkg, ctx, u, d)
        line = [1, 3, 4, 5]
        line[d + 1] = slice(None)
        bad = np.zeros(g.shape, dtype=bool)
        bad[tuple(line)] = True
        assert np.all(np.isnan(got[bad])), d
        assert np.all(np.isfinite(got[~bad])), d
        z = _run(pkg, ctx, np.zeros(g.shape), d)
        assert np.all(z == 0.0), d
    ctx.close()


@pytest.mark.parametrize("contraction", [0, 1])
def test_contraction_sizes(pkg, contraction):
    """Every size class of the tensor-core kernel (output width 16..64 in one pass, 128 in
    two passes of 64 columns) on smooth data, beside the FP64-unit kind.  The bar, 3e-14
    of the bound, is about twice the worst-case bound K 2^-53 of an FP64 dot product of
    length K = 128 (the oracle's own coefficient route is part of the difference)."""
    worst = {}
    for nr, nt, nph in ((4, 5, 4), (16, 17, 16), (24, 33, 34), (40, 48, 64), (64, 20, 48),
                        (8, 72, 8), (8, 100, 8), (8, 8, 96), (8, 8, 128)):
        cfg = config("c1", n_elem=2, n_r=nr, n_theta=nt, n_phi=nph)
        g, ctx = _setup(pkg, cfg, contraction)
        absD = _abs_ops(g)
        ops = (g.d_r, g.d_t, g.d_p)
        u = np.sin(g.R) * np.cos(2 * g.T) * (1.5 + np.sin(3 * g.P)) + 0.1 * g.R
        for d in range(3):
            got = _run(pkg, ctx, u, d)
            err = np.abs(got - ops[d](u)) / _bound(g, absD, u, d)
            worst[f"{(nr, nt, nph)[d]} nodes dir {d}"] = float(err.max())
            assert err.max() <= 3e-14, ((nr, nt, nph), d, float(err.max()))
        ctx.close()
    _report(f"sizes_contraction{contraction}", worst)


@pytest.mark.parametrize("contraction", [0, 1])
def test_contraction_maximum_sizes(pkg, contraction):
    """The largest node counts the library accepts per direction (n_r = 64, n_theta = 128,
    n_phi = 128) and ragged lengths below them, on thin grids, through the test hook
    (the digit-slice kernel whenever it supports the size).  Bar: 2 K 2^-53 of the bound
    (the worst-case rounding of an FP64 dot product of length K), at least 3e-14."""
    worst = {}
    for nr, nt, nph in ((64, 4, 4), (63, 4, 4), (4, 128, 4), (4, 127, 4), (4, 4, 128), (4, 4, 126)):
        cfg = config("c1", n_elem=2, n_r=nr, n_theta=nt, n_phi=nph)
        g, ctx = _setup(pkg, cfg, contraction)
        absD = _abs_ops(g)
        ops = (g.d_r, g.d_t, g.d_p)
        u = np.sin(g.R) * np.cos(2 * g.T) * (1.5 + np.sin(3 * g.P)) + 0.1 * g.R
        for d in range(3):
            k = (nr, nt, nph)[d]
            got = _run(pkg, ctx, u, d)
            err = np.abs(got - ops[d](u)) / _bound(g, absD, u, d)
            worst[f"{k} nodes dir {d}"] = float(err.max())
            assert err.max() <= max(3e-14, 2 * k * 2.0 ** -53), ((nr, nt, nph), d, float(err.max()))
        ctx.close()
    _report(f"maximum_sizes_contraction{contraction}", worst)


def test_maximum_sizes_rhs_and_limits(pkg):
    """Right-hand sides at the largest node counts (thin grids the oracle evaluates in
    seconds) with the default contraction choice against the oracle at the FP64 bar: 64
    radial and 64 Chebyshev theta nodes (digit slices, seven exact accumulators), 128
    Chebyshev theta nodes (FP64 units: measured 9.3e-12 of the bar's normalisation, which
    follows first-derivative rounding, max|U| / dx_min, while Chebyshev second derivatives
    round with the square of the operator norm), 128 Fourier theta and 128 phi nodes
    (digit slices).  Limits: n_phi above 128 or odd, n_theta above 128,
    n_r above 64 are invalid."""
    import torch

    import test_gpu_parity as tp
    for kw in (dict(n_elem=1, n_r=64, n_theta=4, n_phi=4), dict(n_elem=2, n_r=4, n_theta=64, n_phi=4),
               dict(n_elem=2, n_r=4, n_theta=128, n_phi=4),
               dict(n_elem=2, n_r=4, n_theta=128, n_phi=4, theta_min=0.0, theta_max=np.pi, theta_basis=1),
               dict(n_elem=1, n_r=5, n_theta=5, n_phi=128)):
        cfg = config("c1", **kw)
        g, p, U = so.workload_state(cfg)
        ctx = tp._ctx(pkg, cfg)
        R = tp._gpu_rhs(pkg, ctx, U)
        ctx.close()
        tp.assert_parity(R, so.rhs(U, g, p), f"rhs {kw}", lambda X: so.rhs(X, g, p), U, trials=2)
    stream = torch.cuda.current_stream().cuda_stream
    for kw in (dict(n_phi=130), dict(n_phi=256), dict(n_phi=6, n_theta=129), dict(n_r=65), dict(n_phi=7)):
        grid, phys, opts = pkg.make_structs(config("c1", n_elem=1, **kw))
        with pytest.raises(pkg.GrmhdError):
            pkg.Context(grid, phys, opts, stream)


def test_exact_accumulators_reach_fp64_accuracy(pkg):
    """Every digit-order sum has an exact accumulator of its own, so the error is that of
    the dropped digit pairs and the final roundings and stays within a few times the FP64
    units' (an earlier form that folded the sums 6..8 into one rounding accumulator measured
    7.5e-15 and 1.4e-14 of the bound at 64 and 128 nodes), bar 2e-15 of the bound, in
    every direction; the phi lines carry a large constant plus small noise, the case
    where a rounding accumulator's error showed in the right-hand side."""
    worst = {}
    for nr, nt, nph, d in ((24, 4, 4, 0), (32, 4, 4, 0), (40, 4, 4, 0), (64, 4, 4, 0), (4, 32, 4, 1),
                           (4, 48, 4, 1), (4, 128, 4, 1), (4, 4, 64, 2), (4, 4, 128, 2)):
        cfg = config("c1", n_elem=2, n_r=nr, n_theta=nt, n_phi=nph)
        g, ctx = _setup(pkg, cfg, 0)
        absD = _abs_ops(g)
        u = np.sin(g.R) * np.cos(2 * g.T) * (1.5 + np.sin(3 * g.P)) + 0.1 * g.R
        if d == 2:
            rng = np.random.default_rng(nph)
            u = g.R ** 2 * (1.0 + 1e-3 * rng.uniform(-1, 1, g.shape))
        got = _run(pkg, ctx, u, d)
        ctx.close()
        err = np.abs(got - (g.d_r, g.d_t, g.d_p)[d](u)) / _bound(g, absD, u, d)
        worst[f"{(nr, nt, nph)[d]} nodes dir {d}"] = float(err.max())
        assert err.max() <= 2e-15, ((nr, nt, nph), d, float(err.max()))
    _report("exact_accumulators", worst)


@pytest.mark.parametrize("nr,nt,nph", [(24, 32, 64), (8, 12, 16), (32, 32, 32)])
def test_two_accumulator_sets_are_bitwise_equal(pkg, nr, nt, nph):
    """One or two TMEM accumulator sets (the tuning choice) change the schedule, not the
    arithmetic: derivative contractions in every direction give bitwise equal results,
    and an element change of the radial operator under two sets (the operator reload waits
    for the previous tile's MMAs) is covered by the multi-element grid."""
    import torch
    lib = pkg.load()
    cfg = config("c1", n_elem=3, n_r=nr, n_theta=nt, n_phi=nph)
    g, ctx = _setup(pkg, cfg, 0)
    rng = np.random.default_rng(nr + nt + nph)
    u = rng.normal(size=(4,) + g.shape) * 10.0 ** rng.uniform(-3, 3, size=(4, 1, 1, 1, 1))
    src = torch.from_numpy(u.reshape(-1).copy()).cuda()
    ns = (nr, nt, nph)
    try:
        for d in range(3):
            outs = []
            for ts in (1, 2):
                assert lib.grmhd_tune_set(d, ns[d], 0, ts) == pkg.GRMHD_OK
                dst = torch.zeros_like(src)
                ctx.debug_deriv(src, dst, 4, d)
                outs.append(dst.cpu().numpy())
            np.testing.assert_array_equal(outs[0], outs[1])
    finally:
        for d in range(3):
            lib.grmhd_tune_set(d, ns[d], 0, 0)
        ctx.close()
