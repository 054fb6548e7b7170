"""Approximate XCTS initial data on the GPU (grmhd_xcts_init) against the oracle.

Both sides run the same number of fixed-point iterations from the puncture 1 + M/(2r); the
oracle solves the whole 3-D boundary-value problem with one dense matrix built from its own
derivative operators, the library per phi mode through the real Schur form of its angular
operator (a back substitution over radial systems, factorised and solved in the library's
own kernels).  Bars: psi within 1e-11 of max psi (the solves' rounding: the
spectral Laplacian's condition number times 2^-53, measured ~1e-13), the state at the FP64
parity bar.
"""
import numpy as np
import pytest

from oracle import solver as so
from oracle import xcts
from workloads import config, primitive_profiles

import test_gpu_parity as tp
from test_gpu_parity import pkg  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _setup(pkg, cfg):
    import torch
    grid, phys, opts = pkg.make_structs(cfg)
    ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
    p = so.Params.from_config(cfg)
    g = so.Grid(p)
    prim = primitive_profiles(cfg, g.R, g.T, g.P)
    return ctx, g, p, prim


def _call(ctx, prim, iters, tol=0.0):
    return ctx.xcts_init(prim["rho"], prim["p"], prim["vr"], prim["vth"], prim["vph"], prim["A_phi"],
                         iters=iters, tol=tol)


def test_xcts_matches_oracle(pkg):  # noqa: F811
    cfg = config("x1")
    ctx, g, p, prim = _setup(pkg, cfg)
    psi, ch, stats = _call(ctx, prim, iters=10)
    U_ref, psi_ref, ch_ref = xcts.xcts_state(g, p, prim, iters=10)
    assert int(stats[2]) == 10
    err = np.abs(psi.reshape(g.shape) - psi_ref).max() / np.abs(psi_ref).max()
    assert err < 1e-11, err
    # the per-iteration changes follow the oracle's until both reach the rounding floor
    np.testing.assert_allclose(ch[:3], ch_ref[:3], rtol=1e-6)
    got = np.empty(U_ref.size)
    ctx.get_state(got, False)
    # floor of the slice: the oracle's solve again from the density rounded once more
    tp.assert_parity(got.reshape(U_ref.shape), U_ref, "xcts state",
                     lambda rho: xcts.xcts_state(g, p, dict(prim, rho=rho), iters=10)[0], prim["rho"],
                     trials=2)
    ctx.close()


def test_xcts_vacuum_and_early_stop(pkg):  # noqa: F811
    """Zero density: the solve returns the puncture to spectral accuracy after one
    iteration (the second changes nothing, so tol stops it)."""
    cfg = config("x1", n_elem=3, n_r=16, n_theta=8, n_phi=8)
    ctx, g, p, prim = _setup(pkg, cfg)
    prim = dict(prim, rho=np.zeros(g.shape))
    psi, ch, stats = _call(ctx, prim, iters=5, tol=1e-13)
    assert int(stats[2]) == 2 and ch[1] < 1e-13
    assert np.abs(psi.reshape(g.shape) - (1.0 + p.M / (2.0 * g.R))).max() < 1e-8
    ref, _ = xcts.solve_psi(g, p, np.zeros(g.shape), iters=1)
    assert np.abs(psi.reshape(g.shape) - ref).max() < 1e-11 * np.abs(ref).max()
    ctx.close()


def test_xcts_rhs_of_the_slice(pkg):  # noqa: F811
    """The XCTS state through the right-hand side: GPU against oracle at the FP64 bar."""
    cfg = config("x1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    ctx, g, p, prim = _setup(pkg, cfg)
    _call(ctx, prim, iters=6)
    U = np.empty(32 * g.R.size)
    ctx.get_state(U, False)
    U = U.reshape((32,) + g.shape)
    R = tp._gpu_rhs(pkg, ctx, U)
    tp.assert_parity(R, so.rhs(U, g, p), "rhs of the xcts slice", lambda X: so.rhs(X, g, p), U)
    ctx.close()


def test_xcts_errors(pkg):  # noqa: F811
    import torch
    # Chebyshev theta band: no whole sphere
    cfg = config("c1", n_elem=2, n_r=6, n_theta=6, n_phi=4)
    grid, phys, opts = pkg.make_structs(cfg)
    ctx = pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)
    z = np.zeros(ctx.n_points)
    with pytest.raises(pkg.GrmhdError, match="-6"):
        ctx.xcts_init(z, z, z, z, z, z, iters=2)
    ctx.close()
    # a dense source: the plain fixed point diverges and the call says so
    cfg = config("x1", n_elem=2, n_r=8, n_theta=6, n_phi=4, rho0=5.0)
    ctx, g, p, prim = _setup(pkg, cfg)
    with pytest.raises(pkg.GrmhdError, match="-4"):
        _call(ctx, prim, iters=60)
    ctx.close()
