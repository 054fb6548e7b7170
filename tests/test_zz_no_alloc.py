"""grmhd_cfl_dt_noalloc: the CFL time step for callers that cannot allocate device
memory (hosts that own all device memory through their own allocator, latency-bound
loops that cannot afford an allocation's device synchronisation).  It must give the
same dt as the context-based grmhd_cfl_dt, on two calls in a row (the second call
reuses the library's fixed scratch array and must not depend on what the first left
there), and reject inputs beyond its fixed maximum size."""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _hmin(r, th, n_r, n_theta, n_phi, n_elem):
    """Smallest node spacing min(dr, r dtheta, r sin(theta) dphi), the nearer neighbour
    gap along each direction (one-sided at the ends)."""
    def gaps(x):
        d = np.diff(x)
        out = np.empty_like(x)
        out[0], out[-1] = d[0], d[-1]
        out[1:-1] = np.minimum(d[:-1], d[1:])
        return out
    rr = r.reshape(n_elem, n_r, n_theta, n_phi)[:, :, 0, 0]
    tt = th.reshape(n_elem, n_r, n_theta, n_phi)[0, 0, :, 0]
    dr = np.stack([gaps(rr[e]) for e in range(n_elem)])[:, :, None]
    dth = gaps(tt)[None, None, :]
    R = rr[:, :, None]
    h = np.minimum(np.minimum(np.broadcast_to(dr, R.shape[:2] + (n_theta,)), R * dth),
                   R * np.sin(tt)[None, None, :] * (2 * np.pi / n_phi))
    return float(h.min())


def test_cfl_noalloc_matches_context_call():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_18221_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2508_18221_gb300 import _build
        _build.build()
    lib = pkg.load()
    from workloads import config, primitive_profiles

    cfg = config("c2", n_elem=3, n_r=16, n_theta=24, n_phi=32)
    grid, phys, opts = pkg.make_structs(cfg)
    ctx = pkg.Context(grid, phys, opts, 0)
    r, t, ph = ctx.coords()
    shp = cfg.shape
    pr = primitive_profiles(cfg, r.reshape(shp), t.reshape(shp), ph.reshape(shp))
    ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    state = torch.empty(pkg.NV * ctx.n_points, dtype=torch.float64, device="cuda")
    ctx.get_state(state, True)
    dt_ref = ctx.cfl_dt()
    hmin = _hmin(r, t, cfg.n_r, cfg.n_theta, cfg.n_phi, cfg.n_elem)
    outs = [torch.full((1,), -1.0, dtype=torch.float64, device="cuda") for _ in range(3)]
    # a warm-up call (the first call on a device looks up the scratch array's address and
    # may load the library's device code), then the device's free memory must not move
    assert lib.grmhd_cfl_dt_noalloc(state.data_ptr(), ctx.n_points, hmin, cfg.cfl,
                                    outs[2].data_ptr(), None) == pkg.GRMHD_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    dts = []
    for call in range(2):
        st = lib.grmhd_cfl_dt_noalloc(state.data_ptr(), ctx.n_points, hmin, cfg.cfl,
                                      outs[call].data_ptr(), None)
        assert st == pkg.GRMHD_OK, (call, st)
        torch.cuda.synchronize()
        dts.append(float(outs[call].item()))
    assert torch.cuda.mem_get_info()[0] == free_before, "the entry point allocated device memory"
    for dt in dts:
        np.testing.assert_allclose(dt, dt_ref, rtol=1e-13)
    assert dts[0] == dts[1]
    # sizes beyond the fixed scratch are rejected before any device work
    assert lib.grmhd_cfl_dt_noalloc(state.data_ptr(), 16_777_217, hmin, cfg.cfl,
                                    state.data_ptr(), None) == pkg.GRMHD_EINVAL
    assert lib.grmhd_cfl_dt_noalloc(None, ctx.n_points, hmin, cfg.cfl,
                                    state.data_ptr(), None) == pkg.GRMHD_EINVAL
    ctx.close()
