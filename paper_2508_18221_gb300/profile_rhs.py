"""Profiling driver: build a workload through the library and run a bounded number of
right-hand-side evaluations or time steps (for ncu captures and quick timings).

    python -m paper_2508_18221_gb300.profile_rhs --config c2 --rhs 1
    python -m paper_2508_18221_gb300.profile_rhs --config c2 --steps 2 --time
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--rhs", type=int, default=1, help="RHS evaluations")
    ap.add_argument("--steps", type=int, default=0, help="RK steps (one graph)")
    ap.add_argument("--time", action="store_true", help="print per-kernel CUDA-event times")
    ap.add_argument("--precision", type=int, default=0, help="0 FP64, 1 split BF16 x3, 2 TF32")
    ap.add_argument("--coupling", type=int, default=0, help="0 unsplit, 1 split (fluid RK, BSSN Euler)")
    ap.add_argument("--integrator", type=int, default=0, help="0 SSP-RK3, 1 RK4")
    ap.add_argument("--dt-scale", type=float, default=1.0, help="time step as a fraction of the CFL step")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2508_18221_gb300 as pkg
    from workloads import config, primitive_profiles

    cfg = config(a.config)
    grid, phys, opts = pkg.make_structs(cfg, precision=a.precision, coupling=a.coupling,
                                        integrator=a.integrator)
    stream = torch.cuda.Stream()
    ctx = pkg.Context(grid, phys, opts, stream.cuda_stream)
    r, t, ph = ctx.coords()
    shp = cfg.shape
    pr = primitive_profiles(cfg, r.reshape(shp), t.reshape(shp), ph.reshape(shp))
    ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    out = torch.empty(pkg.NV * ctx.n_points, dtype=torch.float64, device="cuda")
    for _ in range(a.rhs):
        ctx.rhs(out, True)
    if a.steps:
        dt = ctx.cfl_dt() * a.dt_scale
        ctx.step(dt, a.steps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(dt, a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"{a.steps} steps: {ms:.3f} ms -> {3 * a.steps * ctx.n_points / ms * 1e3:.4e} "
              f"point-updates/s")
    torch.cuda.synchronize()
    if a.time:
        for k, (ms, fl, by) in ctx.kernel_times(reps=5).items():
            tf = fl / (ms * 1e-3) / 1e12 if fl else 0.0
            gb = by / (ms * 1e-3) / 1e9 if by else 0.0
            print(f"{k:14s} {ms:8.4f} ms  {tf:8.3f} TFLOP/s  {gb:8.1f} GB/s")
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
