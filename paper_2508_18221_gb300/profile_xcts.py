"""Timing driver of the approximate XCTS initial-data solve (grmhd_xcts_init): set-up
(real Schur forms of the angular operators + inverses of the radial systems) and time per fixed-point
iteration.

    python -m paper_2508_18221_gb300.profile_xcts --config x2 --iters 12
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="x2")
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--tol", type=float, default=0.0)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2508_18221_gb300 as pkg
    from workloads import config, primitive_profiles

    cfg = config(a.config)
    grid, phys, opts = pkg.make_structs(cfg)
    stream = torch.cuda.Stream()
    ctx = pkg.Context(grid, phys, opts, stream.cuda_stream)
    r, t, ph = ctx.coords()
    shp = cfg.shape
    pr = primitive_profiles(cfg, r.reshape(shp), t.reshape(shp), ph.reshape(shp))
    psi, ch, st = ctx.xcts_init(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"],
                                iters=a.iters, tol=a.tol)
    n = cfg.n_elem * cfg.n_r * cfg.n_theta
    print(f"{a.config}: {ctx.n_points} nodes, {cfg.n_phi // 2 + 1} phi modes of {n} unknowns")
    print(f"set-up {st[0]:.1f} ms, {st[1]:.3f} ms per iteration, {int(st[2])} iterations, "
          f"last change {ch[-1]:.3e}, psi in [{psi.min():.6f}, {psi.max():.6f}]")
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
