"""Autotuner of the FP64 digit-slice contractions: for every (direction, nodes,
kind) class (kind: derivative or filter) of the given workloads it times the contraction with one and with two
TMEM accumulator sets on a context of that shape (grmhd_tune_contractions) and writes, per
class, the choice with the lower time summed over the shapes that use it (two sets only
when they win by 2 %) to fx_tuning.txt next to the library, which every later process
reads at its first context.

    python -m paper_2508_18221_gb300.autotune --workloads c2,c4,c5 [--out PATH]

Shapes: each single-instance workload as it is; for the batched workload every group shape
(N_r = N_theta in {8, 12, 16, 24, 32}, N_phi in {16, 32, 64}) as an 8-element instance.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="c2,c4")
    ap.add_argument("--out", default=None, help="tuning file (default: fx_tuning.txt next to the library)")
    ap.add_argument("--nfields", type=int, default=21)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2508_18221_gb300 as pkg
    from workloads import config, batch_configs, primitive_profiles

    shapes = []
    for w in a.workloads.split(","):
        if w == "c4":
            seen = set()
            for c in batch_configs(256):
                key = (c.n_r, c.n_theta, c.n_phi)
                if key not in seen:
                    seen.add(key)
                    shapes.append((f"c4 group {key}", config("c2", n_elem=8, n_r=c.n_r, n_theta=c.n_theta,
                                                               n_phi=c.n_phi)))
        else:
            shapes.append((w, config(w)))
    lib = pkg.load()
    # per class: summed ms with one and with two sets over the shapes that use it (shapes of
    # different sizes can disagree; the class takes the choice with the lower total)
    sums = {}
    stream = torch.cuda.Stream()
    for name, cfg in shapes:
        grid, phys, opts = pkg.make_structs(cfg)
        ctx = pkg.Context(grid, phys, opts, stream.cuda_stream)
        r, t, ph = ctx.coords()
        pr = primitive_profiles(cfg, r.reshape(cfg.shape), t.reshape(cfg.shape), ph.reshape(cfg.shape))
        ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
        res = ctx.tune_contractions(nfields=a.nfields, reps=a.reps)
        ns = (cfg.n_r, cfg.n_theta, cfg.n_phi)
        for (d, kind), (m1, m2, ch) in sorted(res.items()):
            key = (d, ns[d], 0 if kind == "derivative" else 1)
            t = sums.setdefault(key, [0.0, 0.0, ch != 0])
            t[0] += m1
            t[1] = t[1] + m2 if (m2 >= 0 and t[1] >= 0) else -1.0
            two = f"{m2:.4f} ms" if m2 >= 0 else "n/a"
            print(f"{name:28s} dir {d} n {ns[d]:3d} {kind:10s} one set {m1:.4f} ms, two sets {two} -> {ch}",
                  flush=True)
        ctx.close()
    # two sets only where they win by 2 % in total (the launch-to-launch spread is about 1 %)
    table = {}
    for key, (s1, s2, tc) in sums.items():
        table[key] = 0 if not tc else (2 if 0 <= s2 < 0.98 * s1 else 1)
    for key in sorted(table):
        s1, s2, _ = sums[key]
        two = f"{s2:.4f} ms" if s2 >= 0 else "n/a"
        print(f"class dir {key[0]} n {key[1]:3d} kind {key[2]}: one set {s1:.4f} ms, two sets {two} in total "
              f"-> {table[key]}", flush=True)
    out = a.out or os.path.join(os.path.dirname(pkg.LIB_PATH), "fx_tuning.txt")
    with open(out, "w") as fh:
        fh.write("# digit-slice contraction tuning: direction nodes kind(0 derivative, 1 filter) sets "
                 "(python -m paper_2508_18221_gb300.autotune)\n")
        for (d, n, kind), ch in sorted(table.items()):
            fh.write(f"{d} {n} {kind} {ch}\n")
    print(f"wrote {out} ({len(table)} classes)")
    assert lib is not None


if __name__ == "__main__":
    main()
