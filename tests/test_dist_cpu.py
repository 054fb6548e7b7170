"""The multi-rank host logic of the benchmark on CPU: two gloo ranks (world_size 2).

Every rank advances its own batch of independent instances (disjoint seeds, the same
sizes), times its region, and the job's figures are the slowest rank's time and all ranks'
units.  No GPU: the collective runs on the gloo backend over 127.0.0.1.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cfgs = bench.rank_batch(8, rank)
    ms_local = 100.0 + 50.0 * rank                       # rank 1 is the slow one
    units_local = sum(c.n_points for c in cfgs) * 3
    ms, units, value = bench.combine(ms_local, units_local, world)
    out.put((rank, [c.seed for c in cfgs], units_local, ms, units, value))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_all_units():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seeds0, u0, ms0, tot0, v0), (r1, seeds1, u1, ms1, tot1, v1) = res
    assert not set(seeds0) & set(seeds1)                 # disjoint instances
    assert ms0 == ms1 == 150.0                           # the slowest rank's time
    assert tot0 == tot1 == float(u0 + u1)                # every rank's units
    assert abs(v0 - (u0 + u1) / 0.150) < 1e-6 * v0
    assert torch is not None


def test_single_rank_combine_is_local():
    import bench
    ms, units, value = bench.combine(200.0, 1000, 1)
    assert (ms, units) == (200.0, 1000.0) and abs(value - 5000.0) < 1e-9
    # rank 0's batch is the single-GPU batch
    from workloads import batch_configs
    assert [c.seed for c in bench.rank_batch(5, 0)] == [c.seed for c in batch_configs(5)]


def test_reference_arm_line_matches_the_benchmark_config():
    """`bench.py --impl reference` times the oracle on the host: one JSON line with the
    benchmark's own metric, unit and config (the sample it times stated in cpu_baseline),
    and an end-to-end figure with no host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, root)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.metric_name(0) and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == bench.WORKLOADS["c2"][0]
    assert d["config"]["nodes"] == 8 * 24 * 32 * 64
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
