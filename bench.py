"""Benchmark: coupled BSSN-Valencia RHS point-updates/s on the GB300.

Default workload (one bench step): the 8-element Kerr-Schild torus instance, spin
a = 0.9, r in [1.5, 100], N_r = 24, N_theta = 32, N_phi = 64 (393,216 nodes, 32 evolved
variables), 100 SSP-RK3 time steps at CFL 0.3 recorded in one CUDA graph, FP64.
value = nodes x RHS evaluations / second (3 RHS per step), summed over ranks.
--precision 1 / 2 runs the mixed modes (tensor-core split-BF16 x3 / TF32 derivative
contractions, FP32 algebra, FP64 state); --workload c5 the 16-element 32 x 64 x 128
instance (4,194,304 nodes, 200 steps per bench step); --workload c2f the c2 instance on
the paper's Fourier theta basis (uniform pole-free theta nodes over the sphere).

--impl reference times the FP64 numpy oracle (the project's CPU reference) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "point-updates/s"
RHS_PER_STEP = 3
PREC_NAME = {0: "FP64", 1: "mixed: split-BF16x3 tensor-core derivatives, FP32 algebra, FP64 "
                           "state/c2p/metric/RK", 2: "mixed: TF32 tensor-core derivatives, FP32 "
                                                      "algebra, FP64 state/c2p/metric/RK"}
DTYPE = {0: "f64", 1: "f64 state + bf16x3/f32 derivatives", 2: "f64 state + tf32/f32 derivatives"}
WORKLOADS = {
    "c2": ("c2: a=0.9, 8 radial elements r in [1.5,100], N_r=24, N_theta=32 Chebyshev-Gauss "
           "nodes on the polar band theta in [pi/8, 7pi/8], N_phi=64, 100 SSP-RK3 steps "
           "(CFL 0.3) per bench step in one CUDA graph", 100),
    "c1": ("c1: a=0.5, 2 radial elements r in [1.8,20], N_r=N_theta=12 (theta band [pi/8, 7pi/8]) "
           "N_phi=16 (4,608 nodes, latency-bound), 100 SSP-RK3 steps (CFL 0.3) per bench step "
           "in one CUDA graph", 100),
    "c2f": ("c2f: c2's instance on the paper's Fourier theta basis (N_theta=32 uniform "
            "pole-free nodes over [0, pi], double-Fourier parity extension), a=0.9, 8 radial "
            "elements r in [1.5,100], N_r=24 N_phi=64, 100 SSP-RK3 steps per bench "
            "step in one CUDA graph; dt = 1e-3 of the CFL step", 100),
    "c5": ("c5: a=0.94, 16 radial elements r in [1.3,500], N_r=32, N_theta=64 (theta band "
           "[pi/8, 7pi/8]), N_phi=128, 200 SSP-RK3 steps (CFL 0.3) per bench step in one CUDA "
           "graph", 200),
    "c4": ("c4: 256 independent instances, a ~ U[0,0.99], 2-8 radial elements, "
           "N_r = N_theta in {8,12,16,24,32} (theta band [pi/8, 7pi/8]), N_phi in {16,32,64}, "
           "Bondi-like profiles; 10 SSP-RK3 steps per bench step, all instances in one CUDA "
           "graph", 10),
}

# Time step as a fraction of the CFL step.  The Fourier theta workload spans the whole
# sphere, where the conformal BSSN fields of the spherical Kerr-Schild slice are not
# smooth across the axis (ln sin(theta), sin(theta)^(+-2/3)): the double-Fourier extension
# makes the right-hand side of the pole-adjacent nodes large and a CFL-sized step moves
# them by O(1).  The throughput does not depend on dt; a small step keeps the 100 steps of
# a bench step near the initial data, like the other workloads.
DT_SCALE = {"c2f": 1e-3}


def rank_batch(n, rank):
    """The rank's own batch: n independent instances drawn from the batch generator with
    seeds disjoint from every other rank's (rank 0 has the single-GPU batch).  Per-GPU work
    stays fixed as ranks are added (weak scaling); the ranks exchange nothing but the
    timing."""
    from workloads import batch_configs
    from workloads.synth import BATCH_BASE_SEED
    return batch_configs(n, base_seed=BATCH_BASE_SEED + n * rank)


def combine(ms_local, units_local, world):
    """Whole-job figures from every rank's timed region: the slowest rank's time and the
    units (point-updates) of all ranks; returns (ms_max, units_total, value per second).
    Uses the initialised default process group when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as tdist
        dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tdist.all_reduce(u, op=tdist.ReduceOp.SUM)
        ms_max, units = float(t.item()), float(u.item())
    else:
        ms_max, units = float(ms_local), float(units_local)
    return ms_max, units, units / (ms_max * 1e-3)


def measure_batch(precision, steps, warmup, world, rank, local, dist_on):
    """The batched workload (256 independent instances per rank, grouped by shape, all
    groups of a step in one CUDA graph): CUDA-event time of `steps` bench steps of 10
    SSP-RK3 steps after `warmup` untimed ones.  Returns the figures of one JSON record
    (aggregate point-updates/s and instance-steps/s over all ranks)."""
    import torch
    import paper_2508_18221_gb300 as pkg
    from workloads import primitive_profiles
    if dist_on:
        import torch.distributed as tdist
    cfgs = rank_batch(256, rank)
    desc, nsteps = WORKLOADS["c4"]
    stream = torch.cuda.Stream()
    batch = pkg.Batch([pkg.make_structs(c, precision=precision) for c in cfgs], stream.cuda_stream)
    npts = 0
    states = []
    for i, c in enumerate(cfgs):
        r, t, ph = batch.coords(i)
        pr = primitive_profiles(c, r.reshape(c.shape), t.reshape(c.shape), ph.reshape(c.shape))
        batch.init_prims(i, pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
        st = torch.empty(pkg.NV * batch.num_points(i), dtype=torch.float64, device="cuda")
        batch.get_state(i, st, True)
        states.append(st)
        npts += batch.num_points(i)
    dts = batch.cfl_dt()

    def one(ev=None):
        for i in range(len(cfgs)):
            batch.set_state(i, states[i], True)
        torch.cuda.synchronize()
        if ev:
            ev[0].record(stream)
        batch.step(dts, nsteps)
        if ev:
            ev[1].record(stream)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if dist_on:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(steps):
            one(evs[k])
        torch.cuda.synchronize()
    if dist_on:
        tdist.barrier()
    ms_local = sum(a.elapsed_time(b) for a, b in evs)
    ms, units, value = combine(ms_local, npts * RHS_PER_STEP * nsteps * steps, world)
    n_inst = len(cfgs) * world
    rec = {"metric": "batched " + metric_name(precision), "value": value, "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
           "instance_steps_per_s": n_inst * nsteps * steps / (ms * 1e-3),
           "dtype": DTYPE[precision],
           "config": {"workload": desc, "precision": precision, "instances": n_inst,
                      "nodes": int(round(units / (RHS_PER_STEP * nsteps * steps))),
                      "groups_rank0": batch.num_groups(),
                      "l2": "inputs (5.4 GB state) far larger than L2",
                      "parallelism": f"{world} rank(s), 256 independent instances each"},
           "gpu_launches": batch.launch_count() * nsteps * steps,
           "clocks": clk.summary()}
    batch.close()
    return rec


def run_batch(args):
    """Batched workload as the main line: value = aggregate point-updates/s, also
    instance-steps/s.  With N ranks every rank advances its own 256-instance batch
    (disjoint seeds; no collective on the data path)."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    rec = measure_batch(args.precision, args.steps, args.warmup, world, rank, local, dist_on)
    line = dict(rec, n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None,
                data="synthetic (seeded Bondi-like profiles, splitmix64 noise)")
    line["config"]["instance_steps_per_s"] = rec["instance_steps_per_s"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist_on:
        tdist.destroy_process_group()


def single_config(cfg, desc, nsteps, precision, world):
    """The `config` record of a single-instance workload, shared by the GPU arm and the
    reference arm (which times a bounded sample of the same workload, stated outside
    `config`)."""
    return {"workload": desc, "precision": precision,
            "nodes": cfg.n_elem * cfg.n_r * cfg.n_theta * cfg.n_phi,
            "rk_steps_per_bench_step": nsteps,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": f"replicas x{world}"}


def metric_name(precision):
    return f"coupled RHS point-updates/s ({PREC_NAME[precision]})"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": smax or None, "reasons": sorted(reasons), "samples": len(sm)}


# ---- the oracle on the host cores (CPU baseline and the reference arm) ----------------
#
# The oracle is numpy FP64 with single-threaded elementwise work.  It runs, as it stands,
# in one process per host core (spawned, never forked from a process that touched the
# GPU), each process evaluating the right-hand side of one radial element of the
# benchmark grid (the element's sub-grid: same N_r, N_theta, N_phi, its own radial range).
# A step is one such evaluation in every process; the throughput is the nodes of all
# processes divided by the step's wall time.

_ORACLE_CACHE = {}


def _oracle_element(workload, e):
    """(grid, params, state) of radial element e of the workload as a one-element grid."""
    key = (workload, e)
    if key not in _ORACLE_CACHE:
        from oracle import solver as so
        from workloads import config
        cfg = config(workload)
        ra = cfg.r_min * (cfg.r_max / cfg.r_min) ** (e / cfg.n_elem)
        rb = cfg.r_min * (cfg.r_max / cfg.r_min) ** ((e + 1) / cfg.n_elem)
        _ORACLE_CACHE[key] = so.workload_state(config(workload, n_elem=1, r_min=ra, r_max=rb))
    return _ORACLE_CACHE[key]


def _oracle_rhs_task(job):
    """One oracle right-hand side of one element (runs in a worker); returns its nodes."""
    from oracle import solver as so
    g, p, U = _oracle_element(*job)
    so.rhs(U, g, p)
    return int(U[0].size)


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


class OraclePool:
    """One spawned process per host core, each running the oracle single-threaded."""

    def __init__(self, workload="c2", workers=None):
        import multiprocessing as mp
        self.workload = workload
        self.workers = workers or os.cpu_count() or 1
        from workloads import config
        self.n_elem = config(workload).n_elem
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def step(self, nproc=None):
        """One oracle RHS of one element in each of nproc processes; (nodes, seconds)."""
        n = nproc or self.workers
        jobs = [(self.workload, w % self.n_elem) for w in range(n)]
        t0 = time.perf_counter()
        nodes = sum(self.pool.map(_oracle_rhs_task, jobs, chunksize=1))
        return nodes, time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline(workload="c2"):
    """The oracle on the host cores: one RHS of one radial element of the benchmark grid
    in every process (after a warm-up pass that builds the elements' states), plus the
    same with one process."""
    pool = OraclePool(workload)
    try:
        pool.step()                                  # warm-up: each worker builds its states
        nodes, sec = pool.step()
        n1, s1 = pool.step(1)
    finally:
        pool.close()
    return {"value": nodes / sec, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "value_1_core": n1 / s1,
            "sample": f"one RHS evaluation of one radial element of the {pool.n_elem}-element "
                      f"grid (as a one-element grid) in each of {pool.workers} spawned "
                      f"processes, {nodes} nodes in {sec:.2f} s; numpy FP64, one thread per "
                      f"process; value_1_core: one process, {n1} nodes in {s1:.2f} s"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from workloads import config
    cfg = config("c2")
    desc, nsteps = WORKLOADS["c2"]
    pool = OraclePool("c2")
    try:
        for _ in range(args.warmup):
            pool.step()
        nodes_total, el = 0, 0.0
        for _ in range(args.steps):
            n, sec = pool.step()
            nodes_total += n
            el += sec
    finally:
        pool.close()
    val = nodes_total / el
    line = {"impl": "reference", "metric": metric_name(0), "value": val, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Kerr-Schild torus, splitmix64 noise)",
            "config": single_config(cfg, desc, nsteps, 0, world),
            "sample_per_step": {"nodes": nodes_total // args.steps, "rhs_evaluations_per_node": 1,
                                "what": f"one RHS of one radial element ({cfg.n_r} x {cfg.n_theta} x "
                                        f"{cfg.n_phi} nodes) in each of {pool.workers} processes"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "cpu_model": _cpu_model(),
                             "sample": f"each step one RHS evaluation of one radial element of the "
                                       f"{cfg.n_elem}-element grid in each of {pool.workers} "
                                       "spawned processes; numpy FP64, one thread per process"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# FP64 work per node of the pointwise kernels: executed FP64 instructions counted by ncu
# (2 x DFMA + DADD + DMUL, smsp__sass_thread_inst_executed_op_d{fma,add,mul}_pred_on.sum)
# on the 393,216-node workload; the kernels recompute nothing, so this is their algorithmic
# FP64 work.  The primitive-recovery count is taken inside the time stepping (Newton
# started from the previous stage's primitives); k_prep<float> (mixed modes) forms the
# fluxes and T^{mu nu} in FP32, so only its metric and primitive recovery count.
FP64_FLOPS_PER_NODE = {"k_rhs<double>": 2501.0, "k_prep<double>": 1050.0, "k_prep<float>": 711.0}
# Nominal FP64 peak of GB300 from its unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop
# x 2.07 GHz (a probe of dependent DFMA chains on all SMs measured 1.198 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# bytes per node of the mixed-precision pointwise RHS: state, stage input and T^{mu nu}
# (FP64), first/second derivatives and flux divergence (FP32) in, stage output out
RHS32_BYTES_PER_NODE = 8 * (32 + 32 + 10) + 4 * (63 + 66 + 8) + 8 * 32


def _kernel_names(cfg, precision):
    """class of grmhd_kernel_times -> kernel (template instance) that runs it."""
    ns = (cfg.n_r, cfg.n_theta, cfg.n_phi)
    names = {"prep": "k_prep<double>" if precision == 0 else "k_prep<float>",
             "iface_d1": "k_iface_avg", "iface_d2": "k_iface_avg",
             "rhs": "k_rhs<double>" if precision == 0 else "k_rhs<float>"}
    for d, dn in enumerate(("r", "theta", "phi")):
        fx = 2 <= ns[d] <= 128 and (d != 2 or ns[d] % 2 == 0)
        fourier = d == 2 or (d == 1 and getattr(cfg, "theta_basis", 0) == 1)
        # derivatives and the filter: the digit-slice kernel (Chebyshev derivatives above 64
        # nodes: the FP64 units)
        fp64_f = f"k_contract_fx<{d}>" if fx else f"k_deriv_eo<{d}>"
        fp64_d = f"k_contract_fx<{d}>" if fx else f"k_deriv_eo<{d}>"
        if fx and not fourier and ns[d] > 64:
            fp64_d = f"k_deriv<{d}>"
        if d == 1 and getattr(cfg, "theta_basis", 0) == 1:
            # Fourier theta: fold, two half-width contractions, unfold (timed together)
            fx_t = fx and cfg.n_phi % 4 == 0
            fp64_f = "theta fold + k_contract_fx<1> x2 + unfold" if fx_t else "theta fold + k_deriv_eo<1> x2 + unfold"
            fp64_d = fp64_f
            tc = "theta fold + k_contract_tc<1> x2 + unfold"
        else:
            tc = f"k_contract_tc<{d}>"
        for c in ("d1", "d2"):
            names[f"{c}_{dn}"] = fp64_d if precision == 0 else tc
        names[f"filter_{dn}"] = fp64_f
    return names


def roofline(kt_full, P, precision, names):
    per_step = {k: (1 if k.startswith("filter") else RHS_PER_STEP) for k in kt_full}
    t_kernel, work = {}, {}
    for k, (ms, fl, by) in kt_full.items():
        kn = names.get(k, k)
        t_kernel[kn] = t_kernel.get(kn, 0.0) + ms * per_step[k]
        f0, b0 = work.get(kn, (0.0, 0.0))
        work[kn] = (f0 + fl * per_step[k], b0 + by * per_step[k])
    t_all = sum(t_kernel.values())
    top = max(t_kernel, key=t_kernel.get)
    t_s = t_kernel[top] * 1e-3
    hbm = _peaks().get("hbm_gbs", 6800.0)
    roof = {"kernel": top, "share_of_step": t_kernel[top] / t_all,
            "kernel_ms_per_step": {kn: round(v, 4) for kn, v in sorted(t_kernel.items(), key=lambda x: -x[1])}}
    launches = sum(per_step[k] for k in kt_full if names.get(k, k) == top)
    if top in FP64_FLOPS_PER_NODE and FP64_FLOPS_PER_NODE[top]:
        achieved = FP64_FLOPS_PER_NODE[top] * P * launches / t_s / 1e12
        roof.update({"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": _traffic(top, P),
                     "peak_source": "GB300 FP64 from unit counts and clock (of nominal)",
                     "work": f"{FP64_FLOPS_PER_NODE[top]:.0f} FP64 flop per node (ncu-counted)"})
    elif top.startswith("k_contract") or top.startswith("k_deriv"):
        if top.startswith("k_deriv_eo"):
            achieved = work[top][0] / t_s / 1e12
            roof.update({"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": _traffic(top, P),
                         "peak_source": "GB300 FP64 from unit counts and clock (of nominal)",
                         "work": "2 N FP64 flop per output node"})
        else:
            achieved = work[top][1] / t_s / 1e9
            roof.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": _traffic(top, P),
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "work": "input read + output written per contracted field"})
    else:
        by = RHS32_BYTES_PER_NODE if top == "k_rhs<float>" else None
        if by is None:
            roof.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                         "traffic": None})
        else:
            achieved = by * P * launches / t_s / 1e9
            roof.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": _traffic(top, P),
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "work": f"{by} bytes per node"})
    if roof.get("traffic") is not None and P != TRAFFIC_NODES:
        roof["traffic_note"] = (f"ncu DRAM bytes of the {TRAFFIC_NODES}-node workload scaled to {P} nodes "
                                "(per-node traffic of a pointwise kernel)")
    return roof


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of
# the current kernel code inside the time stepping of the 393,216-node workload, mean of the
# three stages of a step); absent = not captured since the kernel last changed.  These
# pointwise kernels move a fixed number of bytes per node, so another workload's launch
# is scaled by its node count (traffic_note says so).
# k_rhs<double> moves ~2.8 KB per node, about twice its algorithmic bytes: register spills
# (it is FP64-bound, the bytes are not).
TRAFFIC_NODES = 393216
TRAFFIC = {"k_rhs<double>": 1.10e9, "k_prep<double>": 1.66e8, "k_prep<float>": 1.66e8, "k_rhs<float>": 6.13e8}


def _traffic(kernel, P):
    t = TRAFFIC.get(kernel)
    return None if t is None else t * P / TRAFFIC_NODES


def measure_single(workload, precision, steps, warmup, world, rank, local, dist_on, extras=True):
    """One single-instance workload: `steps` timed bench steps (each `nsteps` SSP-RK3 steps
    recorded in one CUDA graph, from the same initial state, L2 flushed before each) after
    `warmup` untimed ones; then the end-to-end figure through the C ABI with host buffers,
    the bare right-hand side and the per-kernel times behind the roofline.  Returns the
    record and the state after one bench step (a device tensor)."""
    import torch
    import paper_2508_18221_gb300 as pkg
    from workloads import config, primitive_profiles
    if dist_on:
        import torch.distributed as tdist

    cfg = config(workload)
    desc, nsteps = WORKLOADS[workload]
    grid, phys, opts = pkg.make_structs(cfg, precision=precision)
    stream = torch.cuda.Stream()
    ctx = pkg.Context(grid, phys, opts, stream.cuda_stream)
    P = ctx.n_points
    r, t, ph = ctx.coords()
    shp = cfg.shape
    pr = primitive_profiles(cfg, r.reshape(shp), t.reshape(shp), ph.reshape(shp))
    ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    U0 = torch.empty(pkg.NV * P, dtype=torch.float64, device="cuda")
    ctx.get_state(U0, True)
    dt = ctx.cfl_dt() * DT_SCALE.get(workload, 1.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(timed_events=None):
        with torch.cuda.stream(stream):
            ctx.set_state(U0, True)
            flush.fill_(1.0)                      # evict L2 between timed steps
            if timed_events:
                timed_events[0].record(stream)
            ctx.step(dt, nsteps)
            if timed_events:
                timed_events[1].record(stream)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    launches_per_step = ctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if dist_on:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(steps):
            one(evs[k])
        torch.cuda.synchronize()
    if dist_on:
        tdist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max, units, value = combine(ms, P * RHS_PER_STEP * nsteps * steps, world)
    final = torch.empty_like(U0)
    ctx.get_state(final, True)

    # end to end through the C ABI with host buffers (pinned)
    host_in = torch.empty(pkg.NV * P, dtype=torch.float64).pin_memory()
    host_out = torch.empty_like(host_in)
    host_in.copy_(U0.cpu())
    e2e_steps = max(1, min(steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(host_in, False)
        ctx.step(dt, nsteps)
        ctx.get_state(host_out, False)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = P * RHS_PER_STEP * nsteps * e2e_steps * world / e2e_s

    rec = {"metric": metric_name(precision), "value": value, "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": ms_max / steps,
           "dtype": DTYPE[precision], "config": single_config(cfg, desc, nsteps, precision, world),
           "dt": dt,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": pkg.NV * P * 8,
                   "d2h_bytes_per_step": pkg.NV * P * 8},
           "gpu_launches": launches_per_step * steps, "clocks": clk.summary(),
           "us_per_rk_step": ms_max / steps / nsteps * 1e3}
    if extras:
        # bare right-hand side through the C ABI (no graph, device buffers)
        rhs_out = torch.empty_like(U0)
        ctx.set_state(U0, True)
        for _ in range(3):
            ctx.rhs(rhs_out, True)
        torch.cuda.synchronize()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_rhs = 20
        e_a.record(stream)
        for _ in range(n_rhs):
            ctx.rhs(rhs_out, True)
        e_b.record(stream)
        torch.cuda.synchronize()
        rec["rhs_call"] = {"value": P * n_rhs * world / (e_a.elapsed_time(e_b) * 1e-3), "unit": UNIT,
                           "what": "grmhd_rhs on device buffers, no graph, 20 calls"}
    # live per-kernel timing (CUDA events on the library's stream): every RHS class runs
    # RHS_PER_STEP times per step, every filter class once.  The roofline is reported for
    # the kernel with the largest time per step.
    ctx.set_state(U0, True)
    kt_full = ctx.kernel_times(reps=5)
    rec["roofline"] = roofline(kt_full, P, precision, _kernel_names(cfg, precision))
    stats = ctx.diag()
    rec["final_diag"] = {"mass": stats[0], "c2p_floor_points": stats[3]}
    ctx.close()
    return rec, final


# evolved variables grouped by tensor (for the error of the mixed path against FP64)
TENSOR_GROUPS = {"gammatilde": range(0, 6), "phi": [6], "Atilde": range(7, 13), "K": [13],
                 "Gammatilde": range(14, 17), "alpha": [17], "beta": range(18, 21),
                 "B_driver": range(21, 24), "D": [24], "S": range(25, 28), "tau": [28],
                 "B_field": range(29, 32)}


def tensor_rel_l2(a, b, nv):
    """Relative L2 difference of each tensor of two canonical states (device tensors)."""
    A = a.view(nv, -1)
    Bm = b.view(nv, -1)
    out = {}
    for name, idx in TENSOR_GROUPS.items():
        idx = list(idx)
        den = float(Bm[idx].norm())
        out[name] = float((A[idx] - Bm[idx]).norm()) / den if den > 0 else 0.0
    return out


# Relative L2 errors of the split-BF16 x3 mode against the FP64 oracle after 100 SSP-RK3
# steps of the 2-element 12 x 12 x 16 instance, per tensor, from the GPU test
# test_precision_variant_report (asserted there to stay below the spectral truncation
# level of every tensor); the largest and the tightest tensor.
MIXED_STATED_ERROR = {"instance": "2 elements 12 x 12 x 16 (4,608 nodes), 100 SSP-RK3 steps",
                      "max_rel_l2_vs_fp64_oracle": 7.5e-05, "tensor": "B_driver (starts at zero)",
                      "tightest": "K: 2.8e-05 against a truncation level of 2.9e-05 "
                                  "(0.95-1.00 of it over five noise seeds)",
                      "source": "tests/test_gpu_mixed.py::test_precision_variant_report"}


def run_gpu(args):
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    rec, final = measure_single(args.workload, args.precision, args.steps, args.warmup, world, rank,
                                local, dist_on)
    line = dict(rec, n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None,
                data="synthetic (seeded Kerr-Schild torus, splitmix64 noise)")
    extras = not args.no_extras and args.workload == "c2" and args.precision == 0
    if extras:
        # the rest of the headline metric in the same line: the mixed form on the same
        # workload (with its error against the FP64 path after one bench step) and the
        # batched workload in both forms
        mrec, mfinal = measure_single("c2", 1, args.steps, args.warmup, world, rank, local, dist_on,
                                      extras=False)
        nv = final.numel() // (mrec["config"]["nodes"])
        err = tensor_rel_l2(mfinal, final, nv)
        mrec["error_vs_fp64_path"] = {
            "what": "relative L2 per tensor of the state after one bench step (100 SSP-RK3 steps) "
                    "against the FP64 path's state from the same initial data",
            "max": max(err.values()), "per_tensor": err}
        mrec["stated_error"] = MIXED_STATED_ERROR
        mrec["vs_fp64_path"] = mrec["value"] / rec["value"]
        del final, mfinal
        torch.cuda.empty_cache()
        bsteps, bwarm = min(args.steps, 3), max(3, min(args.warmup, 3))
        b64 = measure_batch(0, bsteps, bwarm, world, rank, local, dist_on)
        torch.cuda.empty_cache()
        b32 = measure_batch(1, bsteps, bwarm, world, rank, local, dist_on)
        torch.cuda.empty_cache()
        b64["vs_single_instance_fp64"] = b64["value"] / rec["value"]
        b32["vs_batch_fp64"] = b32["value"] / b64["value"]
        line["mixed"] = mrec
        line["batch"] = {"fp64": b64, "mixed": b32}
    if rank == 0:
        cb = None
        if not args.no_cpu_baseline:
            try:
                cb = cpu_baseline()
            except Exception as exc:  # noqa: BLE001
                cb = {"error": str(exc)}
        line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if dist_on:
        tdist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision and batched records of the default line")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
