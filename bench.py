"""Benchmark: committed spin flips per second of the synchronous-relaxation
n-fold-way Ising simulation on GB300.

Headline workload (one "step" = the whole hot path over the batch): 256
independent periodic 2D Ising lattices, L uniform over {64, 128, 256, 512,
1024}, T uniform in [1, 3.5], h uniform in [-0.2, 0.2], J = 1, fair-coin
initial spins; region shape, region lanes per warp and events per window
chosen by the autotuner; every lattice restarts from its initial state and
runs to t = 100 with window lengths matched to its event rate, then its
observables are reduced.  Beside it: the same lattices one per context (the
"plain" form), the plain single-lattice workloads L = 1024 (window lengths
0.25, 1, 4 to t = 100) and L = 8192 (window length 0.1 to t = 50), f and g
of §6 against log N, and the oracle on a bounded sample of the batch.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 is launched with torch.distributed.run: each rank simulates its own
batch (lattice b of rank r has seed 1000 + 256 r + b) on its own GPU, with no
data exchange ("scaling": "weak"); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "committed spin flips/s on 1 GB300 (batched vs plain), % roofline, iters"
UNIT = "flips/s"
T_END = 100.0
BATCH_N = 256
WORKLOAD = ("256 lattices: L uniform over {64,128,256,512,1024}, T uniform in [1,3.5], h uniform "
            "in [-0.2,0.2], J=1, fair-coin spins, Metropolis rates via the n-fold way, run to "
            "t=100 each (numpy Philox key 4, seeds 1000+b), autotuned region shape, adaptive "
            "window lengths")
PLAIN_L, PLAIN_W, PLAIN_H, PLAIN_T, PLAIN_WINDOWS = 1024, 0.05, 1.0, 100.0, (0.25, 1.0, 4.0)

# Algorithmic work of the method per committed event (counted from the formulas
# of §3 and §5, independent of how this implementation executes them):
#   Philox4x32-10 ~100 integer ops, uniform mapping 6, -log U ~25, the waiting
#   time (sub, divide, add) ~10, Lambda and the class scan ~30, the site rank
#   ~20, the class update of <= 5 sites ~60, the history record ~10
# -> ~260 integer + ~50 floating-point operations = 310 operations; a break
# point adds ~35 (hazard accrual, halo update, class update, new waiting time).
OPS_PER_EVENT = 310
OPS_PER_BREAK = 35
# Integer issue peak: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz.
SMS, LANES_PER_SM, SM_MHZ = 152, 128, 2070.0
INT_PEAK_OPS = SMS * LANES_PER_SM * SM_MHZ * 1e6          # 4.03e13 lane-ops/s
# FP64 pipe (measured on one GB300 with a probe of dependent-free DFMA / DDIV
# streams): 5.0e11 DFMA lane-ops/s; one DDIV takes about 8.6 DFMA slots.
# Per committed event the formulas need -log U (26 add/mul, 1 divide, 1
# integer-to-double conversion) and the waiting time (Lambda conversion and
# scale, subtract, divide, add: 4 add/mul/convert, 1 divide): 32 slots + 2
# divides = 49 DFMA slots.
FP64_PEAK_OPS = 5.0e11
FP64_SLOTS_PER_EVENT = 32 + 2 * 8.6
# History bytes per committed boundary event: f64 time + u8 position, written
# once and read by one neighbour (two for a corner).
HIST_BYTES_PER_BOUNDARY_EVENT = 9 * 2
HBM_GBS_FALLBACK = 6800.0
# DRAM bytes (read + write) per relaxation launch of the batched step, mean
# over the 100 launches of one whole step (one ncu capture on a GB300 of
#   python bench.py --profile-batch --windows 0 --tune-in TUNE, with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:relax_kernel --csv
# and TUNE the autotuner's choice of the same GPU call); valid only for the
# kernel sources they were taken on (hash below) and for the same tuning
# (region shape counts, lanes per warp, kappa).
BATCH_TRAFFIC = {"bytes_per_launch": 14160895882,
                 "tuning": [{"32x16": 127, "32x32": 107, "16x16": 22}, 0, 8.0]}
BATCH_TRAFFIC_SHA = "d591b8aed2c2172c"
# DRAM bytes per launch of the L = 1024 launches, one per window length
#   python bench.py --profile-case --tw TW --windows 100/TW under the same ncu
#   metrics with -s 3 -c 1
PLAIN_TRAFFIC = {0.25: 8675840, 1.0: 107309312, 4.0: 1296592128}
PLAIN_TRAFFIC_SHA = "d591b8aed2c2172c"


def _kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_cs_0405053_gb300/csrc/sr_lib.cu", "paper_cs_0405053_gb300/csrc/sr_state.cuh",
              "paper_cs_0405053_gb300/csrc/sr_region.cuh", "paper_cs_0405053_gb300/csrc/sr_kernel.cuh",
              "paper_cs_0405053_gb300/csrc/sr_device.cuh",
              "paper_cs_0405053_gb300/csrc/sr_softfloat.cuh", "include/sr.h"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- rank bookkeeping
def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed0(rank):
    """First seed of the batch a rank simulates (each rank its own lattices)."""
    return 1000 + BATCH_N * rank


def job_throughput(dist, seconds, committed, device):
    """Whole-job throughput of independent replicas, one per rank: the units
    of all ranks over the slowest rank's time.  Returns (max seconds, value)."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    c = torch.tensor([float(committed)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return t_max, float(c.item()) / t_max


def timed_steps(step, steps, warmup, dist=None, sync=lambda: None, between=lambda: None):
    """W untimed warm-up steps, then exactly K timed steps bracketed by a
    barrier and a synchronize on both sides.  `step()` returns (seconds,
    units) of one step as measured by the caller (CUDA events on the GPU);
    `between()` runs before each timed step, outside its measurement (the L2
    flush).  Returns (per-step seconds, units, wall seconds of the loop)."""
    for _ in range(warmup):
        step()
    sync()
    if dist is not None:
        dist.barrier()
    sync()
    secs, units = [], 0
    w0 = time.perf_counter()
    for _ in range(steps):
        between()
        s, u = step()
        secs.append(s)
        units += u
    sync()
    if dist is not None:
        dist.barrier()
    sync()
    return secs, units, time.perf_counter() - w0


# ---------------------------------------------------------------- clocks
def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None


def _clock_summary(path, gpu_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------- the oracle (CPU baseline)
def _oracle_job(args):
    """One oracle run (plain sequential C, one core): lattice `rep` from t = 0
    to t_end.  Returns (committed events, seconds)."""
    import oracle
    rep, t_end = args
    t0 = time.perf_counter()
    r = oracle.run(rep["L"], rep["J"], rep["h"], rep["T"], rep["W"], rep["H"], rep["seed"],
                   [t_end], keep_spins=False)
    return int(r.counts[-1].sum()), time.perf_counter() - t0


def _oracle_pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)


def oracle_sample(reps, shapes, rates, events_per_job=3.0e6):
    """A bounded sample of the batched workload for the oracle: a stratified
    set of lattices (every side L, cold to hot), each in its region shape
    shapes[b], run from t = 0 to the time at which it has committed about
    `events_per_job` events at its own event rate `rates[b]` (events per unit
    time), at most t = 100."""
    from paper_cs_0405053_gb300 import workloads
    jobs = []
    for b in workloads.stratified(reps, per_side=3):
        t_end = min(T_END, max(0.25, events_per_job / max(rates[b], 1.0)))
        rep = dict(reps[b], W=shapes[b][0], H=shapes[b][1])
        jobs.append((rep, float(t_end)))
    return jobs


def run_oracle_sample(pool, jobs):
    """(committed, wall seconds, per-core events/s) of the jobs run in parallel."""
    w0 = time.perf_counter()
    res = pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - w0
    committed = sum(c for c, _ in res)
    per_core = committed / max(1e-9, sum(s for _, s in res))
    return committed, wall, per_core


def _calibrated_rates(pool, reps, region):
    """Events per unit time of every sampled lattice from a short oracle run
    (t = 0.25), for sizing the reference arm's sample."""
    from paper_cs_0405053_gb300 import workloads
    idx = workloads.stratified(reps, per_side=3)
    res = pool.map(_oracle_job, [(dict(reps[b], W=region[0], H=region[1]), 0.25) for b in idx],
                   chunksize=1)
    rates = {b: c / 0.25 for b, (c, _) in zip(idx, res)}
    return [rates.get(b, 1.0) for b in range(len(reps))]


def run_reference(args):
    """The reference arm: the oracle (the plain CPU simulation the GPU path is
    checked against) timed on this machine's cores on the headline workload,
    each step a bounded sample of it (see oracle_sample)."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas()
    region = (32, 16)
    cores = max(1, min(os.cpu_count() or 1, 16))
    pool = _oracle_pool(cores)
    try:
        rates = _calibrated_rates(pool, reps, region)
        jobs = oracle_sample(reps, [region] * len(reps), rates, events_per_job=1.5e6)
        for _ in range(args.warmup):
            run_oracle_sample(pool, jobs[:cores])
        committed, secs = 0, 0.0
        for _ in range(args.steps):
            c, s, _ = run_oracle_sample(pool, jobs)
            committed += c
            secs += s
    finally:
        pool.terminate()
        pool.join()
    value = committed / secs
    sample = (f"per step {len(jobs)} lattices of the batch (3 per side L: coldest, median, "
              f"hottest), each from t=0 until about 1.5e6 committed events (at most t=100), "
              f"region {region[0]}x{region[1]}, one oracle process per core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def _plain_L1024(sr, torch, stream):
    """The plain single-lattice workload: L = 1024 in 16 x 16 regions, J = 1,
    h = 0.05, T = 1, fair coin; for each window length 0.25, 1, 4: restart,
    windows to t = 100, observables (one persistent launch per window set)."""
    lat = sr.Lattice(PLAIN_L, 1.0, PLAIN_W, PLAIN_H, (16, 16), seed=1)
    out, com, dev = {}, 0, 0.0
    for Tw in PLAIN_WINDOWS:
        n = int(round(PLAIN_T / Tw))
        lat.reset()
        o0 = lat.observables()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        lat.run_windows(Tw, n)
        o = lat.observables()
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        it = [int(v) for v in lat.window_iters(n)]
        kms = o.relax_ms - o0.relax_ms
        out[str(Tw)] = {"ms": round(ms, 3), "kernel_ms": round(kms, 3), "committed": o.committed,
                        "generated": o.generated,
                        "wasted_ratio": (o.generated - o.committed) / max(1, o.committed),
                        "iters_mean": statistics.mean(it) if it else None,
                        "iters_max": max(it) if it else None, "max_f": o.max_f,
                        "breaks": o.breaks, "flips_per_s": o.committed / (ms * 1e-3)}
        com += o.committed
        dev += ms * 1e-3
    kms_all = sum(v["kernel_ms"] for v in out.values())
    ops = com * OPS_PER_EVENT / (kms_all * 1e-3)
    lat.close()
    return {"workload": "L=1024 periodic, 64x64 regions of 16x16, J=1, h=0.05, T=1.0, fair-coin "
                        "spins, Tw in {0.25, 1, 4} to t=100 (one persistent launch each)",
            "flips_per_s": com / dev, "per_window_length": out,
            "roofline": {"bound": "alu", "kernel": "relax_kernel<0,0>", "achieved": ops / 1e12,
                         "peak": INT_PEAK_OPS / 1e12, "unit": "Tops/s", "frac": ops / INT_PEAK_OPS,
                         "traffic": (statistics.mean(PLAIN_TRAFFIC.values())
                                     if PLAIN_TRAFFIC and _kernel_sources_sha() == PLAIN_TRAFFIC_SHA
                                     else None)}}


def _plain_L8192(sr, torch, stream, t_end=50.0):
    """The plain method at scale: L = 8192 in 256 x 256 regions of 32 x 32,
    J = 1, h = 0, T = 2.269, fair coin, window length 0.1 to t = 50."""
    lat = sr.Lattice(8192, 1.0, 0.0, 2.269, (32, 32), seed=1, init="fair")
    n = int(round(t_end / 0.1))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    lat.run_windows(0.1, n)
    o = lat.observables()
    ev[1].record(stream)
    torch.cuda.synchronize()
    s = ev[0].elapsed_time(ev[1]) * 1e-3
    it = lat.window_iters(n)
    lat.close()
    ops = o.committed * OPS_PER_EVENT / (o.relax_ms * 1e-3)
    return {"workload": f"L=8192 periodic, 256x256 regions of 32x32, J=1, h=0, T=2.269, fair-coin "
                        f"spins, Tw=0.1 to t={t_end:g}",
            "flips_per_s": o.committed / s, "s": s, "committed": o.committed,
            "wasted_ratio": (o.generated - o.committed) / max(1, o.committed),
            "iters_mean": float(it.mean()) if len(it) else None, "max_f": o.max_f,
            "roofline": {"bound": "alu", "kernel": "relax_kernel<0,1>", "achieved": ops / 1e12,
                         "peak": INT_PEAK_OPS / 1e12, "unit": "Tops/s",
                         "frac": ops / INT_PEAK_OPS}}


def _one_by_one(sr, torch, stream, reps, tune, every=16):
    """The plain form of the batched workload: a stratified sample of the
    lattices (every `every`-th), each in its own context with the same region
    shape and window rule, run one after the other."""
    com, dev = 0, 0.0
    sample = list(range(0, len(reps), every))
    own = tune.replicas(reps)
    for k in sample:
        one = sr.Batch([own[k]], region=tune.shapes[k])
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        one.run_adaptive(T_END, kappa=tune.kappa)
        o = one.observables(0)
        ev[1].record(stream)
        torch.cuda.synchronize()
        com += o.committed
        dev += ev[0].elapsed_time(ev[1]) * 1e-3
        one.close()
    return {"flips_per_s": com / dev, "s": dev, "committed": com,
            "sample": f"every {every}th lattice ({len(sample)} of {len(reps)}), each in its own "
                      "context with the same region shape and window rule"}


def _fg_vs_log_n(sr):
    """f and g of §6 versus log N: L = 64 .. 2048 in 16x16 regions (N = 16 ..
    16384), T = 3.0, h = 0, T_max = log N / (lambda |boundary|) (Eq. 5.1,
    lambda = 1, 60 boundary sites); 20 windows of warm-up, 60 measured."""
    rows = []
    for L in (64, 128, 256, 512, 1024, 2048):
        N = (L // 16) ** 2
        Tw = math.log(N) / 60.0
        lat = sr.Lattice(L, 1.0, 0.0, 3.0, (16, 16), seed=7)
        lat.run_windows(Tw, 20)
        o0 = lat.observables()
        t0 = time.perf_counter()
        lat.run_windows(Tw, 60)
        dt = time.perf_counter() - t0
        o = lat.observables()
        f = lat.window_f(60)
        g = lat.window_iters(60)
        lat.close()
        lg = math.log(N)
        rows.append({"N": N, "log_N": round(lg, 3), "T_max": round(Tw, 5),
                     "f_mean": float(f.mean()), "f_max": int(f.max()),
                     "g_mean": float(g.mean()), "g_max": int(g.max()),
                     "f_over_log_N": float(f.mean()) / lg, "g_over_log_N": float(g.mean()) / lg,
                     "flips_per_s": (o.committed - o0.committed) / dt})
    return rows


def run_ours(args):
    import numpy as np
    import torch

    import paper_cs_0405053_gb300 as sr
    from paper_cs_0405053_gb300 import workloads

    rank, world, local = _dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    reps = workloads.batch_replicas(seed0=rank_seed0(rank))
    t0 = time.perf_counter()
    tune = sr.autotune(reps, t_trial=1.0)
    tune_s = time.perf_counter() - t0
    bt = sr.Batch(tune.replicas(reps), region=tune.region, lanes_per_warp=tune.lanes_per_warp)
    # every relaxation launch of the batch runs as a replayed CUDA graph (the
    # plan's uploads, the persistent kernel and the status read-back)
    bt.graph_launch(True)
    if args.tune_out:
        with open(args.tune_out, "w") as fh:
            json.dump({"shapes": tune.shapes, "lanes_per_warp": tune.lanes_per_warp,
                       "kappa": tune.kappa, "rate_threshold": tune.rate_threshold}, fh)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    n = len(reps)

    def step():
        """The whole hot path over the batch: every lattice restarts from its
        initial state, runs to t = 100, and its observables are reduced."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        bt.reset()
        bt.run_adaptive(T_END, kappa=tune.kappa)
        obs = [bt.observables(b) for b in range(n)]
        ev[1].record(stream)
        ev[1].synchronize()
        step.last = obs
        return ev[0].elapsed_time(ev[1]) * 1e-3, sum(o.committed for o in obs)

    clock_path = os.path.join(tempfile.gettempdir(), f"sr_clocks_{os.getpid()}.csv")
    for _ in range(args.warmup):
        step()
    o_before = bt.observables(0)
    sampler = _clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    secs, committed, wall = timed_steps(step, args.steps, 0, dist, torch.cuda.synchronize,
                                        flush.zero_)
    if sampler:
        sampler.terminate()
        sampler.wait()
    o_after = bt.observables(0)
    t_max, value = job_throughput(dist, sum(secs), committed, "cuda")
    obs = step.last
    generated = sum(o.generated for o in obs)
    com_step = sum(o.committed for o in obs)
    iters = sum(o.iterations for o in obs) / max(1, sum(o.windows for o in obs))
    relax_ms = o_after.relax_ms - o_before.relax_ms
    relax_n = o_after.relax_launches - o_before.relax_launches
    launches = (o_after.launches - o_before.launches) // max(1, args.steps)

    # ---- end to end through the public API with host buffers: every step
    # uploads each lattice's initial spins from pinned memory (a fair coin of
    # numpy's PCG64 from seed 2000 + b), runs it to t = 100 and reads back the
    # final spins and observables
    sites = [r["L"] ** 2 for r in reps]
    offs = np.concatenate([[0], np.cumsum(sites)])
    rng = np.random.default_rng(2000 + rank)
    init_host = torch.from_numpy(
        np.where(rng.random(int(offs[-1])) < 0.5, 1, -1).astype(np.int8)).pin_memory()
    out_host = torch.empty(int(offs[-1]), dtype=torch.int8).pin_memory()
    base_in, base_out = init_host.data_ptr(), out_host.data_ptr()

    def e2e_step():
        w0 = time.perf_counter()
        for b in range(n):
            bt.set_spins(b, base_in + int(offs[b]))
        bt.run_adaptive(T_END, kappa=tune.kappa)
        c = 0
        for b in range(n):
            bt.spins_into(b, base_out + int(offs[b]))
            c += bt.observables(b).committed
        return time.perf_counter() - w0, c

    e2e_steps = max(3, args.steps // 4)
    e_secs, e_com, _ = timed_steps(e2e_step, e2e_steps, 1, dist, torch.cuda.synchronize)
    _, e2e_value = job_throughput(dist, sum(e_secs), e_com, "cuda")
    g_captures, g_launches = bt.graph_stats()
    launch_shape = {"blocks": bt.blocks, "region_slots_per_block": bt.threads_per_block,
                    "cuda_graph": True, "graph_captures": g_captures, "graph_launches": g_launches}
    bt.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- the plain forms and the measurement context (rank 0)
    one = _one_by_one(sr, torch, stream, reps, tune)
    plain_1024 = _plain_L1024(sr, torch, stream)
    plain_8192 = _plain_L8192(sr, torch, stream)
    fg_rows = _fg_vs_log_n(sr)

    # ---- the oracle on a bounded sample of the batch, one process per core,
    # each lattice sized by its event rate in the GPU run
    rates = [o.committed / T_END for o in obs]
    cores = max(1, min(os.cpu_count() or 1, 16))
    pool = _oracle_pool(cores)
    try:
        jobs = oracle_sample(reps, tune.shapes, rates)
        cpu_com, cpu_wall, cpu_per_core = run_oracle_sample(pool, jobs)
    finally:
        pool.terminate()
        pool.join()

    # ---- roofline of the dominant kernel (the batched relaxation launches):
    # algorithmic integer work of the committed trajectory per launch over the
    # launch's CUDA-event time
    per_launch_ms = relax_ms / max(1, relax_n)
    ev_per_launch = committed / max(1, relax_n)
    achieved = ev_per_launch * OPS_PER_EVENT / (per_launch_ms * 1e-3)
    peaks = _measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_GBS_FALLBACK))
    # boundary sites per site of each lattice's regions, weighted by its committed events
    phi = sum(o.committed * (2 * w + 2 * h - 4) / (w * h)
              for o, (w, h) in zip(obs, tune.shapes)) / max(1, com_step)
    ev_rate = committed / (relax_ms * 1e-3)
    bounds = {"integer_issue": INT_PEAK_OPS / OPS_PER_EVENT,
              "history_bytes_at_hbm": hbm * 1e9 / (HIST_BYTES_PER_BOUNDARY_EVENT * phi),
              "fp64_pipe": FP64_PEAK_OPS / FP64_SLOTS_PER_EVENT}
    traffic = None
    shape_counts = {}
    for w, h in tune.shapes:
        shape_counts[f"{w}x{h}"] = shape_counts.get(f"{w}x{h}", 0) + 1
    if (BATCH_TRAFFIC and _kernel_sources_sha() == BATCH_TRAFFIC_SHA and
            BATCH_TRAFFIC["tuning"] == [shape_counts, tune.lanes_per_warp, tune.kappa]):
        traffic = BATCH_TRAFFIC["bytes_per_launch"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded lattices, fair-coin spins)",
        "config": {"workload": WORKLOAD, "lattices": n, "sites": int(offs[-1]),
                   "tuning": {"region_shapes": shape_counts,
                              "rate_threshold": tune.rate_threshold,
                              "lanes_per_warp": tune.lanes_per_warp or "auto",
                              "kappa": tune.kappa, "trials": tune.trials,
                              "seconds": round(tune_s, 2)},
                   "launch": launch_shape,
                   "l2": "flushed between steps (256 MiB write outside the timed events); the "
                         "batch's device state (several GB) is larger than L2",
                   "parallelism": f"independent batches x{world}" if world > 1 else "1 GPU"},
        "batched": {"flips_per_s": value, "committed_per_step": com_step,
                    "generated_per_step": generated,
                    "wasted_ratio": (generated - com_step) / max(1, com_step),
                    "iters_mean": iters, "relax_launches_per_step": relax_n // max(1, args.steps),
                    "relax_ms_per_step": relax_ms / max(1, args.steps)},
        "one_by_one": one,
        "batched_over_one_by_one": value / one["flips_per_s"],
        "plain_L1024": plain_1024,
        "plain_L8192": plain_8192,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": INT_PEAK_OPS / 1e12,
                     "unit": "Tops/s", "frac": achieved / INT_PEAK_OPS, "traffic": traffic,
                     "traffic_unit": "bytes per launch (DRAM read + write; ncu, mean over the "
                                     "launches of one step)",
                     "peak_source": "derived: 152 SMs x 128 lanes x 2070 MHz integer issue",
                     "kernel": "relax_kernel<0,2>", "kernel_ms_avg": per_launch_ms,
                     "committed_per_launch": ev_per_launch,
                     "ops_per_committed_event": OPS_PER_EVENT,
                     "events_per_s": ev_rate,
                     "events_per_s_bounds": bounds,
                     "frac_of_fp64_bound": ev_rate / bounds["fp64_pipe"],
                     "hbm_peak_gbs": hbm,
                     "hbm_peak_source": "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback"},
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": int(offs[-1]),
                "d2h_bytes_per_step": int(offs[-1]) + n * ctypes.sizeof(sr._Obs)},
        "gpu_launches": int(launches),
        "cpu_baseline": {"value": cpu_com / cpu_wall, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "per_core": cpu_per_core,
                         "sample": f"{len(jobs)} lattices of the batch (3 per side L: coldest, "
                                   "median, hottest), each from t=0 until about 3e6 committed "
                                   "events at its rate in the GPU run (at most t=100), one oracle "
                                   "process per core; committed flips over the wall time"},
        "clocks": _clock_summary(clock_path, local),
        "fg_vs_log_N": fg_rows,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- profiling and reports
def run_profile_case(args):
    """A short slice of the plain workload for profilers: the L=1024 lattice
    from t = 0 through `--windows` windows of length `--tw` (one persistent
    launch)."""
    import torch

    import paper_cs_0405053_gb300 as sr
    torch.cuda.set_device(0)
    lat = sr.Lattice(PLAIN_L, 1.0, PLAIN_W, PLAIN_H, (16, 16), seed=1, lanes_per_region=args.lpr,
                     lanes_per_warp=args.lpw, time_arith=args.arith, replay_records=args.replay,
                     schedule=args.schedule)
    for _ in range(args.warmup):
        lat.reset()
        lat.run_windows(args.tw, args.windows)
    lat.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.run_windows(args.tw, args.windows)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    o = lat.observables()
    mhz = 2070.0
    print(json.dumps({"profile_case": True, "tw": args.tw, "windows": args.windows,
                      "lanes_per_region": args.lpr, "lanes_per_warp": args.lpw, "arith": args.arith,
                      "replay": args.replay,
                      "blocks": lat.blocks, "ms": dt * 1e3,
                      "committed": o.committed, "generated": o.generated,
                      "iterations": o.iterations, "passes": o.region_passes,
                      "skips": o.region_skips,
                      "busy_ms_mean": o.run_cycles / max(1, o.slots) / mhz / 1e3,
                      "busy_ms_max": o.run_cycles_max / mhz / 1e3, "slots": o.slots}))
    return 0


def run_profile_batch(args):
    """The batched workload for profilers, in a fixed configuration (region
    shape --region, --lpw lanes per warp, --kappa): one untimed step from t = 0
    to t = 1, then `--windows` more time units (one launch per time unit), or
    with --windows 0 one whole step (reset, t = 0 to 100)."""
    import torch

    import paper_cs_0405053_gb300 as sr
    from paper_cs_0405053_gb300 import workloads
    torch.cuda.set_device(0)
    reps = workloads.batch_replicas()
    region = tuple(int(v) for v in args.region.split("x"))
    lpw, kappa = args.lpw, args.kappa
    if args.tune_in:
        with open(args.tune_in) as fh:
            t = json.load(fh)
        reps = [dict(r, region=tuple(s)) for r, s in zip(reps, t["shapes"])]
        lpw, kappa = t["lanes_per_warp"], t["kappa"]
    args.kappa = kappa
    bt = sr.Batch(reps, region=region, lanes_per_warp=lpw, schedule=args.schedule)
    bt.run_adaptive(1.0, kappa=args.kappa)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.windows > 0:
        bt.run_adaptive(1.0 + args.windows, kappa=args.kappa)
    else:
        bt.reset()
        bt.run_adaptive(T_END, kappa=args.kappa)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    obs = [bt.observables(b) for b in range(len(reps))]
    com = sum(o.committed for o in obs)
    gen = sum(o.generated for o in obs)
    print(json.dumps({"profile_batch": True, "chunks": args.windows, "s": dt,
                      "committed_total": com, "generated_total": gen,
                      "flips_per_s": com / dt, "launches": obs[0].launches,
                      "relax_launches": obs[0].relax_launches, "relax_ms": obs[0].relax_ms,
                      "blocks": bt.blocks, "region_slots_per_block": bt.threads_per_block,
                      "region": list(region), "lanes_per_warp": lpw, "kappa": kappa,
                      "tune_in": args.tune_in}))
    return 0


def run_scale(args):
    """The plain method at scale: L = 8192 in 256 x 256 regions of 32 x 32, J = 1,
    h = 0, for T in {1.0, 2.269, 3.5} x initial spins {all +1, fair coin} x
    window length in {0.1, 1, 10}, each run from t = 0 to t = args.scale_t
    (50 in the statement).  One line per run: committed flips per second,
    wasted-event ratio and iterations per window."""
    import torch

    import paper_cs_0405053_gb300 as sr
    torch.cuda.set_device(0)
    rows = []
    for T in (1.0, 2.269, 3.5):
        for init in ("up", "fair"):
            for Tw in (0.1, 1.0, 10.0):
                n = max(1, int(round(args.scale_t / Tw)))
                lat = sr.Lattice(8192, 1.0, 0.0, T, (32, 32), seed=1, init=init)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lat.run_windows(Tw, n)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                o = lat.observables()
                it = lat.window_iters(n)
                rows.append({"T": T, "init": init, "Tw": Tw, "windows": n, "s": round(dt, 3),
                             "committed": o.committed, "flips_per_s": o.committed / dt,
                             "wasted_ratio": (o.generated - o.committed) / max(1, o.committed),
                             "iters_mean": float(it.mean()) if len(it) else None,
                             "iters_max": int(it.max()) if len(it) else None,
                             "max_f": o.max_f, "capacity": o.capacity, "m": o.m})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
                lat.close()
    print(json.dumps({"scale": "L=8192, 256x256 regions of 32x32, J=1, h=0, to t=%g" % args.scale_t,
                      "rows": rows}), flush=True)
    return 0


def fluctuation_check(beta, L, ms, fd):
    """The fluctuation relation d<m>/dh = beta N Var(m), N = L^2, in
    equilibrium: Var(m) of the instantaneous m over independent replicas at
    each sample time, averaged over the times (ms [R, times]); its standard
    error by the jackknife over replicas; against the finite differences fd
    [R] of the time-averaged m.  Returns the comparison as a dict."""
    import numpy as np
    R = ms.shape[0]
    var = float(ms.var(axis=0, ddof=1).mean())
    jack = np.array([np.delete(ms, i, axis=0).var(axis=0, ddof=1).mean() for i in range(R)])
    se_var = math.sqrt((R - 1) / R * float(((jack - jack.mean()) ** 2).sum()))
    rel, se_rel = beta * L * L * var, beta * L * L * se_var
    fd_mean, fd_se = float(fd.mean()), float(fd.std(ddof=1) / math.sqrt(R))
    return {"beta_N_var_m": rel, "beta_N_var_m_se": se_rel, "fd_dm_dh": fd_mean, "fd_se": fd_se,
            "ratio": rel / fd_mean if fd_mean else None,
            "z": (fd_mean - rel) / math.hypot(fd_se, se_rel) if (fd_se or se_rel) else None}


def run_grad(args):
    """Gradients of time-averaged m and energy per site with respect to
    (beta, h, J) by the score function (autograd backward through the
    library's kernel), against common-random-number central differences
    (Delta = 1e-3) and, where the chain is in equilibrium above Tc, the
    fluctuation relation dm/dh = beta N Var(m).  Scale "full": 128 replicas
    of L = 512, t in [50, 200]; "small": 64 replicas of L = 128, t in [10, 40]."""
    import numpy as np
    import torch

    from paper_cs_0405053_gb300 import grad
    torch.cuda.set_device(0)
    full = args.grad == "full"
    R, Ls, t1, t2 = (128, 512, 50.0, 200.0) if full else (64, 128, 10.0, 40.0)
    out = []
    for T, h in [(1.8, 0.0), (1.8, 0.05), (2.269, 0.0), (2.269, 0.05), (2.8, 0.0), (2.8, 0.05)]:
        beta = 1.0 / T
        spec = grad.AverageSpec(L=[Ls] * R, seeds=list(range(7000, 7000 + R)), t1=t1, t2=t2,
                                init="up" if T < 2.269 else "fair")
        theta = torch.tensor([[beta, h, 1.0]] * R, dtype=torch.float64, device="cuda",
                             requires_grad=True)
        w0 = time.perf_counter()
        A = grad.time_averages(theta, spec)
        fwd_s = time.perf_counter() - w0
        row = {"T": T, "h": h, "init": spec.init, "forward_s": round(fwd_s, 3)}
        fd_dmdh = None
        # the common-random-number runs at theta +- Delta e_q, shared by both outputs
        sims = []
        for q in range(3):
            tp, tm = theta.detach().clone(), theta.detach().clone()
            tp[:, q] += 1e-3
            tm[:, q] -= 1e-3
            sims.append((grad._simulate(tp.cpu().numpy(), spec)[0],
                         grad._simulate(tm.cpu().numpy(), spec)[0]))
        row["fd_s"] = round(time.perf_counter() - w0 - fwd_s, 3)
        for j, name in enumerate(("m", "e")):
            theta.grad = None
            A[:, j].sum().backward(retain_graph=True)
            g = theta.grad.detach().cpu().numpy()
            est, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(R)
            fds, fdse = [], []
            for q in range(3):
                ap, am = sims[q][0][:, j], sims[q][1][:, j]
                fd = (ap - am) / 2e-3
                if (j, q) == (0, 1):
                    fd_dmdh = fd
                fds.append(float(fd.mean()))
                fdse.append(float(fd.std(ddof=1) / math.sqrt(R)))
            row[f"d{name}"] = {
                "score": [float(v) for v in est], "score_se": [float(v) for v in se],
                "fd": fds, "fd_se": fdse,
                "z": [float((est[q] - fds[q]) / math.hypot(se[q], fdse[q])) for q in range(3)]}
        if T > 2.269:          # equilibrium above Tc: the fluctuation relation of m
            _, _, _, ms = grad._simulate(theta.detach().cpu().numpy(), spec, samples=30)
            row["fluctuation"] = fluctuation_check(beta, Ls, ms, fd_dmdh)
        out.append(row)
    zs = [abs(z) for r in out for k in ("dm", "de") for z in r[k]["z"]]
    print(json.dumps({"grad": args.grad, "replicas": R, "L": Ls, "t": [t1, t2],
                      "params": "theta = (beta, h, J); d/d theta of the time averages of m and "
                                "energy per site", "max_abs_z": max(zs), "rows": out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only a short slice of the plain workload (for ncu)")
    ap.add_argument("--tw", type=float, default=1.0)
    ap.add_argument("--windows", type=int, default=5)
    ap.add_argument("--lpr", type=int, default=0,
                    help="lanes per region: 1, 32 or 0 (automatic)")
    ap.add_argument("--lpw", type=int, default=0, help="region lanes per warp (lane mapping)")
    ap.add_argument("--arith", type=int, default=0, help="time arithmetic: 1 FP64, 2 integer")
    ap.add_argument("--schedule", type=int, default=0,
                    help="profile cases: 0 automatic, 1 static, 2 dynamic, 3 asynchronous")
    ap.add_argument("--region", default="32x16", help="profile-batch: region shape WxH")
    ap.add_argument("--kappa", type=float, default=8.0, help="profile-batch: events per window")
    ap.add_argument("--tune-out", default=None, help="write the autotuner's choice to this file")
    ap.add_argument("--tune-in", default=None,
                    help="profile-batch: region shapes, lanes per warp and kappa from this file")
    ap.add_argument("--replay", type=int, default=0,
                    help="checkpoint records per region for incremental replay (0 auto, -1 off)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run only a slice of the batched workload (for ncu)")
    ap.add_argument("--grad", choices=["small", "full"], default=None,
                    help="gradient check of the score-function backward (separate report)")
    ap.add_argument("--scale", action="store_true",
                    help="the L = 8192 runs of the plain method at scale (separate report)")
    ap.add_argument("--scale-t", type=float, default=50.0)
    args = ap.parse_args()
    if args.scale:
        return run_scale(args)
    if args.grad:
        return run_grad(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
