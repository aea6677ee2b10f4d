"""Benchmark: committed spin flips per second of the synchronous-relaxation
n-fold-way Ising simulation on GB300.

Workload (one "step" = the whole hot path over the lattice, for each window
length): L = 1024 periodic 2D Ising, 64 x 64 regions of 16 x 16, J = 1,
h = 0.05, T = 1.0, fair-coin initial spins from the seed; for each window
length Tw in {0.25, 1, 4}: initialise (spins, class counts, first waiting
times), run synchronous relaxation windows to t = 100, reduce the observables.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 is launched with torch.distributed.run: each rank simulates its own
replica (seed 1 + rank) on its own GPU, with no data exchange ("scaling":
"weak"); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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
L, RW, RH, J, H_FIELD, TEMP, T_END = 1024, 16, 16, 1.0, 0.05, 1.0, 100.0
WINDOWS = (0.25, 1.0, 4.0)
WORKLOAD = ("L=1024 periodic 2D Ising, 64x64 regions of 16x16, J=1, h=0.05, T=1.0, fair-coin "
            "spins, Metropolis rates via the n-fold way, run to t=100 for each window length "
            "Tw in {0.25, 1, 4}")

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
# History bytes per committed boundary event: f64 time + u8 position, written
# once and read by one neighbour (two for a corner); the HBM bound uses the
# measured copy bandwidth of this part.
HIST_BYTES_PER_BOUNDARY_EVENT = 9 * 2
HBM_GBS = 6788.3
# DRAM bytes (read + write) of one relaxation launch of each window length,
# from one ncu capture of the full launch on a GB300:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
#       --clock-control none -k regex:relax_kernel -s 3 -c 1 \
#       python bench.py --profile-case --tw TW --windows 100/TW
# valid only for the kernel sources they were taken on (hash below; carried
# over host-only changes to sr_lib.cu and sr.h -- the checkpoint calls, the
# wording of the timeout -- with identical resource usage reported by ptxas
# for every kernel)
TRAFFIC_BYTES = {0.25: 3482112 + 4785152, 1.0: 27091456 + 77085440, 4.0: 408394496 + 842041600}
TRAFFIC_SOURCES_SHA = "6b70cf6667816189"


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


def replica_seed(rank):
    """Seed of the lattice simulated by a rank (each rank its own replica)."""
    return 1 + rank


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


def _oracle_baseline(Tw=1.0):
    """The oracle (plain sequential C) on the workload for one window length:
    the lattice to t = 100 with window ends every Tw."""
    import oracle
    oracle.build()
    n = int(round(T_END / Tw))
    ends, t = [], 0.0
    for _ in range(n):
        t = t + Tw
        ends.append(t)
    t0 = time.perf_counter()
    r = oracle.run(L, J, H_FIELD, TEMP, RW, RH, 1, ends, keep_spins=False)
    dt = time.perf_counter() - t0
    committed = int(r.counts[-1].sum())
    return committed, dt


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        _oracle_baseline(WINDOWS[0])
    times, committed = [], 0
    for _ in range(args.steps):
        step_t = 0.0
        for Tw in WINDOWS:                     # one oracle run per window length, as a step
            c, dt = _oracle_baseline(Tw)
            committed += c
            step_t += dt
        times.append(step_t)
    total = sum(times)
    value = committed / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "the full workload: per step one oracle run to t=100 for each "
                                   "window length (0.25, 1, 4), every committed flip counted once"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _batched_vs_plain(args, sr, torch, stream):
    """The batched workload: 256 independent lattices (L uniform over
    {64 .. 1024}, T uniform in [1, 3.5], h uniform in [-0.2, 0.2], J = 1,
    fair-coin spins) run to t = args.batch_t in one context, with the region
    shape, lanes per warp and events per window chosen by the autotuner and
    window lengths matched to each lattice's event rate; against the same
    lattices run one per context (a stratified sample of every 8th lattice)."""
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas()
    t0 = time.perf_counter()
    tune = sr.autotune(reps, t_trial=1.0)
    tune_s = time.perf_counter() - t0
    t_end = float(args.batch_t)

    def timed(b, lpw):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        ev0.record(stream)
        b.run_adaptive(t_end, kappa=tune.kappa)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        obs = [b.observables(k) for k in range(len(b))]
        return ev0.elapsed_time(ev1) * 1e-3, wall, obs

    bt = sr.Batch(reps, region=tune.region, lanes_per_warp=tune.lanes_per_warp)
    bt.run_adaptive(min(1.0, t_end), kappa=tune.kappa)      # warm-up
    bt.reset()
    clock_path = os.path.join(tempfile.gettempdir(), f"sr_clocks_batch_{os.getpid()}.csv")
    sampler = _clock_sampler(clock_path)
    time.sleep(0.3 if sampler else 0)
    dev_s, wall_s, obs = timed(bt, tune.lanes_per_warp)
    if sampler:
        sampler.terminate()
        sampler.wait()
    committed = sum(o.committed for o in obs)
    generated = sum(o.generated for o in obs)
    iters = sum(o.iterations for o in obs) / max(1, sum(o.windows for o in obs))
    launches = obs[0].launches
    bt.close()
    batched = committed / dev_s

    sample = list(range(0, len(reps), 8))
    p_com, p_s = 0, 0.0
    for k in sample:
        one = sr.Batch([reps[k]], region=tune.region)
        d, _, o = timed(one, 0)
        p_com += o[0].committed
        p_s += d
        one.close()
    plain = p_com / p_s
    ops = committed * OPS_PER_EVENT / dev_s
    return {
        "workload": "256 lattices: L uniform over {64,128,256,512,1024}, T uniform in [1,3.5], "
                    "h uniform in [-0.2,0.2], J=1, fair-coin spins, Metropolis, run to "
                    f"t={t_end:g} each (numpy Philox key 4, seeds 1000+b)",
        "sites": int(sum(r["L"] ** 2 for r in reps)),
        "tuning": {"region": list(tune.region), "lanes_per_warp": tune.lanes_per_warp or "auto",
                   "kappa": tune.kappa, "trials": tune.trials, "seconds": round(tune_s, 2)},
        "batched": {"flips_per_s": batched, "s": dev_s, "wall_s": wall_s, "committed": committed,
                    "generated": generated, "wasted_ratio": (generated - committed) / committed,
                    "iters_mean": iters, "launches": launches},
        "one_by_one": {"flips_per_s": plain, "s": p_s, "committed": p_com,
                       "sample": f"every 8th lattice ({len(sample)} of {len(reps)}), each in its "
                                 "own context with the same shape and window rule"},
        "batched_over_one_by_one": batched / plain,
        "clocks": _clock_summary(clock_path, torch.cuda.current_device()),
        "roofline": {"bound": "alu", "achieved": ops / 1e12, "peak": INT_PEAK_OPS / 1e12,
                     "unit": "Tops/s", "frac": ops / INT_PEAK_OPS},
    }


def _fg_vs_log_n(sr):
    """f and g of §6 versus log N: L = 64 .. 2048 in 16x16 regions (N = 16 ..
    16384), T = 3.0, h = 0, T_max = log N / (lambda |boundary|) (Eq. 5.1,
    lambda = 1, 60 boundary sites); 20 windows of warm-up, 60 measured."""
    rows = []
    for L in (64, 128, 256, 512, 1024, 2048):
        N = (L // RW) ** 2
        Tw = math.log(N) / 60.0
        lat = sr.Lattice(L, 1.0, 0.0, 3.0, (RW, RH), seed=7)
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

    rank, world, local = _dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    seed = replica_seed(rank)
    stream = torch.cuda.current_stream()
    lat = sr.Lattice(L, J, H_FIELD, TEMP, (RW, RH), seed=seed, lanes_per_region=args.lpr,
                     lanes_per_warp=args.lpw, time_arith=args.arith)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def one_pass(record):
        """One step: for each window length, init + windows to t=100 + observables."""
        out = []
        for Tw in WINDOWS:
            n = int(round(T_END / Tw))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            lat.reset()
            ev[1].record(stream)
            lat.run_windows(Tw, n)
            ev[2].record(stream)
            obs = lat.observables()
            ev[3].record(stream)
            out.append((Tw, ev, obs, lat.window_iters(n)))
        return out

    for _ in range(args.warmup):
        one_pass(False)
    torch.cuda.synchronize()

    clock_path = os.path.join(tempfile.gettempdir(), f"sr_clocks_{os.getpid()}.csv")
    sampler = _clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    step_ms, kernel_ms, per_tw = [], [], {Tw: [] for Tw in WINDOWS}
    committed_total = 0
    launches0 = lat.observables().launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                         # L2 flush between timed steps (outside the events)
        res = one_pass(True)
        torch.cuda.synchronize()
        ms = 0.0
        for Tw, ev, obs, iters in res:
            ms += ev[0].elapsed_time(ev[3])
            kernel_ms.append(ev[1].elapsed_time(ev[2]))
            committed_total += obs.committed          # counters restart at each reset
            launches_last = obs.launches
            per_tw[Tw].append((ev[0].elapsed_time(ev[3]), ev[1].elapsed_time(ev[2]), obs, iters))
        step_ms.append(ms)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    launches = launches_last - launches0
    if sampler:
        sampler.terminate()
        sampler.wait()
    total_ms = sum(step_ms)
    t_max, value = job_throughput(dist, total_ms / 1e3, committed_total, "cuda")

    # ---- end to end through the public API with host buffers: upload the
    # initial spins from pinned memory, run, read back observables and spins
    rng = np.random.default_rng(1000 + rank)
    init_host = torch.from_numpy(np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)).pin_memory()
    out_host = torch.empty((L, L), dtype=torch.int8).pin_memory()
    e2e_lat = sr.Lattice(L, J, H_FIELD, TEMP, (RW, RH), seed=seed, lanes_per_region=args.lpr,
                         lanes_per_warp=args.lpw, time_arith=args.arith)
    e2e_committed, e2e_time = 0, 0.0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        c_step = 0
        for Tw in WINDOWS:
            e2e_lat.set_spins(init_host.numpy())
            e2e_lat.run_windows(Tw, int(round(T_END / Tw)))
            o = e2e_lat.observables()
            sr.library().sr_get_spins(e2e_lat._ctx, out_host.data_ptr(), L * L)
            c_step += o.committed
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_committed += c_step
            e2e_time += dt
    e2e_lat.close()
    e2e_value = e2e_committed / e2e_time if e2e_time > 0 else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (the persistent relaxation kernel):
    # algorithmic integer work of the committed trajectory per launch / launch time
    kms = sum(kernel_ms) / len(kernel_ms)
    last = {Tw: per_tw[Tw][-1] for Tw in WINDOWS}
    ev_per_launch = statistics.mean(o.committed for (_, _, o, _) in (last[t] for t in WINDOWS))
    ops = ev_per_launch * OPS_PER_EVENT
    achieved = ops / (kms * 1e-3)
    peak = INT_PEAK_OPS
    # the other bound of the statement: boundary history bytes at HBM bandwidth
    # (boundary fraction of 16x16 regions at uniform rates, 60/256)
    hbm_bound_events = HBM_GBS * 1e9 / (HIST_BYTES_PER_BOUNDARY_EVENT * 60 / 256)
    cpu_committed, cpu_dt = _oracle_baseline()
    batch_info = None if args.no_batch else _batched_vs_plain(args, sr, torch, stream)
    fg_rows = None if args.no_batch else _fg_vs_log_n(sr)
    tw_detail = {}
    for Tw in WINDOWS:
        ms, kms_tw, o, iters = per_tw[Tw][-1]
        it = [int(v) for v in iters]
        tw_detail[str(Tw)] = {
            "ms": round(ms, 3), "kernel_ms": round(kms_tw, 3), "committed": o.committed,
            "generated": o.generated, "wasted_ratio": (o.generated - o.committed) / max(1, o.committed),
            "iters_mean": statistics.mean(it) if it else None, "iters_max": max(it) if it else None,
            "windows": len(it), "max_f": o.max_f, "breaks": o.breaks,
            "flips_per_s": o.committed / (ms * 1e-3)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded fair-coin lattice)",
        "config": {"workload": WORKLOAD, "regions": lat.n_regions,
                   "launch": {"region_slots_per_block": lat.threads_per_block, "blocks": lat.blocks,
                              "lanes_per_region": args.lpr or "auto"},
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "per_window_length": tw_detail},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "Tops/s", "frac": achieved / peak,
                     "traffic": (statistics.mean(TRAFFIC_BYTES[t] for t in WINDOWS)
                                 if _kernel_sources_sha() == TRAFFIC_SOURCES_SHA else None),
                     "traffic_unit": "bytes per launch (DRAM read + write, mean over the "
                                     "three window lengths; ncu)",
                     "peak_source": "derived: 152 SMs x 128 lanes x 2070 MHz integer issue",
                     "kernel": "relax_kernel", "kernel_ms_avg": kms,
                     "ops_per_committed_event": OPS_PER_EVENT,
                     "events_per_s_bounds": {"integer_issue": peak / OPS_PER_EVENT,
                                             "history_bytes_at_hbm": hbm_bound_events}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": L * L * len(WINDOWS),
                "d2h_bytes_per_step": (L * L + 64) * len(WINDOWS)},
        "gpu_launches": launches,
        "cpu_baseline": {"value": cpu_committed / cpu_dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one oracle run of the full workload to t=100 (window "
                                   "length 1); committed flips over its run time"},
        "clocks": _clock_summary(clock_path, local),
        "batched": batch_info,
        "fg_vs_log_N": fg_rows,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A short slice of the workload for profilers: the L=1024 lattice from
    t = 0 through `--windows` windows of length `--tw` (one persistent launch)."""
    import torch

    import paper_cs_0405053_gb300 as sr
    torch.cuda.set_device(0)
    lat = sr.Lattice(L, J, H_FIELD, TEMP, (RW, RH), seed=1, lanes_per_region=args.lpr,
                     lanes_per_warp=args.lpw, time_arith=args.arith, replay_records=args.replay,
                     schedule=args.schedule)
    t0 = None
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
    """A short slice of the batched workload for profilers: the 256 lattices
    in 32x16 regions (32 region lanes per warp, 16 events per window target),
    one chunk [0, 1) untimed, then `--windows` chunks of one time unit, each
    chunk one persistent launch."""
    import torch

    import paper_cs_0405053_gb300 as sr
    from paper_cs_0405053_gb300 import workloads
    torch.cuda.set_device(0)
    reps = workloads.batch_replicas()
    bt = sr.Batch(reps, region=(32, 16), lanes_per_warp=32, schedule=args.schedule)
    bt.run_adaptive(1.0, kappa=16.0, chunk=1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt.run_adaptive(1.0 + args.windows, kappa=16.0, chunk=1.0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    obs = [bt.observables(b) for b in range(len(reps))]
    com = sum(o.committed for o in obs)
    print(json.dumps({"profile_batch": True, "chunks": args.windows, "s": dt,
                      "committed_total": com, "launches": obs[0].launches,
                      "blocks": bt.blocks, "region_slots_per_block": bt.threads_per_block}))
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


def run_grad(args):
    """Gradients of time-averaged m and energy per site with respect to
    (beta, h, J) by the score function (autograd backward through the
    library's kernel), against common-random-number central differences
    (Delta = 1e-3) and, where the chain is in equilibrium, the fluctuation
    relation dm/dh = beta N Var(m).  Scale "full": 128 replicas of L = 512,
    t in [50, 200]; "small": 64 replicas of L = 128, t in [10, 40]."""
    import numpy as np
    import torch

    import paper_cs_0405053_gb300 as sr
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
        for j, name in enumerate(("m", "e")):
            theta.grad = None
            A[:, j].sum().backward(retain_graph=True)
            g = theta.grad.detach().cpu().numpy()
            est, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(R)
            fds, fdse = [], []
            for q in range(3):
                tp, tm = theta.detach().clone(), theta.detach().clone()
                tp[:, q] += 1e-3
                tm[:, q] -= 1e-3
                ap = grad._simulate(tp.cpu().numpy(), spec)[0][:, j]
                am = grad._simulate(tm.cpu().numpy(), spec)[0][:, j]
                fd = (ap - am) / 2e-3
                fds.append(float(fd.mean()))
                fdse.append(float(fd.std(ddof=1) / math.sqrt(R)))
            row[f"d{name}"] = {
                "score": [float(v) for v in est], "score_se": [float(v) for v in se],
                "fd": fds, "fd_se": fdse,
                "z": [float((est[q] - fds[q]) / math.hypot(se[q], fdse[q])) for q in range(3)]}
        if T != 2.269:          # equilibrium: the fluctuation relation of the magnetisation
            _, _, _, ms = grad._simulate(theta.detach().cpu().numpy(), spec, samples=30)
            # variance over independent replicas at each sample time, averaged
            row["beta_N_var_m"] = float(beta * Ls * Ls * ms.var(axis=0, ddof=1).mean())
        out.append(row)
    print(json.dumps({"grad": args.grad, "replicas": R, "L": Ls, "t": [t1, t2],
                      "params": "theta = (beta, h, J); d/d theta of the time averages of m and "
                                "energy per site", "rows": out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-case", action="store_true",
                    help="run only a short slice of the workload (for ncu)")
    ap.add_argument("--tw", type=float, default=1.0)
    ap.add_argument("--windows", type=int, default=5)
    ap.add_argument("--lpr", type=int, default=0,
                    help="lanes per region: 1, 32 or 0 (automatic)")
    ap.add_argument("--lpw", type=int, default=0, help="region lanes per warp (lane mapping)")
    ap.add_argument("--arith", type=int, default=0, help="time arithmetic: 1 FP64, 2 integer")
    ap.add_argument("--schedule", type=int, default=0,
                    help="profile cases: 0 automatic, 1 static, 2 dynamic, 3 asynchronous")
    ap.add_argument("--batch-t", type=float, default=100.0,
                    help="simulated time of the batched section")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched section")
    ap.add_argument("--replay", type=int, default=0,
                    help="checkpoint records per region for incremental replay (0 auto, -1 off)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run only a short slice of the batched workload (for ncu)")
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
