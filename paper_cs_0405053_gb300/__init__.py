"""GB300 (sm_103a) synchronous relaxation of the continuous-time n-fold-way
Ising simulation (Lubachevsky & Weiss, "Synchronous Relaxation for Parallel
Ising Spin Simulations").

This module is a thin ctypes binding of ``libsr`` (C ABI in ``include/sr.h``);
every step of the simulation runs in the library's CUDA kernels.  PyTorch, when
present, only supplies the CUDA stream and device buffers.  There is no CPU
fallback: without the compiled library or a GPU every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

from . import _build

__all__ = ["SRError", "Lattice", "Batch", "Replica", "Observables", "Tuning", "autotune",
           "library", "eval_draws", "SR_OK"]

SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA = 0, -1, -2, -3
SR_NOT_CONVERGED, SR_CAPACITY, SR_TIMEOUT, SR_EUNSUPPORTED = -4, -5, -6, -7
INIT_MODES = {"fair": 0, "up": 1, "down": 2}
RATES = {"metropolis": 0, "glauber": 1}


class SRError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {library().sr_strerror(code).decode()} ({code})")


class _Params(C.Structure):
    _fields_ = [("L", C.c_int), ("J", C.c_double), ("h", C.c_double), ("T", C.c_double),
                ("region_w", C.c_int), ("region_h", C.c_int), ("seed", C.c_uint64),
                ("init_mode", C.c_int), ("rates", C.c_int), ("capacity", C.c_int),
                ("max_iters", C.c_int), ("trace_capacity", C.c_int),
                ("lanes_per_region", C.c_int), ("lanes_per_warp", C.c_int), ("time_arith", C.c_int),
                ("threads_per_block", C.c_int), ("blocks", C.c_int),
                ("barrier_timeout_ms", C.c_int), ("replay_records", C.c_int),
                ("fresh_steps", C.c_int), ("score", C.c_int), ("schedule", C.c_int),
                ("test_barrier_skip_block", C.c_int),
                ("stream", C.c_void_p)]


class _Replica(C.Structure):
    _fields_ = [("L", C.c_int), ("J", C.c_double), ("h", C.c_double), ("T", C.c_double),
                ("seed", C.c_uint64), ("init_mode", C.c_int), ("rates", C.c_int),
                ("region_w", C.c_int), ("region_h", C.c_int)]


@dataclass
class Replica:
    """One lattice of a Batch; region = None takes the batch's region shape."""
    L: int
    J: float = 1.0
    h: float = 0.0
    T: float = 1.0
    seed: int = 1
    init: str = "fair"
    rates: str = "metropolis"
    region: Optional[Tuple[int, int]] = None


class _Adapt(C.Structure):
    _fields_ = [("kappa", C.c_double), ("chunk", C.c_double), ("tw_first", C.c_double),
                ("tw_min", C.c_double), ("tw_max", C.c_double)]


class _Tune(C.Structure):
    _fields_ = [("region_w", C.c_int), ("region_h", C.c_int), ("lanes_per_warp", C.c_int),
                ("kappa", C.c_double), ("flips_per_s", C.c_double), ("trials", C.c_int),
                ("rate_threshold", C.c_double)]


class _Obs(C.Structure):
    _fields_ = [("t_c", C.c_double), ("mag", C.c_int64), ("bonds", C.c_int64), ("m", C.c_double),
                ("E", C.c_double), ("int_mag", C.c_double), ("int_bonds", C.c_double),
                ("committed", C.c_uint64), ("generated", C.c_uint64), ("breaks", C.c_uint64),
                ("windows", C.c_uint64), ("iterations", C.c_uint64), ("sum_f", C.c_uint64),
                ("last_iters", C.c_uint32),
                ("max_iters_seen", C.c_uint32), ("max_f", C.c_uint32), ("capacity", C.c_uint32),
                ("launches", C.c_uint64), ("region_passes", C.c_uint64),
                ("region_skips", C.c_uint64), ("run_cycles", C.c_uint64),
                ("run_cycles_max", C.c_uint64), ("slots", C.c_uint64),
                ("relax_ms", C.c_double), ("relax_launches", C.c_uint64)]


@dataclass
class Observables:
    t_c: float
    mag: int
    bonds: int
    m: float
    E: float
    int_mag: float
    int_bonds: float
    committed: int
    generated: int
    breaks: int
    windows: int
    iterations: int
    sum_f: int
    last_iters: int
    max_iters_seen: int
    max_f: int
    capacity: int
    launches: int
    region_passes: int
    region_skips: int
    run_cycles: int
    run_cycles_max: int
    slots: int
    relax_ms: float
    relax_launches: int


_lib = None
_P = C.c_void_p


def library(build_if_missing: bool = True) -> C.CDLL:
    """Load libsr (building it in-tree first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(path):
            raise OSError(f"libsr is not built: {path} is missing (run __graft_entry__.build())")
        lib = C.CDLL(path)
        sig = {
            "sr_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_uint64]),
            "sr_create_ex": (C.c_int, [C.POINTER(_P), C.POINTER(_Params)]),
            "sr_run_window": (C.c_int, [_P, C.c_double, C.c_double]),
            "sr_run_windows": (C.c_int, [_P, C.c_double, C.c_double, C.c_int]),
            "sr_observables": (C.c_int, [_P, C.POINTER(_Obs)]),
            "sr_destroy": (None, [_P]),
            "sr_get_spins": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_get_spins_device": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_set_spins": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_set_spins_device": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_reset": (C.c_int, [_P]),
            "sr_get_carry": (C.c_int, [_P, _P, _P, _P, _P, C.c_size_t]),
            "sr_get_trace": (C.c_int, [_P, _P, _P, _P, C.c_size_t, C.c_size_t]),
            "sr_get_window_iters": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_get_window_f": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_eval_draws": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint64, C.c_size_t, _P, _P]),
            "sr_get_info": (C.c_int, [_P, _P, _P, _P, _P, _P]),
            "sr_eval_softfloat": (C.c_int, [C.c_int, _P, _P, _P, C.c_size_t]),
            "sr_strerror": (C.c_char_p, [C.c_int]),
            "sr_create_batch": (C.c_int, [C.POINTER(_P), _P, C.c_int, C.POINTER(_Params)]),
            "sr_run_batch": (C.c_int, [_P, _P, _P]),
            "sr_set_graph_launch": (C.c_int, [_P, C.c_int]),
            "sr_get_graph_stats": (C.c_int, [_P, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
            "sr_observables_replica": (C.c_int, [_P, C.c_int, C.POINTER(_Obs)]),
            "sr_get_spins_replica": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
            "sr_set_spins_replica": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
            "sr_get_carry_replica": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_size_t]),
            "sr_run_batch_adaptive": (C.c_int, [_P, _P, C.POINTER(_Adapt), _P]),
            "sr_score": (C.c_int, [_P, _P]),
            "sr_score_stats": (C.c_int, [_P, C.c_int, _P, _P]),
            "sr_score_grad": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P]),
            "sr_autotune": (C.c_int, [_P, C.c_int, C.POINTER(_Params), C.c_double,
                                      C.POINTER(_Tune), _P]),
            "sr_checkpoint_size": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
            "sr_checkpoint_save": (C.c_int, [_P, _P, C.c_size_t]),
            "sr_checkpoint_load": (C.c_int, [_P, C.c_char_p, C.c_size_t]),
            "sr_run_noalloc": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                         C.c_int, C.c_uint64, _P, C.c_double, C.c_int, _P, _P,
                                         _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _checkpoint(ctx) -> bytes:
    lib = library()
    n = C.c_size_t()
    _check(lib.sr_checkpoint_size(ctx, C.byref(n)), "sr_checkpoint_size")
    buf = C.create_string_buffer(n.value)
    _check(lib.sr_checkpoint_save(ctx, buf, n.value), "sr_checkpoint_save")
    return buf.raw


def _load_checkpoint(ctx, data: bytes) -> None:
    data = bytes(data)
    _check(library().sr_checkpoint_load(ctx, data, len(data)), "sr_checkpoint_load")


def _graph_launch(ctx, on: bool) -> None:
    _check(library().sr_set_graph_launch(ctx, 1 if on else 0), "sr_set_graph_launch")


def _graph_stats(ctx) -> Tuple[int, int]:
    cap, rep = C.c_ulonglong(), C.c_ulonglong()
    _check(library().sr_get_graph_stats(ctx, C.byref(cap), C.byref(rep)), "sr_get_graph_stats")
    return cap.value, rep.value


def _check(code: int, what: str) -> None:
    if code != SR_OK:
        raise SRError(code, what)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _torch_stream():
    try:
        import torch
    except ImportError:       # the library creates its own stream
        return None
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream().cuda_stream


def eval_draws(seed: int, region: int, i0: int, n: int) -> Tuple[np.ndarray, np.ndarray]:
    """(x = -log U_i, kV_i) for events i0 .. i0+n-1 of a region, on the GPU."""
    x = np.zeros(n, dtype=np.float64)
    kv = np.zeros(n, dtype=np.uint64)
    _check(library().sr_eval_draws(seed, region, i0, n, _ptr(x), _ptr(kv)), "sr_eval_draws")
    return x, kv


def eval_softfloat(op: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The integer-emulated double operation `op` of the event loop, on the GPU."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros_like(a)
    _check(library().sr_eval_softfloat(op, _ptr(a), _ptr(b), _ptr(out), a.size), "sr_eval_softfloat")
    return out


class Lattice:
    """One L x L periodic lattice split into region_w x region_h regions."""

    def __init__(self, L: int, J: float = 1.0, h: float = 0.0, T: float = 1.0,
                 region: Tuple[int, int] = (16, 16), seed: int = 1, init: str = "fair",
                 rates: str = "metropolis", capacity: int = 0, max_iters: int = 0,
                 trace_capacity: int = 0, lanes_per_region: int = 0, lanes_per_warp: int = 0,
                 time_arith: int = 0, threads_per_block: int = 0,
                 blocks: int = 0,
                 barrier_timeout_ms: int = 0, replay_records: int = 0,
                 fresh_steps: bool = False, score: bool = False, schedule: int = 0,
                 test_barrier_skip_block: int = -1,
                 stream: Optional[int] = None, use_torch_stream: bool = True):
        lib = library()
        if stream is None and use_torch_stream:
            stream = _torch_stream()
        self.L, self.J, self.h, self.T = L, J, h, T
        self.region = region
        self.seed = seed
        self.trace_capacity = trace_capacity
        prm = _Params(L, J, h, T, region[0], region[1], seed, INIT_MODES[init], RATES[rates],
                      capacity, max_iters, trace_capacity, lanes_per_region, lanes_per_warp,
                      time_arith, threads_per_block, blocks,
                      barrier_timeout_ms, replay_records, int(fresh_steps), int(score),
                      schedule, test_barrier_skip_block, stream)
        self._ctx = _P()
        _check(lib.sr_create_ex(C.byref(self._ctx), C.byref(prm)), "sr_create_ex")
        n_regions = C.c_int()
        frac = C.c_int()
        tpb = C.c_int()
        blk = C.c_int()
        P = np.zeros(10, dtype=np.uint64)
        _check(lib.sr_get_info(self._ctx, C.byref(n_regions), C.byref(frac), _ptr(P), C.byref(tpb),
                               C.byref(blk)), "sr_get_info")
        self.n_regions = n_regions.value
        self.frac_bits = frac.value
        self.P = P
        self.threads_per_block = tpb.value
        self.blocks = blk.value
        self.t_c = 0.0

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_ctx", None):
            library().sr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the method
    def run_window(self, Tw: float) -> None:
        """One synchronous-relaxation step of length Tw from the committed time."""
        code = library().sr_run_window(self._ctx, self.t_c, Tw)
        self.t_c = self.t_c + Tw if code == SR_OK else self.observables().t_c
        _check(code, "sr_run_window")

    def run_windows(self, Tw: float, n: int) -> None:
        code = library().sr_run_windows(self._ctx, self.t_c, Tw, n)
        if code == SR_OK:
            for _ in range(n):
                self.t_c = self.t_c + Tw
        else:
            self.t_c = self.observables().t_c
        _check(code, "sr_run_windows")

    def observables(self) -> Observables:
        o = _Obs()
        _check(library().sr_observables(self._ctx, C.byref(o)), "sr_observables")
        return Observables(*[getattr(o, f) for f, _ in _Obs._fields_])

    def spins(self) -> np.ndarray:
        out = np.zeros((self.L, self.L), dtype=np.int8)
        _check(library().sr_get_spins(self._ctx, _ptr(out), out.size), "sr_get_spins")
        return out

    def spins_into(self, dev_ptr: int) -> None:
        """Unpack the committed spins into a caller-owned device buffer of L*L int8."""
        _check(library().sr_get_spins_device(self._ctx, dev_ptr, self.L * self.L),
               "sr_get_spins_device")

    def set_spins(self, spins: np.ndarray) -> None:
        a = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        _check(library().sr_set_spins(self._ctx, _ptr(a), a.size), "sr_set_spins")
        self.t_c = 0.0

    def set_spins_from(self, dev_ptr: int) -> None:
        _check(library().sr_set_spins_device(self._ctx, dev_ptr, self.L * self.L),
               "sr_set_spins_device")
        self.t_c = 0.0

    def reset(self) -> None:
        _check(library().sr_reset(self._ctx), "sr_reset")
        self.t_c = 0.0

    def graph_launch(self, on: bool = True) -> None:
        """Run every later relaxation launch as a replayed CUDA graph (see
        sr_set_graph_launch); off frees the graph."""
        _graph_launch(self._ctx, on)

    def graph_stats(self) -> Tuple[int, int]:
        """(graph captures, graph launches) of this context."""
        return _graph_stats(self._ctx)

    def checkpoint(self) -> bytes:
        """The committed state (spins, clock carry, integrals, counters) as
        bytes; load_checkpoint on a context of the same lattice resumes it."""
        return _checkpoint(self._ctx)

    def load_checkpoint(self, data: bytes) -> None:
        _load_checkpoint(self._ctx, data)
        self.t_c = self.observables().t_c

    def carry(self):
        n = self.n_regions
        i = np.zeros(n, dtype=np.uint64)
        x = np.zeros(n, dtype=np.float64)
        b = np.zeros(n, dtype=np.float64)
        t = np.zeros(n, dtype=np.float64)
        _check(library().sr_get_carry(self._ctx, _ptr(i), _ptr(x), _ptr(b), _ptr(t), n),
               "sr_get_carry")
        return i, x, b, t

    def trace(self):
        """(lens[n_regions], times[n_regions, cap], sites[n_regions, cap])."""
        n, cap = self.n_regions, self.trace_capacity
        lens = np.zeros(n, dtype=np.uint64)
        times = np.zeros((n, cap), dtype=np.float64)
        sites = np.zeros((n, cap), dtype=np.uint32)
        _check(library().sr_get_trace(self._ctx, _ptr(lens), _ptr(times), _ptr(sites), n, cap),
               "sr_get_trace")
        return lens, times, sites

    def window_iters(self, n: int = 4096) -> np.ndarray:
        """Iterations g of each of the last n windows of the last run call."""
        out = np.zeros(n, dtype=np.uint32)
        m = library().sr_get_window_iters(self._ctx, _ptr(out), n)
        if m < 0:
            raise SRError(m, "sr_get_window_iters")
        return out[:m]

    def score(self) -> np.ndarray:
        """d log L / d(beta, h, J) of the committed path (score mode)."""
        out = np.zeros(3, dtype=np.float64)
        _check(library().sr_score(self._ctx, _ptr(out)), "sr_score")
        return out

    def score_stats(self):
        """(C_k, I_k): committed events by class and integrals of N_k dt."""
        c = np.zeros(10, dtype=np.uint64)
        occ = np.zeros(10, dtype=np.float64)
        _check(library().sr_score_stats(self._ctx, 0, _ptr(c), _ptr(occ)), "sr_score_stats")
        return c, occ

    def window_f(self, n: int = 4096) -> np.ndarray:
        """f of §6 (most boundary events of a region in an iteration) of each
        of the last n windows of the last run call."""
        out = np.zeros(n, dtype=np.uint32)
        m = library().sr_get_window_f(self._ctx, _ptr(out), n)
        if m < 0:
            raise SRError(m, "sr_get_window_f")
        return out[:m]


def _common_params(region, capacity=0, max_iters=0, lanes_per_region=0, lanes_per_warp=0,
                   time_arith=0, threads_per_block=0, blocks=0, barrier_timeout_ms=0,
                   replay_records=0, stream=None, fresh_steps=False, score=False,
                   schedule=0) -> _Params:
    return _Params(0, 0.0, 0.0, 0.0, region[0], region[1], 0, 0, 0, capacity, max_iters, 0,
                   lanes_per_region, lanes_per_warp, time_arith, threads_per_block, blocks,
                   barrier_timeout_ms, replay_records, int(fresh_steps), int(score), schedule,
                   -1, stream)


def _replica_array(replicas):
    reps = [r if isinstance(r, Replica) else Replica(**r) for r in replicas]
    arr = (_Replica * len(reps))(*[
        _Replica(r.L, r.J, r.h, r.T, r.seed, INIT_MODES[r.init], RATES[r.rates],
                 *(r.region if r.region else (0, 0))) for r in reps])
    return reps, arr


@dataclass
class Tuning:
    """Choice of the autotuner (sr_autotune): a region shape per lattice
    (shapes[b]; region is lattice 0's), lanes per warp and kappa."""
    region: Tuple[int, int]
    lanes_per_warp: int
    kappa: float
    flips_per_s: float
    trials: int
    rate_threshold: float
    shapes: list

    def replicas(self, replicas) -> list:
        """The lattices with their chosen region shapes, for Batch(...)."""
        reps = [r if isinstance(r, Replica) else Replica(**r) for r in replicas]
        return [Replica(r.L, r.J, r.h, r.T, r.seed, r.init, r.rates, tuple(s))
                for r, s in zip(reps, self.shapes)]


def autotune(replicas, t_trial: float = 1.0, **settings) -> Tuning:
    """Region shape, region lanes per warp and events per window for a batch,
    chosen by timing short trial runs of these lattices on the GPU."""
    lib = library()
    _, arr = _replica_array(replicas)
    stream = settings.pop("stream", None)
    if stream is None:
        stream = _torch_stream()
    prm = _common_params((16, 16), stream=stream, **settings)
    t = _Tune()
    wh = np.zeros(2 * len(arr), dtype=np.int32)
    _check(lib.sr_autotune(C.cast(arr, C.c_void_p), len(arr), C.byref(prm), t_trial, C.byref(t),
                           _ptr(wh)), "sr_autotune")
    shapes = [(int(wh[2 * b]), int(wh[2 * b + 1])) for b in range(len(arr))]
    return Tuning((t.region_w, t.region_h), t.lanes_per_warp, t.kappa, t.flips_per_s, t.trials,
                  t.rate_threshold, shapes)


class Batch:
    """Independent lattices simulated together: every lattice follows the
    synchronous-relaxation procedure on its own (own windows, iterations and
    results, the same as a Lattice of its own), while their regions share one
    persistent launch.  All lattices use one region shape."""

    def __init__(self, replicas, region: Tuple[int, int] = (16, 16), capacity: int = 0,
                 max_iters: int = 0, lanes_per_region: int = 0, lanes_per_warp: int = 0,
                 time_arith: int = 0, threads_per_block: int = 0, blocks: int = 0,
                 barrier_timeout_ms: int = 0, replay_records: int = 0,
                 fresh_steps: bool = False, score: bool = False, schedule: int = 0,
                 test_barrier_skip_block: int = -1,
                 stream: Optional[int] = None, use_torch_stream: bool = True):
        lib = library()
        if stream is None and use_torch_stream:
            stream = _torch_stream()
        self.replicas, arr = _replica_array(replicas)
        self.region = region
        prm = _common_params(region, capacity, max_iters, lanes_per_region, lanes_per_warp,
                             time_arith, threads_per_block, blocks, barrier_timeout_ms,
                             replay_records, stream, fresh_steps, score, schedule)
        prm.test_barrier_skip_block = test_barrier_skip_block
        self._arr = arr
        self._ctx = _P()
        _check(lib.sr_create_batch(C.byref(self._ctx), C.cast(arr, C.c_void_p), len(arr),
                                   C.byref(prm)), "sr_create_batch")
        tpb = C.c_int()
        blk = C.c_int()
        _check(lib.sr_get_info(self._ctx, None, None, None, C.byref(tpb), C.byref(blk)),
               "sr_get_info")
        self.threads_per_block = tpb.value
        self.blocks = blk.value
        self.t_c = np.zeros(len(self.replicas), dtype=np.float64)

    def __len__(self) -> int:
        return len(self.replicas)

    def close(self) -> None:
        if getattr(self, "_ctx", None):
            library().sr_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, Tw, n_windows) -> None:
        """n_windows[b] windows of length Tw[b] for every lattice b (scalars
        broadcast), all in one persistent launch."""
        n = len(self.replicas)
        tw = np.ascontiguousarray(np.broadcast_to(np.asarray(Tw, dtype=np.float64), (n,)))
        nw = np.ascontiguousarray(np.broadcast_to(np.asarray(n_windows, dtype=np.int32), (n,)))
        code = library().sr_run_batch(self._ctx, _ptr(tw), _ptr(nw))
        for b in range(n):
            self.t_c[b] = self.observables(b).t_c
        _check(code, "sr_run_batch")

    def run_adaptive(self, t_end, kappa: float = 0.0, chunk: float = 0.0, tw_first: float = 0.0,
                     tw_min: float = 0.0, tw_max: float = 0.0) -> np.ndarray:
        """Advance every lattice to t_end[b] with window lengths matched to its
        event rate; returns each lattice's last window length."""
        n = len(self.replicas)
        te = np.ascontiguousarray(np.broadcast_to(np.asarray(t_end, dtype=np.float64), (n,)))
        last = np.zeros(n, dtype=np.float64)
        o = _Adapt(kappa, chunk, tw_first, tw_min, tw_max)
        code = library().sr_run_batch_adaptive(self._ctx, _ptr(te), C.byref(o), _ptr(last))
        for b in range(n):
            self.t_c[b] = self.observables(b).t_c
        _check(code, "sr_run_batch_adaptive")
        return last

    def reset(self) -> None:
        _check(library().sr_reset(self._ctx), "sr_reset")
        self.t_c[:] = 0.0

    def graph_launch(self, on: bool = True) -> None:
        """Run every later relaxation launch as a replayed CUDA graph (see
        sr_set_graph_launch); off frees the graph."""
        _graph_launch(self._ctx, on)

    def graph_stats(self) -> Tuple[int, int]:
        """(graph captures, graph launches) of this context."""
        return _graph_stats(self._ctx)

    def checkpoint(self) -> bytes:
        """The committed state of every lattice as bytes (see Lattice.checkpoint)."""
        return _checkpoint(self._ctx)

    def load_checkpoint(self, data: bytes) -> None:
        _load_checkpoint(self._ctx, data)
        for b in range(len(self.replicas)):
            self.t_c[b] = self.observables(b).t_c

    def observables(self, b: int) -> Observables:
        o = _Obs()
        _check(library().sr_observables_replica(self._ctx, b, C.byref(o)), "sr_observables_replica")
        return Observables(*[getattr(o, f) for f, _ in _Obs._fields_])

    def spins(self, b: int) -> np.ndarray:
        L = self.replicas[b].L
        out = np.zeros((L, L), dtype=np.int8)
        _check(library().sr_get_spins_replica(self._ctx, b, _ptr(out), out.size),
               "sr_get_spins_replica")
        return out

    def spins_into(self, b: int, host_ptr: int) -> None:
        """Committed spins of lattice b into a caller-owned host buffer of L_b^2 int8."""
        L = self.replicas[b].L
        _check(library().sr_get_spins_replica(self._ctx, b, host_ptr, L * L),
               "sr_get_spins_replica")

    def set_spins(self, b: int, spins) -> None:
        """Restart lattice b alone from the given spins (t_c = 0)."""
        L = self.replicas[b].L
        if isinstance(spins, int):          # a host pointer (e.g. pinned memory)
            ptr = spins
        else:
            a = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
            if a.size != L * L:
                raise ValueError(f"lattice {b} has {L * L} sites, got {a.size}")
            ptr = _ptr(a)
        _check(library().sr_set_spins_replica(self._ctx, b, ptr, L * L), "sr_set_spins_replica")
        self.t_c[b] = 0.0

    def score(self) -> np.ndarray:
        """[n, 3]: d log L / d(beta, h, J) of every lattice's committed path."""
        out = np.zeros((len(self.replicas), 3), dtype=np.float64)
        _check(library().sr_score(self._ctx, _ptr(out)), "sr_score")
        return out

    def score_stats(self, b: int):
        c = np.zeros(10, dtype=np.uint64)
        occ = np.zeros(10, dtype=np.float64)
        _check(library().sr_score_stats(self._ctx, b, _ptr(c), _ptr(occ)), "sr_score_stats")
        return c, occ

    def region_of(self, b: int) -> Tuple[int, int]:
        """The region shape of lattice b."""
        r = self.replicas[b]
        return tuple(r.region) if r.region else tuple(self.region)

    def carry(self, b: int):
        r = self.replicas[b]
        W, H = self.region_of(b)
        n = (r.L // W) * (r.L // H)
        i = np.zeros(n, dtype=np.uint64)
        x = np.zeros(n, dtype=np.float64)
        bb = np.zeros(n, dtype=np.float64)
        t = np.zeros(n, dtype=np.float64)
        _check(library().sr_get_carry_replica(self._ctx, b, _ptr(i), _ptr(x), _ptr(bb), _ptr(t), n),
               "sr_get_carry_replica")
        return i, x, bb, t
