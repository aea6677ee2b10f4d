"""CPU oracle for the synchronous-relaxation n-fold-way Ising simulation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code allowed to import this package.
It loads ``sr_oracle.c`` (plain C, compiled with gcc, no FMA contraction) and
shares nothing with the CUDA library.

Every function follows the paper (Lubachevsky & Weiss):
  * ``philox``       -- the counter-based random numbers that make the
                        "presimulated list" of §4 deterministic;
  * ``neglog_unit``  -- -log U_i of Eq. 3.4;
  * ``rates``        -- p_k of Eqs. 2.2 / 2.3 for the ten classes of §3;
  * ``select``       -- class and site choice of Eqs. 3.5-3.8;
  * ``tau``          -- the waiting time with break points of Eqs. 3.4, 5.2-5.6;
  * ``run``          -- the global time-order simulation whose trajectory the
                        converged relaxation (§4 boxed procedure, §5) must equal.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sr_oracle.c")
_LIB = os.path.join(_HERE, "_sr_oracle.so")

INIT_FAIR_COIN, INIT_ALL_UP, INIT_ALL_DOWN, INIT_GIVEN = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("L", C.c_int), ("J", C.c_double), ("h", C.c_double), ("T", C.c_double),
                ("region_w", C.c_int), ("region_h", C.c_int), ("seed", C.c_uint64),
                ("init_mode", C.c_int), ("glauber", C.c_int), ("debug", C.c_int),
                ("fresh_steps", C.c_int)]


class _Outputs(C.Structure):
    _fields_ = [("spins", C.c_void_p), ("counts", C.c_void_p), ("mag", C.c_void_p),
                ("bonds", C.c_void_p), ("int_mag", C.c_void_p), ("int_bonds", C.c_void_p),
                ("carry_i", C.c_void_p), ("carry_x", C.c_void_p), ("carry_b", C.c_void_p),
                ("carry_t", C.c_void_p),
                ("trace_cap", C.c_int64), ("trace_len", C.c_int64),
                ("tr_region", C.c_void_p), ("tr_index", C.c_void_p), ("tr_time", C.c_void_p),
                ("tr_site", C.c_void_p), ("debug_failures", C.c_int64),
                ("ev_class", C.c_void_p), ("occupancy", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_unit_from_bits.argtypes = [C.c_uint64]
        _lib.orc_unit_from_bits.restype = C.c_double
        _lib.orc_neglog_unit.argtypes = [C.c_uint64]
        _lib.orc_neglog_unit.restype = C.c_double
        _lib.orc_rates.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p]
        _lib.orc_frac_bits.argtypes = [C.c_int]
        _lib.orc_frac_bits.restype = C.c_int
        _lib.orc_rates_fixed.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        _lib.orc_select.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]
        _lib.orc_select.restype = C.c_int
        _lib.orc_lambda.argtypes = [C.c_uint64, C.c_int]
        _lib.orc_lambda.restype = C.c_double
        _lib.orc_tau.argtypes = [C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_int]
        _lib.orc_tau.restype = C.c_double
        _lib.orc_run.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_int, C.c_void_p,
                                 C.POINTER(_Outputs)]
        _lib.orc_run.restype = C.c_int
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def philox(ctr: Sequence[int], key: Sequence[int]) -> tuple:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return tuple(int(v) for v in out)


def unit_from_bits(k52: int) -> float:
    return lib().orc_unit_from_bits(k52)


def neglog_unit(k52: int) -> float:
    """-log U for U = (2 k52 + 1) 2^-53 (Eq. 3.4's -log U_i)."""
    return lib().orc_neglog_unit(k52)


def rates(J: float, h: float, T: float, glauber: bool = False) -> np.ndarray:
    p = np.zeros(10, dtype=np.float64)
    lib().orc_rates(J, h, T, int(glauber), _ptr(p))
    return p


def frac_bits(sites: int) -> int:
    return lib().orc_frac_bits(sites)


def rates_fixed(p: np.ndarray, F: int) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    P = np.zeros(10, dtype=np.uint64)
    lib().orc_rates_fixed(_ptr(p), F, _ptr(P))
    return P


def select(N: Sequence[int], P: np.ndarray, kV: int) -> tuple:
    """(k*, 0-based position in class k*) of Eqs. 3.5-3.8, exact."""
    n = np.ascontiguousarray(N, dtype=np.int32)
    P = np.ascontiguousarray(P, dtype=np.uint64)
    pos = np.zeros(1, dtype=np.uint64)
    k = lib().orc_select(_ptr(n), _ptr(P), kV, _ptr(pos))
    return k, int(pos[0])


def lam(lam_fixed: int, F: int) -> float:
    return lib().orc_lambda(lam_fixed, F)


def tau(t_last: float, x: float, b: float, lam_fixed: int, F: int) -> float:
    return lib().orc_tau(t_last, x, b, lam_fixed, F)


@dataclass
class RunResult:
    spins: Optional[np.ndarray]        # [n_windows, L, L] int8
    counts: Optional[np.ndarray]       # [n_windows, n_regions] uint64 (cumulative)
    mag: np.ndarray                    # [n_windows] int64
    bonds: np.ndarray                  # [n_windows] int64
    int_mag: np.ndarray                # [n_windows] float64
    int_bonds: np.ndarray              # [n_windows] float64
    carry_i: np.ndarray
    carry_x: np.ndarray
    carry_b: np.ndarray
    carry_t: np.ndarray
    trace_len: int
    tr_region: Optional[np.ndarray]
    tr_index: Optional[np.ndarray]
    tr_time: Optional[np.ndarray]
    tr_site: Optional[np.ndarray]
    debug_failures: int
    ev_class: np.ndarray               # [n_regions, 10] uint64 events by class before the flip
    occupancy: np.ndarray              # [n_regions, 10] float64 integral of N_k dt


def score_tables(J: float, h: float, T: float, glauber: bool = False):
    """d log p_k / d theta and d p_k / d theta for theta = (beta, h, J), beta =
    1/T, for the ten classes k = 5*[s=+1] + n_up (Eqs. 2.1-2.3): the flip of
    class k changes the energy by dE = 2 s (J (2 n_up - 4) + h).  Metropolis
    p = min(1, exp(-beta dE)) (Eq. 2.2) has d log p = -d(beta dE) where dE > 0
    and 0 where dE < 0 (p = 1 there).  At dE = 0 p has a kink: moving theta_q
    one way puts the class on the exp branch (one-sided derivative
    -d(beta dE)/d theta_q), the other way on the p = 1 branch (derivative 0).
    The table takes the mean of the two, -d(beta dE)/d theta_q / 2, so the
    score's expectation is the mean of the left and right derivatives, which is
    what a central difference measures.  Glauber p = e / (1 + e), e =
    exp(-beta dE) (Eq. 2.3), is smooth: d log p = -(1 - p) d(beta dE).
    Returns (dlogp, dp), each [3, 10]."""
    beta = 1.0 / T
    dlogp = np.zeros((3, 10))
    dp = np.zeros((3, 10))
    p = rates(J, h, T, glauber)
    for k in range(10):
        s = 1.0 if k >= 5 else -1.0
        nb = 2.0 * (k % 5) - 4.0
        dE = 2.0 * s * (J * nb + h)
        d_bdE = np.array([dE, beta * 2.0 * s, beta * 2.0 * s * nb])   # d(beta dE)/d(beta, h, J)
        if glauber:
            dlogp[:, k] = -(1.0 - p[k]) * d_bdE
        elif dE > 0.0:
            dlogp[:, k] = -d_bdE
        elif dE == 0.0:                  # the kink of min(1, theta): both sides, averaged
            dlogp[:, k] = -0.5 * d_bdE
        dp[:, k] = p[k] * dlogp[:, k]
    return dlogp, dp


def score(r: "RunResult", J: float, h: float, T: float, glauber: bool = False) -> np.ndarray:
    """The score d log L / d(beta, h, J) of the simulated path: the sum over
    events of d log p_k minus the integral of sum_k N_k dp_k / dtheta."""
    dlogp, dp = score_tables(J, h, T, glauber)
    c = r.ev_class.sum(axis=0).astype(np.float64)
    occ = r.occupancy.sum(axis=0)
    return dlogp @ c - dp @ occ


def run(L: int, J: float, h: float, T: float, region_w: int, region_h: int, seed: int,
        t_end: Sequence[float], init_mode: int = INIT_FAIR_COIN,
        init_spins: Optional[np.ndarray] = None, glauber: bool = False, debug: bool = False,
        keep_spins: bool = True, keep_counts: bool = True, trace_cap: int = 0,
        fresh_steps: bool = False) -> RunResult:
    """Run the global time-order simulation from t = 0 through each t_end.
    fresh_steps: the alternate step rule of §5 (clocks restart with new
    random numbers at every t_end but the last)."""
    t_end = np.ascontiguousarray(t_end, dtype=np.float64)
    nw = len(t_end)
    nreg = (L // region_w) * (L // region_h)
    prm = _Params(L, J, h, T, region_w, region_h, seed, init_mode, int(glauber), int(debug),
                  int(fresh_steps))
    spins = np.zeros((nw, L, L), dtype=np.int8) if keep_spins else None
    counts = np.zeros((nw, nreg), dtype=np.uint64) if keep_counts else None
    mag = np.zeros(nw, dtype=np.int64)
    bonds = np.zeros(nw, dtype=np.int64)
    int_mag = np.zeros(nw, dtype=np.float64)
    int_bonds = np.zeros(nw, dtype=np.float64)
    ci = np.zeros(nreg, dtype=np.uint64)
    cx = np.zeros(nreg, dtype=np.float64)
    cb = np.zeros(nreg, dtype=np.float64)
    ct = np.zeros(nreg, dtype=np.float64)
    trr = np.zeros(trace_cap, dtype=np.uint32) if trace_cap else None
    tri = np.zeros(trace_cap, dtype=np.uint64) if trace_cap else None
    trt = np.zeros(trace_cap, dtype=np.float64) if trace_cap else None
    trs = np.zeros(trace_cap, dtype=np.uint32) if trace_cap else None
    init = None
    if init_spins is not None:
        init = np.ascontiguousarray(init_spins, dtype=np.int8).reshape(L * L)
        prm.init_mode = INIT_GIVEN
    evc = np.zeros((nreg, 10), dtype=np.uint64)
    occ = np.zeros((nreg, 10), dtype=np.float64)
    out = _Outputs(_ptr(spins), _ptr(counts), _ptr(mag), _ptr(bonds), _ptr(int_mag),
                   _ptr(int_bonds), _ptr(ci), _ptr(cx), _ptr(cb), _ptr(ct),
                   trace_cap, 0, _ptr(trr), _ptr(tri), _ptr(trt), _ptr(trs), 0,
                   _ptr(evc), _ptr(occ))
    rc = lib().orc_run(C.byref(prm), _ptr(init), nw, _ptr(t_end), C.byref(out))
    if rc != 0:
        raise ValueError(f"oracle run failed with code {rc}")
    n = min(out.trace_len, trace_cap)
    return RunResult(spins, counts, mag, bonds, int_mag, int_bonds, ci, cx, cb, ct,
                     int(out.trace_len),
                     trr[:n] if trr is not None else None, tri[:n] if tri is not None else None,
                     trt[:n] if trt is not None else None, trs[:n] if trs is not None else None,
                     int(out.debug_failures), evc, occ)
