"""The four calls of the boundary (sr_create, sr_run_window, sr_observables,
sr_destroy) through ctypes, with nothing but their own arguments: the small
workload of the statement (L = 64 in 4 x 4 regions of 16 x 16, J = 1,
h = 0.05, T = 1.5, fair-coin spins, windows of length 1 to t = 10) against
the oracle's run of the same lattice: spins and per-region event counts at
the end, and every observable the call reports."""
import ctypes as C

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")


def test_four_call_boundary_against_the_oracle():
    lib = sr.library()
    L, J, h, T, W, H, seed = 64, 1.0, 0.05, 1.5, 16, 16, 1
    ctx = C.c_void_p()
    assert lib.sr_create(C.byref(ctx), L, J, h, T, W, H, seed) == sr.SR_OK
    t, ends = 0.0, []
    for _ in range(10):
        assert lib.sr_run_window(ctx, t, 1.0) == sr.SR_OK
        t = t + 1.0
        ends.append(t)
    assert lib.sr_run_window(ctx, 0.5, 1.0) == sr.SR_EINVAL       # t0 is not the committed time
    assert lib.sr_run_window(ctx, t, 0.0) == sr.SR_EINVAL         # Tw <= 0
    obs = sr._Obs()
    assert lib.sr_observables(ctx, C.byref(obs)) == sr.SR_OK
    spins = np.zeros(L * L, dtype=np.int8)
    assert lib.sr_get_spins(ctx, spins.ctypes.data, spins.size) == sr.SR_OK
    counts = np.zeros((L // W) * (L // H), dtype=np.uint64)
    assert lib.sr_get_carry(ctx, counts.ctypes.data, None, None, None, counts.size) == sr.SR_OK
    lib.sr_destroy(ctx)
    lib.sr_destroy(None)                                          # NULL-safe

    ref = oracle.run(L, J, h, T, W, H, seed, ends)
    assert np.array_equal(spins.reshape(L, L), ref.spins[-1])
    assert np.array_equal(counts, ref.counts[-1])
    assert obs.t_c == 10.0 and obs.windows == 10
    assert obs.mag == ref.mag[-1] and obs.bonds == ref.bonds[-1]
    assert obs.m == ref.mag[-1] / L ** 2
    assert obs.E == -J * ref.bonds[-1] - h * ref.mag[-1]
    assert obs.committed == int(ref.counts[-1].sum())
    assert obs.generated >= obs.committed and obs.iterations >= obs.windows
    for got, want in ((obs.int_mag, ref.int_mag[-1]), (obs.int_bonds, ref.int_bonds[-1])):
        assert abs(got - want) <= 1e-9 * L * L * 10.0, (got, want)
    assert obs.relax_launches == 10 and obs.relax_ms > 0.0


def test_create_refuses_bad_arguments():
    lib = sr.library()
    ctx = C.c_void_p()
    for args in ((2, 1.0, 0.0, 1.5, 1, 1, 1),                                          # L < 3
                 (64, 1.0, 0.0, 1.5, 10, 16, 1),                                     # 10 does not divide 64
                 (64, 1.0, 0.0, 0.0, 16, 16, 1),                                     # T <= 0
                 (64, 1.0, 0.0, float("nan"), 16, 16, 1),
                 (64, float("inf"), 0.0, 1.5, 16, 16, 1)):
        assert lib.sr_create(C.byref(ctx), *args) == sr.SR_EINVAL
        assert not ctx.value
    assert lib.sr_create(C.byref(ctx), 128, 1.0, 0.0, 1.5, 64, 64, 1) == sr.SR_EUNSUPPORTED
