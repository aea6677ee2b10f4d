"""GPU path (libsr through its C ABI) against the CPU oracle, element by
element on the same seeded inputs.

The bar (fixed by the deterministic random streams and the exact rate grid):
spins at every window end, per-region event counts, the clock carry and every
committed event's time and site are bit-identical.  Event times are compared
as exact doubles, which is stricter than the 1e-12 relative tolerance the
method's statement allows."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")


def _ends(Tw, n, t0=0.0):
    out, t = [], t0
    for _ in range(n):
        t = t + Tw
        out.append(t)
    return out


def _compare(L, W, H, J=1.0, h=0.05, T=1.5, seed=1, Tw=1.0, nwin=3, init="fair", rates="metropolis",
             trace=True, given=None, **kw):
    cap = 1 << 14 if trace else 0
    lat = sr.Lattice(L, J, h, T, (W, H), seed=seed, init=init, rates=rates, trace_capacity=cap, **kw)
    if given is not None:
        lat.set_spins(given)
    gpu = []
    for _ in range(nwin):
        lat.run_window(Tw)
        gpu.append(lat.spins())
    ends = _ends(Tw, nwin)
    mode = {"fair": oracle.INIT_FAIR_COIN, "up": oracle.INIT_ALL_UP, "down": oracle.INIT_ALL_DOWN}[init]
    ref = oracle.run(L, J, h, T, W, H, seed, ends, init_mode=mode, init_spins=given,
                     glauber=(rates == "glauber"), trace_cap=(1 << 22) if trace else 0)
    for w in range(nwin):
        assert np.array_equal(gpu[w], ref.spins[w]), f"spins differ at window {w}"
    i, x, b, tl = lat.carry()
    assert np.array_equal(i, ref.carry_i)
    assert np.array_equal(x, ref.carry_x)
    assert np.array_equal(b, ref.carry_b)
    assert np.array_equal(tl, ref.carry_t)
    obs = lat.observables()
    assert obs.mag == ref.mag[-1] and obs.bonds == ref.bonds[-1]
    assert obs.committed == int(ref.counts[-1].sum())
    scale_m = max(1.0, abs(ref.int_mag[-1]), L * L * ends[-1] * 1e-3)
    assert abs(obs.int_mag - ref.int_mag[-1]) <= 1e-9 * scale_m
    scale_b = max(1.0, abs(ref.int_bonds[-1]), L * L * ends[-1] * 1e-3)
    assert abs(obs.int_bonds - ref.int_bonds[-1]) <= 1e-9 * scale_b
    if trace:
        lens, times, sites = lat.trace()
        assert np.array_equal(lens, ref.counts[-1])
        for q in range(lat.n_regions):
            sel = ref.tr_region == q
            n = int(lens[q])
            assert np.array_equal(times[q, :n], ref.tr_time[sel]), f"times of region {q}"
            assert np.array_equal(sites[q, :n], ref.tr_site[sel]), f"sites of region {q}"
    return lat, ref


# ----------------------------------------------------------------- numerics
def test_draws_bitwise():
    for seed, region, i0 in [(1, 0, 0), (2**63 + 12345, 77, 10**12), (7, 4095, 2**40 - 100)]:
        x, kv = sr.eval_draws(seed, region, i0, 4096)
        for j in range(0, 4096, 1):
            w = oracle.philox([(i0 + j) & 0xFFFFFFFF, (i0 + j) >> 32, region, 0],
                              [seed & 0xFFFFFFFF, seed >> 32])
            ku = ((w[1] << 32) | w[0]) >> 12
            assert int(kv[j]) == ((w[3] << 32) | w[2]) >> 12
            assert x[j] == oracle.neglog_unit(ku)


def test_initial_spins_match():
    for seed in (1, 2, 3):
        lat = sr.Lattice(64, 1.0, 0.05, 1.5, (16, 16), seed=seed)
        ref = oracle.run(64, 1.0, 0.05, 1.5, 16, 16, seed, [0.0])
        assert np.array_equal(lat.spins(), ref.spins[0])
    lat = sr.Lattice(12, 1.0, 0.0, 2.0, (4, 3), init="up")
    assert np.all(lat.spins() == 1)


def test_rate_table_matches():
    for T, h, rates in [(1.5, 0.05, "metropolis"), (1.0, 0.0, "glauber"), (3.5, -0.2, "metropolis")]:
        lat = sr.Lattice(32, 1.0, h, T, (16, 16), rates=rates)
        F = oracle.frac_bits(256)
        assert lat.frac_bits == F
        assert np.array_equal(lat.P, oracle.rates_fixed(oracle.rates(1.0, h, T, rates == "glauber"), F))


# ----------------------------------------------------------------- trajectories
# mappings: (lanes per region, region lanes per warp, time arithmetic)
MAPS = [dict(lanes_per_region=1, lanes_per_warp=32, time_arith=1),
        dict(lanes_per_region=1, lanes_per_warp=3, time_arith=2),
        dict(lanes_per_region=32),
        dict(lanes_per_region=1, lanes_per_warp=2, time_arith=1, replay_records=-1),
        dict(lanes_per_region=1, lanes_per_warp=5, time_arith=1, replay_records=2),
        dict(lanes_per_region=1, lanes_per_warp=4, schedule=2),
        dict(lanes_per_region=32, schedule=2),
        dict(lanes_per_region=1, lanes_per_warp=3, schedule=3)]
LPR = list(range(len(MAPS)))


@pytest.mark.parametrize("lpr", LPR)
@pytest.mark.parametrize("L,W,H", [(3, 1, 1), (4, 2, 2), (8, 4, 4), (8, 8, 8), (6, 3, 2), (12, 4, 3),
                                   (16, 16, 4), (16, 4, 16), (16, 1, 16), (9, 3, 1), (32, 8, 8),
                                   (30, 10, 6), (32, 32, 32), (64, 32, 32)])
def test_small_lattices_bit_exact(L, W, H, lpr):
    _compare(L, W, H, seed=L * 31 + W, T=1.7, Tw=0.7, nwin=4, **MAPS[lpr])


@pytest.mark.parametrize("T,h,J,rates,init", [(1.0, 0.0, 1.0, "metropolis", "fair"),
                                              (2.269, 0.0, 1.0, "metropolis", "up"),
                                              (3.5, 0.0, 1.0, "metropolis", "fair"),
                                              (1.2, -0.2, 0.8, "glauber", "down"),
                                              (1e300, 0.0, 1.0, "metropolis", "fair"),
                                              (2.0, 0.3, 0.0, "metropolis", "fair"),
                                              (0.005, 0.05, 1.0, "metropolis", "fair")])
@pytest.mark.parametrize("lpr", LPR)
def test_parameters_bit_exact(T, h, J, rates, init, lpr):
    _compare(24, 8, 6, J=J, h=h, T=T, rates=rates, init=init, seed=5, Tw=0.5, nwin=4,
             **MAPS[lpr])


def test_given_initial_spins():
    rng = np.random.default_rng(3)
    given = np.where(rng.random((16, 16)) < 0.3, 1, -1).astype(np.int8)
    _compare(16, 4, 4, given=given, seed=9, nwin=3)


@pytest.mark.parametrize("lpr", LPR)
@pytest.mark.parametrize("seed", range(1, 9))
def test_small_config_L64_bit_exact(seed, lpr):
    """L = 64, 4 x 4 regions of 16 x 16, J = 1, h = 0.05, T = 1.5, fair coin,
    window 1.0, run to t = 10."""
    _compare(64, 16, 16, h=0.05, T=1.5, seed=seed, Tw=1.0, nwin=10, **MAPS[lpr])


def test_window_length_does_not_change_the_trajectory():
    """Window ends are not break points (§5, 'Subsequent steps'): the
    converged fixed point is the same for any window length."""
    res = []
    for Tw, n in [(0.25, 16), (1.0, 4), (4.0, 1), (0.5, 8)]:
        lat = sr.Lattice(64, 1.0, 0.05, 1.0, (16, 16), seed=4, trace_capacity=1 << 12)
        lat.run_windows(Tw, n)
        res.append((lat.spins(), lat.carry(), lat.trace()))
    for other in res[1:]:
        assert np.array_equal(res[0][0], other[0])
        for a, b in zip(res[0][1], other[1]):
            assert np.array_equal(a, b)
        lens, times, sites = res[0][2]
        assert np.array_equal(lens, other[2][0])
        for q in range(len(lens)):       # entries past a region's count are not events
            n = int(lens[q])
            assert np.array_equal(times[q, :n], other[2][1][q, :n])
            assert np.array_equal(sites[q, :n], other[2][2][q, :n])


def test_single_region_is_the_serial_n_fold_way():
    """One region = plain serial n-fold way (§5, first iteration): every window
    converges in one iteration and nothing is discarded."""
    lat, _ = _compare(32, 32, 32, T=2.0, h=0.05, seed=3, Tw=1.0, nwin=5)
    obs = lat.observables()
    assert obs.iterations == 5 and obs.max_iters_seen == 1
    assert obs.generated == obs.committed and obs.breaks == 0


def test_iterations_follow_the_canonical_assumption():
    """Iteration 1 assumes no neighbour flips (§5): a window with no boundary
    event converges in one iteration, any boundary event forces a second.
    Each iteration settles at least the next boundary event in time order
    (the events before it see correct inputs), so a window with B boundary
    events converges in at most B + 1 iterations."""
    lat = sr.Lattice(64, 1.0, 0.05, 1.5, (16, 16), seed=2, trace_capacity=1 << 12)
    lat.run_windows(1.0, 5)
    g = lat.window_iters()
    lens, times, sites = lat.trace()
    xs, ys = sites % 64, sites // 64
    on_edge = (xs % 16 == 0) | (xs % 16 == 15) | (ys % 16 == 0) | (ys % 16 == 15)
    for w in range(5):
        nb = 0
        for q in range(lat.n_regions):
            n = int(lens[q])
            sel = (times[q, :n] >= w) & (times[q, :n] < w + 1)
            nb += int(on_edge[q, :n][sel].sum())
        assert (g[w] == 1) == (nb == 0), (w, g[w], nb)
        assert g[w] <= nb + 1, (w, g[w], nb)


@pytest.mark.parametrize("lpr", LPR)
def test_medium_lattice_bit_exact(lpr):
    _compare(256, 16, 16, h=0.05, T=1.0, seed=1, Tw=1.0, nwin=3, trace=False, **MAPS[lpr])


@pytest.mark.parametrize("lpr", LPR)
def test_capacity_growth_exact_both_mappings(lpr):
    _compare(64, 16, 16, T=3.5, seed=6, Tw=2.0, nwin=2, **MAPS[lpr])


# ----------------------------------------------------------------- failure paths
def test_capacity_growth_is_exact_and_fixed_capacity_fails():
    # automatic capacity starting small enough to overflow: grows, same result
    _compare(64, 16, 16, T=3.5, seed=6, Tw=2.0, nwin=2)
    lat = sr.Lattice(64, 1.0, 0.0, 3.5, (16, 16), seed=6, capacity=1)
    with pytest.raises(sr.SRError) as e:
        lat.run_window(2.0)
    assert e.value.code == sr.SR_CAPACITY
    assert lat.t_c == 0.0
    # the committed state is untouched: a bigger context reproduces the oracle
    ref = oracle.run(64, 1.0, 0.0, 3.5, 16, 16, 6, [0.0])
    assert np.array_equal(lat.spins(), ref.spins[0])


def test_iteration_cap_reports_not_converged():
    lat = sr.Lattice(64, 1.0, 0.05, 2.5, (16, 16), seed=7, max_iters=1)
    with pytest.raises(sr.SRError) as e:
        lat.run_window(2.0)
    assert e.value.code == sr.SR_NOT_CONVERGED


def test_barrier_wait_times_out_instead_of_hanging():
    # one block never arrives at the grid barrier; every wait is bounded
    lat = sr.Lattice(64, 1.0, 0.05, 1.5, (8, 8), seed=1, threads_per_block=32,
                     barrier_timeout_ms=100, test_barrier_skip_block=0)
    assert lat.blocks >= 2
    with pytest.raises(sr.SRError) as e:
        lat.run_window(1.0)
    assert e.value.code == sr.SR_TIMEOUT
    lat.close()
    # the GPU context is still usable
    _compare(16, 4, 4, seed=2, nwin=2)


def test_bad_arguments():
    with pytest.raises(sr.SRError):
        sr.Lattice(64, 1.0, 0.0, 1.0, (10, 16))
    with pytest.raises(sr.SRError):
        sr.Lattice(2, 1.0, 0.0, 1.0, (1, 1))
    with pytest.raises(sr.SRError):
        sr.Lattice(64, 1.0, 0.0, -1.0, (16, 16))
    lat = sr.Lattice(32, 1.0, 0.0, 1.0, (16, 16))
    lib = sr.library()
    assert lib.sr_run_window(lat._ctx, 1.0, 1.0) == sr.SR_EINVAL      # t0 != t_c
    assert lib.sr_run_window(lat._ctx, 0.0, -1.0) == sr.SR_EINVAL


def test_reset_reproduces_the_run():
    lat = sr.Lattice(64, 1.0, 0.05, 1.5, (16, 16), seed=11)
    lat.run_windows(1.0, 3)
    a = lat.spins()
    lat.reset()
    lat.run_windows(1.0, 3)
    assert np.array_equal(a, lat.spins())
