"""Batches of independent lattices in one persistent launch, each lattice
against the oracle's run of that lattice alone.

Each lattice of a batch follows the synchronous-relaxation procedure of §4 on
its own (its own windows, iterations and fixed point), so its trajectory must
be bit-identical to the single-lattice run: spins, per-region event counts,
the clock carry and the exact integer observables."""
import numpy as np
import pytest

import oracle
import oracle_pool

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")

INIT = {"fair": oracle.INIT_FAIR_COIN, "up": oracle.INIT_ALL_UP, "down": oracle.INIT_ALL_DOWN}


def _ends(Tw, n):
    out, t = [], 0.0
    for _ in range(n):
        t = t + Tw
        out.append(t)
    return out


def _check_lattice(batch, b, W, H, Tw, nwin_total):
    r = batch.replicas[b]
    ends = _ends(Tw, nwin_total) if nwin_total else [0.0]
    ref = oracle.run(r.L, r.J, r.h, r.T, W, H, r.seed, ends, init_mode=INIT[r.init],
                     glauber=(r.rates == "glauber"))
    assert np.array_equal(batch.spins(b), ref.spins[-1]), f"spins of lattice {b}"
    i, x, bb, t = batch.carry(b)
    if nwin_total:
        assert np.array_equal(i, ref.carry_i), f"event index of lattice {b}"
        assert np.array_equal(x, ref.carry_x)
        assert np.array_equal(bb, ref.carry_b)
        assert np.array_equal(t, ref.carry_t)
    else:
        assert not i.any() and not bb.any() and not t.any()
    o = batch.observables(b)
    assert o.mag == ref.mag[-1] and o.bonds == ref.bonds[-1]
    assert o.committed == int(ref.counts[-1].sum())
    assert o.windows == nwin_total
    assert o.t_c == (ends[-1] if nwin_total else 0.0)


REPS = [dict(L=32, J=1.0, h=0.05, T=1.5, seed=11),
        dict(L=16, J=0.8, h=-0.2, T=1.2, seed=12, rates="glauber", init="down"),
        dict(L=48, J=1.0, h=0.0, T=2.269, seed=13, init="up"),
        dict(L=24, J=1.0, h=0.2, T=3.5, seed=14),
        dict(L=8, J=1.0, h=0.0, T=1.0, seed=15),
        dict(L=40, J=0.0, h=0.3, T=2.0, seed=16)]
TW = [1.0, 0.5, 0.25, 2.0, 0.7, 1.0]
NW = [3, 5, 2, 1, 4, 0]

MAPS = [dict(),
        dict(lanes_per_region=1, lanes_per_warp=3, time_arith=2),
        dict(lanes_per_region=1, lanes_per_warp=32, time_arith=1, replay_records=2),
        dict(lanes_per_region=32),
        dict(lanes_per_region=1, lanes_per_warp=32, schedule=1),
        dict(lanes_per_region=1, lanes_per_warp=32, schedule=3),
        dict(lanes_per_region=1, lanes_per_warp=5, time_arith=2, schedule=3, replay_records=2)]


@pytest.mark.parametrize("m", range(len(MAPS)))
def test_mixed_batch_bit_exact(m):
    with sr.Batch(REPS, region=(8, 8), **MAPS[m]) as batch:
        batch.run(TW, NW)
        for b in range(len(REPS)):
            _check_lattice(batch, b, 8, 8, TW[b], NW[b])


@pytest.mark.parametrize("m", range(len(MAPS)))
def test_batch_runs_continue(m):
    """Two run calls with different window counts: each lattice continues
    from its own committed time."""
    with sr.Batch(REPS, region=(8, 8), **MAPS[m]) as batch:
        batch.run(TW, NW)
        more = [1, 0, 3, 2, 1, 2]
        batch.run(TW, more)
        for b in range(len(REPS)):
            _check_lattice(batch, b, 8, 8, TW[b], NW[b] + more[b])
        assert batch.t_c[5] == _ends(TW[5], 2)[-1]


def test_many_small_lattices():
    """Sixty lattices of 4 regions each, spread over blocks and lanes."""
    reps = [dict(L=16, J=1.0, h=0.05 * ((b % 5) - 2), T=1.0 + 0.05 * b, seed=100 + b)
            for b in range(60)]
    nw = [1 + (b % 4) for b in range(60)]
    with sr.Batch(reps, region=(8, 8)) as batch:
        batch.run(0.5, nw)
        for b in range(60):
            _check_lattice(batch, b, 8, 8, 0.5, nw[b])


def test_batch_equals_separate_lattices():
    """Observables and counters of a lattice in a batch equal those of the
    same lattice simulated alone."""
    reps = REPS[:4]
    with sr.Batch(reps, region=(8, 8)) as batch:
        batch.run(TW[:4], NW[:4])
        for b, r in enumerate(reps):
            lat = sr.Lattice(r["L"], r["J"], r["h"], r["T"], (8, 8), seed=r["seed"],
                             init=r.get("init", "fair"), rates=r.get("rates", "metropolis"))
            lat.run_windows(TW[b], NW[b])
            o1, o2 = batch.observables(b), lat.observables()
            assert np.array_equal(batch.spins(b), lat.spins())
            for f in ("t_c", "mag", "bonds", "committed", "generated", "breaks", "windows",
                      "iterations", "max_iters_seen", "max_f", "int_mag", "int_bonds"):
                assert getattr(o1, f) == getattr(o2, f), f
            lat.close()


def test_batch_capacity_growth():
    """Long windows at high temperature overflow the initial history capacity
    of one lattice; the retry re-runs only what did not commit."""
    reps = [dict(L=32, T=3.5, h=0.0, seed=21), dict(L=16, T=1.0, h=0.1, seed=22)]
    with sr.Batch(reps, region=(16, 16)) as batch:
        batch.run([8.0, 1.0], [2, 3])
        assert batch.observables(0).capacity > 64
        _check_lattice(batch, 0, 16, 16, 8.0, 2)
        _check_lattice(batch, 1, 16, 16, 1.0, 3)


def test_batch_reset_and_bad_arguments():
    with sr.Batch(REPS[:2], region=(8, 8)) as batch:
        batch.run(1.0, 2)
        s0 = batch.spins(0)
        batch.reset()
        batch.run(1.0, 2)
        assert np.array_equal(batch.spins(0), s0)
        with pytest.raises(sr.SRError):
            batch.run([1.0, -1.0], [1, 1])
        with pytest.raises(sr.SRError):
            batch.observables(2)
    with pytest.raises(sr.SRError):
        sr.Batch([dict(L=20)], region=(8, 8))      # 20 is not a multiple of 8
    with pytest.raises(sr.SRError):
        sr.Batch([], region=(8, 8))


# ----------------------------------------------------------------- adaptive windows
def _check_at(batch, b, W, H, t_final, n_windows_min=1):
    r = batch.replicas[b]
    ref = oracle.run(r.L, r.J, r.h, r.T, W, H, r.seed, [t_final], init_mode=INIT[r.init],
                     glauber=(r.rates == "glauber"))
    assert np.array_equal(batch.spins(b), ref.spins[-1]), f"spins of lattice {b}"
    i, x, bb, t = batch.carry(b)
    assert np.array_equal(i, ref.carry_i)
    assert np.array_equal(x, ref.carry_x)
    assert np.array_equal(bb, ref.carry_b)
    assert np.array_equal(t, ref.carry_t)
    o = batch.observables(b)
    assert o.committed == int(ref.counts[-1].sum())
    assert o.windows >= n_windows_min


@pytest.mark.parametrize("m", [0, 1])
def test_adaptive_windows_bit_exact(m):
    """Window lengths chosen from each lattice's event rate do not change its
    trajectory; every lattice ends exactly at its own target time."""
    t_end = [3.0, 2.0, 4.0, 1.5, 2.5, 0.0]
    with sr.Batch(REPS, region=(8, 8), **MAPS[m]) as batch:
        last = batch.run_adaptive(t_end, kappa=4.0, chunk=0.5)
        for b in range(len(REPS)):
            assert batch.t_c[b] == t_end[b]
            if t_end[b] > 0:
                assert last[b] > 0 and last[b] == 2.0 ** round(np.log2(last[b]))
                _check_at(batch, b, 8, 8, t_end[b])
        # continue to non-dyadic ends
        t2 = [3.3, 2.7, 4.0, 1.9, 2.5, 0.7]
        batch.run_adaptive(t2)
        for b in range(len(REPS)):
            assert batch.t_c[b] == t2[b]
            _check_at(batch, b, 8, 8, t2[b])


def test_adaptive_argument_checks():
    with sr.Batch(REPS[:2], region=(8, 8)) as batch:
        batch.run_adaptive([1.0, 1.0])
        with pytest.raises(sr.SRError):
            batch.run_adaptive([0.5, 2.0])          # before the committed time
        with pytest.raises(sr.SRError):
            batch.run_adaptive([2.0, 2.0], kappa=-1.0)
        with pytest.raises(sr.SRError):
            batch.run_adaptive([2.0, 2.0], tw_min=1.0, tw_max=0.5)


MIXED = [dict(L=32, T=2.8, h=0.05, seed=81, region=(8, 8)),
         dict(L=64, T=1.5, h=0.0, seed=82, region=(32, 16)),
         dict(L=48, T=3.3, h=-0.1, seed=83, region=(16, 8), init="up"),
         dict(L=64, T=2.2, h=0.1, seed=84),                       # the batch's shape
         dict(L=32, T=1.2, h=0.2, seed=85, region=(32, 32), rates="glauber"),
         dict(L=24, T=2.5, h=0.0, seed=86, region=(8, 12))]
MIXED_TW = [0.5, 0.25, 0.5, 1.0, 0.5, 0.25]
MIXED_NW = [4, 6, 3, 2, 4, 8]


@pytest.mark.parametrize("m", range(len(MAPS)))
def test_lattices_with_their_own_region_shapes(m):
    """Each lattice of a batch partitioned into its own region shape (§5: the
    subsets G_i); the launch lays its state out for the largest shape.  Every
    lattice against the oracle with that lattice's shape, in every mapping
    and schedule."""
    with sr.Batch(MIXED, region=(16, 16), **MAPS[m]) as batch:
        batch.run(MIXED_TW, MIXED_NW)
        for b in range(len(MIXED)):
            W, H = batch.region_of(b)
            assert (W, H) == MIXED[b].get("region", (16, 16))
            _check_lattice(batch, b, W, H, MIXED_TW[b], MIXED_NW[b])


def test_own_region_shapes_checkpoint_and_score():
    reps = [dict(r) for r in MIXED[:4]]
    with sr.Batch(reps, region=(16, 16), score=True) as a:
        a.run(MIXED_TW[:4], [2, 3, 2, 1])
        data = a.checkpoint()
        a.run(MIXED_TW[:4], [2, 3, 1, 1])
        S_a = a.score()
        spins_a = [a.spins(b) for b in range(4)]
    with sr.Batch(reps, region=(16, 16), score=True) as b2:
        b2.load_checkpoint(data)
        b2.run(MIXED_TW[:4], [2, 3, 1, 1])
        assert np.array_equal(b2.score(), S_a)
        for b in range(4):
            assert np.array_equal(b2.spins(b), spins_a[b])
    other = [dict(r) for r in reps]
    other[1]["region"] = (16, 16)            # a different shape: the checkpoint does not fit
    with sr.Batch(other, region=(16, 16), score=True) as b3:
        with pytest.raises(sr.SRError):
            b3.load_checkpoint(data)


def test_autotune_small_batch():
    reps = [dict(L=32, T=1.5, h=0.05, seed=31), dict(L=64, T=3.0, h=0.0, seed=32),
            dict(L=96, T=2.2, h=-0.1, seed=33)]
    t = sr.autotune(reps, t_trial=0.5)
    # 96 is not a multiple of 64 but every candidate shape divides 32, 64, 96
    shapes = [(16, 16), (8, 8), (32, 32), (16, 8), (32, 16)]
    assert (t.region[0], t.region[1]) in shapes and t.region == t.shapes[0]
    assert all(s in shapes for s in t.shapes) and len(t.shapes) == 3
    assert t.rate_threshold in (0.0, 32.0, 64.0, 128.0, 256.0)
    if t.rate_threshold == 0.0:
        assert len(set(t.shapes)) == 1          # one common shape won
    assert t.lanes_per_warp in (0, 8, 16, 32)
    assert t.kappa in (4.0, 8.0, 16.0, 32.0)
    assert t.trials == 5 + 4 + 3 + 3
    assert t.flips_per_s > 0
    with sr.Batch(t.replicas(reps), region=t.region, lanes_per_warp=t.lanes_per_warp) as batch:
        batch.run_adaptive(1.0, kappa=t.kappa)
        for b in range(3):
            W, H = batch.region_of(b)
            assert (W, H) == t.shapes[b]
            _check_at(batch, b, W, H, 1.0)
    with pytest.raises(sr.SRError):
        sr.autotune([dict(L=36, T=2.0)])              # no candidate shape divides 36


def test_batched_workload_sample_bit_exact():
    """The 256-lattice batched workload (L from 64 to 1024, T in [1, 3.5],
    h in [-0.2, 0.2]) to t = 0.25 with adaptive windows; a stratified sample
    of lattices against their oracle runs."""
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas()
    with sr.Batch(reps, region=(16, 16)) as batch:
        batch.run_adaptive(0.25, kappa=8.0, chunk=0.125)
        assert np.all(batch.t_c == 0.25)
        for b in range(0, len(reps), 11):
            _check_at(batch, b, 16, 16, 0.25)


def test_benched_batch_configuration_against_the_oracle():
    """The batched workload exactly as the benchmark runs it: the autotuner's
    region shape of each lattice, lanes per warp and kappa, the automatic (asynchronous)
    schedule, adaptive window lengths, a warm-up run and a reset, then every
    lattice to t = 10.  A stratified sample of 15 lattices (the coldest, the
    median and the hottest of each side L) against their oracle runs: spins,
    clock carry, counts and observables."""
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas()
    sample = workloads.stratified(reps, per_side=3)
    assert len(sample) == 15
    tune = sr.autotune(reps, t_trial=1.0)
    pool = oracle_pool.pool(len(sample))
    try:
        jobs = {b: pool.apply_async(oracle_pool.run, (dict(
            L=reps[b]["L"], J=reps[b]["J"], h=reps[b]["h"], T=reps[b]["T"],
            region_w=tune.shapes[b][0], region_h=tune.shapes[b][1], seed=reps[b]["seed"],
            t_end=[10.0]),)) for b in sample}
        with sr.Batch(tune.replicas(reps), region=tune.region,
                      lanes_per_warp=tune.lanes_per_warp) as bt:
            bt.run_adaptive(1.0, kappa=tune.kappa)
            bt.reset()
            bt.run_adaptive(10.0, kappa=tune.kappa)
            assert np.all(bt.t_c == 10.0)
            for b in sample:
                ref = jobs[b].get(timeout=1800)
                assert np.array_equal(oracle_pool.pack(bt.spins(b)), ref["spins"][0]), b
                for got, want in zip(bt.carry(b), ref["carry"]):
                    assert np.array_equal(got, want), b
                o = bt.observables(b)
                assert o.committed == int(ref["counts"][0].sum())
                assert (o.mag, o.bonds) == (int(ref["mag"][0]), int(ref["bonds"][0]))
                n = reps[b]["L"] ** 2
                assert abs(o.int_mag - ref["int_mag"][0]) <= 1e-9 * n * 10.0
                assert abs(o.int_bonds - ref["int_bonds"][0]) <= 1e-9 * n * 10.0
    finally:
        pool.terminate()
        pool.join()


def test_many_short_asynchronous_launches_from_coarsened_spins():
    """The task queue of the asynchronous schedule under many short launches:
    the 256-lattice workload with a region shape per lattice, restarted 30
    times from coarsened spins (the state at t = 4) and run to t = 1 in
    chunks of 1/4.  Every launch must end normally (a lost or repeated task
    would leave a lattice waiting until the bounded wait ends it with
    SR_TIMEOUT), and the last run of three lattices equals the oracle from
    the same spins."""
    from paper_cs_0405053_gb300 import workloads
    reps = workloads.batch_replicas()
    shapes = [(8, 8), (16, 8), (16, 16), (32, 16)]
    own = [dict(r, region=shapes[b % 4]) for b, r in enumerate(reps)]
    with sr.Batch(own, region=(16, 16)) as bt:
        bt.run_adaptive(4.0, kappa=8.0)
        late = [bt.spins(b) for b in range(len(reps))]
        for _ in range(30):
            for b in range(len(reps)):
                bt.set_spins(b, late[b])
            bt.run_adaptive(1.0, kappa=4.0, chunk=0.25)
            assert np.all(bt.t_c == 1.0)
        for b in (0, 101, 255):
            W, H = shapes[b % 4]
            r = reps[b]
            ref = oracle.run(r["L"], r["J"], r["h"], r["T"], W, H, r["seed"], [1.0],
                             init_spins=late[b])
            assert np.array_equal(bt.spins(b), ref.spins[-1]), b
            assert np.array_equal(bt.carry(b)[0], ref.carry_i), b


# ----------------------------------------------------------------- errors in a batch
def _consistent_with_oracle(batch, W, H):
    """Every lattice's committed state equals the oracle at its own t_c."""
    for b, r in enumerate(batch.replicas):
        t = float(batch.t_c[b])
        ref = oracle.run(r.L, r.J, r.h, r.T, W, H, r.seed, [t], init_mode=INIT[r.init],
                         glauber=(r.rates == "glauber"))
        assert np.array_equal(batch.spins(b), ref.spins[-1]), (b, t)
        i, x, bb, tl = batch.carry(b)
        if t > 0:
            assert np.array_equal(i, ref.carry_i), (b, t)


@pytest.mark.parametrize("schedule", [2, 3])
def test_batch_capacity_overflow_keeps_every_lattice_consistent(schedule):
    reps = [dict(L=16, T=1.0, h=0.1, seed=41), dict(L=64, T=3.5, h=0.0, seed=42),
            dict(L=8, T=2.0, h=0.0, seed=43)]
    with sr.Batch(reps, region=(8, 8), capacity=2, schedule=schedule) as bt:
        with pytest.raises(sr.SRError) as e:
            bt.run([0.5, 2.0, 0.5], [4, 3, 4])
        assert e.value.code == sr.SR_CAPACITY
        assert bt.t_c[1] == 0.0            # the hot lattice never committed a window
        _consistent_with_oracle(bt, 8, 8)


@pytest.mark.parametrize("schedule", [2, 3])
def test_batch_iteration_cap_keeps_every_lattice_consistent(schedule):
    # the single-region lattice converges in one iteration, the others cannot
    reps = [dict(L=8, T=2.0, h=0.1, seed=51), dict(L=32, T=2.5, h=0.05, seed=52)]
    with sr.Batch(reps, region=(8, 8), max_iters=1, schedule=schedule) as bt:
        with pytest.raises(sr.SRError) as e:
            bt.run(1.0, 3)
        assert e.value.code == sr.SR_NOT_CONVERGED
        assert bt.t_c[1] == 0.0
        _consistent_with_oracle(bt, 8, 8)


def test_async_waits_outlast_a_long_tail():
    """When one small hot lattice is left, each of its iterations publishes one
    task and the waiting warps (here about 1200) are served one per iteration;
    their waits, bounded at 25 ms, must count time without any progress only."""
    reps = [dict(L=64, T=3.5, h=0.0, seed=71), dict(L=32, T=1.0, h=0.1, seed=72)]
    with sr.Batch(reps, region=(32, 32), schedule=3, blocks=300, threads_per_block=128,
                  barrier_timeout_ms=25) as bt:
        bt.run([1.0, 1.0], [3, 1])
        assert bt.t_c[0] == 3.0 and bt.t_c[1] == 1.0
        _consistent_with_oracle(bt, 32, 32)


@pytest.mark.parametrize("schedule", [2, 3])
def test_batch_wait_times_out_instead_of_hanging(schedule):
    reps = [dict(L=32, T=2.0, h=0.0, seed=61), dict(L=16, T=1.5, h=0.1, seed=62)]
    with sr.Batch(reps, region=(8, 8), schedule=schedule, threads_per_block=32,
                  barrier_timeout_ms=100, test_barrier_skip_block=0) as bt:
        assert bt.blocks >= 2
        with pytest.raises(sr.SRError) as e:
            bt.run(1.0, 2)
        assert e.value.code == sr.SR_TIMEOUT
    # the GPU context is still usable
    with sr.Batch(reps, region=(8, 8), schedule=schedule) as bt:
        bt.run(1.0, 2)
        _consistent_with_oracle(bt, 8, 8)
