"""The alternate step rule of §5 on the GPU against the oracle: at every
committed time each region's clock restarts with new random numbers
(event j of window w: Philox counter (j, w, region, 2)).  Spins at every
window end, event counts, the clock state after the last window and every
committed event's time and site must be bit-identical."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")

MAPS = [dict(lanes_per_region=1, lanes_per_warp=32, time_arith=1),
        dict(lanes_per_region=1, lanes_per_warp=3, time_arith=2),
        dict(lanes_per_region=1, lanes_per_warp=2, time_arith=1, replay_records=-1),
        dict(lanes_per_region=1, lanes_per_warp=5, time_arith=1, replay_records=2),
        dict(lanes_per_region=1, lanes_per_warp=4, schedule=3)]


def _ends(Tw, n, t0=0.0):
    out, t = [], t0
    for _ in range(n):
        t = t + Tw
        out.append(t)
    return out


def _compare(L, W, H, J=1.0, h=0.05, T=1.5, seed=1, Tw=0.5, nwin=4, calls=1, **kw):
    lat = sr.Lattice(L, J, h, T, (W, H), seed=seed, trace_capacity=1 << 14, fresh_steps=True,
                     **kw)
    spins = []
    per = nwin // calls
    for _ in range(calls):
        for _ in range(per):
            lat.run_window(Tw)
            spins.append(lat.spins())
    ends = _ends(Tw, per * calls)
    ref = oracle.run(L, J, h, T, W, H, seed, ends, trace_cap=1 << 22, fresh_steps=True)
    for w in range(len(ends)):
        assert np.array_equal(spins[w], ref.spins[w]), f"window {w}"
    i, x, b, tl = lat.carry()
    assert np.array_equal(i, ref.carry_i)
    assert np.array_equal(x, ref.carry_x)
    assert np.array_equal(b, ref.carry_b)
    assert np.array_equal(tl, ref.carry_t)
    lens, times, sites = lat.trace()
    assert np.array_equal(lens, ref.counts[-1])
    for q in range(lat.n_regions):
        sel = ref.tr_region == q
        n = int(lens[q])
        assert np.array_equal(times[q, :n], ref.tr_time[sel])
        assert np.array_equal(sites[q, :n], ref.tr_site[sel])
    o = lat.observables()
    assert o.mag == ref.mag[-1] and o.bonds == ref.bonds[-1]
    lat.close()


@pytest.mark.parametrize("m", range(len(MAPS)))
@pytest.mark.parametrize("L,W,H", [(8, 4, 4), (12, 4, 3), (16, 16, 4), (32, 8, 8), (30, 10, 6),
                                   (64, 16, 16)])
def test_fresh_steps_bit_exact(L, W, H, m):
    _compare(L, W, H, seed=L + W, T=1.7, Tw=0.6, nwin=5, **MAPS[m])


@pytest.mark.parametrize("T,h,rates", [(1.0, 0.05, "metropolis"), (3.5, 0.0, "metropolis"),
                                       (1.2, -0.2, "glauber")])
def test_fresh_steps_parameters(T, h, rates):
    L, W, H = 24, 8, 6
    lat = sr.Lattice(L, 1.0, h, T, (W, H), seed=9, rates=rates, fresh_steps=True)
    lat.run_windows(0.25, 8)
    ref = oracle.run(L, 1.0, h, T, W, H, 9, _ends(0.25, 8), glauber=(rates == "glauber"),
                     fresh_steps=True)
    assert np.array_equal(lat.spins(), ref.spins[-1])
    assert lat.observables().committed == int(ref.counts[-1].sum())


def test_fresh_steps_window_count_continues_across_calls():
    """Window indices of the random streams keep counting across run calls."""
    _compare(32, 8, 8, seed=4, Tw=0.5, nwin=6, calls=3)


def test_fresh_steps_in_a_batch():
    reps = [dict(L=32, T=1.5, h=0.05, seed=5), dict(L=16, T=3.0, h=0.0, seed=6),
            dict(L=24, T=2.0, h=-0.1, seed=7, rates="glauber")]
    tw, nw = [0.5, 0.25, 1.0], [4, 6, 2]
    with sr.Batch(reps, region=(8, 8), fresh_steps=True) as batch:
        batch.run(tw, nw)
        for b, r in enumerate(reps):
            ref = oracle.run(r["L"], 1.0, r["h"], r["T"], 8, 8, r["seed"], _ends(tw[b], nw[b]),
                             glauber=(r.get("rates") == "glauber"), fresh_steps=True)
            assert np.array_equal(batch.spins(b), ref.spins[-1]), b
            i, x, bb, t = batch.carry(b)
            assert np.array_equal(i, ref.carry_i)
            assert np.array_equal(x, ref.carry_x)


def test_fresh_steps_differ_from_the_carry_rule_and_need_lanes():
    a = sr.Lattice(32, 1.0, 0.05, 1.5, (8, 8), seed=3, fresh_steps=True)
    c = sr.Lattice(32, 1.0, 0.05, 1.5, (8, 8), seed=3)
    a.run_windows(0.5, 4)
    c.run_windows(0.5, 4)
    assert not np.array_equal(a.spins(), c.spins())
    with pytest.raises(sr.SRError):
        sr.Lattice(32, 1.0, 0.05, 1.5, (8, 8), seed=3, fresh_steps=True, lanes_per_region=32)
