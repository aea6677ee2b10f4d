"""Checkpoint and resume (§5, "Subsequent steps": the state one window hands
to the next).  A context loaded from a checkpoint must continue bit for bit as
the saved one would have: same spins, clock carry, integrals, counters and
score statistics as a run that never stopped, and the oracle's trajectory."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")


def _state(lat):
    o = lat.observables()
    return (lat.spins(), lat.carry(),
            (o.t_c, o.mag, o.bonds, o.int_mag, o.int_bonds, o.committed, o.generated, o.breaks,
             o.windows, o.iterations, o.sum_f, o.max_f))


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    assert a[2] == b[2]


@pytest.mark.parametrize("kw", [dict(), dict(score=True), dict(fresh_steps=True),
                                dict(lanes_per_region=32), dict(lanes_per_warp=3, time_arith=2)])
def test_resume_is_bit_identical(kw):
    args = (64, 1.0, 0.05, 1.5, (16, 16))
    full = sr.Lattice(*args, seed=3, **kw)
    full.run_windows(0.5, 6)
    want = _state(full)
    want_score = full.score_stats() if kw.get("score") else None
    full.close()

    first = sr.Lattice(*args, seed=3, **kw)
    first.run_windows(0.5, 3)
    ck = first.checkpoint()
    first.close()
    resumed = sr.Lattice(*args, seed=3, **kw)
    resumed.load_checkpoint(ck)
    assert resumed.t_c == 1.5
    resumed.run_windows(0.5, 3)
    _same(_state(resumed), want)
    if want_score is not None:
        c, occ = resumed.score_stats()
        assert np.array_equal(c, want_score[0]) and np.array_equal(occ, want_score[1])
    # the oracle's window ends matter only under the alternate step rule
    ends = [0.5 * k for k in range(1, 7)]
    ref = oracle.run(64, 1.0, 0.05, 1.5, 16, 16, 3, ends, fresh_steps=bool(kw.get("fresh_steps")))
    assert np.array_equal(resumed.spins(), ref.spins[-1])
    resumed.close()


def test_batch_resume_is_bit_identical():
    reps = [dict(L=32, J=1.0, h=0.1, T=2.0, seed=21), dict(L=48, J=1.0, h=0.0, T=3.0, seed=22),
            dict(L=16, J=0.8, h=-0.2, T=1.2, seed=23, rates="glauber")]
    tw = [0.5, 0.25, 1.0]
    with sr.Batch(reps, region=(8, 8)) as full:
        full.run(tw, [4, 6, 2])
        want = [(full.spins(b), full.carry(b), full.observables(b)) for b in range(3)]
    with sr.Batch(reps, region=(8, 8)) as first:
        first.run(tw, [2, 3, 1])
        ck = first.checkpoint()
    with sr.Batch(reps, region=(8, 8)) as resumed:
        resumed.load_checkpoint(ck)
        assert list(resumed.t_c) == [1.0, 0.75, 1.0]
        resumed.run(tw, [2, 3, 1])
        for b in range(3):
            assert np.array_equal(resumed.spins(b), want[b][0])
            for x, y in zip(resumed.carry(b), want[b][1]):
                assert np.array_equal(x, y)
            o, w = resumed.observables(b), want[b][2]
            assert (o.t_c, o.committed, o.generated, o.windows, o.int_mag) == \
                   (w.t_c, w.committed, w.generated, w.windows, w.int_mag)


def test_a_checkpoint_only_loads_into_its_own_lattice():
    a = sr.Lattice(32, 1.0, 0.05, 1.5, (16, 16), seed=5)
    a.run_windows(1.0, 2)
    ck = a.checkpoint()
    other = sr.Lattice(32, 1.0, 0.05, 1.5, (16, 16), seed=6)
    other.run_windows(1.0, 1)
    before = _state(other)
    lib = sr.library()
    for bad in (ck[:-1], ck + b"\0", b"\0" * len(ck)):
        assert lib.sr_checkpoint_load(other._ctx, bad, len(bad)) == sr.SR_EINVAL
    with pytest.raises(sr.SRError) as e:          # another seed: another trajectory
        other.load_checkpoint(ck)
    assert e.value.code == sr.SR_EINVAL
    _same(_state(other), before)                  # a refused load changes nothing
    for kw in (dict(score=True), dict(region=(8, 8))):
        args = dict(L=32, J=1.0, h=0.05, T=1.5, region=(16, 16), seed=5)
        args.update(kw)
        with pytest.raises(sr.SRError):
            sr.Lattice(**args).load_checkpoint(ck)
