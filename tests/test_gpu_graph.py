"""Relaxation launches replayed from a CUDA graph (sr_set_graph_launch).

The graph holds the same uploads, kernel and read-back as a direct launch, so
every lattice's trajectory must be the oracle's, bit for bit, and equal to
the direct launches of an identical context: spins, the clock carry, the
exact integer observables and the counters of the procedure of §4.  The
graph is captured once and replayed while the kernel parameters stay the
same; a new ring length or history capacity recaptures it."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")

INIT = {"fair": oracle.INIT_FAIR_COIN, "up": oracle.INIT_ALL_UP}

REPS = [dict(L=32, J=1.0, h=0.05, T=1.5, seed=21),
        dict(L=16, J=0.8, h=-0.2, T=1.2, seed=22, rates="glauber"),
        dict(L=48, J=1.0, h=0.0, T=2.269, seed=23, init="up"),
        dict(L=24, J=1.0, h=0.2, T=3.5, seed=24),
        dict(L=40, J=0.0, h=0.3, T=2.0, seed=25)]
TW = [1.0, 0.5, 0.25, 0.5, 1.0]
NW = [2, 3, 4, 2, 1]

MAPS = [dict(),                                             # asynchronous schedule
        dict(lanes_per_region=1, lanes_per_warp=32, schedule=1),
        dict(lanes_per_region=32)]


def _same(a, b, n):
    for q in range(n):
        assert np.array_equal(a.spins(q), b.spins(q)), f"spins of lattice {q}"
        for u, v in zip(a.carry(q), b.carry(q)):
            assert np.array_equal(u, v), f"clock carry of lattice {q}"
        oa, ob = a.observables(q), b.observables(q)
        for f in ("t_c", "mag", "bonds", "int_mag", "int_bonds", "committed", "generated",
                  "breaks", "windows", "iterations", "sum_f", "max_f"):
            assert getattr(oa, f) == getattr(ob, f), f"{f} of lattice {q}"


@pytest.mark.parametrize("m", range(len(MAPS)))
def test_graph_replays_match_direct_launches_and_oracle(m):
    with sr.Batch(REPS, region=(8, 8), **MAPS[m]) as direct, \
            sr.Batch(REPS, region=(8, 8), **MAPS[m]) as graph:
        graph.graph_launch(True)
        for _ in range(3):                      # the same plan: one capture, then replays
            direct.run(TW, NW)
            graph.run(TW, NW)
        captures, replays = graph.graph_stats()
        assert replays >= 3 and 1 <= captures < replays
        _same(direct, graph, len(REPS))
        for q, r in enumerate(REPS):
            ends, t = [], 0.0
            for _ in range(3 * NW[q]):
                t = t + TW[q]
                ends.append(t)
            ref = oracle.run(r["L"], r["J"], r["h"], r["T"], 8, 8, r["seed"], ends,
                             init_mode=INIT[r.get("init", "fair")],
                             glauber=r.get("rates") == "glauber")
            assert np.array_equal(graph.spins(q), ref.spins[-1]), f"lattice {q} against the oracle"
            o = graph.observables(q)
            assert o.mag == ref.mag[-1] and o.bonds == ref.bonds[-1]
            assert o.committed == int(ref.counts[-1].sum())
        assert direct.graph_stats() == (0, 0)


def test_graph_adaptive_runs_match():
    """The adaptive runner changes window lengths from chunk to chunk; the
    graph's staged plan carries them, and a new ring length recaptures it."""
    with sr.Batch(REPS, region=(8, 8)) as direct, sr.Batch(REPS, region=(8, 8)) as graph:
        graph.graph_launch(True)
        direct.run_adaptive(6.0, kappa=8.0)
        graph.run_adaptive(6.0, kappa=8.0)
        _same(direct, graph, len(REPS))
        captures, replays = graph.graph_stats()
        assert replays >= 6 and captures >= 1


def test_graph_recaptures_after_capacity_growth():
    """Windows long enough to overflow the first history capacity: the
    capacity doubles, the kernel parameters change and the graph is captured
    again; the trajectory is still the direct one."""
    # regions of 32 x 2 sites: every flip is on the north or south edge, so a
    # window of 4 time units at T = 3.5 puts about 75 entries on each list
    reps = [dict(L=32, J=1.0, h=0.0, T=3.5, seed=31)]
    with sr.Batch(reps, region=(32, 2)) as direct, sr.Batch(reps, region=(32, 2)) as graph:
        graph.graph_launch(True)
        direct.run([0.25], [2])
        graph.run([0.25], [2])
        c0, _ = graph.graph_stats()
        direct.run([4.0], [1])
        graph.run([4.0], [1])
        _same(direct, graph, 1)
        assert graph.observables(0).capacity > 64
        c1, _ = graph.graph_stats()
        assert c1 > c0


def test_single_lattice_graph_and_off_again():
    with sr.Lattice(64, 1.0, 0.05, 1.5, (16, 16), seed=41) as direct, \
            sr.Lattice(64, 1.0, 0.05, 1.5, (16, 16), seed=41) as graph:
        graph.graph_launch(True)
        direct.run_windows(1.0, 3)
        graph.run_windows(1.0, 3)
        graph.graph_launch(False)               # frees the graph; direct launches again
        direct.run_windows(1.0, 2)
        graph.run_windows(1.0, 2)
        assert np.array_equal(direct.spins(), graph.spins())
        oa, ob = direct.observables(), graph.observables()
        assert (oa.mag, oa.bonds, oa.committed, oa.iterations) == \
               (ob.mag, ob.bonds, ob.committed, ob.iterations)
        assert graph.graph_stats()[1] >= 1
