"""The paper's efficiency theorems (§6), measured: with T_max chosen by
Eq. 5.1 (log N / (lambda |boundary|)), f (the most boundary events of a region
in an iteration) and g (iterations per step) grow no faster than log N as the
number of regions N grows with the region size fixed.

Theorem 1: E(f) <= C e log N + 1/(C - 1); Theorem 2: E(g) <= C e K log N +
1/(C - 1), for every C > 1, K = 13 (a region, its 4 neighbours and their 8
further neighbours on the square lattice).  Checked with C = 2."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")

BOUNDARY_16 = 60          # boundary sites of a 16 x 16 region
K_SET = 13


def _measure(L, T=3.0, windows=60, warm=20, seed=7):
    N = (L // 16) ** 2
    Tw = math.log(N) / (1.0 * BOUNDARY_16)    # Metropolis: the largest rate is 1
    lat = sr.Lattice(L, 1.0, 0.0, T, (16, 16), seed=seed)
    if warm:
        lat.run_windows(Tw, warm)
    lat.run_windows(Tw, windows)
    f = lat.window_f(windows).astype(np.float64)
    g = lat.window_iters(windows).astype(np.float64)
    o = lat.observables()
    lat.close()
    assert len(f) == windows and len(g) == windows
    return N, f, g, o


def test_window_f_matches_the_totals():
    N, f, g, o = _measure(128, windows=30, warm=0)
    assert int(f.sum()) == o.sum_f
    assert int(g.sum()) == o.iterations
    assert f.max() == o.max_f


def test_f_and_g_grow_like_log_N():
    rows = [_measure(L) for L in (64, 256, 1024)]
    rf, rg = [], []
    for N, f, g, _ in rows:
        lg = math.log(N)
        assert f.mean() <= 2 * math.e * lg + 1.0, (N, f.mean())
        assert g.mean() <= 2 * math.e * K_SET * lg + 1.0, (N, g.mean())
        rf.append(f.mean() / lg)
        rg.append(g.mean() / lg)
    # from N = 16 to N = 4096 regions (log N x 3), f / log N and g / log N stay
    # within a factor of 3 of each other: no faster than logarithmic growth
    assert max(rf) / min(rf) < 3.0, rf
    assert max(rg) / min(rg) < 3.0, rg
