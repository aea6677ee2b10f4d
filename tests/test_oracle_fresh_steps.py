"""The alternate step rule of §5 ("An alternate approach to subsequent
steps") in the oracle: at every committed time all clocks restart with new
random numbers.  The paper states that for the Ising model this stays
unbiased (exponential waiting times are memoryless); these tests pin that
against the exact law of the chain, independently of the oracle's code."""
import math

import numpy as np
import pytest
from scipy import linalg, stats

import oracle
from test_oracle_physics import _codes, _generator


@pytest.mark.parametrize("rw,rh,J,h,T,glauber", [
    (3, 3, 1.0, 0.05, 2.5, False),
    (1, 1, 1.0, 0.05, 2.5, False),
    (1, 3, 0.8, 0.3, 1.8, True),
])
def test_transition_law_with_restarts(rw, rh, J, h, T, glauber):
    """Restarting every clock at each sample time leaves the lag-dt transition
    matrix exp(Q dt) of the chain unchanged."""
    L, dt, nwin = 3, 0.3, 40000
    P = linalg.expm(_generator(L, J, h, T, glauber) * dt)
    r = oracle.run(L, J, h, T, rw, rh, 23, [dt * (i + 1) for i in range(nwin)], glauber=glauber,
                   keep_counts=False, fresh_steps=True)
    codes = _codes(r.spins)
    src, dst = codes[:-1], codes[1:]
    chi2, dof = 0.0, 0
    for s in np.unique(src):
        nxt = dst[src == s]
        n = len(nxt)
        expect = n * P[s]
        obs = np.bincount(nxt, minlength=P.shape[0]).astype(float)
        big = expect >= 5
        if big.sum() == 0:
            continue
        e_rest, o_rest = n - expect[big].sum(), n - obs[big].sum()
        chi2 += (((obs[big] - expect[big]) ** 2) / expect[big]).sum()
        bins = int(big.sum())
        if e_rest >= 1:
            chi2 += (o_rest - e_rest) ** 2 / e_rest
            bins += 1
        dof += bins - 1
    assert dof > 20
    assert stats.chi2.sf(chi2, dof) > 1e-3, (chi2, dof)


def test_restarts_keep_poisson_counts():
    """T -> infinity with a restart every 0.05: each region's count on [0, t]
    is still Poisson(|G_i| t)."""
    L, rw, t = 64, 8, 1.0
    ends = [0.05 * (i + 1) for i in range(20)]
    r = oracle.run(L, 1.0, 0.0, 1e300, rw, rw, 43, ends, fresh_steps=True)
    counts = r.counts[-1].astype(np.float64)
    mu = rw * rw * t
    n = len(counts)
    assert abs(counts.mean() - mu) < 4 * math.sqrt(mu / n)
    disp = ((counts - mu) ** 2 / mu).sum()
    assert stats.chi2.sf(disp, n) > 1e-3 and stats.chi2.cdf(disp, n) > 1e-3


@pytest.mark.parametrize("L,rw,rh", [(6, 2, 3), (8, 4, 4), (6, 6, 6), (9, 3, 1)])
def test_invariants_and_trace_with_restarts(L, rw, rh):
    ends = [0.4 * (i + 1) for i in range(10)]
    r = oracle.run(L, 1.0, 0.05, 1.7, rw, rh, 13, ends, debug=True, trace_cap=100000,
                   fresh_steps=True)
    assert r.debug_failures == 0
    nreg = (L // rw) * (L // rh)
    for q in range(nreg):
        sel = r.tr_region == q
        assert np.array_equal(r.tr_index[sel], np.arange(sel.sum()))
        assert np.all(np.diff(r.tr_time[sel]) > 0)
    init = oracle.run(L, 1.0, 0.05, 1.7, rw, rh, 13, [0.0]).spins[0].ravel().copy()
    for site in r.tr_site:
        init[site] = -init[site]
    assert np.array_equal(init, r.spins[-1].ravel())


def test_restarts_depend_on_the_window_ends():
    """Unlike the carry rule, the trajectory now depends on where the steps
    end; with a single step both rules draw from different streams."""
    base = dict(L=16, J=1.0, h=0.05, T=1.5, region_w=4, region_h=4, seed=3, fresh_steps=True)
    a = oracle.run(t_end=[float(i) for i in range(1, 11)], **base)
    b = oracle.run(t_end=[2.5, 5.0, 7.5, 10.0], **base)
    assert not np.array_equal(a.spins[-1], b.spins[-1])
    # the first window is common to a run with one more window
    c = oracle.run(t_end=[1.0], **base)
    assert np.array_equal(a.spins[0], c.spins[0])
    assert np.array_equal(a.counts[0], c.counts[0])
