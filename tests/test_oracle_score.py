"""The path statistics behind the score function (differentiation of time
averages with respect to beta = 1/T, h and J), pinned against exact
mathematics.

For the continuous-time chain of §3 the log-likelihood of a path on [0, t]
is sum_events log p_k(event) - integral sum_k N_k p_k ds, so its score is
S = sum_k C_k dlog p_k - sum_k dp_k I_k with C_k the events of class k and
I_k the integral of N_k.  Checked here: the bookkeeping identities, the
compensator (C_k - p_k I_k has mean zero), and d E[M(t)] / d theta =
E[M(t) S] against finite differences of the exact matrix exponential."""
import math

import numpy as np
import pytest
from scipy import linalg

import oracle
from test_oracle_physics import _all_states, _generator


def test_bookkeeping_identities():
    L, rw, rh, t = 24, 8, 6, 3.0
    r = oracle.run(L, 1.0, 0.05, 2.0, rw, rh, 5, [1.0, 2.0, t])
    assert np.array_equal(r.ev_class.sum(axis=1), r.counts[-1])
    sites = rw * rh
    assert np.allclose(r.occupancy.sum(axis=1), sites * t, rtol=1e-12, atol=0)
    # window ends split the integrals but do not change them
    r1 = oracle.run(L, 1.0, 0.05, 2.0, rw, rh, 5, [t])
    assert np.array_equal(r.ev_class, r1.ev_class)
    assert np.allclose(r.occupancy, r1.occupancy, rtol=1e-12, atol=1e-12)


def test_compensator_has_mean_zero():
    """C_k - p_k I_k is a martingale started at 0 (the events of class k come
    at rate N_k p_k): summed over 256 regions it is within a few standard
    deviations (its variance is E[C_k]) of zero for every class."""
    L, T, h = 128, 2.2, 0.1
    r = oracle.run(L, 1.0, h, T, 8, 8, 9, [4.0])
    p = oracle.rates(1.0, h, T)
    c = r.ev_class.sum(axis=0).astype(np.float64)
    occ = r.occupancy.sum(axis=0)
    for k in range(10):
        if c[k] < 50:
            continue
        z = (c[k] - p[k] * occ[k]) / math.sqrt(c[k])
        assert abs(z) < 5.0, (k, c[k], p[k] * occ[k], z)


def _exact_mean_m(J, h, T, glauber, t, L=3):
    """E[M(t)] from the all-up state, exactly: e_up^T exp(Q t) M."""
    S = _all_states(L)
    M = S.sum(axis=1).astype(np.float64)
    up = int(np.argmax(M))
    P = linalg.expm(_generator(L, J, h, T, glauber) * t)
    return float(P[up] @ M)


@pytest.mark.parametrize("J,h,T,glauber", [(1.0, 0.2, 2.5, False), (0.8, -0.1, 2.0, True)])
def test_score_derivative_matches_exact_dynamics(J, h, T, glauber):
    L, t, n = 3, 0.8, 20000
    ms, ss = np.zeros(n), np.zeros((n, 3))
    for i in range(n):
        r = oracle.run(L, J, h, T, L, L, 1000 + i, [t], init_mode=oracle.INIT_ALL_UP,
                       glauber=glauber, keep_spins=False, keep_counts=False)
        ms[i] = r.mag[-1]
        ss[i] = oracle.score(r, J, h, T, glauber)
    # the score has mean zero
    assert np.all(np.abs(ss.mean(axis=0)) < 4.5 * ss.std(axis=0) / math.sqrt(n))
    # d E[M] / d (beta, h, J): score estimate vs exact central differences
    est = (ms[:, None] * ss).mean(axis=0)
    se = (ms[:, None] * ss).std(axis=0) / math.sqrt(n)
    d = 1e-5
    beta = 1.0 / T
    exact = np.array([
        (_exact_mean_m(J, h, 1.0 / (beta + d), glauber, t)
         - _exact_mean_m(J, h, 1.0 / (beta - d), glauber, t)) / (2 * d),
        (_exact_mean_m(J, h + d, T, glauber, t) - _exact_mean_m(J, h - d, T, glauber, t)) / (2 * d),
        (_exact_mean_m(J + d, h, T, glauber, t) - _exact_mean_m(J - d, h, T, glauber, t)) / (2 * d)])
    assert np.all(np.abs(est - exact) < 4.0 * se + 1e-6), (est, exact, se)


def _exact_mean_m_start(J, h, T, t, init, L=3):
    """E[M(t)] exactly for the Metropolis chain: from the all-up state, or from
    fair-coin spins (every state equally likely)."""
    S = _all_states(L)
    M = S.sum(axis=1).astype(np.float64)
    P = linalg.expm(_generator(L, J, h, T, False) * t)
    if init == "up":
        return float(P[int(np.argmax(M))] @ M)
    return float(P.mean(axis=0) @ M)


@pytest.mark.parametrize("init,T,t,n", [("up", 3.5, 3.0, 160000), ("fair", 2.5, 0.8, 40000)])
def test_score_at_the_metropolis_kink(init, T, t, n):
    """h = 0 puts the n_up = 2 classes exactly on the kink of Eq. 2.2
    (dE = 2 s h = 0), where p = min(1, exp(-beta dE)) has different left and
    right derivatives in h.  Pinned against the exact chain of the 3x3
    lattice: the score built with the right-hand (left-hand) derivative at the
    kink estimates the exact right (left) derivative of E[M(t)] in h, and the
    table's mean of the two estimates the central difference.  From the all-up
    state the left and right derivatives differ; from fair-coin spins they are
    equal by symmetry, and a table that takes the right derivative for one
    spin sign and the left for the other misses by tens of standard errors."""
    J, h, beta = 1.0, 0.0, 1.0 / T
    mode = oracle.INIT_ALL_UP if init == "up" else oracle.INIT_FAIR_COIN
    ms, C, O = np.zeros(n), np.zeros((n, 10)), np.zeros((n, 10))
    for i in range(n):
        r = oracle.run(3, J, h, T, 3, 3, 1000 + i, [t], init_mode=mode, keep_spins=False,
                       keep_counts=False)
        ms[i] = r.mag[-1]
        C[i] = r.ev_class.sum(axis=0)
        O[i] = r.occupancy.sum(axis=0)
    dlogp, dp = oracle.score_tables(J, h, T)
    p = oracle.rates(J, h, T)
    # the kink classes: s = -1 (k = 2) and s = +1 (k = 7) with two up neighbours
    assert p[2] == 1.0 and p[7] == 1.0
    assert dlogp[1, 7] == -beta and dlogp[1, 2] == beta       # mean of -2 beta | 0 and 0 | 2 beta
    assert dlogp[0, 2] == dlogp[0, 7] == dlogp[2, 2] == dlogp[2, 7] == 0.0   # d(beta dE) = 0

    def estimate(tab_h):
        S = C @ tab_h - O @ (p * tab_h)
        a = ms * S
        return a.mean(), a.std() / math.sqrt(n)

    d = 1e-6
    e0 = _exact_mean_m_start(J, 0.0, T, t, init)
    right = (_exact_mean_m_start(J, d, T, t, init) - e0) / d
    left = (e0 - _exact_mean_m_start(J, -d, T, t, init)) / d
    central = 0.5 * (right + left)
    tab_right, tab_left, tab_mixed = dlogp[1].copy(), dlogp[1].copy(), dlogp[1].copy()
    tab_right[7], tab_right[2] = -2 * beta, 0.0
    tab_left[7], tab_left[2] = 0.0, 2 * beta
    tab_mixed[7], tab_mixed[2] = 0.0, 0.0
    for tab, want in ((dlogp[1], central), (tab_right, right), (tab_left, left)):
        est, se = estimate(tab)
        assert abs(est - want) < 4.0 * se + 1e-6, (init, est, want, se)
    if init == "fair":
        est, se = estimate(tab_mixed)
        assert abs(est - central) > 20.0 * se, (est, central, se)
    else:
        assert right - left > 0.3          # a real kink: one-sided tables would be biased
