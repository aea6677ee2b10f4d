"""Pins for the oracle's building blocks against definitions that do not come
from the oracle itself: published Philox known-answer vectors, libm's log, the
closed-form Metropolis/Glauber rates of Eqs. 2.2-2.3, and the selection rule of
Eqs. 3.5-3.8 re-derived with exact rationals."""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle


def test_philox_known_answers():
    # Known-answer vectors published with the Random123 library (Salmon et
    # al., SC'11) for Philox4x32 with 10 rounds.
    with open(__file__.replace("test_oracle_numerics.py", "golden/philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 3
    for row in rows:
        vals = [int(v, 16) for v in row]
        ctr, key, want = vals[0:4], vals[4:6], tuple(vals[6:10])
        assert oracle.philox(ctr, key) == want


def test_unit_is_exact_and_open():
    for k in [0, 1, 2, 2**51, 2**52 - 1, 987654321]:
        u = oracle.unit_from_bits(k)
        assert Fraction(u) == Fraction(2 * k + 1, 2**53)
        assert 0.0 < u < 1.0


def _ulp(x):
    return math.ulp(x)


def test_neglog_close_to_libm():
    rng = random.Random(5)
    ks = [0, 1, 2, 3, 2**51 - 1, 2**51, 2**52 - 1, 2**52 - 2, 3 << 49, 1 << 30]
    ks += [rng.getrandbits(52) for _ in range(20000)]
    ks += [rng.getrandbits(rng.randint(1, 52)) for _ in range(5000)]
    worst = 0.0
    for k in ks:
        u = oracle.unit_from_bits(k)
        want = -math.log(u)
        got = oracle.neglog_unit(k)
        err = abs(got - want) / _ulp(want)
        worst = max(worst, err)
    assert worst <= 4.0, worst


def test_neglog_is_positive_and_monotone():
    rng = random.Random(6)
    ks = sorted(rng.getrandbits(52) for _ in range(3000))
    vals = [oracle.neglog_unit(k) for k in ks]
    assert all(v > 0 for v in vals)
    assert all(a >= b for a, b in zip(vals, vals[1:]))


@pytest.mark.parametrize("J,h,T", [(1.0, 0.05, 1.5), (1.0, 0.05, 1.0), (1.0, 0.0, 1.0),
                                   (1.0, 0.0, 2.269), (1.0, 0.0, 3.5), (0.7, -0.2, 2.0),
                                   (0.0, 0.3, 1.0)])
def test_metropolis_and_glauber_rates(J, h, T):
    p = oracle.rates(J, h, T)
    g = oracle.rates(J, h, T, glauber=True)
    for k in range(10):
        s = 1 if k >= 5 else -1
        n_up = k % 5
        nb = n_up - (4 - n_up)
        dE = 2 * s * (J * nb + h)
        theta = math.exp(-dE / T)
        assert p[k] == pytest.approx(min(1.0, theta), rel=1e-15)
        assert g[k] == pytest.approx(theta / (1 + theta), rel=1e-15)
    # detailed balance between a site's two spin states with the same neighbours:
    # p(s -> -s) / p(-s -> s) = exp(-dE/T)
    for n_up in range(5):
        nb = 2 * n_up - 4
        dE_down_to_up = 2 * (-1) * (J * nb + h)
        assert p[n_up] / p[5 + n_up] == pytest.approx(math.exp(-dE_down_to_up / T), rel=1e-12)


def test_fixed_point_rates():
    for sites, F in [(256, 54), (1024, 52), (9, 59), (1, 62), (1 << 20, 42)]:
        assert oracle.frac_bits(sites) == F
        assert sites * (1 << F) < (1 << 63)
    p = oracle.rates(1.0, 0.05, 1.5)
    P = oracle.rates_fixed(p, 54)
    for k in range(10):
        assert abs(Fraction(int(P[k]), 1 << 54) - Fraction(p[k])) <= Fraction(1, 1 << 55)


def _select_rational(N, P, kV):
    """Eqs. 3.5-3.8 with exact rationals: W(k) = sum_{j<=k} N_j p_j / Lambda,
    class k with W(k-1) < V <= W(k), R = (V - W(k-1)) / (N_k p_k / Lambda),
    0-based index = floor(R N_k) (Eq. 3.8 minus one), at most N_k - 1."""
    p = [Fraction(int(x)) for x in P]
    lam = sum(n * q for n, q in zip(N, p))
    V = Fraction(2 * kV + 1, 2**53)
    W_prev = Fraction(0)
    for k in range(10):
        W = W_prev + N[k] * p[k] / lam
        if W_prev < V <= W:
            R = (V - W_prev) / (N[k] * p[k] / lam)
            idx = math.floor(R * N[k])
            return k, min(idx, N[k] - 1)
        W_prev = W
    raise AssertionError("no class found")


def test_select_matches_rational_definition():
    rng = random.Random(7)
    for trial in range(3000):
        sites = rng.choice([9, 16, 256, 1024])
        F = oracle.frac_bits(sites)
        T = rng.choice([0.5, 1.0, 1.5, 2.269, 3.5])
        h = rng.choice([0.0, 0.05, -0.2])
        P = oracle.rates_fixed(oracle.rates(1.0, h, T, glauber=bool(trial % 2)), F)
        cut = sorted(rng.randint(0, sites) for _ in range(9))
        N = [b - a for a, b in zip([0] + cut, cut + [sites])]
        kV = rng.getrandbits(52)
        if trial % 10 == 0:
            kV = rng.choice([0, 2**52 - 1])
        assert oracle.select(N, P, kV) == _select_rational(N, P, kV)


def test_select_frequencies_are_proportional_to_rates():
    # Over a uniform grid of V, each (class, position) pair must be chosen with
    # frequency p_k / Lambda: the n-fold way picks a site with probability
    # proportional to its own flip rate (§3).
    F = oracle.frac_bits(16)
    P = oracle.rates_fixed(oracle.rates(1.0, 0.05, 1.5), F)
    N = [1, 0, 3, 2, 0, 4, 0, 2, 3, 1]
    lam = sum(n * int(q) for n, q in zip(N, P))
    M = 200000
    counts = {}
    for j in range(M):
        kV = ((2 * j + 1) << 52) // (2 * M)      # V close to (j + 1/2) / M
        key = oracle.select(N, P, kV)
        counts[key] = counts.get(key, 0) + 1
    for k in range(10):
        for pos in range(N[k]):
            want = int(P[k]) / lam
            got = counts.get((k, pos), 0) / M
            assert abs(got - want) <= 2.0 / M + 1e-12, (k, pos, got, want)
    assert sum(counts.values()) == M


def test_tau_without_break_points_is_eq_3_4():
    F = oracle.frac_bits(256)
    rng = random.Random(8)
    for _ in range(2000):
        lamf = rng.randint(1, 256 << F)
        lam = oracle.lam(lamf, F)
        assert lam == math.ldexp(float(lamf), -F)
        t0 = rng.uniform(0, 100)
        x = oracle.neglog_unit(rng.getrandbits(52))
        t = oracle.tau(t0, x, 0.0, lamf, F)
        assert t == max(t0 + x / lam, math.nextafter(t0, math.inf))
    assert oracle.tau(1.0, 1.0, 0.0, 0, F) == math.inf


def test_tau_with_break_point_solves_eq_5_2():
    # Integral of Lambda from the last event to tau equals -log U (Eq. 5.2),
    # with one break point at t_b where the rate changes from lam1 to lam2.
    F = oracle.frac_bits(256)
    rng = random.Random(9)
    for _ in range(500):
        l1 = rng.randint(1 << F, 200 << F)
        l2 = rng.randint(1 << F, 200 << F)
        x = oracle.neglog_unit(rng.getrandbits(52))
        t_prev = rng.uniform(0, 10)
        tau1 = oracle.tau(t_prev, x, 0.0, l1, F)
        tb = t_prev + (tau1 - t_prev) * rng.uniform(0.01, 0.99)
        b = 0.0 + oracle.lam(l1, F) * (tb - t_prev)
        tau2 = oracle.tau(tb, x, b, l2, F)
        integral = oracle.lam(l1, F) * (tb - t_prev) + oracle.lam(l2, F) * (tau2 - tb)
        assert integral == pytest.approx(x, rel=1e-12, abs=1e-12)
        assert tau2 > tb
