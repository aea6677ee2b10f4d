"""Pins for the oracle's dynamics against results fixed by the mathematics of
the model, not by the oracle: the exact transition law of the 3x3 periodic
lattice (matrix exponential of its generator), exact Boltzmann weights by
enumeration (Eq. 2.1), the T -> infinity and J = 0 closed forms, Onsager's
spontaneous magnetisation, and the book-keeping invariants of §3."""
import math

import numpy as np
import pytest
from scipy import linalg, stats

import oracle


# ----------------------------------------------------------------- helpers
def _neighbours(L):
    idx = np.arange(L * L).reshape(L, L)
    return [np.roll(idx, -1, axis=1).ravel(), np.roll(idx, 1, axis=1).ravel(),
            np.roll(idx, -1, axis=0).ravel(), np.roll(idx, 1, axis=0).ravel()]


def _all_states(L):
    n = L * L
    codes = np.arange(1 << n, dtype=np.int64)
    return np.where((codes[:, None] >> np.arange(n)) & 1, 1, -1).astype(np.int64)


def _energy(spins, L, J, h):
    """Eq. 2.1 with every nearest-neighbour bond counted once."""
    nb = _neighbours(L)
    bonds = (spins * spins[:, nb[0]]).sum(1) + (spins * spins[:, nb[2]]).sum(1)
    return -J * bonds - h * spins.sum(1), bonds, spins.sum(1)


def _generator(L, J, h, T, glauber):
    S = _all_states(L)
    n = L * L
    nb = _neighbours(L)
    Q = np.zeros((1 << n, 1 << n))
    rows = np.arange(1 << n)
    for v in range(n):
        field = sum(S[:, nb[d][v]] for d in range(4))
        dE = 2.0 * S[:, v] * (J * field + h)
        theta = np.exp(-dE / T)
        rate = theta / (1 + theta) if glauber else np.minimum(1.0, theta)
        Q[rows, rows ^ (1 << v)] += rate
    Q[rows, rows] = -Q.sum(1)
    return Q


def _codes(spins):
    flat = spins.reshape(spins.shape[0], -1)
    return ((flat > 0).astype(np.int64) << np.arange(flat.shape[1])).sum(1)


# ----------------------------------------------------------------- invariants
@pytest.mark.parametrize("L,rw,rh", [(6, 1, 1), (6, 2, 3), (6, 3, 2), (6, 6, 6), (6, 6, 1),
                                     (6, 1, 6), (8, 4, 4), (8, 8, 2), (8, 2, 8), (3, 1, 1),
                                     (4, 2, 2), (9, 3, 3)])
def test_invariants_after_every_event(L, rw, rh):
    """N_k sums, classes, Lambda = sum N_k p_k, spin and bond sums recounted
    from scratch after every event (§3)."""
    ends = [0.5 * (i + 1) for i in range(8)]
    r = oracle.run(L, 1.0, 0.05, 1.7, rw, rh, 11, ends, debug=True, trace_cap=100000)
    assert r.debug_failures == 0
    nreg = (L // rw) * (L // rh)
    assert r.trace_len == int(r.counts[-1].sum())
    for q in range(nreg):
        sel = r.tr_region == q
        assert np.array_equal(r.tr_index[sel], np.arange(sel.sum()))
        assert np.all(np.diff(r.tr_time[sel]) > 0)          # strictly increasing
        # every event of region q flips a site of region q
        xs, ys = r.tr_site[sel] % L, r.tr_site[sel] // L
        assert np.all((ys // rh) * (L // rw) + xs // rw == q)
    assert np.all(np.diff(r.tr_time) >= 0)                    # global time order
    assert np.all(r.tr_time < ends[-1])
    # spins after the trace replayed from the initial state
    init = oracle.run(L, 1.0, 0.05, 1.7, rw, rh, 11, [0.0]).spins[0].ravel().copy()
    for site in r.tr_site:
        init[site] = -init[site]
    assert np.array_equal(init, r.spins[-1].ravel())


def test_window_ends_do_not_change_the_trajectory():
    """Window ends are not break points (§5, 'Subsequent steps')."""
    base = dict(L=16, J=1.0, h=0.05, T=1.5, region_w=4, region_h=4, seed=3, trace_cap=200000)
    a = oracle.run(t_end=[float(i) for i in range(1, 11)], **base)
    b = oracle.run(t_end=[2.5, 5.0, 7.5, 10.0], **base)
    c = oracle.run(t_end=[10.0], **base)
    for other in (b, c):
        assert np.array_equal(a.spins[-1], other.spins[-1])
        assert np.array_equal(a.tr_time, other.tr_time)
        assert np.array_equal(a.tr_site, other.tr_site)
        for f in ("carry_i", "carry_x", "carry_b", "carry_t"):
            assert np.array_equal(getattr(a, f), getattr(other, f))


# ----------------------------------------------------------------- exact dynamics
@pytest.mark.parametrize("rw,rh,J,h,T,glauber", [
    (3, 3, 1.0, 0.05, 2.5, False),
    (1, 1, 1.0, 0.05, 2.5, False),
    (3, 1, 1.0, -0.2, 2.0, False),
    (1, 3, 0.8, 0.3, 1.8, True),
    (1, 1, 1.0, 0.0, 3.5, True),
])
def test_transition_law_matches_matrix_exponential(rw, rh, J, h, T, glauber):
    """The sampled chain at lag dt must have the transition matrix exp(Q dt)
    of the continuous-time Markov chain of §3 (site v flips at rate p(v))."""
    L, dt, nwin = 3, 0.3, 40000
    P = linalg.expm(_generator(L, J, h, T, glauber) * dt)
    r = oracle.run(L, J, h, T, rw, rh, 21, [dt * (i + 1) for i in range(nwin)], glauber=glauber,
                   keep_counts=False)
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
    pval = stats.chi2.sf(chi2, dof)
    assert dof > 20
    assert pval > 1e-3, (chi2, dof, pval)


@pytest.mark.parametrize("rw,rh,T,h", [(2, 2, 3.0, 0.05), (4, 4, 2.5, 0.0), (1, 4, 5.0, 0.05)])
def test_boltzmann_by_enumeration_4x4(rw, rh, T, h):
    """Long-run occupation of the (E, M) levels of the 4x4 periodic lattice
    equals exact Boltzmann weights exp(-E/T) summed over the 65536 states."""
    L, J = 4, 1.0
    S = _all_states(L)
    E, _, M = _energy(S, L, J, h)
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    levels = {}
    for e, m, pw in zip(E, M, w):
        key = (round(e, 9), int(m))
        levels[key] = levels.get(key, 0.0) + pw
    dt, nwin = 15.0, 6000
    r = oracle.run(L, J, h, T, rw, rh, 31, [dt * (i + 1) for i in range(nwin)], keep_counts=False)
    Es, _, Ms = _energy(r.spins.reshape(nwin, -1).astype(np.int64), L, J, h)
    keys = sorted(levels)
    index = {k: i for i, k in enumerate(keys)}
    obs = np.zeros(len(keys))
    for e, m in zip(Es, Ms):
        obs[index[(round(e, 9), int(m))]] += 1
    expect = np.array([levels[k] for k in keys]) * nwin
    big = expect >= 5
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(expect[big], expect[~big].sum())
    chi2 = ((o - e) ** 2 / e).sum()
    pval = stats.chi2.sf(chi2, len(o) - 1)
    assert pval > 1e-3, (chi2, len(o), pval)


# ----------------------------------------------------------------- closed forms
def test_infinite_temperature_poisson_counts_and_correlation():
    """T -> infinity: every p_k = 1, Lambda = |G_i| is constant, each region's
    event count on [0, t] is Poisson(|G_i| t) and <s(0) s(t)> = exp(-2 t)."""
    L, rw = 64, 8
    ts = [0.25, 0.5, 1.0]
    r0 = oracle.run(L, 1.0, 0.0, 1e300, rw, rw, 41, [0.0])
    r = oracle.run(L, 1.0, 0.0, 1e300, rw, rw, 41, ts)
    s0 = r0.spins[0].astype(np.float64).ravel()
    for i, t in enumerate(ts):
        c = float((s0 * r.spins[i].ravel()).mean())
        assert abs(c - math.exp(-2 * t)) < 4.0 / L, (t, c)
    counts = r.counts[-1].astype(np.float64)
    mu = rw * rw * ts[-1]
    n = len(counts)
    assert abs(counts.mean() - mu) < 4 * math.sqrt(mu / n)
    # dispersion test: sum (c - mu)^2 / mu ~ chi2(n)
    disp = ((counts - mu) ** 2 / mu).sum()
    assert stats.chi2.sf(disp, n) > 1e-3 and stats.chi2.cdf(disp, n) > 1e-3


def test_field_only_relaxation_closed_form():
    """J = 0: independent two-state chains with r(- -> +) = min(1, e^{2h/T})
    and r(+ -> -) = min(1, e^{-2h/T}); m(t) = m_eq + (m_0 - m_eq) e^{-(r+ + r-) t}."""
    L, h, T = 128, 0.3, 1.0
    ts = [0.2, 0.5, 1.0, 2.0, 4.0]
    r = oracle.run(L, 0.0, h, T, 16, 16, 51, ts, init_mode=oracle.INIT_ALL_DOWN)
    up = min(1.0, math.exp(2 * h / T))
    down = min(1.0, math.exp(-2 * h / T))
    m_eq = (up - down) / (up + down)
    assert m_eq == pytest.approx(math.tanh(h / T))
    for i, t in enumerate(ts):
        want = m_eq + (-1.0 - m_eq) * math.exp(-(up + down) * t)
        got = r.mag[i] / (L * L)
        assert abs(got - want) < 4.0 / L, (t, got, want)


@pytest.mark.parametrize("T,tol", [(1.5, 2e-3), (1.8, 4e-3)])
def test_onsager_spontaneous_magnetisation(T, tol):
    """J = 1, h = 0, T < T_c = 2/ln(1+sqrt 2): |m| -> (1 - sinh(2/T)^-4)^(1/8)."""
    L = 512
    ends = [float(t) for t in range(1, 41)]
    r = oracle.run(L, 1.0, 0.0, T, 32, 32, 61, ends, init_mode=oracle.INIT_ALL_UP,
                   keep_spins=False, keep_counts=False)
    m = np.abs(r.mag[15:]) / (L * L)
    m0 = (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125
    assert abs(m.mean() - m0) < tol, (m.mean(), m0)


def test_energy_bookkeeping_matches_recount():
    L = 32
    r = oracle.run(L, 1.0, 0.05, 2.0, 8, 8, 71, [1.0, 2.0, 3.0])
    for w in range(3):
        s = r.spins[w].astype(np.int64)
        bonds = (s * np.roll(s, -1, 0)).sum() + (s * np.roll(s, -1, 1)).sum()
        assert r.bonds[w] == bonds and r.mag[w] == s.sum()
