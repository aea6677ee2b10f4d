"""Pins for the oracle's time integrals of the spin sum M and the bond sum
(the integrals of the observables of Eq. 2.1 along the piecewise-constant
path of §3, which the score-function averages are built from).

* Recount: M(t) and the bond sum are recounted from the spins themselves
  (not from the oracle's running sums) after every event of the oracle's
  trace, and integrated segment by segment between events and up to each
  window end; the result must equal int_mag and int_bonds bit for bit.
* Closed form: with J = 0 every spin is an independent two-state chain
  (rates min(1, e^{-2 beta h}) down and min(1, e^{2 beta h}) up), so E[m(t)],
  its integral and the integral of E[bonds] = 2 L^2 m(t)^2 are known exactly."""
import math

import numpy as np
import pytest

import oracle


def _recount(spins):
    s = spins.astype(np.int64)
    bonds = (s * np.roll(s, -1, axis=1)).sum() + (s * np.roll(s, -1, axis=0)).sum()
    return int(s.sum()), int(bonds)


@pytest.mark.parametrize("L,rw,rh,T,h,init", [(12, 4, 4, 2.0, 0.1, oracle.INIT_FAIR_COIN),
                                              (12, 6, 3, 2.8, -0.2, oracle.INIT_ALL_UP),
                                              (9, 3, 3, 3.0, 0.0, oracle.INIT_FAIR_COIN),
                                              (8, 8, 8, 3.5, 0.05, oracle.INIT_ALL_DOWN)])
def test_integrals_equal_a_recount_along_the_trace(L, rw, rh, T, h, init):
    ends = [0.5, 1.0, 1.75, 3.0, 4.0]
    r = oracle.run(L, 1.0, h, T, rw, rh, 21, ends, init_mode=init, trace_cap=1 << 20)
    assert r.trace_len == len(r.tr_time) >= 50
    spins = oracle.run(L, 1.0, h, T, rw, rh, 21, [0.0], init_mode=init).spins[0].copy()
    M, B = _recount(spins)
    im, ib, t_prev, j = 0.0, 0.0, 0.0, 0
    for w, te in enumerate(ends):
        while j < len(r.tr_time) and r.tr_time[j] < te:
            t = float(r.tr_time[j])
            im += float(M) * (t - t_prev)           # the value held before the flip
            ib += float(B) * (t - t_prev)
            t_prev = t
            site = int(r.tr_site[j])
            spins.flat[site] = -spins.flat[site]
            M, B = _recount(spins)
            j += 1
        im += float(M) * (te - t_prev)              # the last segment, closed at the window end
        ib += float(B) * (te - t_prev)
        t_prev = te
        assert (M, B) == (int(r.mag[w]), int(r.bonds[w]))
        assert np.array_equal(spins, r.spins[w])
        assert im == r.int_mag[w] and ib == r.int_bonds[w], (w, im, r.int_mag[w], ib, r.int_bonds[w])
    assert j == len(r.tr_time)


@pytest.mark.parametrize("h,T,init,m0", [(0.3, 1.0, oracle.INIT_ALL_UP, 1.0),
                                         (0.3, 1.0, oracle.INIT_ALL_DOWN, -1.0),
                                         (-0.2, 2.0, oracle.INIT_ALL_UP, 1.0)])
def test_integrals_against_the_field_only_closed_form(h, T, init, m0):
    L, ends, n = 64, [0.25, 1.0, 2.5], 48
    beta = 1.0 / T
    r_dn = min(1.0, math.exp(-2 * beta * h))       # + -> -
    r_up = min(1.0, math.exp(2 * beta * h))        # - -> +
    rate = r_dn + r_up
    m_eq = (r_up - r_dn) / rate
    a = m0 - m_eq
    im = np.zeros((n, len(ends)))
    ib = np.zeros((n, len(ends)))
    for i in range(n):
        res = oracle.run(L, 0.0, h, T, 16, 16, 300 + i, ends, init_mode=init, keep_spins=False)
        im[i] = res.int_mag / L ** 2
        ib[i] = res.int_bonds / L ** 2
    for w, t in enumerate(ends):
        e = math.exp(-rate * t)
        want_m = m_eq * t + a * (1 - e) / rate
        want_b = 2 * (m_eq ** 2 * t + 2 * m_eq * a * (1 - e) / rate
                      + a * a * (1 - e * e) / (2 * rate))
        for got, want in ((im[:, w], want_m), (ib[:, w], want_b)):
            se = got.std(ddof=1) / math.sqrt(n)
            assert abs(got.mean() - want) < 4.0 * se + 1e-12, (w, got.mean(), want, se)
