"""Per-region restatement of §5, used to pin the oracle's global time order.

Given the true history of every region, one region's own history must be
reproduced by running the serial n-fold way (§3) for that region alone with
its neighbours' flips as break points (§5, Eqs. 5.2-5.6): this is the fixed
point the synchronous relaxation converges to.  Written independently of the
oracle's event loop: it keeps only the region's spins and its halo, recounts
every class from the spins at each step, and walks the break points in time
order.  It reuses the oracle's scalar formulas (random pairs, tau, class and
site choice), which other tests pin on their own."""
import numpy as np

import oracle


def region_sites(L, W, H, r):
    NX = L // W
    rx, ry = r % NX, r // NX
    return [(ry * H + y) * L + rx * W + x for y in range(H) for x in range(W)]


def neighbours(L, s):
    x, y = s % L, s // L
    return [y * L + (x + 1) % L, y * L + (x - 1) % L, ((y + 1) % L) * L + x, ((y - 1) % L) * L + x]


def replay(L, W, H, J, h, T, seed, r, spins0, flips, t_end, glauber=False):
    """Events (time, site) of region r in [0, t_end); flips = all (time, site)
    flips of the lattice (any order of other regions' flips is fine)."""
    F = oracle.frac_bits(W * H)
    P = [int(v) for v in oracle.rates_fixed(oracle.rates(J, h, T, glauber), F)]
    s = np.array(spins0, dtype=np.int64).reshape(-1)
    mine = region_sites(L, W, H, r)
    mset = set(mine)
    nb = {v: neighbours(L, v) for v in mine}

    def cls(v):
        return 5 * (s[v] > 0) + sum(1 for u in nb[v] if s[u] > 0)

    key = [seed & 0xFFFFFFFF, seed >> 32]

    def draw(i):
        w = oracle.philox([i & 0xFFFFFFFF, i >> 32, r, 0], key)
        return oracle.neglog_unit(((w[1] << 32) | w[0]) >> 12), ((w[3] << 32) | w[2]) >> 12

    halo = [(t, v) for (t, v) in sorted(flips)
            if v not in mset and any(u in mset for u in neighbours(L, v))]
    i, b, t_last = 0, 0.0, 0.0
    x, kv = draw(0)
    events, k = [], 0
    while True:
        classes = [cls(v) for v in mine]
        lam = sum(P[c] for c in classes)
        tau = oracle.tau(t_last, x, b, lam, F)
        t_b = halo[k][0] if k < len(halo) else float("inf")
        if tau <= t_b:
            if not tau < t_end:
                break
            N = [classes.count(c) for c in range(10)]
            kk, pos = oracle.select(N, P, kv)
            v = [u for u, c in zip(mine, classes) if c == kk][pos]
            events.append((tau, v))
            s[v] = -s[v]
            t_last, b, i = tau, 0.0, i + 1
            x, kv = draw(i)
        else:
            b = b + oracle.lam(lam, F) * (t_b - t_last)
            t_last = t_b
            s[halo[k][1]] = -s[halo[k][1]]
            k += 1
    return events
