"""The oracle's global time-order simulation against the per-region
definition of §5: every region's history is reproduced exactly by the region
alone, given its neighbours' flips as break points, and events come out in
non-decreasing time order whatever the number of regions."""
import numpy as np
import pytest

import oracle
from region_replay import replay


@pytest.mark.parametrize("L,W,H,T,h,glauber,Tw", [
    (32, 8, 8, 1.7, 0.05, False, 0.5),
    (24, 6, 4, 3.0, -0.1, False, 0.4),
    (16, 4, 4, 1.2, 0.0, True, 1.0),
    (12, 3, 12, 2.3, 0.05, False, 0.6),
])
def test_every_region_replays_its_own_history(L, W, H, T, h, glauber, Tw):
    ref = oracle.run(L, 1.0, h, T, W, H, 3, [0.0, Tw], glauber=glauber, trace_cap=1 << 20)
    flips = list(zip(ref.tr_time.tolist(), ref.tr_site.tolist()))
    for r in range((L // W) * (L // H)):
        sel = ref.tr_region == r
        want = list(zip(ref.tr_time[sel].tolist(), ref.tr_site[sel].tolist()))
        got = replay(L, W, H, 1.0, h, T, 3, r, ref.spins[0], flips, Tw, glauber)
        assert got == want, f"region {r}"


@pytest.mark.parametrize("L,W,H", [(64, 4, 4), (128, 8, 2), (96, 3, 3), (256, 16, 16)])
def test_global_time_order_with_many_regions(L, W, H):
    r = oracle.run(L, 1.0, 0.05, 2.0, W, H, 5, [0.3, 0.6], trace_cap=1 << 22)
    assert r.trace_len <= (1 << 22)
    assert np.all(np.diff(r.tr_time) >= 0)
