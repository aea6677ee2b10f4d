"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (automatic launch shape, one persistent launch per call).

L = 1024 (64 x 64 regions of 16 x 16, J = 1, h = 0.05, T = 1.0, fair coin):
the oracle finishes t = 100 in seconds, so spins, counts, carry and every
event are compared for each window length.  L = 8192 (256 x 256 regions of
32 x 32, h = 0): the oracle covers a short interval at full size; longer runs
are checked through a property that holds at any size (the trajectory does
not depend on the window length)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")


@pytest.mark.parametrize("lpr", [1, 32])
@pytest.mark.parametrize("Tw,per_call", [(0.25, 40), (1.0, 10), (4.0, 1)])
def test_L1024_to_t100_bit_exact(Tw, per_call, lpr):
    L, W = 1024, 16
    trace = Tw == 1.0
    lat = sr.Lattice(L, 1.0, 0.05, 1.0, (W, W), seed=1, trace_capacity=4096 if trace else 0,
                     lanes_per_region=lpr)
    checkpoints, gpu = [], []
    t = 0.0
    n_total = int(round(100 / Tw))
    done = 0
    while done < n_total:
        lat.run_windows(Tw, per_call)
        for _ in range(per_call):
            t = t + Tw
        done += per_call
        checkpoints.append(t)
        gpu.append(lat.spins())
    ref = oracle.run(L, 1.0, 0.05, 1.0, W, W, 1, checkpoints, trace_cap=(1 << 24) if trace else 0)
    for k in range(len(checkpoints)):
        assert np.array_equal(gpu[k], ref.spins[k]), f"spins differ at t = {checkpoints[k]}"
    i, x, b, tl = lat.carry()
    assert np.array_equal(i, ref.carry_i)
    assert np.array_equal(x, ref.carry_x)
    assert np.array_equal(b, ref.carry_b)
    assert np.array_equal(tl, ref.carry_t)
    if trace:
        lens, times, sites = lat.trace()
        assert int(lens.max()) <= 4096
        order = np.argsort(ref.tr_region, kind="stable")
        bounds = np.searchsorted(ref.tr_region[order], np.arange(lat.n_regions + 1))
        for q in range(lat.n_regions):
            sel = order[bounds[q]:bounds[q + 1]]
            n = int(lens[q])
            assert n == len(sel)
            assert np.array_equal(times[q, :n], ref.tr_time[sel])
            assert np.array_equal(sites[q, :n], ref.tr_site[sel])
    obs = lat.observables()
    assert obs.committed == int(ref.counts[-1].sum())
    assert obs.generated >= obs.committed


@pytest.mark.parametrize("T,init", [(1.0, "up"), (1.0, "fair"), (2.269, "up"), (2.269, "fair"),
                                    (3.5, "up"), (3.5, "fair")])
def test_L8192_short_interval_bit_exact(T, init):
    L, W = 8192, 32
    lat = sr.Lattice(L, 1.0, 0.0, T, (W, W), seed=1, init=init,
                     lanes_per_region=32 if T == 2.269 else 0)
    lat.run_windows(0.1, 2)
    mode = oracle.INIT_ALL_UP if init == "up" else oracle.INIT_FAIR_COIN
    ends = [0.1, 0.1 + 0.1]
    ref = oracle.run(L, 1.0, 0.0, T, W, W, 1, ends[1:], init_mode=mode)
    assert np.array_equal(lat.spins(), ref.spins[0])
    i, x, b, tl = lat.carry()
    assert np.array_equal(i, ref.carry_i)
    assert np.array_equal(tl, ref.carry_t)
    assert np.array_equal(b, ref.carry_b)


@pytest.mark.parametrize("T", [1.0, 3.5])
def test_L8192_window_length_independence(T):
    """Tw in {0.1, 1, 10} reach the same committed state at t = 10."""
    L, W = 8192, 32
    out = []
    for Tw, n in [(0.1, 100), (1.0, 10), (10.0, 1)]:
        lat = sr.Lattice(L, 1.0, 0.0, T, (W, W), seed=1, init="fair")
        lat.run_windows(Tw, n)
        out.append((lat.spins(), lat.carry(), lat.observables()))
        lat.close()
    # Tw = 1 and Tw = 10 both end at exactly 10.0
    for a, b in zip(out[1][1], out[2][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[1][0], out[2][0])
    assert out[1][2].committed == out[2][2].committed
    # 0.1 added 100 times ends at 9.99999999999998; with no event or break
    # point in [that, 10.0) the states agree as well
    t01 = 0.0
    for _ in range(100):
        t01 = t01 + 0.1
    assert float(out[1][1][3].max()) < t01
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][0], out[1][0])
