"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (automatic launch shape, one persistent launch per call).

L = 1024 (64 x 64 regions of 16 x 16, J = 1, h = 0.05, T = 1.0, fair coin):
the oracle finishes t = 100 in seconds, so spins, counts, carry and every
event are compared for each window length.  L = 8192 (256 x 256 regions of
32 x 32, h = 0): every (T, initial spins) pair against the oracle to t = 1 at
window lengths 0.1 and 1, and T = 1 from all up to t = 10 in one window of
10 (the oracle runs in worker processes while the GPU tests run); longer runs
are checked through a property that holds at any size (the trajectory does
not depend on the window length)."""
import numpy as np
import pytest

import oracle
import oracle_pool

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")

C3_CASES = [(T, init) for T in (1.0, 2.269, 3.5) for init in ("up", "fair")]


def _tenths():
    """The ten window ends of Tw = 0.1 (repeated addition), then 1.0."""
    ends, t = [], 0.0
    for _ in range(10):
        t = t + 0.1
        ends.append(t)
    return ends + [1.0]


@pytest.fixture(scope="module", autouse=True)
def c3_reference():
    """Oracle runs of the L = 8192 cases, started when the module starts."""
    pool = oracle_pool.pool(len(C3_CASES) + 1)
    jobs = {}
    for T, init in C3_CASES:
        mode = oracle.INIT_ALL_UP if init == "up" else oracle.INIT_FAIR_COIN
        jobs[(T, init)] = pool.apply_async(oracle_pool.run, (dict(
            L=8192, J=1.0, h=0.0, T=T, region_w=32, region_h=32, seed=1, t_end=_tenths(),
            init_mode=mode),))
    jobs["t10"] = pool.apply_async(oracle_pool.run, (dict(
        L=8192, J=1.0, h=0.0, T=1.0, region_w=32, region_h=32, seed=1, t_end=[10.0],
        init_mode=oracle.INIT_ALL_UP),))
    yield jobs
    pool.terminate()
    pool.join()


def _same_state(lat, ref, w):
    """Spins, per-region counts and observables of lat equal the oracle's at end w."""
    assert np.array_equal(oracle_pool.pack(lat.spins()), ref["spins"][w])
    i, x, b, tl = lat.carry()
    assert np.array_equal(i, ref["counts"][w])
    o = lat.observables()
    assert (o.mag, o.bonds) == (int(ref["mag"][w]), int(ref["bonds"][w]))
    for got, want in ((o.int_mag, ref["int_mag"][w]), (o.int_bonds, ref["int_bonds"][w])):
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want)) * 8192 ** 2, (got, want)
    return i, x, b, tl


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


@pytest.mark.parametrize("T,init", C3_CASES)
def test_L8192_to_t1_bit_exact(T, init, c3_reference):
    """Tw = 0.1: spins, counts and observables at every window end; Tw = 1:
    the same at t = 1 plus the clock carry of every region."""
    L, W = 8192, 32
    lpr = 32 if T == 2.269 else 0          # the warp mapping at full size too
    ref = c3_reference[(T, init)].get(timeout=3600)
    lat = sr.Lattice(L, 1.0, 0.0, T, (W, W), seed=1, init=init, lanes_per_region=lpr)
    for w in range(10):
        lat.run_window(0.1)
        _same_state(lat, ref, w)
    lat.close()
    lat = sr.Lattice(L, 1.0, 0.0, T, (W, W), seed=1, init=init, lanes_per_region=lpr)
    lat.run_window(1.0)
    carry = _same_state(lat, ref, 10)
    for got, want in zip(carry, ref["carry"]):
        assert np.array_equal(got, want)
    lat.close()


def test_L8192_all_up_T1_to_t10_in_one_window(c3_reference):
    L, W = 8192, 32
    ref = c3_reference["t10"].get(timeout=3600)
    lat = sr.Lattice(L, 1.0, 0.0, 1.0, (W, W), seed=1, init="up")
    lat.run_window(10.0)
    carry = _same_state(lat, ref, 0)
    for got, want in zip(carry, ref["carry"]):
        assert np.array_equal(got, want)
    assert lat.observables().committed > 100000
    lat.close()


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
