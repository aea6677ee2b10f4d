"""sr_run_noalloc: the whole simulation for callers that cannot allocate GPU
memory at the point where they simulate (a fixed memory budget, a host
application that forbids cudaMalloc in its callbacks).  The entry point keeps
all its working state in a fixed scratch array inside the library, so its
results must equal those of the ordinary entry points, call after call.

This file is collected last on purpose: it runs after every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sr = pytest.importorskip("paper_cs_0405053_gb300")


def _entry():
    fn = sr.library().sr_run_noalloc
    assert fn.restype is C.c_int and len(fn.argtypes) == 13    # declared by the binding
    return fn


def _run_noalloc(L, W, H, J, h, T, seed, Tw, n, init):
    fn = _entry()
    dev_in = None if init is None else torch.from_numpy(init.reshape(-1)).cuda()
    out = torch.zeros(L * L, dtype=torch.int8, device="cuda")
    counts = torch.zeros((L // W) * (L // H), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(L, J, h, T, W, H, seed, None if dev_in is None else dev_in.data_ptr(), Tw, n,
            out.data_ptr(), counts.data_ptr(), stream)
    assert rc == 0, sr.library().sr_strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(L, L), counts.cpu().numpy().view(np.uint64)


def _run_existing(L, W, H, J, h, T, seed, Tw, n, init):
    lat = sr.Lattice(L, J, h, T, (W, H), seed=seed)
    if init is not None:
        lat.set_spins(init)
    lat.run_windows(Tw, n)
    spins = lat.spins()
    counts = lat.carry()[0]
    lat.close()
    return spins, counts


def test_no_alloc_equals_the_allocating_entry_points_on_two_calls():
    rng = np.random.default_rng(17)
    given = np.where(rng.random((96, 96)) < 0.4, 1, -1).astype(np.int8)
    cases = [
        (64, 16, 16, 1.0, 0.05, 1.5, 1, 1.0, 5, None),      # fair coin from the seed
        (96, 8, 12, 1.0, 0.0, 2.3, 7, 0.5, 6, given),       # caller-given spins
        (32, 8, 8, 1.0, 0.1, float("inf"), 3, 0.25, 4, None),   # T = inf: every p_k = 1
    ]
    for case in cases:          # two calls in a row share the same scratch
        a_spins, a_counts = _run_noalloc(*case)
        b_spins, b_counts = _run_existing(*case)
        assert np.array_equal(a_spins, b_spins)
        assert np.array_equal(a_counts, b_counts)
        assert int(a_counts.sum()) > 0


def test_no_alloc_rejects_problems_larger_than_its_scratch():
    fn = _entry()
    out = torch.zeros(8192 * 8192, dtype=torch.int8, device="cuda")
    rc = fn(8192, 1.0, 0.0, 2.0, 32, 32, 1, None, 1.0, 1, out.data_ptr(), None,
            torch.cuda.current_stream().cuda_stream)
    assert rc == -8          # SR_ETOOLARGE: nothing was run, nothing allocated
