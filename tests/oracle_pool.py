"""Oracle runs in worker processes, so that the long CPU reference runs of a
GPU test module overlap its GPU work.  Test infrastructure: it only calls the
oracle.  The pool uses the spawn start method (a process forked after the
parent has touched the GPU can hang)."""
import multiprocessing as mp
import os

import numpy as np


def run(kwargs):
    """oracle.run(**kwargs), returned compactly: spins at every window end as
    packed bits (1 = up), the per-region counts at every end, the final
    clock carry and the observables."""
    import oracle
    r = oracle.run(**kwargs)
    return {
        "spins": [np.packbits(r.spins[w].reshape(-1) > 0) for w in range(r.spins.shape[0])],
        "counts": r.counts,
        "carry": (r.carry_i, r.carry_x, r.carry_b, r.carry_t),
        "mag": r.mag, "bonds": r.bonds, "int_mag": r.int_mag, "int_bonds": r.int_bonds,
    }


def pack(spins):
    """The packed form of a spin array, as run() returns it."""
    return np.packbits(np.asarray(spins).reshape(-1) > 0)


def pool(n=None):
    n = n or max(1, min(16, os.cpu_count() or 1))
    return mp.get_context("spawn").Pool(n)
