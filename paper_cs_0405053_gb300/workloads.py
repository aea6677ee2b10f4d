"""Seeded synthetic workloads shaped like the paper's problem statement (§2):
periodic square lattices with their couplings, fields, temperatures and
seeds.  Input generation only; nothing here computes any step of the method.
"""
from __future__ import annotations

from typing import List

import numpy as np

# Plain single lattice: L = 1024 in 64 x 64 regions of 16 x 16, J = 1,
# h = 0.05, T = 1.0 (below Tc ~ 2.269), fair-coin spins, run to t = 100 with
# window lengths 0.25, 1 and 4.
PLAIN_L1024 = dict(L=1024, region=(16, 16), J=1.0, h=0.05, T=1.0, t_end=100.0,
                   windows=(0.25, 1.0, 4.0))

BATCH_SIDES = (64, 128, 256, 512, 1024)
BATCH_KEY = 4          # Philox key of the batch draw
BATCH_SEED0 = 1000     # lattice b simulates with seed BATCH_SEED0 + b


def batch_replicas(n: int = 256, key: int = BATCH_KEY, seed0: int = BATCH_SEED0) -> List[dict]:
    """n independent lattices: L uniform over {64, 128, 256, 512, 1024}, T
    uniform in [1.0, 3.5], h uniform in [-0.2, 0.2], J = 1, fair-coin spins,
    Metropolis rates; drawn in that order from numpy's Philox generator keyed
    by `key`.  Lattice b simulates with seed seed0 + b."""
    g = np.random.Generator(np.random.Philox(key=key))
    Ls = g.choice(np.array(BATCH_SIDES), size=n)
    Ts = g.uniform(1.0, 3.5, size=n)
    hs = g.uniform(-0.2, 0.2, size=n)
    return [dict(L=int(Ls[b]), J=1.0, h=float(hs[b]), T=float(Ts[b]), seed=seed0 + b)
            for b in range(n)]


def stratified(reps: List[dict], per_side: int = 3) -> List[int]:
    """Indices of a sample that covers every side L and the range of T: for
    each side, `per_side` lattices spread evenly over its T order (the
    coldest and the hottest among them)."""
    by_side = {}
    for b, r in enumerate(reps):
        by_side.setdefault(r["L"], []).append(b)
    out = []
    for L in sorted(by_side):
        ids = sorted(by_side[L], key=lambda b: reps[b]["T"])
        k = min(per_side, len(ids))
        picks = sorted({round(j * (len(ids) - 1) / max(1, k - 1)) for j in range(k)})
        out += [ids[p] for p in picks]
    return out
