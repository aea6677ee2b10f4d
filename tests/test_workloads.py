"""The seeded synthetic workloads: the 256-lattice batch is reproducible and
follows its stated recipe (L over {64, ..., 1024}, T in [1, 3.5], h in
[-0.2, 0.2], J = 1, seeds 1000 + b), about 7.4e7 sites in total."""
import numpy as np

from paper_cs_0405053_gb300 import workloads


def test_batch_draw_is_reproducible_and_in_range():
    a = workloads.batch_replicas()
    b = workloads.batch_replicas()
    assert a == b and len(a) == 256
    assert {r["L"] for r in a} <= set(workloads.BATCH_SIDES)
    assert len({r["L"] for r in a}) == len(workloads.BATCH_SIDES)
    assert all(1.0 <= r["T"] <= 3.5 and -0.2 <= r["h"] <= 0.2 and r["J"] == 1.0 for r in a)
    assert [r["seed"] for r in a] == [workloads.BATCH_SEED0 + i for i in range(256)]
    sites = sum(r["L"] ** 2 for r in a)
    assert 6.5e7 < sites < 8.5e7
    assert workloads.batch_replicas(key=5) != a


def test_plain_workload_constants():
    w = workloads.PLAIN_L1024
    assert (w["L"], w["region"], w["J"], w["h"], w["T"], w["t_end"]) == (1024, (16, 16), 1.0, 0.05,
                                                                          1.0, 100.0)
    assert w["windows"] == (0.25, 1.0, 4.0)
    assert all(np.isclose(w["t_end"] / tw, round(w["t_end"] / tw)) for tw in w["windows"])
