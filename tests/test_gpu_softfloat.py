"""The integer-emulated IEEE double operations of the event loop against the
IEEE result (numpy's float64, correctly rounded by definition), bit for bit,
over random and boundary operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")


def _operands(rng, n):
    out = []
    # normal numbers over a wide exponent range
    e = rng.integers(1, 2046, n, dtype=np.int64)
    m = rng.integers(0, 1 << 52, n, dtype=np.int64)
    out.append(((e << 52) | m).view(np.float64))
    # exponents near 1, low significand bits cleared (ties, exact results)
    e = rng.integers(1000, 1046, n, dtype=np.int64)
    m = rng.integers(0, 1 << 52, n, dtype=np.int64) & ~((1 << rng.integers(0, 52, n)) - 1)
    out.append(((e << 52) | m).view(np.float64))
    # times, rates and hazards of the workloads
    out.append(rng.uniform(0, 200, n))
    out.append(rng.exponential(1.0, n))
    return np.concatenate(out)


def _pairs(rng, n):
    a = _operands(rng, n)
    b = _operands(rng, n)
    rng.shuffle(b)
    # near-equal operands (cancellation) and neighbours
    k = len(a) // 4
    b[:k] = a[:k] * (1 + rng.integers(-8, 9, k) * 2.0**-52)
    b[k:2 * k] = np.nextafter(a[k:2 * k], 0)
    sp = np.array([0.0, 1.0, 2.0, 0.5, 1.5, 3.0, 1 + 2**-52, 2 - 2**-52, 2.0**-1000, 2.0**1000, 1e-300,
                   1e300, 0.1, 36.7368005696771, 5e-324, 2.2250738585072014e-308])
    A, B = np.meshgrid(sp, sp)
    return np.concatenate([a, A.ravel(), B.ravel()]), np.concatenate([b, B.ravel(), A.ravel()])


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_soft_double_matches_ieee(op):
    rng = np.random.default_rng(10 + op)
    a, b = _pairs(rng, 1 << 20)
    a, b = np.abs(a), np.abs(b)
    if op == 3:
        b = np.where(b == 0, 1.0, b)
    with np.errstate(all="ignore"):
        want = {0: a + b, 1: a - b, 2: a * b, 3: a / b}[op]
    got = sr.eval_softfloat(op, a, b)
    assert np.array_equal(got.view(np.int64), want.view(np.int64))


def test_scaled_integer_matches_ieee():
    rng = np.random.default_rng(3)
    v = rng.integers(1, np.iinfo(np.int64).max, 1 << 20, dtype=np.int64)
    v = v >> rng.integers(0, 63, v.size)
    v = np.maximum(v, 1)
    F = rng.integers(0, 64, v.size).astype(np.float64)
    got = sr.eval_softfloat(4, v.view(np.float64), F)
    want = v.astype(np.float64) * np.ldexp(1.0, -F.astype(np.int64))
    assert np.array_equal(got.view(np.int64), want.view(np.int64))
