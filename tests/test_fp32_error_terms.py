"""The FP32-propensity mode forms the rounding error of each binary32 sum in
its compensated a0 scan by Fast2Sum on (max, min) of the two non-negative
operands, where the oracle writes TwoSum.  The two agree bit for bit because
the error of a rounded sum is unique and both are exact (Fast2Sum when the
first operand is the larger).  Checked here in numpy binary32 arithmetic
(round to nearest even, no contraction) over random magnitudes, equal
operands, zeros, neighbouring values and far-apart exponents."""
import numpy as np


def _two_sum(a, b):
    s = a + b
    bp = s - a
    return s, (a - (s - bp)) + (b - bp)


def _fast_two_sum_max_min(a, b):
    hi, lo = np.maximum(a, b), np.minimum(a, b)
    s = hi + lo
    return s, lo - (s - hi)


def test_fast2sum_on_max_min_equals_two_sum_for_non_negative_binary32():
    rng = np.random.default_rng(7)
    n = 1_000_000
    e = rng.integers(-40, 40, size=(2, n))
    m = rng.uniform(1.0, 2.0, size=(2, n))
    x = (m * np.exp2(e)).astype(np.float32)
    a, b = x[0], x[1]
    # special cases: zeros, equal values, neighbours, one ulp, far apart
    z = np.float32(0.0)
    one = np.float32(1.0)
    extra_a = np.array([z, z, one, one, one, np.float32(3.0), np.float32(1e30), np.float32(1e-30)], dtype=np.float32)
    extra_b = np.array([z, one, one, np.nextafter(one, np.float32(2)), np.float32(2 ** -24),
                        np.float32(3.0), np.float32(1e-30), np.float32(1e30)], dtype=np.float32)
    a = np.concatenate([a, extra_a, np.nextafter(a[:1000], np.float32(np.inf))])
    b = np.concatenate([b, extra_b, a[:1000]])
    with np.errstate(over="ignore"):
        s1, e1 = _two_sum(a, b)
        s2, e2 = _fast_two_sum_max_min(a, b)
    assert s1.dtype == np.float32 and e2.dtype == np.float32
    assert np.array_equal(s1.view(np.uint32), s2.view(np.uint32))
    assert np.array_equal(e1.view(np.uint32), e2.view(np.uint32))
    # the error is exact: a + b == s + e in rational arithmetic (a sample,
    # the special cases included)
    from fractions import Fraction
    idx = np.concatenate([rng.integers(0, n, size=2000), np.arange(n, n + len(extra_a))])
    for i in idx:
        if np.isfinite(s2[i]):
            assert Fraction(float(a[i])) + Fraction(float(b[i])) == Fraction(float(s2[i])) + Fraction(float(e2[i]))
