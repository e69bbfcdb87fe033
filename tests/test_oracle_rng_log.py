"""Pins for the oracle's random source and logarithm (no GPU).

* Philox4x64-10 is checked against numpy's ``Philox`` bit generator, an
  independent implementation of the same published generator (Salmon et al.,
  SC'11).  numpy advances its 256-bit counter before producing a block, so
  block(c) of the oracle equals numpy's first block started at c - 1.
* The fixed-point -ln(u) is checked against mpmath at 200-bit precision and
  against libm.  Bound (derived in the design notes): |E - E_true| <=
  0.52 ulp(E_true) + 2^-57, i.e. within about half an ulp wherever E >= 1/16
  and within 2^-57 absolute for the tiny values E takes as u -> 1.
* Its integer constants are checked against mpmath (independent of the
  Python-integer series that produces them).
"""
import math

import numpy as np
import pytest

import oracle


def _numpy_block(ctr, key):
    cint = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    g = np.random.Philox(key=int(key[0]) | (int(key[1]) << 64), counter=(cint - 1) % (1 << 256))
    return g.random_raw(4)


def test_philox_matches_numpy_random_counters():
    rng = np.random.default_rng(2024)
    for _ in range(300):
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        ctr = [c * 2 + int(b) for c, b in zip(ctr, rng.integers(0, 2, size=4))]
        key = [int(v) * 2 + 1 for v in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_block(ctr, key))


def test_philox_matches_numpy_edge_counters():
    cases = [((0, 0, 0, 0), (0, 0)), ((2**64 - 1,) * 4, (2**64 - 1,) * 2),
             ((1, 0, 0, 0), (1, 0)), ((0, 65535, 0, 0), (1, 7)), ((123, 2**40, 0, 0), (99, 0))]
    for ctr, key in cases:
        assert np.array_equal(oracle.philox4x64(ctr, key), _numpy_block(ctr, key))


def test_philox_event_words_uniformity():
    """Top 8 bits of the words used by events are uniform (chi-square, 255 dof)."""
    words = []
    for m in range(2000):
        words.extend(oracle.philox4x64((m, 17, 0, 0), (1, 0)).tolist())
    top = np.array(words, dtype=np.uint64) >> np.uint64(56)
    counts = np.bincount(top.astype(np.int64), minlength=256)
    exp = len(words) / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 255 dof: mean 255, sd ~22.6; 5.5 sd bound
    assert chi2 < 255 + 5.5 * math.sqrt(2 * 255)


def test_log_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(7)
    qs = [np.array([1, 3, 5, 7, (1 << 53) - 1, (1 << 53) - 3, (1 << 52) + 1, (1 << 52) - 1], dtype=np.uint64)]
    for e in range(1, 53):
        qs.append(rng.integers(1 << e, 1 << (e + 1), size=40, dtype=np.uint64) | np.uint64(1))
    qs.append(((1 << 53) - 2 * rng.integers(1, 1 << 30, size=400, dtype=np.uint64) + 1).astype(np.uint64))
    # table cell boundaries: q = 2^52 (1 + i/128) +- 1
    for i in range(128):
        base = (1 << 52) + i * (1 << 45)
        qs.append(np.array([base + 1, max(base - 1, 1)], dtype=np.uint64))
    q = np.concatenate(qs)
    E = oracle.neg_log_u(q)
    for qi, ei in zip(q.tolist(), E.tolist()):
        true = -mpmath.log(mpmath.mpf(qi) / mpmath.mpf(2) ** 53)
        err = float(abs(mpmath.mpf(ei) - true))
        assert err <= 0.52 * math.ulp(float(true)) + 2.0 ** -57, (qi, ei, float(true))


def test_log_against_libm():
    rng = np.random.default_rng(11)
    q = rng.integers(0, 1 << 52, size=200000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    E = oracle.neg_log_u(q)
    ref = -np.log(q.astype(np.float64) * 2.0 ** -53)  # q < 2^53: exact conversion
    ulp = np.spacing(ref)
    # libm is itself within ~1 ulp, so allow 1.6 ulp between the two plus the absolute term
    assert np.all(np.abs(E - ref) <= 1.6 * ulp + 2.0 ** -57)


def test_log_monotone_and_range():
    q = np.arange(1, 1 << 16, 2, dtype=np.uint64)
    E = oracle.neg_log_u(q)
    assert np.all(np.diff(E) < 0)
    top = ((1 << 53) - 2 * np.arange(0, 1 << 15, dtype=np.uint64) - 1).astype(np.uint64)[::-1]
    Et = oracle.neg_log_u(top)
    assert np.all(np.diff(Et) <= 0) and np.all(Et > 0)
    assert abs(oracle.neg_log_u([1])[0] - 53 * math.log(2)) < 1e-14


def test_log_constants_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 300
    inv, lnf, ln2, horner = oracle.log_constants()
    two64 = mpmath.mpf(2) ** 64
    for i in range(128):
        F = 1 + mpmath.mpf(2 * i + 1) / 256
        assert inv[i] == int(mpmath.nint(two64 / F))
        assert lnf[i] == int(mpmath.nint(two64 * mpmath.log(F)))
    assert ln2 == int(mpmath.nint(two64 * mpmath.log(2)))
    for m in range(1, 8):
        assert horner[m] == int(mpmath.nint(mpmath.mpf(2) ** 62 / m)) * (1 if m % 2 else -1)


def test_uniform_map_is_exact_and_open():
    """u(w) = (2 (w >> 12) + 1) 2^-53 lies in (0, 1) and is exact in double."""
    for w in [0, 2**64 - 1, 2**12 - 1, 2**12, 2**63]:
        q = ((w >> 12) << 1) | 1
        u = q * 2.0 ** -53
        assert 0.0 < u < 1.0
        assert int(u * 2.0 ** 53) == q


def test_uniform_grid_formula():
    g = oracle.uniform_grid(3001, 30.0)
    k = np.arange(3001, dtype=np.float64)
    assert np.array_equal(g, (k * 30.0) / 3000.0)
    assert g[0] == 0.0 and g[-1] == 30.0
