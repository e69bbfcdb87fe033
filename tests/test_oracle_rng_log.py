"""Pins for the oracle's random source and logarithm (no GPU).

* Philox4x32-10 is checked against triton's implementation of the same
  published generator (Salmon et al., SC'11), run on the CPU by triton's
  interpreter; it is written independently of the oracle.
* The fixed-point -ln(u) is checked against mpmath at 200-bit precision and
  against libm.  Bound: |E - E_true| <= 0.5 ulp(E_true) + 2^-57.  The fixed-
  point sum is within about 1.8 * 2^-58 of -ln(u) (floors of the products,
  the 32-bit series tail, the omitted r^6/6, the rounding of the table and of
  n ln 2, and the 6-bit shift above 1), then rounded once to double.  So the
  result is within half an ulp plus that, and within 2^-57 absolute for the
  tiny values E takes as u -> 1.
* Its integer constants are checked against mpmath (independent of the
  Python-integer series that produces them).
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle


def _triton_blocks(cases):
    """Philox4x32-10 blocks from triton's implementation (CPU interpreter), in
    a subprocess so the interpreter setting cannot leak into this process."""
    pytest.importorskip("triton")
    script = os.path.join(os.path.dirname(__file__), "philox_triton_reference.py")
    r = subprocess.run([sys.executable, script], input=json.dumps(cases), capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    return np.array(json.loads(r.stdout), dtype=np.uint64)


def test_philox4x32_matches_triton():
    rng = np.random.default_rng(2024)
    cases = [[int(v) for v in rng.integers(0, 2**32, size=6, dtype=np.uint64)] for _ in range(250)]
    cases += [[0, 0, 0, 0, 0, 0], [2**32 - 1] * 6, [1, 0, 0, 0, 1, 0], [0, 65535, 0, 7, 1, 7],
              [5, 17, 0, 0, 1, 0], [123, 2**31, 2**31 - 1, 3, 99, 0]]
    ref = _triton_blocks(cases)
    for case, want in zip(cases, ref):
        got = oracle.philox4x32(case[:4], case[4:])
        assert np.array_equal(got.astype(np.uint64), want), case


def test_philox_event_words_uniformity():
    """Top 8 bits of the words of consecutive event blocks are uniform (chi-square, 255 dof)."""
    words = []
    for n in range(2000):
        words.extend(oracle.philox4x32((n, 17, 0, 0), (1, 0)).tolist())
    top = np.array(words, dtype=np.uint64) >> np.uint64(24)
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
    # cell boundaries and centres: q = 2^52 (1 + i/512) +- 1, + half a cell
    for i in range(512):
        base = (1 << 52) + i * (1 << 43)
        qs.append(np.array([base + 1, max(base - 1, 1), base + (1 << 42) + 1], dtype=np.uint64))
    q = np.concatenate(qs)
    E = oracle.neg_log_u(q)
    for qi, ei in zip(q.tolist(), E.tolist()):
        true = -mpmath.log(mpmath.mpf(qi) / mpmath.mpf(2) ** 53)
        err = float(abs(mpmath.mpf(ei) - true))
        assert err <= 0.5 * math.ulp(float(true)) + 2.0 ** -57, (qi, ei, float(true))


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
    inv, lnf, ln2, k3, k5 = oracle.log_constants()
    two64 = mpmath.mpf(2) ** 64
    for i in range(512):
        F = 1 + mpmath.mpf(2 * i + 1) / 1024
        assert inv[i] == int(mpmath.nint(two64 / F))
        assert lnf[i] == int(mpmath.nint(two64 * mpmath.log(F)))
    assert ln2 == int(mpmath.nint(two64 * mpmath.log(2)))
    assert k3 == int(mpmath.nint(mpmath.mpf(2) ** 31 / 3)) and k5 == int(mpmath.nint(mpmath.mpf(2) ** 31 / 5))


def test_uniform_map_is_exact_and_open():
    """u(a, b) = (2 ((a << 20) | (b >> 12)) + 1) 2^-53 lies in (0, 1) and is exact in double."""
    for a, b in [(0, 0), (2**32 - 1, 2**32 - 1), (0, 2**12 - 1), (0, 2**12), (2**31, 0)]:
        q = ((((a << 20) | (b >> 12))) << 1) | 1
        u = q * 2.0 ** -53
        assert 0.0 < u < 1.0
        assert int(u * 2.0 ** 53) == q


def test_uniform_grid_formula():
    g = oracle.uniform_grid(3001, 30.0)
    k = np.arange(3001, dtype=np.float64)
    assert np.array_equal(g, (k * 30.0) / 3000.0)
    assert g[0] == 0.0 and g[-1] == 30.0
