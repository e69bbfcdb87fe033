"""Pins for the oracle's FP32-propensity mode (no GPU).

The mode keeps time and a0 in FP64 and moves the propensities and the
selection sums to binary32.  Each test checks it against something fixed
outside the oracle:
  * where every product and sum is exact in binary32 (dyadic rates, small
    counts) the mode must reproduce the FP64 mode's trajectories bit for bit,
    in both summation schedules;
  * hand-built cases whose binary32 and FP64 results differ, checked against
    numpy's IEEE binary32 / binary64 arithmetic: the first event time uses
    a0 formed in FP64 from error-compensated binary32 chunk sums (so rounding
    losses of the binary32 sums do not reach a0), and each propensity is
    (float)c * (float)h rounded in binary32;
  * the closed forms of the birth-death and isomerisation processes.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

FP32 = oracle.PRECISION_FP32
SCHEDULES = [oracle.SCHEDULE_L, oracle.SCHEDULE_W32]


def _z(est, mu, se):
    return np.abs(est - mu) / se


def _dyadic(net, seed):
    """The same network with rates snapped to {1/8, 1/4, 1/2, 1, 2}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rates = 2.0 ** rng.integers(-3, 2, size=net.n_reactions)
    return net.with_rates(rates.astype(np.float64))


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_exact_binary32_arithmetic_reproduces_fp64_mode(schedule):
    cases = [
        (W.birth_death(8.0, 0.125, 0), 20.0, 60),
        (W.isomerisation(1.0, 0.5, 6, 3), 3.0, 60),
        (_dyadic(W.random_network(11, n_species=12, n_reactions=40, x0_hi=12), 4), 0.3, 40),
        (_dyadic(W.random_network(12, n_species=32, n_reactions=128, x0_hi=15), 5), 0.2, 24),
    ]
    for net, T, N in cases:
        kw = dict(schedule=schedule, per_traj=True, max_events=3000, threads=4)
        r64 = oracle.run(net, N, T, 41, 7, **kw)
        r32 = oracle.run(net, N, T, 41, 7, precision=FP32, **kw)
        # exactness precondition: every a_j is a multiple of 1/8 below 2 x_max^2 and the
        # sum of M of them stays below 2^21, so binary32 represents every product and sum
        assert net.n_reactions * 2 * max(r64.max_x, 2) ** 2 * 8 < 2 ** 24, net.name
        assert np.array_equal(r32.traj_hash, r64.traj_hash), net.name
        assert np.array_equal(r32.traj_events, r64.traj_events)
        assert np.array_equal(r32.S1, r64.S1) and np.array_equal(r32.S2, r64.S2)
        assert r64.events > N


def _first_event(net, seed, traj=0, precision=FP32, schedule=oracle.SCHEDULE_L):
    rt, rj, _, _, ne = oracle.trace(net, traj, 1e9, 1, seed, grid=[1e9], max_events=1, precision=precision,
                                    schedule=schedule)
    assert ne == 1
    w = oracle.philox4x32([0, traj, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
    q1 = ((((int(w[0]) << 20) | (int(w[1]) >> 12)) << 1) | 1)
    E = float(oracle.neg_log_u(q1)[0])
    return float(rt[0]), int(rj[0]), E


def test_time_step_uses_the_fp64_sum_of_the_binary32_propensities():
    # a = (2^24, 1): the binary32 total rounds to 2^24 (tie to even), the FP64 one is 2^24 + 1
    R = np.zeros((2, 1), np.int32)
    P = np.zeros((2, 1), np.int32)
    net = W.Network("two_sources", ["X"], R, P, np.array([2.0 ** 24, 1.0]), np.array([0], np.int32))
    assert np.float32(2.0 ** 24) + np.float32(1.0) == np.float32(2.0 ** 24)
    for schedule in SCHEDULES:
        for seed in (1, 2, 3):
            t, j, E = _first_event(net, seed, schedule=schedule)
            assert t == E / (2.0 ** 24 + 1.0)
            assert t != E / 2.0 ** 24
            assert j == 0  # reaction 1 is absorbed by the binary32 total's rounding


def test_a0_sums_each_lane_chunk_with_compensation():
    # 64 reactions (two per lane); reactions 0 and 1 share lane 0 with
    # a = (2^24, 1): the binary32 running sum rounds to 2^24, its TwoSum error
    # is 1, so a0 = 2^24 + 1 under W32; under L the whole list is one
    # compensated sum and gives the same.  Zero rates elsewhere.
    M = 64
    R = np.zeros((M, 1), np.int32)
    P = np.zeros((M, 1), np.int32)
    rates = np.zeros(M)
    rates[0], rates[1] = 2.0 ** 24, 1.0
    net = W.Network("chunk_pair", ["X"], R, P, rates, np.array([0], np.int32))
    for schedule in SCHEDULES:
        for seed in (7, 8):
            t, j, E = _first_event(net, seed, schedule=schedule)
            assert t == E / (2.0 ** 24 + 1.0), schedule
            assert j == 0
    # three values whose binary32 sum loses 2^-24 twice over: the compensated
    # FP64 value keeps both
    rates = np.zeros(M)
    rates[0], rates[1], rates[2] = 1.0, 2.0 ** -24, 2.0 ** -24
    assert np.float32(np.float32(1.0) + np.float32(2.0 ** -24)) == np.float32(1.0)
    net = W.Network("chunk_small", ["X"], R, P, rates, np.array([0], np.int32))
    t, _, E = _first_event(net, 9, schedule=oracle.SCHEDULE_L)
    assert t == E / (1.0 + 2.0 ** -23)


def test_propensity_is_a_binary32_product_of_rounded_factors():
    # X -> 0 with c = 0.1 and x = 3: a = RN32(RN32(0.1) * 3), widened exactly
    R = np.array([[1]], np.int32)
    P = np.array([[0]], np.int32)
    net = W.Network("decay", ["X"], R, P, np.array([0.1]), np.array([3], np.int32))
    a32 = float(np.float32(np.float32(0.1) * np.float32(3.0)))
    assert a32 != 0.1 * 3.0
    for seed in (4, 5):
        t, j, E = _first_event(net, seed)
        assert j == 0 and t == E / a32
        t64, _, _ = _first_event(net, seed, precision=oracle.PRECISION_FP64)
        assert t64 == E / (0.1 * 3.0)
    # a second-order propensity: C(x, 2) in int64, then (float) and the binary32 product
    R = np.array([[2]], np.int32)
    net = W.Network("dimer", ["X"], R, P, np.array([0.3]), np.array([5000], np.int32))
    h = 5000 * 4999 // 2
    a32 = float(np.float32(np.float32(0.3) * np.float32(h)))
    t, _, E = _first_event(net, 6)
    assert t == E / a32


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_fp32_birth_death_poisson_law(schedule):
    net = W.birth_death(10.0, 0.1, 0)
    N, G, T = 12000, 51, 100.0
    r = oracle.run(net, N, T, G, seed=1, threads=8, precision=FP32, schedule=schedule)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    lam = (10.0 / 0.1) * (1.0 - np.exp(-0.1 * g))
    assert mean[0, 0] == 0.0 and var[0, 0] == 0.0
    m, v, lam1 = mean[1:, 0], var[1:, 0], lam[1:]
    assert np.max(_z(m, lam1, np.sqrt(lam1 / N))) < 4.5
    assert np.max(_z(v, lam1, np.sqrt((lam1 + 2 * lam1 * lam1) / N))) < 4.5


def test_fp32_isomerisation_binomial_law():
    c1, c2, A0, B0 = 1.3, 0.7, 30, 10
    net = W.isomerisation(c1, c2, A0, B0)
    N, G, T = 12000, 41, 4.0
    r = oracle.run(net, N, T, G, seed=9, threads=8, precision=FP32, schedule=oracle.SCHEDULE_W32)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    k = c1 + c2
    p = (c2 + c1 * np.exp(-k * g)) / k
    q = c2 * (1.0 - np.exp(-k * g)) / k
    mu = A0 * p + B0 * q
    sig2 = A0 * p * (1 - p) + B0 * q * (1 - q)
    assert np.all(mean[:, 0] + mean[:, 1] == A0 + B0)
    assert _z(mean[1:, 0], mu[1:], np.sqrt(sig2[1:] / N)).max() < 4.5
    assert _z(var[1:, 0], sig2[1:], sig2[1:] * np.sqrt(2.2 / N)).max() < 5.0


def test_moment_sums_match_traces():
    net = W.hiv_shaped()
    N, G, T = 6, 11, 5.0
    r = oracle.run(net, N, T, G, seed=3, moments=True, precision=FP32, schedule=oracle.SCHEDULE_W32)
    s3 = np.zeros((G, 4))
    s4 = np.zeros((G, 4))
    for i in range(N):
        _, _, xs, _, _ = oracle.trace(net, i, T, G, seed=3, precision=FP32, schedule=oracle.SCHEDULE_W32)
        s3 += xs.astype(np.float64) ** 3
        s4 += xs.astype(np.float64) ** 4
    assert np.allclose(r.S3, s3, rtol=1e-12) and np.allclose(r.S4, s4, rtol=1e-12)
    assert r.S1[0, 0] == N * 1000 and math.isclose(r.S3[0, 0], N * 1e9)


def _fp64_lane_scan(a32):
    """The former reading, for contrast only: each lane's compensated chunk
    widened to FP64 on its own, the 32 lane values scanned in FP64."""
    M = len(a32)
    ch = (M + 31) // 32
    lanes = []
    for l in range(32):
        c = [np.float32(v) for v in a32[l * ch:min(M, (l + 1) * ch)]]
        if not c:
            lanes.append(0.0)
            continue
        s, err = c[0], np.float32(0.0)
        for x in c[1:]:
            t = np.float32(s + x)
            bp = np.float32(t - s)
            err = np.float32(err + np.float32(np.float32(s - np.float32(t - bp)) + np.float32(x - bp)))
            s = t
        lanes.append(float(s) + float(err))
    v = lanes[:]
    off = 1
    while off < 32:
        prev = v[:]
        for l in range(off, 32):
            v[l] = prev[l] + prev[l - off]
        off *= 2
    return v[31]


def test_w32_a0_pair_scan_is_exact_where_every_error_is_representable():
    """Lane sums that leave FP64 rounding in a plain FP64 scan of the lanes
    but whose errors are exact binary32 values: the pair scan keeps every
    error until the one final FP64 addition, so a0 is the exact sum (an
    integer here), and the first event time is E / a0."""
    from fractions import Fraction
    M = 64  # two reactions per lane
    cases = []
    a = np.zeros(M, np.float32)
    a[0], a[2], a[4] = 2.0 ** 53, 1.0, 1.0          # lanes 0, 1, 2
    cases.append(a)
    a = np.zeros(M, np.float32)
    a[0], a[1], a[6], a[9] = 2.0 ** 40, 3.0, 2.0 ** 13, 1.0
    cases.append(a)
    a = np.zeros(M, np.float32)
    a[::2] = 2.0 ** 52
    a[1::2] = 1.0                                     # 32 lanes of (2^52, 1)
    cases.append(a)
    differs = 0
    for a in cases:
        exact = sum(Fraction(float(v)) for v in a)
        assert exact == int(exact) and float(exact) == exact  # representable in FP64
        got = oracle.fp32_a0(a, oracle.SCHEDULE_W32)
        assert Fraction(got) == exact
        differs += _fp64_lane_scan(a) != got
    assert differs >= 1  # the cases tell the pair scan from a plain FP64 scan of the lanes
    # the same through a trajectory's first event: order-0 reactions with these rates
    a = cases[0]
    R = np.zeros((M, 1), np.int32)
    P = np.zeros((M, 1), np.int32)
    net = W.Network("pair_scan", ["X"], R, P, a.astype(np.float64), np.array([0], np.int32))
    for seed in (3, 4):
        t, _, E = _first_event(net, seed, schedule=oracle.SCHEDULE_W32)
        assert t == E / (2.0 ** 53 + 2.0)


@pytest.mark.parametrize("M", [8, 64, 128, 300, 512])
def test_w32_a0_is_within_the_pair_summation_bound(M):
    """Random non-negative binary32 propensities over 20 binades: the pair
    scan's a0 is within 2^-40 (relative) of the exact sum -- the bound of
    compensated summation in binary32 pairs ((n u)^2 with u = 2^-24, n <= 512
    terms, plus one FP64 rounding) -- far inside what a plain binary32 sum
    reaches on the same data."""
    from fractions import Fraction
    rng = np.random.default_rng(M)
    worst, worst32 = 0.0, 0.0
    for _ in range(40):
        a = (rng.random(M) * 2.0 ** rng.integers(-10, 10, size=M)).astype(np.float32)
        a[rng.random(M) < 0.2] = 0.0
        exact = sum(Fraction(float(v)) for v in a)
        if exact == 0:
            continue
        got = oracle.fp32_a0(a, oracle.SCHEDULE_W32)
        worst = max(worst, abs(float((Fraction(got) - exact) / exact)))
        s32 = np.float32(0.0)
        for v in a:
            s32 = np.float32(s32 + v)
        worst32 = max(worst32, abs(float((Fraction(float(s32)) - exact) / exact)))
        assert got == oracle.fp32_a0(a[::-1].copy()[::-1].copy(), oracle.SCHEDULE_W32)  # deterministic
    assert worst <= 2.0 ** -40
    assert worst32 > 2.0 ** -30  # the data do exercise binary32 rounding
