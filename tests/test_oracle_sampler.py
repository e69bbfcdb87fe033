"""Pins for the oracle's sampler and reduction (no GPU).

Each test checks the oracle against something fixed outside it:
  * closed forms: the birth-death process from X0 = 0 is Poisson with mean
    (k1/k2)(1 - e^{-k2 t}); the expected event count over [0, T] is
    k1 T + k2 int_0^T E X(s) ds = 1900.0045 for k1 = 10, k2 = 0.1, T = 100;
    isomerisation A <-> B gives A(t) = Bin(A0, p) + Bin(B0, q);
  * the exact CTMC transient of tiny networks (matrix exponential of the
    generator, scipy's expm_multiply);
  * the first-step law: tau ~ Exp(a0) and P(j) = a_j / a0, with a_j worked
    out by hand for the initial states;
  * the grid-alignment definition (state after all events with time <= g_k)
    evaluated from the recorded event list, and integer sums over
    per-trajectory traces;
  * exact rational arithmetic for the finalisation and the summation
    schedules.
Statistical tests use fixed seeds; thresholds are 4.5-5 standard errors.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


def _z(est, mu, se):
    return np.abs(est - mu) / se


def test_birth_death_poisson_mean_and_variance():
    net = W.birth_death(10.0, 0.1, 0)
    N, G, T = 20000, 101, 100.0
    r = oracle.run(net, N, T, G, seed=1, threads=8)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    lam = (10.0 / 0.1) * (1.0 - np.exp(-0.1 * g))
    assert mean[0, 0] == 0.0 and var[0, 0] == 0.0
    m, v, l = mean[1:, 0], var[1:, 0], lam[1:]
    assert np.max(_z(m, l, np.sqrt(l / N))) < 4.5
    assert np.max(_z(v, l, np.sqrt((l + 2 * l * l) / N))) < 4.5


def test_birth_death_expected_event_count():
    net = W.birth_death(10.0, 0.1, 0)
    N = 4000
    r = oracle.run(net, N, 100.0, 11, seed=3, per_traj=True, threads=8)
    expected = 1000.0 + 1000.0 - 100.0 * (1.0 - math.exp(-10.0))  # = 1900.0045...
    assert abs(expected - 1900.0045) < 1e-4
    ev = r.traj_events.astype(np.float64)
    assert r.events == int(ev.sum())
    se = ev.std(ddof=1) / math.sqrt(N)
    assert abs(ev.mean() - expected) < 4.5 * se


def test_birth_death_final_state_is_poisson():
    scipy_stats = pytest.importorskip("scipy.stats")
    net = W.birth_death(10.0, 0.1, 0)
    lam = 100.0 * (1.0 - math.exp(-10.0))
    finals = []
    for i in range(4000):
        _, _, xs, flags, _ = oracle.trace(net, i, 100.0, 2, seed=5, record_max=1)
        assert flags == 0
        finals.append(int(xs[1, 0]))
    finals = np.array(finals)
    edges = [0, 80, 85, 88, 91, 94, 97, 100, 103, 106, 109, 112, 115, 120, 10**6]
    obs = np.histogram(finals, bins=edges)[0]
    cdf = scipy_stats.poisson.cdf(np.array(edges[1:]) - 1, lam)
    probs = np.diff(np.concatenate([[0.0], cdf]))
    exp = probs * len(finals)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    dof = len(obs) - 1
    assert scipy_stats.chi2.sf(chi2, dof) > 1e-4


def test_isomerisation_binomial_law():
    c1, c2, A0, B0 = 1.0, 0.5, 30, 10
    net = W.isomerisation(c1, c2, A0, B0)
    N, G, T = 20000, 41, 4.0
    r = oracle.run(net, N, T, G, seed=9, threads=8)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    k = c1 + c2
    p = (c2 + c1 * np.exp(-k * g)) / k
    q = c2 * (1.0 - np.exp(-k * g)) / k
    mu = A0 * p + B0 * q
    sig2 = A0 * p * (1 - p) + B0 * q * (1 - q)
    assert mean[0, 0] == A0 and var[0, 0] == 0.0
    assert np.all(mean[:, 0] + mean[:, 1] == A0 + B0)   # conservation, exactly
    zm = _z(mean[1:, 0], mu[1:], np.sqrt(sig2[1:] / N))
    zv = _z(var[1:, 0], sig2[1:], sig2[1:] * np.sqrt(2.2 / N))
    assert zm.max() < 4.5 and zv.max() < 5.0


def _ctmc_moments(net, times, cap=60):
    """Exact mean/var/4th central moment of every species at `times` by
    uniformised matrix exponential of the (truncated) CTMC generator."""
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    R = np.asarray(net.reactants, dtype=np.int64)
    Pm = np.asarray(net.products, dtype=np.int64)
    nu = Pm - R
    c = np.asarray(net.rates, dtype=np.float64)
    x0 = tuple(int(v) for v in net.x0)
    index = {x0: 0}
    states = [x0]
    rows, cols, vals = [], [], []
    head = 0
    while head < len(states):
        x = states[head]
        for j in range(R.shape[0]):
            h = 1
            for s in range(R.shape[1]):
                if R[j, s] == 1:
                    h *= x[s]
                elif R[j, s] == 2:
                    h *= x[s] * (x[s] - 1) // 2
            if h == 0 or c[j] == 0.0:
                continue
            y = tuple(int(v) for v in np.asarray(x) + nu[j])
            if max(y) > cap:
                continue
            if y not in index:
                index[y] = len(states)
                states.append(y)
            rate = c[j] * h
            rows.append(index[x]); cols.append(index[y]); vals.append(rate)
            rows.append(index[x]); cols.append(index[x]); vals.append(-rate)
        head += 1
    n = len(states)
    Q = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    p0 = np.zeros(n); p0[0] = 1.0
    X = np.array(states, dtype=np.float64)
    out = []
    for t in times:
        p = spl.expm_multiply(Q.T * t, p0) if t > 0 else p0
        mu = p @ X
        d = X - mu
        out.append((mu, p @ d ** 2, p @ d ** 4))
    return out


@pytest.mark.parametrize("case", range(3))
def test_tiny_networks_match_exact_transient(case):
    net, T = W.tiny_networks()[case]
    N, G = 40000, 9
    r = oracle.run(net, N, T, G, seed=21 + case, threads=8)
    mean, var = oracle.finalize(N, r.S1, r.S2)
    g = oracle.uniform_grid(G, T)
    mom = _ctmc_moments(net, g)
    for k in range(1, G):
        mu, s2, m4 = mom[k]
        for s in range(net.n_species):
            if s2[s] < 1e-12:
                assert abs(mean[k, s] - mu[s]) < 1e-9
                continue
            zm = abs(mean[k, s] - mu[s]) / math.sqrt(s2[s] / N)
            se_v = math.sqrt(max(m4[s] - s2[s] ** 2 * (N - 3) / (N - 1), 1e-30) / N)
            zv = abs(var[k, s] - s2[s]) / se_v
            assert zm < 4.5 and zv < 4.5, (net.name, k, s, zm, zv)


def _first_steps(net, n, seed, schedule=oracle.SCHEDULE_L):
    taus, js = [], []
    for i in range(n):
        rt, rj, _, _, ne = oracle.trace(net, i, 1e9, 1, seed, grid=[1e9], max_events=1,
                                        schedule=schedule, record_max=1)
        assert ne == 1
        taus.append(rt[0]); js.append(rj[0])
    return np.array(taus), np.array(js)


@pytest.mark.parametrize("schedule", [oracle.SCHEDULE_L, oracle.SCHEDULE_W32])
def test_first_step_law_hiv_shaped(schedule):
    stats = pytest.importorskip("scipy.stats")
    net = W.hiv_shaped()
    # a_j at x0 = (T 1000, I 0, V 100, E 10), by hand:
    #   10, 0.01*1000, 2e-5*1000*100, 0.5*0, 50*0, 3*100, 1e-3*0*10, 1e-4*0*10, 1, 0.1*10
    a = np.array([10.0, 10.0, 2.0, 0.0, 0.0, 300.0, 0.0, 0.0, 1.0, 1.0])
    a0 = 324.0
    taus, js = _first_steps(net, 20000, seed=4, schedule=schedule)
    assert stats.kstest(taus * a0, "expon").pvalue > 1e-3
    counts = np.bincount(js, minlength=10)
    assert np.all(counts[a == 0] == 0)
    nz = a > 0
    exp = a[nz] / a0 * len(js)
    chi2 = float(((counts[nz] - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, nz.sum() - 1) > 1e-3


def test_first_step_law_second_order():
    stats = pytest.importorskip("scipy.stats")
    net = W.dimerisation(0.3, 0.2, 0.05, 8, 5)
    # 2A -> C: 0.3 * C(8,2) = 8.4 ; C -> 2A: 0 ; A + B -> C: 0.05 * 8 * 5 = 2.0
    a0 = 10.4
    taus, js = _first_steps(net, 20000, seed=8)
    assert stats.kstest(taus * a0, "expon").pvalue > 1e-3
    counts = np.bincount(js, minlength=3)
    assert counts[1] == 0
    exp = np.array([8.4, 2.0]) / a0 * len(js)
    chi2 = float(((counts[[0, 2]] - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, 1) > 1e-3


def _states_from_events(net, rt, rj, grid):
    nu = np.asarray(net.products, dtype=np.int64) - np.asarray(net.reactants, dtype=np.int64)
    x = np.zeros((len(rt) + 1, net.n_species), dtype=np.int64)
    x[0] = net.x0
    for e, j in enumerate(rj):
        x[e + 1] = x[e] + nu[j]
    # state at g = after all events with time <= g (right-continuous)
    idx = np.searchsorted(rt, grid, side="right")
    return x[idx]


def test_grid_alignment_is_right_continuous():
    net = W.hiv_shaped()
    T, G = 30.0, 301
    for traj in range(5):
        rt, rj, xs, flags, ne = oracle.trace(net, traj, T, G, seed=1)
        assert flags == 0 and len(rt) == ne and np.all(np.diff(rt) > 0)
        assert np.array_equal(xs, _states_from_events(net, rt, rj, oracle.uniform_grid(G, T)))
        # a grid that hits event times exactly: the post-event state must be seen
        grid = np.unique(np.concatenate([[0.0], rt[:50], [T]]))
        rt2, rj2, xs2, _, _ = oracle.trace(net, traj, T, 0, seed=1, grid=grid)
        assert np.array_equal(rt2, rt) and np.array_equal(rj2, rj)
        assert np.array_equal(xs2, _states_from_events(net, rt, rj, grid))


def test_reduction_equals_sum_of_traces_and_is_order_free():
    net = W.hiv_shaped()
    T, G, N = 30.0, 61, 48
    r = oracle.run(net, N, T, G, seed=2, per_traj=True)
    s1 = np.zeros((G, 4), dtype=np.int64)
    s2 = np.zeros((G, 4), dtype=np.int64)
    for i in range(N):
        rt, rj, xs, _, ne = oracle.trace(net, i, T, G, seed=2)
        assert ne == r.traj_events[i]
        s1 += xs
        s2 += xs * xs
    assert np.array_equal(r.S1, s1) and np.array_equal(r.S2, s2)
    perm = np.random.default_rng(0).permutation(N)
    rp = oracle.run(net, N, T, G, seed=2, ids=perm.tolist(), threads=3)
    assert np.array_equal(rp.S1, s1) and np.array_equal(rp.S2, s2)
    # shards by trajectory offset add up exactly
    a = oracle.run(net, 20, T, G, seed=2, traj_begin=0)
    b = oracle.run(net, N - 20, T, G, seed=2, traj_begin=20)
    assert np.array_equal(a.S1 + b.S1, s1) and np.array_equal(a.S2 + b.S2, s2)


def test_finalize_matches_exact_rationals():
    rng = np.random.default_rng(3)
    for N in [2, 3, 1000, 65536, 1 << 20]:
        S1 = rng.integers(0, 1 << 40, size=(7, 3), dtype=np.int64)
        S2 = S1 * 3 + rng.integers(0, 1 << 20, size=(7, 3), dtype=np.int64)
        mean, var = oracle.finalize(N, S1, S2)
        for k in range(7):
            for s in range(3):
                assert mean[k, s] == float(Fraction(int(S1[k, s]), N))
                exact = Fraction(N * int(S2[k, s]) - int(S1[k, s]) ** 2, N * (N - 1))
                assert abs(var[k, s] - float(exact)) <= 2 * math.ulp(float(exact)) + 1e-300
    mean, var = oracle.finalize(1, np.array([[5]], dtype=np.int64), np.array([[25]], dtype=np.int64))
    assert mean[0, 0] == 5.0 and math.isnan(var[0, 0])


def test_truncation_and_absorbing_state():
    net = W.hiv_shaped()
    r = oracle.run(net, 16, 30.0, 31, seed=1, max_events=5, per_traj=True)
    assert r.truncated == 16 and np.all(r.traj_events == 5)
    assert np.all(r.traj_flags == oracle.FLAG_TRUNCATED)
    rt, rj, xs, flags, ne = oracle.trace(net, 3, 30.0, 31, seed=1, max_events=5)
    assert flags == oracle.FLAG_TRUNCATED and ne == 5
    assert np.array_equal(xs, _states_from_events(net, rt, rj, oracle.uniform_grid(31, 30.0)))
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32),
                      np.array([1.0]), np.array([3], np.int32))
    rt, rj, xs, flags, ne = oracle.trace(death, 0, 1e6, 5, seed=1)
    assert ne == 3 and flags == 0 and xs[-1, 0] == 0


def test_overflow_is_flagged_not_fired():
    # 0 -> 2^31-1 molecules can't be exceeded: X near the limit, 0 -> X
    net = W.Network("grow", ["X"], np.array([[0]], np.int32), np.array([[1]], np.int32),
                    np.array([1.0]), np.array([2147483645], np.int32))
    rt, rj, xs, flags, ne = oracle.trace(net, 0, 100.0, 3, seed=1)
    assert flags == oracle.FLAG_OVERFLOW and ne == 2 and xs[-1, 0] == 2147483647


@pytest.mark.parametrize("M", [1, 5, 31, 32, 33, 100, 128, 512])
def test_summation_schedules_exact_on_integers(M):
    """With small integer propensities every partial sum is exact, so any
    schedule must reproduce the exact prefix sums; a wrong lane offset or chunk
    index would change an integer."""
    rng = np.random.default_rng(M)
    a = rng.integers(0, 1000, size=M).astype(np.float64)
    want = np.cumsum(a)
    for sch in (oracle.SCHEDULE_L, oracle.SCHEDULE_W32):
        pre, a0 = oracle.prefix_sums(a, sch)
        assert np.array_equal(pre, want) and a0 == want[-1]


def test_w32_rounding_within_bound():
    rng = np.random.default_rng(1)
    for M in [64, 128, 500]:
        a = np.exp(rng.uniform(-7, 14, size=M))
        pre, a0 = oracle.prefix_sums(a, oracle.SCHEDULE_W32)
        exact = np.cumsum([Fraction(float(v)) for v in a])
        for j in range(M):
            assert abs(Fraction(float(pre[j])) - exact[j]) <= exact[j] * Fraction(64, 2 ** 53)


def test_w32_selection_never_picks_a_zero_propensity_reaction():
    """Under W32 a lane's exclusive scan value can exceed the previous lane's
    last prefix by rounding, so the prefixes are not monotone at lane
    boundaries.  A zero-propensity reaction opening a lane must still never
    be chosen (Sec. 2: only possible transitions fire), for any target."""
    rng = np.random.default_rng(5)
    M = 64  # two reactions per lane
    found = 0
    for _ in range(200):
        a = rng.uniform(0.1, 1.0, size=M) * 10.0 ** rng.integers(-3, 4, size=M)
        for lane in range(1, 32):
            j0 = 2 * lane
            b = a.copy()
            b[j0] = 0.0
            pre, a0 = oracle.prefix_sums(b, oracle.SCHEDULE_W32)
            if not pre[j0] > pre[j0 - 1]:
                continue
            found += 1
            lo = pre[j0 - 1]
            for target in (lo, np.nextafter(lo, np.inf), np.nextafter(pre[j0], -np.inf)):
                j = oracle.select(b, target, oracle.SCHEDULE_W32)
                assert j != j0 and b[j] > 0.0
                assert j > j0 - 1  # prefix_{j0-1} <= target: nothing at or before j0 - 1 qualifies
            j = oracle.select(b, np.nextafter(lo, -np.inf), oracle.SCHEDULE_W32)
            assert j <= j0 - 1 and b[j] > 0.0
        if found >= 5:
            break
    assert found >= 5
    # all-zero propensities: nothing to choose
    assert oracle.select(np.zeros(40), 0.0, oracle.SCHEDULE_W32) == -1
