"""Pins for the oracle's selective memory along the time axis (Sec. 3.2.1,
Fig. 3): Avg-Y on the union of every trajectory's event times and Avg-XY,
the average of k successive Avg-Y points in time and value (no GPU).

  * a Python restatement from the recorded event lists (union of times with
    0, right-continuous states, windows of k union points), in exact
    integer and Fraction arithmetic;
  * the grid path: with the union times as the grid, the grid sums give the
    same Avg-Y values (two independent constructions in the oracle);
  * conservation in the isomerisation network at every point.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


def _python_avg_xy(net, N, T, seed, k, schedule):
    nu = (net.products - net.reactants).astype(np.int64)
    events = []
    for i in range(N):
        rt, rj, _, _, ne = oracle.trace(net, i, T, 1, seed, grid=[T], schedule=schedule, record_max=100000)
        assert ne == len(rt)
        events.append((rt, rj))
    union = sorted({0.0} | {float(t) for rt, _ in events for t in rt})
    U = len(union)
    S1 = np.zeros((U, net.n_species), dtype=object)
    S2 = np.zeros((U, net.n_species), dtype=object)
    for rt, rj in events:
        x = [int(v) for v in net.x0]
        e = 0
        for q, tq in enumerate(union):
            while e < len(rt) and rt[e] <= tq:
                x = [x[s] + int(nu[rj[e], s]) for s in range(net.n_species)]
                e += 1
            for s in range(net.n_species):
                S1[q, s] += x[s]
                S2[q, s] += x[s] * x[s]
    out_t, out_m, out_q = [], [], []
    for a in range(0, U, k):
        b = min(U, a + k)
        tsum = 0.0
        for q in range(a, b):
            tsum += union[q]
        out_t.append(tsum / (b - a))
        out_m.append([float(Fraction(int(sum(S1[a:b, s])), N * (b - a))) for s in range(net.n_species)])
        out_q.append([float(Fraction(int(sum(S2[a:b, s])), N * (b - a))) for s in range(net.n_species)])
    return np.array(out_t), np.array(out_m), np.array(out_q), U


@pytest.mark.parametrize("k", [1, 3, 7])
@pytest.mark.parametrize("schedule", [oracle.SCHEDULE_L, oracle.SCHEDULE_W32])
def test_avg_xy_matches_restatement_from_event_lists(k, schedule):
    net = W.isomerisation(1.3, 0.7, 6, 3)
    N, T, seed = 5, 2.0, 4
    t, m, q, U = oracle.avg_xy(net, N, T, seed, k, schedule=schedule)
    pt, pm, pq, pU = _python_avg_xy(net, N, T, seed, k, schedule)
    assert U == pU and len(t) == -(-U // k)
    assert np.array_equal(t, pt) and np.array_equal(m, pm) and np.array_equal(q, pq)


def test_avg_y_equals_the_grid_path_on_the_union_times():
    net = W.hiv_shaped()
    N, T, seed = 6, 3.0, 2
    t, m, q, U = oracle.avg_xy(net, N, T, seed, 1, schedule=oracle.SCHEDULE_L)
    assert t[0] == 0.0 and np.all(np.diff(t) > 0) and len(t) == U
    r = oracle.run(net, N, T, U, seed, grid=t)
    mean, _ = oracle.finalize(N, r.S1, r.S2)
    assert np.array_equal(mean, m)
    assert np.array_equal(r.S2.astype(np.float64) / N, q)


def test_conservation_and_window_count():
    net = W.isomerisation(1.0, 0.5, 30, 10)
    N, T = 40, 4.0
    t, m, q, U = oracle.avg_xy(net, N, T, 3, 40)
    assert len(t) == -(-U // 40) and np.all(np.diff(t) > 0)
    assert np.allclose(m.sum(axis=1), 40.0, rtol=0, atol=1e-12)
    assert m[0, 0] > 29.0 and t[-1] < T
