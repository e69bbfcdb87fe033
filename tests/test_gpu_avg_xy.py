"""GPU checks of selective memory along the time axis (ssa_ensemble_avg_xy):
Avg-Y on the union of event times and Avg-XY windows, against the oracle
bit for bit (the same trajectories -- thread schedule L or warp schedule W32
-- the same integer window sums, the same ascending FP64 time sums), against
the grid path on the union times, and at the bench size (65,536
trajectories) through properties that hold at any size."""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(net, n, T, seed, k, **kw):
    model = ssa.Model.from_network(net)
    try:
        return ssa.ensemble_avg_xy(model, n, T, seed, k, **kw)
    finally:
        model.close()


SCHED = {"thread": oracle.SCHEDULE_L, "warp": oracle.SCHEDULE_W32}


@pytest.mark.parametrize("case", ["birth_death", "hiv", "hiv_warp", "random", "fp32"])
def test_bit_exact_with_oracle(case):
    sched = "thread"
    if case == "birth_death":
        net, n, T, ks, prec = W.birth_death(), 64, 10.0, [1, 7, 64], "fp64"
    elif case == "hiv":
        net, n, T, ks, prec = W.hiv_shaped(), 48, 5.0, [1, 48], "fp64"
    elif case == "hiv_warp":
        net, n, T, ks, prec, sched = W.hiv_shaped(), 48, 5.0, [1, 48], "fp64", "warp"
    elif case == "random":
        net, n, T, ks, prec, sched = W.random_network(3), 16, 0.5, [1, 16], "fp64", "warp"
    else:
        net, n, T, ks, prec, sched = W.random_network(3), 16, 0.5, [3], "fp32", "warp"
    oprec = oracle.PRECISION_FP32 if prec == "fp32" else oracle.PRECISION_FP64
    for k in ks:
        # AUTO picks the thread schedule for the small FP64 networks
        t, m, q, U = _gpu(net, n, T, 5, k, precision=prec, schedule="auto" if sched == "thread" else "warp")
        ot, om, oq, oU = oracle.avg_xy(net, n, T, 5, k, schedule=SCHED[sched], precision=oprec)
        assert U == oU and len(t) == len(ot) == -(-U // k), (case, k)
        assert np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq), (case, k)


@pytest.mark.parametrize("sched", ["thread", "warp"])
def test_avg_y_equals_grid_path_on_union_times(sched):
    net = W.hiv_shaped()
    n, T = 200, 4.0
    t, m, q, U = _gpu(net, n, T, 8, 1, schedule=sched)
    model = ssa.Model.from_network(net)
    r = ssa.ensemble_run(model, n, T, len(t), 8, grid=t, schedule=sched)
    model.close()
    assert np.array_equal(r.mean, m)
    assert np.array_equal(r.sum2.astype(np.float64) / n, q)


def test_bench_size_properties():
    w = W.workload_hiv_shaped()
    n = w.n_traj
    t, m, q, U = _gpu(w.net, n, w.t_end, 1, n)
    model = ssa.Model.from_network(w.net)
    r = ssa.ensemble_run(model, n, w.t_end, 2, 1)  # the same (thread-schedule) trajectories
    model.close()
    # distinct event times: at most one per event, nearly all distinct
    assert 0.999 * r.events <= U - 1 <= r.events
    assert len(t) == -(-U // n) and np.all(np.diff(t) > 0) and 0.0 < t[0] and t[-1] < w.t_end
    assert np.all(q >= m * m - 1e-9 * np.maximum(1.0, q))  # E[x^2] >= E[x]^2 in every window
    # window k from Avg-Y: the same means up to the final rounding
    t1, m1, q1, U1 = _gpu(w.net, 4096, w.t_end, 1, 1)
    t8, m8, q8, U8 = _gpu(w.net, 4096, w.t_end, 1, 8)
    assert U1 == U8
    assert t1[0] == 0.0 and np.all(np.diff(t1) > 0)  # sorted and deduplicated (Avg-Y)
    t1b, m1b, _, U1b = _gpu(w.net, 4096, w.t_end, 1, 1)
    assert U1b == U1 and np.array_equal(t1b, t1) and np.array_equal(m1b, m1)  # repeatable
    P = len(t8)
    for p in [0, 1, P // 2, P - 1]:
        sl = slice(8 * p, min(U1, 8 * p + 8))
        assert np.allclose(m8[p], m1[sl].mean(axis=0), rtol=1e-12, atol=0)
        assert np.isclose(t8[p], t1[sl].mean(), rtol=1e-12, atol=0)


def test_log_capacity_pilot_hint_and_retry():
    """The event log's capacity: estimated from a pilot (more trajectories
    than the pilot's 4,096), given exactly enough, or given far too little
    (one record: the logging run overflows and is repeated with the count it
    reports) -- the results are the oracle's in every case."""
    net, n, T = W.hiv_shaped(), 4200, 0.1
    for sched in ("thread", "warp"):
        ot, om, oq, oU = oracle.avg_xy(net, n, T, 4, 1, schedule=SCHED[sched])
        for hint in (0, 1, 10 ** 7):
            t, m, q, U = _gpu(net, n, T, 4, 1, log_records=hint, schedule=sched)
            assert U == oU and np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq), hint
        # one model, two calls: the second sizes the log from the first one's count
        model = ssa.Model.from_network(net)
        try:
            for _ in range(2):
                t, m, q, U = ssa.ensemble_avg_xy(model, n, T, 4, 1, schedule=sched)
                assert U == oU and np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq)
        finally:
            model.close()
    ssa.release_cached_memory()
    with pytest.raises(ssa.SSAError) as e:
        _gpu(net, 16, T, 4, 1, log_records=-1)
    assert e.value.status == ssa.binding.SSA_EINVAL


@pytest.mark.parametrize("sched", ["thread", "warp"])
def test_wide_small_network_both_schedules(sched):
    """12 species and 15 reactions: the thread kernel's widest template
    bucket (16 x 16) for the thread schedule, and the warp schedule."""
    net = W.random_network(21, n_species=12, n_reactions=15, x0_hi=30)
    for k in (1, 5, 200):
        t, m, q, U = _gpu(net, 200, 3.0, 3, k, schedule=sched, max_events=200000)
        ot, om, oq, oU = oracle.avg_xy(net, 200, 3.0, 3, k, schedule=SCHED[sched], max_events=200000)
        assert U == oU and np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq), (sched, k)
