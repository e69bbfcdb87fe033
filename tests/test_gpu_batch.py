"""GPU checks of batched ensembles (ssa_batch_*): every network of a batch
must give exactly the results of running it alone (ssa_ensemble_run in the
schedule the batch reports for it, stream id = batch stream id + its index),
whatever the launch shape and schedules the autotuner picks; the captured
graph must replay correctly for new seeds; networks are also checked against
the oracle directly in their recorded schedule."""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu


def _mixed():
    nets = [W.birth_death(), W.hiv_shaped(), W.random_network(3),
            W.random_network(41, n_species=64, n_reactions=512, x0_hi=60),
            W.random_network(42, n_species=4, n_reactions=8, x0_hi=30), W.isomerisation(1.3, 0.7, 30, 10),
            W.random_network(43, n_species=20, n_reactions=70, x0_hi=40)]
    n = [300, 257, 64, 29, 500, 111, 90]
    t_end = [100.0, 30.0, 2.0, 1.0, 5.0, 4.0, 1.5]
    G = [101, 301, 201, 51, 11, 41, 76]
    return nets, n, t_end, G


SCHED_NAME = {1: "thread", 2: "warp"}
ORACLE_SCHED = {1: oracle.SCHEDULE_L, 2: oracle.SCHEDULE_W32}


def _alone(net, n, t_end, G, seed, stream_id, precision, grid=None, max_events=4000, schedule="warp"):
    model = ssa.Model.from_network(net)
    try:
        r = ssa.ensemble_run(model, n, t_end, G, seed, grid=grid, schedule=schedule, precision=precision,
                             stream_id=stream_id, max_events=max_events)
    finally:
        model.close()
    return r


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_each_network_alone(precision):
    nets, n, t_end, G = _mixed()
    hiv_grid = np.unique(np.concatenate([[0.0, 0.5], np.linspace(1.0, 30.0, 299)]))
    grids = [None, hiv_grid, None, None, None, None, None]
    G[1] = len(hiv_grid)
    models = [ssa.Model.from_network(x) for x in nets]
    batch = ssa.Batch(models, n, t_end, G, grids, precision=precision, max_events=4000, stream_id=3)
    outs, st = batch.launch(11, want_sums=True)
    total = 0
    scheds = []
    for b, net in enumerate(nets):
        ns = batch.network_stats(b)
        scheds.append(ns.schedule)
        r = _alone(net, n[b], t_end[b], G[b], 11, 3 + b, precision, grid=grids[b], schedule=SCHED_NAME[ns.schedule])
        assert r.schedule == ns.schedule
        for k in ("sum1", "sum2", "mean", "var"):
            assert np.array_equal(outs[b][k].view(np.int64), getattr(r, k).view(np.int64)), (b, k)
        assert ns.events == r.events and ns.max_x == r.max_x
        total += r.events
    assert st.events == total
    # schedule AUTO before tuning: the rule of ssa_ensemble_run (the thread
    # schedule for small FP64 networks; FP32 batches run every network per warp)
    if precision == "fp64":
        assert scheds == [1, 1, 2, 2, 1, 1, 2]
    else:
        assert scheds == [2] * len(nets)
    # two networks straight against the oracle (same schedule and precision)
    prec = oracle.PRECISION_FP32 if precision == "fp32" else oracle.PRECISION_FP64
    for b in (1, 3):
        o = oracle.run(nets[b], n[b], t_end[b], G[b], 11, grid=grids[b], stream=3 + b,
                       schedule=ORACLE_SCHED[scheds[b]], precision=prec, max_events=4000, threads=16)
        assert np.array_equal(outs[b]["sum1"], o.S1) and np.array_equal(outs[b]["sum2"], o.S2)
    batch.close()
    for m in models:
        m.close()


def test_graph_replay_tuning_and_device_outputs():
    import torch
    nets, n, t_end, G = _mixed()
    models = [ssa.Model.from_network(x) for x in nets]
    host = ssa.Batch(models, n, t_end, G, precision="fp32", max_events=4000)
    a, _ = host.launch(5, want_sums=True)
    b, _ = host.launch(6, want_sums=True)
    c, _ = host.launch(5, want_sums=True)
    for i in range(len(nets)):
        assert np.array_equal(a[i]["sum2"], c[i]["sum2"])
    assert any(not np.array_equal(a[i]["sum2"], b[i]["sum2"]) for i in range(len(nets)))
    threads, split, ms = host.tune()
    assert threads in (64, 128, 256) and ms > 0
    d, _ = host.launch(5, want_sums=True)
    for i in range(len(nets)):
        assert np.array_equal(a[i]["sum1"], d[i]["sum1"]) and np.array_equal(a[i]["sum2"], d[i]["sum2"])
    dev = ssa.Batch(models, n, t_end, G, device="cuda:0", precision="fp32", max_events=4000, block_threads=64)
    e, _ = dev.launch(5, want_sums=True)
    torch.cuda.synchronize()
    for i in range(len(nets)):
        assert np.array_equal(e[i]["sum2"].cpu().numpy(), a[i]["sum2"])
        assert np.array_equal(e[i]["mean"].cpu().numpy().view(np.int64), a[i]["mean"].view(np.int64))
    host.close()
    dev.close()
    for m in models:
        m.close()


def test_uneven_256_network_batch_sampled():
    """The uneven 256-network batch (trajectory counts / 64): every network's
    t = 0 sums, and eight networks spread over the batch against running them
    alone."""
    ws = W.batch_networks(traj_div=64)
    assert len(ws) == 256
    models = [ssa.Model.from_network(w.net) for w in ws]
    batch = ssa.Batch(models, [w.n_traj for w in ws], [w.t_end for w in ws], [w.n_grid for w in ws],
                      precision="fp32", max_events=200000)
    outs, st = batch.launch(1, want_sums=True)
    assert st.overflowed == 0
    for b, w in enumerate(ws):
        x0 = w.net.x0.astype(np.int64)
        assert np.array_equal(outs[b]["sum1"][0], w.n_traj * x0)
    for b in np.linspace(0, 255, 8).astype(int):
        w = ws[b]
        r = _alone(w.net, w.n_traj, w.t_end, w.n_grid, 1, int(b), "fp32", max_events=200000)
        assert np.array_equal(outs[b]["sum2"], r.sum2) and np.array_equal(outs[b]["sum1"], r.sum1)
    batch.close()
    for m in models:
        m.close()


def test_tuner_picks_a_schedule_per_network_and_results_follow_it():
    """FP64 batch: ssa_batch_tune times the thread and the warp schedule of
    every network that fits both and records the faster; each network then
    equals the oracle in its recorded schedule (L or W32), launches repeat
    bit for bit, and fixed schedules are left alone by the tuner."""
    nets, n, t_end, G = _mixed()
    models = [ssa.Model.from_network(x) for x in nets]
    fits = [True, True, False, False, True, True, False]  # at most 16 reactions and species
    batch = ssa.Batch(models, n, t_end, G, precision="fp64", max_events=4000, stream_id=5)
    threads, split, ms = batch.tune()
    assert threads in (64, 128, 256) and ms > 0
    outs, _ = batch.launch(21, want_sums=True)
    again, _ = batch.launch(21, want_sums=True)
    for b, net in enumerate(nets):
        sched = batch.network_stats(b).schedule
        assert sched in (1, 2) and (fits[b] or sched == 2), (b, sched)
        o = oracle.run(net, n[b], t_end[b], G[b], 21, stream=5 + b, schedule=ORACLE_SCHED[sched],
                       max_events=4000, threads=16, per_traj=True)
        assert np.array_equal(outs[b]["sum1"], o.S1) and np.array_equal(outs[b]["sum2"], o.S2), (b, sched)
        om, ov = oracle.finalize(n[b], o.S1, o.S2)
        assert np.array_equal(outs[b]["mean"].view(np.int64), om.view(np.int64))
        assert np.array_equal(again[b]["sum2"], outs[b]["sum2"])
        assert batch.network_stats(b).events == o.events
    batch.close()
    # fixed schedules: every network per warp, or (small networks only) per thread
    for sched, idx in (("warp", list(range(len(nets)))), ("thread", [0, 1, 4, 5])):
        sub = [models[i] for i in idx]
        fixed = ssa.Batch(sub, [n[i] for i in idx], [t_end[i] for i in idx], [G[i] for i in idx], precision="fp64",
                          max_events=4000, stream_id=5, schedule=sched)
        fixed.tune()
        res, _ = fixed.launch(22, want_sums=True)
        for q, i in enumerate(idx):
            ns = fixed.network_stats(q)
            assert SCHED_NAME[ns.schedule] == sched
            r = _alone(nets[i], n[i], t_end[i], G[i], 22, 5 + q, "fp64", schedule=sched)
            assert np.array_equal(res[q]["sum2"], r.sum2) and np.array_equal(res[q]["sum1"], r.sum1)
        fixed.close()
    for m in models:
        m.close()

