"""GPU edge cases of the newer paths, against the oracle: Avg-XY with
truncated and absorbing trajectories, a batch of networks with explicit grids
and truncation, the gradient with device buffers and a device grid, and the
FP32 warp kernel on an explicit grid."""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu
W32 = oracle.SCHEDULE_W32


@pytest.mark.parametrize("sched", ["thread", "warp"])
def test_avg_xy_truncation_and_absorbing_states(sched):
    osched = oracle.SCHEDULE_L if sched == "thread" else W32
    net = W.hiv_shaped()
    model = ssa.Model.from_network(net)
    t, m, q, U = ssa.ensemble_avg_xy(model, 40, 30.0, 3, 7, max_events=25, schedule=sched)
    ot, om, oq, oU = oracle.avg_xy(net, 40, 30.0, 3, 7, max_events=25, schedule=osched)
    assert U == oU <= 40 * 25 + 1 and np.array_equal(t, ot) and np.array_equal(m, om) and np.array_equal(q, oq)
    model.close()
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32), np.array([2.0]),
                      np.array([5], np.int32))
    model = ssa.Model.from_network(death)
    t, m, q, U = ssa.ensemble_avg_xy(model, 33, 50.0, 4, 1, schedule=sched)
    ot, om, oq, oU = oracle.avg_xy(death, 33, 50.0, 4, 1, schedule=osched)
    assert U == oU == 33 * 5 + 1 and np.array_equal(m, om) and m[-1, 0] == 0.0
    if sched == "thread":  # the thread schedule is FP64 only
        with pytest.raises(ssa.SSAError) as e:
            ssa.ensemble_avg_xy(model, 33, 50.0, 4, 5, precision="fp32", schedule="thread")
        assert e.value.status == ssa.binding.SSA_EUNSUPPORTED
        model.close()
        return
    # FP32 mode
    t, m, q, U = ssa.ensemble_avg_xy(model, 33, 50.0, 4, 5, precision="fp32")
    ot, om, oq, oU = oracle.avg_xy(death, 33, 50.0, 4, 5, schedule=W32, precision=oracle.PRECISION_FP32)
    assert U == oU and np.array_equal(t, ot) and np.array_equal(m, om)
    model.close()


def test_batch_explicit_grids_and_truncation():
    nets = [W.hiv_shaped(), W.random_network(3), W.birth_death()]
    grids = [np.array([0.0, 0.1, 0.1, 2.5, 29.0, 30.0]), None, np.linspace(0.0, 5.0, 17)]
    n, T = [50, 20, 64], [30.0, 0.5, 5.0]
    G = [len(grids[0]), 41, len(grids[2])]
    models = [ssa.Model.from_network(x) for x in nets]
    batch = ssa.Batch(models, n, T, G, grids, precision="fp64", max_events=300)
    outs, st = batch.launch(21, want_sums=True)
    for b, net in enumerate(nets):
        o = oracle.run(net, n[b], T[b], G[b], 21, grid=grids[b], stream=b, schedule=W32, max_events=300,
                       threads=8)
        assert np.array_equal(outs[b]["sum1"], o.S1) and np.array_equal(outs[b]["sum2"], o.S2), b
        assert batch.network_stats(b).truncated == o.truncated
    batch.close()
    for mdl in models:
        mdl.close()


def test_gradient_with_device_buffers_and_grid():
    import torch
    net = W.hiv_shaped()
    model = ssa.Model.from_network(net)
    grid = np.concatenate([[0.0], np.sort(np.random.default_rng(2).uniform(0.0, 30.0, 60)), [30.0]])
    f = ssa.ensemble_run(model, 256, 30.0, len(grid), 6, grid=grid)
    w = np.zeros((len(grid), 4))
    w[:, 1] = 0.1
    g_host, se_host, _ = ssa.ensemble_grad(model, 256, 30.0, len(grid), 6, w, f.mean, grid=grid)
    g_dev, se_dev, traj = ssa.ensemble_grad(model, 256, 30.0, len(grid), 6, torch.as_tensor(w, device="cuda:0"),
                                            torch.as_tensor(f.mean, device="cuda:0"), grid=grid, device="cuda:0",
                                            per_traj=True)
    torch.cuda.synchronize()
    assert np.array_equal(g_host, g_dev.cpu().numpy()) and np.array_equal(se_host, se_dev.cpu().numpy())
    og = oracle.grad(net, 256, 30.0, len(grid), 6, w, f.mean, grid=grid, threads=8)
    scale = np.abs(og).max(axis=0) + 1e-300
    assert np.all(np.abs(traj.cpu().numpy().T - og) <= 1e-9 * scale)
    model.close()


def test_fp32_warp_kernel_explicit_grid():
    net = W.random_network(3)
    grid = np.linspace(0.0, 1.0, 23) ** 2
    model = ssa.Model.from_network(net)
    g = ssa.ensemble_run(model, 40, 1.0, len(grid), 8, grid=grid, precision="fp32", per_traj=True)
    o = oracle.run(net, 40, 1.0, len(grid), 8, grid=grid, schedule=W32, precision=oracle.PRECISION_FP32,
                   per_traj=True, threads=8)
    assert np.array_equal(g.sum2, o.S2) and np.array_equal(g.traj_hash, o.traj_hash)
    model.close()
