"""GPU parity of the warp-per-trajectory kernel (summation schedule W32)
against the oracle run with the same schedule, through the C ABI.

Bit-exact in FP64: int64 grid sums, mean, variance, per-trajectory event
counts, flags and event-sequence hashes.  Cases cover every chunk width
(ceil(M / 32) = 1, 2, 3, 7, 16, with empty lanes and ragged last chunks),
networks small enough for the thread kernel forced onto the warp kernel,
explicit grids, shards, truncation and overflow, and the random
32-species / 128-reaction network at its full size (262,144 trajectories,
1001-point grid) on sampled trajectory ids.
"""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu

W32 = oracle.SCHEDULE_W32


def _gpu(net, n, t_end, G, seed, device=True, **kw):
    model = ssa.Model.from_network(net)
    try:
        r = ssa.ensemble_run(model, n, t_end, G, seed, device="cuda:0" if device else None, per_traj=True,
                             schedule="warp", **kw)
    finally:
        model.close()
    keys = ("mean", "var", "sum1", "sum2", "traj_events", "traj_hash", "traj_flags")
    if device:
        import torch
        torch.cuda.synchronize()
        out = {k: getattr(r, k).cpu().numpy() for k in keys}
        out["traj_hash"] = out["traj_hash"].view(np.uint64)
    else:
        out = {k: getattr(r, k) for k in keys}
    out["stats"] = r
    return out


def _oracle(net, n, t_end, G, seed, threads=16, **kw):
    r = oracle.run(net, n, t_end, G, seed, per_traj=True, threads=threads, schedule=W32, **kw)
    mean, var = oracle.finalize(n, r.S1, r.S2)
    return r, mean, var


def _assert_same(g, r, mean, var):
    assert np.array_equal(g["traj_events"], r.traj_events)
    assert np.array_equal(g["traj_hash"], r.traj_hash)
    assert np.array_equal(g["traj_flags"], r.traj_flags)
    assert np.array_equal(g["sum1"], r.S1)
    assert np.array_equal(g["sum2"], r.S2)
    assert np.array_equal(g["mean"].view(np.int64), mean.view(np.int64))
    assert np.array_equal(g["var"].view(np.int64), var.view(np.int64))
    assert g["stats"].events == r.events


def test_random_32x128_network_bit_exact():
    w = W.workload_random(n_traj=200)
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    r, mean, var = _oracle(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    _assert_same(g, r, mean, var)
    assert r.truncated == 0 and r.overflowed == 0 and r.events > 200 * 1000


@pytest.mark.parametrize("S,M", [(5, 1), (8, 31), (8, 32), (12, 33), (16, 70), (24, 100), (40, 200), (64, 512)])
def test_every_chunk_width_bit_exact(S, M):
    net = W.random_network(500 + M, n_species=S, n_reactions=M, x0_hi=60)
    n = 8 * 3 + 5  # several warps of one CTA plus a ragged CTA
    g = _gpu(net, n, 1.0, 101, 7, max_events=4000)
    r, mean, var = _oracle(net, n, 1.0, 101, 7, max_events=4000)
    _assert_same(g, r, mean, var)


@pytest.mark.parametrize("device", [True, False])
def test_small_networks_forced_onto_the_warp_kernel(device):
    net = W.hiv_shaped()
    g = _gpu(net, 300, 30.0, 301, 5, device=device)
    r, mean, var = _oracle(net, 300, 30.0, 301, 5)
    _assert_same(g, r, mean, var)
    w = W.workload_birth_death(n_traj=257)
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed, device=device)
    r, mean, var = _oracle(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    _assert_same(g, r, mean, var)


def test_launch_shapes_do_not_change_results():
    net = W.random_network(3)
    base = _gpu(net, 64, 2.0, 201, 9)
    for threads, blocks in [(32, 0), (64, 3), (256, 1), (128, 0)]:
        g = _gpu(net, 64, 2.0, 201, 9, block_threads=threads, grid_blocks=blocks)
        for k in ("sum1", "sum2", "traj_hash", "traj_events"):
            assert np.array_equal(g[k], base[k]), (threads, blocks, k)
    r, mean, var = _oracle(net, 64, 2.0, 201, 9)
    _assert_same(base, r, mean, var)


def test_explicit_grid_shards_and_stream_id():
    net = W.random_network(3)
    rt, _, _, _, _ = oracle.trace(net, 0, 2.0, 2, seed=9, schedule=W32)
    grid = np.unique(np.concatenate([[0.0], rt[:30], np.linspace(0.25, 2.0, 20)]))
    g = _gpu(net, 48, 2.0, len(grid), 9, grid=grid, stream_id=5)
    r, mean, var = _oracle(net, 48, 2.0, len(grid), 9, grid=grid, stream=5)
    _assert_same(g, r, mean, var)
    a = _gpu(net, 40, 2.0, 101, 9, traj_offset=0)
    b = _gpu(net, 24, 2.0, 101, 9, traj_offset=40)
    full = _gpu(net, 64, 2.0, 101, 9)
    assert np.array_equal(a["sum1"] + b["sum1"], full["sum1"])
    assert np.array_equal(a["sum2"] + b["sum2"], full["sum2"])
    assert np.array_equal(np.concatenate([a["traj_hash"], b["traj_hash"]]), full["traj_hash"])


def test_truncation_absorbing_and_overflow():
    net = W.random_network(3)
    g = _gpu(net, 70, 10.0, 101, 1, max_events=33)
    r, mean, var = _oracle(net, 70, 10.0, 101, 1, max_events=33)
    _assert_same(g, r, mean, var)
    assert g["stats"].truncated == 70
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32), np.array([2.0]),
                      np.array([5], np.int32))
    g = _gpu(death, 45, 50.0, 51, 3)
    r, mean, var = _oracle(death, 45, 50.0, 51, 3)
    _assert_same(g, r, mean, var)
    grow = W.Network("grow", ["X"], np.array([[0]], np.int32), np.array([[1]], np.int32), np.array([1.0]),
                     np.array([2147483645], np.int32))
    with pytest.raises(ssa.SSAError) as e:
        _gpu(grow, 3, 100.0, 3, 1, device=False)
    assert e.value.status == ssa.binding.SSA_EOVERFLOW


def test_random_network_full_size_sampled_ids():
    """The random 32 x 128 network at 262,144 trajectories in the launch
    configuration the library picks: sampled ids against the oracle, and the
    properties that hold at any size."""
    w = W.workload_random()
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    ids = np.unique(np.linspace(0, w.n_traj - 1, 192).astype(np.int64))
    r = oracle.run(w.net, 0, w.t_end, w.n_grid, w.seed, per_traj=True, threads=16, schedule=W32, ids=ids)
    assert np.array_equal(g["traj_events"][ids], r.traj_events)
    assert np.array_equal(g["traj_hash"][ids], r.traj_hash)
    assert np.array_equal(g["traj_flags"][ids], r.traj_flags)
    x0 = w.net.x0.astype(np.int64)
    assert np.array_equal(g["sum1"][0], w.n_traj * x0)
    assert np.array_equal(g["sum2"][0], w.n_traj * x0 * x0)
    assert int(g["traj_events"].sum()) == g["stats"].events
    assert np.all(g["traj_flags"] == 0)
    # finalisation of sampled cells from the int64 sums, in exact integers
    n = w.n_traj
    for k, s in [(1, 0), (500, 7), (1000, 31)]:
        s1, s2 = int(g["sum1"][k, s]), int(g["sum2"][k, s])
        assert g["mean"][k, s] == float(s1) / float(n)
        assert g["var"][k, s] == float(n * s2 - s1 * s1) / float(n * (n - 1))
