"""GPU parity: libssa's CUDA path against the oracle, through the C ABI.

FP64 exact mode must agree bit for bit: int64 grid sums S1 / S2, mean and
variance (same finalisation formula), per-trajectory event counts, flags
and event-sequence hashes.  Cases span several CTAs and ragged tails, both
reduction placements, several launch shapes, explicit grids, shards, and the
degenerate cases (one trajectory, one grid point, absorbing states,
truncation, overflow).
"""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu

FNV_OFFSET = 0xCBF29CE484222325


def _gpu(net, n, t_end, G, seed, device=True, **kw):
    model = ssa.Model.from_network(net)
    try:
        r = ssa.ensemble_run(model, n, t_end, G, seed, device="cuda:0" if device else None, per_traj=True, **kw)
    finally:
        model.close()
    if device:
        import torch
        torch.cuda.synchronize()
        out = {k: getattr(r, k).cpu().numpy() for k in ("mean", "var", "sum1", "sum2", "traj_events", "traj_hash",
                                                        "traj_flags")}
        out["traj_hash"] = out["traj_hash"].view(np.uint64)
    else:
        out = {k: getattr(r, k) for k in ("mean", "var", "sum1", "sum2", "traj_events", "traj_hash", "traj_flags")}
    out["stats"] = r
    return out


def _oracle(net, n, t_end, G, seed, grid=None, threads=8, **kw):
    r = oracle.run(net, n, t_end, G, seed, grid=grid, per_traj=True, threads=threads, **kw)
    mean, var = oracle.finalize(n, r.S1, r.S2)
    return r, mean, var


def _assert_same(g, r, mean, var):
    assert np.array_equal(g["sum1"], r.S1)
    assert np.array_equal(g["sum2"], r.S2)
    assert np.array_equal(g["mean"].view(np.int64), mean.view(np.int64))
    assert np.array_equal(g["var"].view(np.int64), var.view(np.int64))
    assert np.array_equal(g["traj_events"], r.traj_events)
    assert np.array_equal(g["traj_hash"], r.traj_hash)
    assert np.array_equal(g["traj_flags"], r.traj_flags)
    assert g["stats"].events == r.events


@pytest.mark.parametrize("device", [True, False])
def test_birth_death_full_bit_exact(device):
    w = W.workload_birth_death()
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed, device=device)
    r, mean, var = _oracle(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    _assert_same(g, r, mean, var)


def test_hiv_shaped_bit_exact_several_ctas_ragged():
    net = W.hiv_shaped()
    n = 3 * 152 + 77  # ragged against any block size
    g = _gpu(net, n, 30.0, 3001, 5, block_threads=64)
    r, mean, var = _oracle(net, n, 30.0, 3001, 5)
    _assert_same(g, r, mean, var)


@pytest.mark.parametrize("reduce,threads", [("shared", 128), ("global", 96), ("global", 512), ("auto", 0)])
def test_launch_shape_and_reduction_placement_do_not_change_results(reduce, threads):
    net = W.hiv_shaped()
    n = 2000
    g = _gpu(net, n, 30.0, 601, 11, reduce=reduce, block_threads=threads)
    r, mean, var = _oracle(net, n, 30.0, 601, 11)
    _assert_same(g, r, mean, var)


def test_hiv_shaped_full_size_bench_configuration():
    """The benchmark's workload (65,536 trajectories, 3001 grid points) in the
    launch configuration bench.py times, against the full oracle.  Warps hand
    trajectories to one another in that configuration."""
    w = W.workload_hiv_shaped()
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    r, mean, var = _oracle(w.net, w.n_traj, w.t_end, w.n_grid, w.seed, threads=16)
    _assert_same(g, r, mean, var)
    assert r.truncated == 0 and r.overflowed == 0
    assert g["stats"].handoffs > 0


def test_handoff_with_more_ctas_than_fit_at_once():
    """A grid larger than one wave: CTAs that start after the first ones have
    finished find the work counter empty and join the hand-off pool late (or
    find it closed); every trajectory still ends once, equal to the oracle."""
    net = W.hiv_shaped()
    g = _gpu(net, 4000, 30.0, 601, 24, block_threads=64, grid_blocks=2000)
    r, mean, var = _oracle(net, 4000, 30.0, 601, 24, threads=16)
    _assert_same(g, r, mean, var)


@pytest.mark.parametrize("n,seed,threads", [(16384, 21, 0), (4000, 22, 64), (9000, 23, 512)])
def test_trajectories_handed_between_warps_stay_bit_exact(n, seed, threads):
    """Heavy-tailed trajectory lengths leave warps idle while others still
    run several trajectories; the idle warps take handed-off trajectories
    (counted in the run's stats) and every per-trajectory result, grid sum
    and moment stays equal to the oracle's."""
    net = W.hiv_shaped()
    g = _gpu(net, n, 30.0, 3001, seed, block_threads=threads)
    r, mean, var = _oracle(net, n, 30.0, 3001, seed, threads=16)
    _assert_same(g, r, mean, var)
    assert g["stats"].handoffs > 0


@pytest.mark.parametrize("case", range(3))
def test_tiny_networks_bit_exact(case):
    net, T = W.tiny_networks()[case]
    g = _gpu(net, 3000, T, 41, 100 + case)
    r, mean, var = _oracle(net, 3000, T, 41, 100 + case)
    _assert_same(g, r, mean, var)


@pytest.mark.parametrize("M", [1, 3, 7, 12, 16])
def test_random_small_networks_bit_exact(M):
    net = W.random_network(77 + M, n_species=6, n_reactions=M, x0_hi=40)
    g = _gpu(net, 700, 2.0, 201, 3, max_events=20000)
    r, mean, var = _oracle(net, 700, 2.0, 201, 3, max_events=20000)
    _assert_same(g, r, mean, var)


def test_explicit_nonuniform_grid_with_event_times():
    net = W.hiv_shaped()
    rt, _, _, _, _ = oracle.trace(net, 0, 30.0, 2, seed=9)
    grid = np.unique(np.concatenate([[0.0], rt[:40], np.linspace(0.5, 30.0, 50)]))
    for device in (True, False):
        g = _gpu(net, 300, 30.0, len(grid), 9, device=device, grid=grid)
        r, mean, var = _oracle(net, 300, 30.0, len(grid), 9, grid=grid)
        _assert_same(g, r, mean, var)


def test_shards_by_offset_add_up():
    net = W.hiv_shaped()
    a = _gpu(net, 700, 30.0, 301, 4, traj_offset=0)
    b = _gpu(net, 500, 30.0, 301, 4, traj_offset=700)
    full = _gpu(net, 1200, 30.0, 301, 4)
    assert np.array_equal(a["sum1"] + b["sum1"], full["sum1"])
    assert np.array_equal(a["sum2"] + b["sum2"], full["sum2"])
    assert np.array_equal(np.concatenate([a["traj_hash"], b["traj_hash"]]), full["traj_hash"])
    r = oracle.run(net, 500, 30.0, 301, 4, traj_begin=700, per_traj=True)
    assert np.array_equal(b["sum1"], r.S1) and np.array_equal(b["traj_hash"], r.traj_hash)


def test_stream_id_changes_the_stream_and_matches_oracle():
    net = W.hiv_shaped()
    g = _gpu(net, 400, 30.0, 101, 4, stream_id=9)
    r, mean, var = _oracle(net, 400, 30.0, 101, 4, stream=9)
    _assert_same(g, r, mean, var)
    g0 = _gpu(net, 400, 30.0, 101, 4)
    assert not np.array_equal(g0["traj_hash"], g["traj_hash"])


def test_single_trajectory_and_single_grid_point():
    net = W.hiv_shaped()
    g = _gpu(net, 1, 30.0, 1, 2)
    r, mean, var = _oracle(net, 1, 30.0, 1, 2)
    _assert_same(g, r, mean, var)
    assert np.isnan(g["var"]).all()


def test_truncation_absorbing_and_no_event_cases():
    net = W.hiv_shaped()
    g = _gpu(net, 333, 30.0, 301, 1, max_events=7)
    r, mean, var = _oracle(net, 333, 30.0, 301, 1, max_events=7)
    _assert_same(g, r, mean, var)
    assert g["stats"].truncated == 333 and np.all(g["traj_flags"] == ssa.binding.TRAJ_TRUNCATED)
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32), np.array([2.0]),
                      np.array([5], np.int32))
    g = _gpu(death, 257, 50.0, 51, 3)
    r, mean, var = _oracle(death, 257, 50.0, 51, 3)
    _assert_same(g, r, mean, var)
    # an empty network state with only zero rates: no events at all
    idle = W.Network("idle", ["X"], np.array([[1]], np.int32), np.array([[2]], np.int32), np.array([0.0]),
                     np.array([4], np.int32))
    g = _gpu(idle, 65, 1.0, 5, 3)
    assert np.all(g["traj_events"] == 0) and np.all(g["sum1"] == 65 * 4)
    assert np.all(g["traj_hash"] == np.uint64(FNV_OFFSET))


def test_overflow_is_reported():
    net = W.Network("grow", ["X"], np.array([[0]], np.int32), np.array([[1]], np.int32), np.array([1.0]),
                    np.array([2147483645], np.int32))
    with pytest.raises(ssa.SSAError) as e:
        _gpu(net, 3, 100.0, 3, 1, device=False)
    assert e.value.status == ssa.binding.SSA_EOVERFLOW


def test_repeatable_and_seed_sensitive():
    net = W.hiv_shaped()
    a = _gpu(net, 1000, 30.0, 301, 7)
    b = _gpu(net, 1000, 30.0, 301, 7)
    c = _gpu(net, 1000, 30.0, 301, 8)
    assert np.array_equal(a["sum2"], b["sum2"]) and np.array_equal(a["traj_hash"], b["traj_hash"])
    assert not np.array_equal(a["sum2"], c["sum2"])


def test_shards_finalised_on_the_host_match_one_run():
    from paper_1007_1768_gb300.shards import finalize_sums, shard_range
    net = W.hiv_shaped()
    n, world = 3001, 3
    s1 = s2 = 0
    for rank in range(world):
        off, cnt = shard_range(n, rank, world)
        g = _gpu(net, cnt, 30.0, 301, 12, device=False, traj_offset=off)
        s1, s2 = s1 + g["sum1"], s2 + g["sum2"]
    full = _gpu(net, n, 30.0, 301, 12, device=False)
    assert np.array_equal(s1, full["sum1"]) and np.array_equal(s2, full["sum2"])
    mean, var = finalize_sums(s1, s2, n)
    assert np.array_equal(mean.view(np.int64), full["mean"].view(np.int64))
    assert np.array_equal(var.view(np.int64), full["var"].view(np.int64))


def test_cooperative_batches_ending_inside_a_batch():
    """A warp holding at most 4 trajectories runs them cooperatively, 8 events
    per batch, from the first event (1, 3 or 4 trajectories here): truncation
    at max_events, an absorbing state and the int32 overflow land at various
    places inside a batch, and the later events of that batch are undone."""
    net = W.hiv_shaped()
    for n in (1, 3, 4):
        for me in (1, 8, 13, 21, 100):
            g = _gpu(net, n, 30.0, 301, 5, max_events=me)
            r, mean, var = _oracle(net, n, 30.0, 301, 5, max_events=me)
            _assert_same(g, r, mean, var)
    death = W.Network("death", ["X"], np.array([[1]], np.int32), np.array([[0]], np.int32), np.array([2.0]),
                      np.array([11], np.int32))
    g = _gpu(death, 3, 50.0, 51, 3)
    r, mean, var = _oracle(death, 3, 50.0, 51, 3)
    _assert_same(g, r, mean, var)
    assert np.all(g["traj_events"] == 11)
    # births from 2^31 - 1 - 20: the 21st would leave int32 (device buffers,
    # no stats: the call does not wait, so no status for the overflow; two
    # trajectories keep the sums of x^2 inside int64)
    grow = W.Network("grow", ["X"], np.array([[0]], np.int32), np.array([[1]], np.int32), np.array([5.0]),
                     np.array([2147483647 - 20], np.int32))
    g = _gpu(grow, 2, 100.0, 11, 4, stats=False)
    r, mean, var = _oracle(grow, 2, 100.0, 11, 4)
    for key, want in (("sum1", r.S1), ("sum2", r.S2), ("traj_events", r.traj_events), ("traj_hash", r.traj_hash),
                      ("traj_flags", r.traj_flags)):
        assert np.array_equal(g[key], want), key
    assert np.all(r.traj_events == 20) and np.all(r.traj_flags == ssa.binding.TRAJ_OVERFLOW)


def test_explicit_uniform_grid_takes_the_same_path():
    """A host grid equal to the uniform grid bit for bit locates grid cells by
    the uniform estimate; the results are those of the implicit grid and of
    the oracle with the explicit grid (and a grid off by one ulp at one point
    still matches the oracle through the general path)."""
    net = W.hiv_shaped()
    grid = (np.arange(301, dtype=np.float64) * 30.0) / 300.0
    a = _gpu(net, 600, 30.0, 301, 3)
    b = _gpu(net, 600, 30.0, 0, 3, grid=grid, device=False)
    for key in ("sum1", "sum2", "traj_hash", "traj_events"):
        assert np.array_equal(a[key], b[key]), key
    r, mean, var = _oracle(net, 600, 30.0, 0, 3, grid=grid)
    _assert_same(b, r, mean, var)
    g2 = grid.copy()
    g2[150] = np.nextafter(g2[150], 0.0)
    c = _gpu(net, 600, 30.0, 0, 3, grid=g2, device=False)
    r2, mean2, var2 = _oracle(net, 600, 30.0, 0, 3, grid=g2)
    _assert_same(c, r2, mean2, var2)


@pytest.mark.parametrize("n", [3, 200, 1000])
def test_wide_small_network_thread_kernel(n):
    """The thread kernel's widest template bucket (12 species, 15 reactions
    run as 16 x 16), with cooperative mode from the first event (3
    trajectories) and at the end of a fuller launch."""
    net = W.random_network(21, n_species=12, n_reactions=15, x0_hi=30)
    g = _gpu(net, n, 3.0, 31, 9, schedule="thread", max_events=200000)
    r, mean, var = _oracle(net, n, 3.0, 31, 9, max_events=200000)
    _assert_same(g, r, mean, var)
