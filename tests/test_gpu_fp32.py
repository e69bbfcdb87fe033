"""GPU checks of the FP32-propensity mode.

(1) Parity: the warp kernel in FP32 mode against the oracle's FP32 mode
    (same schedule W32), bit for bit: int64 sums, mean, variance, event
    counts, flags and sequence hashes.
(2) Statistics: grid mean and variance of the FP32 mode within 4 standard
    errors of the FP64 oracle at every grid point and species, with the
    standard error of a difference of two means sqrt(v32/N + v64/N) and, for
    the variances, sqrt(2) times the standard error of one sample variance
    from the oracle's 4th central moments.  Cells with zero standard error
    (deterministic, e.g. t = 0) must agree exactly.  Both runs use the same
    random numbers, so most trajectories coincide.
"""
import numpy as np
import pytest

import oracle
import paper_1007_1768_gb300 as ssa
import workloads as W

pytestmark = pytest.mark.gpu

W32 = oracle.SCHEDULE_W32
FP32 = oracle.PRECISION_FP32


def _gpu(net, n, t_end, G, seed, precision="fp32", **kw):
    model = ssa.Model.from_network(net)
    try:
        r = ssa.ensemble_run(model, n, t_end, G, seed, device="cuda:0", per_traj=True, precision=precision, **kw)
    finally:
        model.close()
    import torch
    torch.cuda.synchronize()
    out = {k: getattr(r, k).cpu().numpy() for k in ("mean", "var", "sum1", "sum2", "traj_events", "traj_hash",
                                                    "traj_flags")}
    out["traj_hash"] = out["traj_hash"].view(np.uint64)
    out["stats"] = r
    return out


def _assert_same(g, r, n):
    mean, var = oracle.finalize(n, r.S1, r.S2)
    assert np.array_equal(g["traj_events"], r.traj_events)
    assert np.array_equal(g["traj_hash"], r.traj_hash)
    assert np.array_equal(g["traj_flags"], r.traj_flags)
    assert np.array_equal(g["sum1"], r.S1) and np.array_equal(g["sum2"], r.S2)
    assert np.array_equal(g["mean"].view(np.int64), mean.view(np.int64))
    assert np.array_equal(g["var"].view(np.int64), var.view(np.int64))


def test_fp32_random_32x128_bit_exact():
    w = W.workload_random(n_traj=160)
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    r = oracle.run(w.net, w.n_traj, w.t_end, w.n_grid, w.seed, per_traj=True, threads=16, schedule=W32,
                   precision=FP32)
    _assert_same(g, r, w.n_traj)


@pytest.mark.parametrize("S,M", [(4, 10), (8, 31), (12, 33), (16, 70), (40, 200), (64, 512)])
def test_fp32_chunk_widths_bit_exact(S, M):
    net = W.hiv_shaped() if M == 10 else W.random_network(600 + M, n_species=S, n_reactions=M, x0_hi=60)
    n, T = 29, (30.0 if M == 10 else 1.0)
    g = _gpu(net, n, T, 101, 3, max_events=4000)
    r = oracle.run(net, n, T, 101, 3, per_traj=True, threads=16, schedule=W32, precision=FP32, max_events=4000)
    _assert_same(g, r, n)


def test_fp32_full_size_random_sampled_ids():
    w = W.workload_random()
    g = _gpu(w.net, w.n_traj, w.t_end, w.n_grid, w.seed)
    ids = np.unique(np.linspace(0, w.n_traj - 1, 128).astype(np.int64))
    r = oracle.run(w.net, 0, w.t_end, w.n_grid, w.seed, per_traj=True, threads=16, schedule=W32, precision=FP32,
                   ids=ids)
    assert np.array_equal(g["traj_events"][ids], r.traj_events)
    assert np.array_equal(g["traj_hash"][ids], r.traj_hash)
    assert int(g["traj_events"].sum()) == g["stats"].events
    # no trajectory runs away (a zero-propensity reaction firing would drive counts negative)
    assert np.all(g["traj_flags"] == 0) and g["stats"].max_x < 2000
    assert int(g["traj_events"].max()) < 20000


def _four_se_report(m32, v32, m64, v64, s3, s4, n):
    """z of the FP32 - FP64 differences of mean and variance per cell, from
    the FP64 sample's central moments."""
    mu = m64
    mu2 = v64 * (n - 1) / n
    raw3, raw4 = s3 / n, s4 / n
    raw2 = mu2 + mu * mu
    mu4 = raw4 - 4 * mu * raw3 + 6 * mu * mu * raw2 - 3 * mu ** 4
    se_var1 = np.sqrt(np.maximum(mu4 - mu2 * mu2 * (n - 3) / (n - 1), 0.0) / n)
    se_m = np.sqrt(np.maximum(v32, 0) / n + np.maximum(v64, 0) / n)
    se_v = np.sqrt(2.0) * se_var1
    zero_m, zero_v = se_m == 0, se_v == 0
    assert np.array_equal(m32[zero_m], m64[zero_m])
    assert np.array_equal(v32[zero_v], v64[zero_v])
    zm = np.where(zero_m, 0.0, np.abs(m32 - m64) / np.where(zero_m, 1.0, se_m))
    zv = np.where(zero_v, 0.0, np.abs(v32 - v64) / np.where(zero_v, 1.0, se_v))
    return zm, zv


@pytest.mark.parametrize("workload", ["random", "hiv_shaped"])
def test_fp32_within_four_standard_errors_of_fp64_oracle(workload):
    if workload == "random":
        w = W.workload_random(n_traj=8192)
    else:
        w = W.workload_hiv_shaped(n_traj=16384)
    n = w.n_traj
    g = _gpu(w.net, n, w.t_end, w.n_grid, w.seed)
    r = oracle.run(w.net, n, w.t_end, w.n_grid, w.seed, threads=16, moments=True)
    m64, v64 = oracle.finalize(n, r.S1, r.S2)
    zm, zv = _four_se_report(g["mean"], g["var"], m64, v64, r.S3, r.S4, n)
    print(f"{workload}: cells {zm.size}, max z mean {zm.max():.3f}, max z var {zv.max():.3f}, "
          f"cells above 4 SE {(zm > 4).sum() + (zv > 4).sum()}")
    assert zm.max() < 4.0 and zv.max() < 4.0
    # same random numbers: most trajectories keep the FP64 event sequence
    assert g["stats"].events > 0
