"""Host-side helpers for running one ensemble as shards (one process per
GPU, or several runs on one GPU): contiguous trajectory-id ranges, and the
finalisation of int64 sums added across shards.

Trajectory i is fixed by (seed, id, stream id) alone, so shards that cover
[0, N) with ssa_ensemble_run(traj_offset=offset, n_traj=count) add up to the
int64 sums of one run of N trajectories, bit for bit, in any order.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_traj: int, rank: int, world: int):
    """(traj_offset, count) of shard `rank` of `world`: contiguous ranges whose
    sizes differ by at most one, covering [0, n_traj) in rank order."""
    if world < 1 or not (0 <= rank < world) or n_traj < world:
        raise ValueError("need 0 <= rank < world <= n_traj")
    base, extra = divmod(n_traj, world)
    offset = rank * base + min(rank, extra)
    return offset, base + (1 if rank < extra else 0)


def finalize_sums(sum1, sum2, n_traj: int):
    """mean = sum1 / N and var = (N sum2 - sum1^2) / (N (N - 1)) from int64 sums,
    with the numerator formed exactly (Python integers) and rounded once --
    the same values the library's finalisation kernel writes."""
    s1 = np.asarray(sum1, dtype=np.int64)
    s2 = np.asarray(sum2, dtype=np.int64)
    mean = s1.astype(np.float64) / float(n_traj)
    var = np.empty(s1.shape, dtype=np.float64)
    if n_traj < 2:
        var[...] = np.nan
        return mean, var
    den = float(n_traj) * float(n_traj - 1)
    flat1, flat2, out = s1.ravel(), s2.ravel(), var.ravel()
    for q in range(flat1.size):
        a, b = int(flat1[q]), int(flat2[q])
        out[q] = float(n_traj * b - a * a) / den
    return mean, var
