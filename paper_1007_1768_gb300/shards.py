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
    """mean = sum1 / N and var = (N sum2 - sum1^2) / (N (N - 1)) from int64 sums
    added across shards: libssa's ssa_finalize_sums (exact 128-bit numerator,
    one rounding), the same values the device finalisation writes."""
    from . import binding
    s1 = np.ascontiguousarray(sum1, dtype=np.int64)
    s2 = np.ascontiguousarray(sum2, dtype=np.int64)
    if s1.shape != s2.shape or s1.ndim != 2:
        raise ValueError("sum1 and sum2 must be [n_grid, n_species] arrays of one shape")
    mean = np.empty(s1.shape, dtype=np.float64)
    var = np.empty(s1.shape, dtype=np.float64)
    binding._check(binding.lib().ssa_finalize_sums(int(n_traj), s1.shape[0], s1.shape[1], s1.ctypes.data,
                                                   s2.ctypes.data, mean.ctypes.data, var.ctypes.data))
    return mean, var
