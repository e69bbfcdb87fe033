"""The sharded path on CPU ranks (gloo, world size 2): each rank runs its
contiguous id range (the oracle stands in for the GPU, which this host does
not have), the int64 sums are added with an all-reduce, and the result must
equal one full run bit for bit; the host finalisation must equal the
oracle's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_1007_1768_gb300.shards import finalize_sums, shard_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, out_path):
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = W.hiv_shaped()
    off, cnt = shard_range(n, rank, world)
    r = oracle.run(net, cnt, 30.0, 301, 7, traj_begin=off)
    s = torch.from_numpy(np.stack([r.S1, r.S2]))
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, s.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_the_ids():
    for n, world in [(10, 3), (1000, 7), (65536, 8), (5, 5)]:
        ranges = [shard_range(n, r, world) for r in range(world)]
        assert ranges[0][0] == 0
        for (o1, c1), (o2, _) in zip(ranges, ranges[1:]):
            assert o1 + c1 == o2
        assert sum(c for _, c in ranges) == n
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard_range(3, 0, 4)


def test_two_gloo_ranks_add_up_to_one_run(tmp_path):
    n = 601
    out = str(tmp_path / "sums.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), n, out), nprocs=2, start_method="spawn", join=True)
    s = np.load(out)
    full = oracle.run(W.hiv_shaped(), n, 30.0, 301, 7)
    assert np.array_equal(s[0], full.S1) and np.array_equal(s[1], full.S2)
    mean, var = finalize_sums(s[0], s[1], n)
    om, ov = oracle.finalize(n, full.S1, full.S2)
    assert np.array_equal(mean.view(np.int64), om.view(np.int64))
    assert np.array_equal(var.view(np.int64), ov.view(np.int64))
