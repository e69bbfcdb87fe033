"""ssa_ensemble_run_noalloc: the entry point for callers that cannot allocate
device memory during a call (memory owned and pre-sized by another runtime,
plugins barred from the allocator, loops that must not block on an
allocation).  Its scratch is a fixed device array inside libssa.

Checked through the C ABI: two calls in a row (the second reuses what the
first left in the shared array) must each match ssa_ensemble_run on the same
arguments bit for bit (the tolerance the parity tests use for FP64 exact
mode), and sizes beyond the fixed scratch must be refused with
SSA_EINVAL.  This file is collected last so that a failure here cannot hide
the results of the other tests.
"""
import ctypes

import numpy as np
import pytest

import paper_1007_1768_gb300 as ssa
import workloads as W
from paper_1007_1768_gb300 import binding

pytestmark = pytest.mark.gpu


def _device_buffers(torch, G, S, N):
    dev = torch.device("cuda", 0)
    return {
        "mean": torch.empty((G, S), dtype=torch.float64, device=dev),
        "var": torch.empty((G, S), dtype=torch.float64, device=dev),
        "sum1": torch.empty((G, S), dtype=torch.int64, device=dev),
        "sum2": torch.empty((G, S), dtype=torch.int64, device=dev),
        "hash": torch.empty(N, dtype=torch.int64, device=dev),
    }


def _call(fn, model, n, t_end, G, seed, bufs, opts):
    opts.traj_hash = bufs["hash"].data_ptr()
    st = binding.RunStats()
    rc = fn(model.handle, n, t_end, G, None, seed, ctypes.byref(opts), bufs["mean"].data_ptr(),
            bufs["var"].data_ptr(), bufs["sum1"].data_ptr(), bufs["sum2"].data_ptr(), ctypes.byref(st))
    assert rc == binding.SSA_OK, ssa.lib().ssa_last_error().decode()
    return {k: v.cpu().numpy().copy() for k, v in bufs.items()}, st


def test_noalloc_matches_ensemble_run_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    L = ssa.lib()
    net = W.hiv_shaped()
    n, t_end, G = 3000, 30.0, 3001
    model = ssa.Model.from_network(net)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    # the library's own allocation path, for reference
    ref_bufs = _device_buffers(torch, G, net.n_species, n)
    na_bufs = _device_buffers(torch, G, net.n_species, n)
    for seed in (11, 12):
        ref_opts = ssa.make_opts(memory=binding.MEM_DEVICE, cuda_stream=stream.cuda_stream)
        ref, ref_st = _call(L.ssa_ensemble_run, model, n, t_end, G, seed, ref_bufs, ref_opts)
        na_opts = ssa.make_opts(memory=binding.MEM_DEVICE, cuda_stream=stream.cuda_stream)
        got, got_st = _call(L.ssa_ensemble_run_noalloc, model, n, t_end, G, seed, na_bufs, na_opts)
        for key in ("sum1", "sum2", "hash"):
            assert np.array_equal(got[key], ref[key]), key
        for key in ("mean", "var"):
            assert np.array_equal(got[key].view(np.int64), ref[key].view(np.int64)), key
        assert got_st.events == ref_st.events and got_st.max_x == ref_st.max_x
    model.close()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    L = ssa.lib()
    net = W.hiv_shaped()
    model = ssa.Model.from_network(net)
    opts = ssa.make_opts(memory=binding.MEM_DEVICE)
    G = 200000  # 16 * G * 4 species bytes > 4 MiB
    rc = L.ssa_ensemble_run_noalloc(model.handle, 10, 1.0, G, None, 1, ctypes.byref(opts), ctypes.c_void_p(8),
                                    ctypes.c_void_p(8), None, None, None)
    assert rc == binding.SSA_EINVAL
    assert b"SSA_NOALLOC_SCRATCH_BYTES" in L.ssa_last_error()
    host = ssa.make_opts(memory=binding.MEM_HOST)
    rc = L.ssa_ensemble_run_noalloc(model.handle, 10, 1.0, 11, None, 1, ctypes.byref(host), ctypes.c_void_p(8),
                                    ctypes.c_void_p(8), None, None, None)
    assert rc == binding.SSA_EINVAL
    model.close()
