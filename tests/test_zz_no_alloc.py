"""ssa_ensemble_run_noalloc: the entry point for callers that cannot allocate
device memory during a call (memory owned and pre-sized by another runtime,
plugins barred from the allocator, loops that must not block on an
allocation).  Its scratch is a fixed device array inside libssa.

Checked through the C ABI: two calls in a row (the second reuses what the
first left in the shared array) must each match ssa_ensemble_run on the same
arguments bit for bit (the tolerance the parity tests use for FP64 exact
mode), on the implicit uniform grid and on an explicit non-uniform device
grid, and the sums must equal the oracle's.  Sizes beyond the fixed scratch,
host buffers and models it does not serve must be refused.  This file is
collected last so that a failure here cannot hide the results of the other
tests.
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


def _call(fn, model, n, t_end, G, seed, bufs, opts, grid=None):
    opts.traj_hash = bufs["hash"].data_ptr()
    st = binding.RunStats()
    gp = None if grid is None else ctypes.c_void_p(grid.data_ptr())
    rc = fn(model.handle, n, t_end, G, gp, seed, ctypes.byref(opts), bufs["mean"].data_ptr(),
            bufs["var"].data_ptr(), bufs["sum1"].data_ptr(), bufs["sum2"].data_ptr(), ctypes.byref(st))
    assert rc == binding.SSA_OK, ssa.lib().ssa_last_error().decode()
    return {k: v.cpu().numpy().copy() for k, v in bufs.items()}, st


@pytest.mark.parametrize("grid_kind", ["uniform", "explicit"])
def test_noalloc_matches_ensemble_run_on_two_calls_in_a_row(grid_kind):
    torch = pytest.importorskip("torch")
    import oracle
    L = ssa.lib()
    net = W.hiv_shaped()
    n, t_end, G = 3000, 30.0, 3001
    model = ssa.Model.from_network(net)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    grid_h = None
    grid_d = None
    if grid_kind == "explicit":  # ascending, uneven spacing, denser early
        G = 777
        grid_h = t_end * (np.linspace(0.0, 1.0, G) ** 2)
        grid_d = torch.as_tensor(grid_h, device="cuda:0")
    # the library's own allocation path, for reference
    ref_bufs = _device_buffers(torch, G, net.n_species, n)
    na_bufs = _device_buffers(torch, G, net.n_species, n)
    for seed in (11, 12):
        ref_opts = ssa.make_opts(memory=binding.MEM_DEVICE, cuda_stream=stream.cuda_stream)
        ref, ref_st = _call(L.ssa_ensemble_run, model, n, t_end, G, seed, ref_bufs, ref_opts, grid_d)
        na_opts = ssa.make_opts(memory=binding.MEM_DEVICE, cuda_stream=stream.cuda_stream)
        got, got_st = _call(L.ssa_ensemble_run_noalloc, model, n, t_end, G, seed, na_bufs, na_opts, grid_d)
        for key in ("sum1", "sum2", "hash"):
            assert np.array_equal(got[key], ref[key]), key
        for key in ("mean", "var"):
            assert np.array_equal(got[key].view(np.int64), ref[key].view(np.int64)), key
        assert got_st.events == ref_st.events and got_st.max_x == ref_st.max_x
        o = oracle.run(net, n, t_end, G, seed, grid=grid_h, per_traj=True, threads=8)
        assert np.array_equal(got["sum1"], o.S1) and np.array_equal(got["sum2"], o.S2)
        assert np.array_equal(got["hash"].view(np.uint64), o.traj_hash)
        om, ov = oracle.finalize(n, o.S1, o.S2)
        assert np.array_equal(got["mean"].view(np.int64), om.view(np.int64))
        assert np.array_equal(got["var"].view(np.int64), ov.view(np.int64))
        assert got_st.events == o.events
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
    # a model with rate modifiers runs on the warp schedule only: refused with its own message
    pnet = W.paper_hiv()
    pmodel = ssa.Model.from_network(pnet)
    rc = L.ssa_ensemble_run_noalloc(pmodel.handle, 10, 1.0, 11, None, 1, ctypes.byref(opts), ctypes.c_void_p(8),
                                    ctypes.c_void_p(8), None, None, None)
    assert rc == binding.SSA_EUNSUPPORTED
    assert b"rate modifiers" in L.ssa_last_error()
    pmodel.close()
    # an out-of-range reduce mode is refused as ssa_ensemble_run refuses it
    bad = ssa.make_opts(memory=binding.MEM_DEVICE)
    bad.reduce = 7
    rc = L.ssa_ensemble_run_noalloc(model.handle, 10, 1.0, 11, None, 1, ctypes.byref(bad), ctypes.c_void_p(8),
                                    ctypes.c_void_p(8), None, None, None)
    assert rc == binding.SSA_EINVAL
    model.close()
