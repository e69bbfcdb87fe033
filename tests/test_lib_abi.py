"""C-ABI checks that need no GPU: libssa loads, exports every function that
include/ssa.h declares, rejects bad models with SSA_EINVAL and a message, and
the ctypes structs match the C layout (checked by compiling a probe of the
header with the host compiler)."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_1007_1768_gb300 as ssa
from paper_1007_1768_gb300 import binding
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ssa.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ssa_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_and_binding_list_agree():
    assert sorted(binding.EXPORTS) == _declared_functions()


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(ssa.library_path() if os.path.exists(ssa.library_path()) else ssa.lib()._name)
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_status_strings_and_defaults():
    L = ssa.lib()
    assert L.ssa_status_string(0) == b"ok"
    assert L.ssa_status_string(1) == b"invalid argument"
    o = binding.RunOpts()
    L.ssa_run_opts_init(ctypes.byref(o))
    assert o.precision == 0 and o.schedule == 0 and o.memory == 0 and o.max_events == 100000000
    assert o.workspace is None and o.cuda_stream is None


def _create(R, P, c, x0):
    L = ssa.lib()
    R = np.ascontiguousarray(R, np.int32)
    P = np.ascontiguousarray(P, np.int32)
    c = np.ascontiguousarray(c, np.float64)
    x0 = np.ascontiguousarray(x0, np.int32)
    h = ctypes.c_void_p()
    st = L.ssa_model_create(R.shape[1], R.shape[0], R.ctypes.data, P.ctypes.data, c.ctypes.data, x0.ctypes.data,
                            ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("R,P,c,x0", [
    ([[3]], [[0]], [1.0], [1]),                 # multiplicity > 2
    ([[1, 2]], [[0, 0]], [1.0], [1, 1]),        # order 3
    ([[1]], [[-1]], [1.0], [1]),                # negative product
    ([[1]], [[0]], [-1.0], [1]),                # negative rate
    ([[1]], [[0]], [float("nan")], [1]),        # NaN rate
    ([[1]], [[0]], [float("inf")], [1]),        # infinite rate
    ([[1]], [[0]], [1.0], [-5]),                # negative initial count
])
def test_model_create_rejects_bad_models(R, P, c, x0):
    st, h = _create(R, P, c, x0)
    assert st == binding.SSA_EINVAL and not h.value
    assert len(ssa.lib().ssa_last_error()) > 0


def test_model_create_and_info():
    L = ssa.lib()
    st, h = _create([[0], [1]], [[1], [0]], [10.0, 0.1], [0])
    assert st == 0 and h.value
    S, M = ctypes.c_int32(), ctypes.c_int32()
    assert L.ssa_model_info(h, ctypes.byref(S), ctypes.byref(M)) == 0
    assert (S.value, M.value) == (1, 2)
    nbytes = ctypes.c_size_t()
    o = binding.RunOpts()
    L.ssa_run_opts_init(ctypes.byref(o))
    assert L.ssa_ensemble_workspace_size(h, 1000, 1001, ctypes.byref(o), ctypes.byref(nbytes)) == 0
    assert nbytes.value >= 2 * 1001 * 8
    L.ssa_model_destroy(h)
    L.ssa_model_destroy(None)


def test_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "ssa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ssa_run_opts), offsetof(ssa_run_opts, max_events),
         offsetof(ssa_run_opts, cuda_stream), offsetof(ssa_run_opts, workspace_bytes),
         offsetof(ssa_run_opts, traj_flags), sizeof(ssa_run_stats), offsetof(ssa_run_stats, kernel_ms),
         offsetof(ssa_run_stats, schedule), offsetof(ssa_run_stats, handoffs));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + os.path.dirname(HEADER), "-o", exe, c], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    R, S = binding.RunOpts, binding.RunStats
    assert vals == [ctypes.sizeof(R), R.max_events.offset, R.cuda_stream.offset, R.workspace_bytes.offset,
                    R.traj_flags.offset, ctypes.sizeof(S), S.kernel_ms.offset, S.schedule.offset,
                    S.handoffs.offset]


def test_host_run_rejects_bad_arguments_before_touching_the_gpu():
    net_R, net_P = [[0], [1]], [[1], [0]]
    model = ssa.Model(net_R, net_P, [10.0, 0.1], [0])
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(model, 0, 10.0, 11, seed=1)
    assert e.value.status == binding.SSA_EINVAL
    with pytest.raises(ssa.SSAError):
        ssa.ensemble_run(model, 10, -1.0, 11, seed=1)
    with pytest.raises(ssa.SSAError):
        ssa.ensemble_run(model, 10, 10.0, 3, seed=1, grid=[0.0, 5.0, 4.0])
    with pytest.raises(ssa.SSAError):
        ssa.ensemble_run(model, 10, 10.0, 2, seed=1, grid=[0.0, 11.0])
    with pytest.raises(ssa.SSAError):
        ssa.ensemble_run(model, 10, 10.0, 11, seed=1, block_threads=48)
    model.close()


def test_schedule_limits_are_refused_before_touching_the_gpu():
    import workloads as W
    big = ssa.Model.from_network(W.random_network(3))  # 32 species, 128 reactions
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(big, 10, 1.0, 11, seed=1, schedule="thread")
    assert e.value.status == binding.SSA_EUNSUPPORTED and "thread schedule" in str(e.value)
    big.close()
    huge = ssa.Model.from_network(W.random_network(4, n_species=8, n_reactions=513))
    for sched in ("auto", "warp"):
        with pytest.raises(ssa.SSAError) as e:
            ssa.ensemble_run(huge, 10, 1.0, 11, seed=1, schedule=sched)
        assert e.value.status == binding.SSA_EUNSUPPORTED and "512" in str(e.value)
    huge.close()


def test_fp32_mode_limits_are_refused_before_touching_the_gpu():
    net_R, net_P = [[0], [1]], [[1], [0]]
    model = ssa.Model(net_R, net_P, [10.0, 0.1], [0])
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(model, 10, 1.0, 11, seed=1, precision="fp32", schedule="thread")
    assert e.value.status == binding.SSA_EUNSUPPORTED and "warp schedule" in str(e.value)
    model.close()
    model = ssa.Model(net_R, net_P, [1e39, 0.1], [0])
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(model, 10, 1.0, 11, seed=1, precision="fp32")
    assert e.value.status == binding.SSA_EINVAL and "binary32" in str(e.value)
    model.close()


def test_batch_arguments_are_refused_before_touching_the_gpu():
    net_R, net_P = [[0], [1]], [[1], [0]]
    m = ssa.Model(net_R, net_P, [10.0, 0.1], [0])
    with pytest.raises(ssa.SSAError) as e:
        ssa.Batch([m, m], [10, 10], [1.0, 1.0], [11, 11], stream_id=(1 << 32) - 1)
    assert e.value.status == binding.SSA_EINVAL
    # the thread schedule takes FP64 networks of at most 16 reactions and species only
    with pytest.raises(ssa.SSAError) as e:
        ssa.Batch([m], [10], [1.0], [11], schedule="thread", precision="fp32")
    assert e.value.status == binding.SSA_EUNSUPPORTED
    big = ssa.Model.from_network(W.random_network(5, n_species=8, n_reactions=20))
    with pytest.raises(ssa.SSAError) as e:
        ssa.Batch([m, big], [10, 10], [1.0, 1.0], [11, 11], schedule="thread")
    assert e.value.status == binding.SSA_EUNSUPPORTED
    big.close()
    bad = ssa.make_opts()
    bad.schedule = 7
    hp = binding._ptr_array([m.handle.value])
    n, te, g = np.array([10], np.int64), np.array([1.0]), np.array([11], np.int32)
    h = ctypes.c_void_p()
    assert ssa.lib().ssa_batch_create(1, hp, n.ctypes.data, te.ctypes.data, g.ctypes.data, None, ctypes.byref(bad),
                                      ctypes.byref(h)) == binding.SSA_EINVAL
    with pytest.raises(ssa.SSAError) as e:
        ssa.Batch([m], [0], [1.0], [11])
    assert e.value.status == binding.SSA_EINVAL
    with pytest.raises(ssa.SSAError) as e:
        ssa.Batch([m], [10], [1.0], [11], block_threads=96)
    assert e.value.status == binding.SSA_EINVAL
    m.close()


def test_rate_modifier_arguments_are_checked_before_touching_the_gpu():
    m = ssa.Model([[1, 0]], [[0, 0]], [0.5], [4, 3])
    for args in [(1, 1, 0.1, 0.0, 1.0), (0, 2, 0.1, 0.0, 1.0), (0, 1, float("nan"), 0.0, 1.0),
                 (0, 1, 0.1, -1.0, 1.0), (0, 1, 0.1, 2.0, 1.0)]:
        with pytest.raises(ssa.SSAError) as e:
            m.set_rate_modifier(*args)
        assert e.value.status == binding.SSA_EINVAL, args
    m.set_rate_modifier(0, 1, 0.1, 0.0, float("inf"))
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(m, 10, 1.0, 3, seed=1, schedule="thread")
    assert e.value.status == binding.SSA_EUNSUPPORTED and "modifier" in str(e.value)
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run(m, 10, 1.0, 3, seed=1, precision="fp32")
    assert e.value.status == binding.SSA_EUNSUPPORTED
    m.set_rate_modifier(0, -1, 0.0, 0.0, 0.0)  # removed again
    m.close()


def test_finalize_sums_on_the_host_equals_the_oracle():
    """ssa_finalize_sums (host, no GPU) against the oracle's finalisation,
    bit for bit, on sums of real ensembles and on hand-built extremes (sums
    whose 128-bit numerator needs more than 64 bits, N = 1 and N = 2)."""
    import oracle
    import workloads as W
    from paper_1007_1768_gb300.shards import finalize_sums
    r = oracle.run(W.hiv_shaped(), 301, 30.0, 101, 9)
    for n, s1, s2 in [(301, r.S1, r.S2)]:
        mean, var = finalize_sums(s1, s2, n)
        om, ov = oracle.finalize(n, s1, s2)
        assert np.array_equal(mean.view(np.int64), om.view(np.int64))
        assert np.array_equal(var.view(np.int64), ov.view(np.int64))
    rng = np.random.default_rng(5)
    n = 3_000_000_000  # N * sum2 needs about 125 bits
    x = rng.integers(0, 2**31 - 1, size=(7, 3), dtype=np.int64)
    s1 = x * 40
    s2 = (x // 2**16) * (x // 2**16) * 2**20 + rng.integers(0, 2**40, size=(7, 3), dtype=np.int64)
    for nn in (n, 2, 1):
        mean, var = finalize_sums(s1, s2, nn)
        om, ov = oracle.finalize(nn, s1, s2)
        assert np.array_equal(mean.view(np.int64), om.view(np.int64))
        assert np.array_equal(np.isnan(var), np.isnan(ov))
        assert np.array_equal(var[~np.isnan(var)].view(np.int64), ov[~np.isnan(ov)].view(np.int64))
    L = ssa.lib()
    d = np.zeros((2, 2))
    z = np.zeros((2, 2), dtype=np.int64)
    assert L.ssa_finalize_sums(0, 2, 2, z.ctypes.data, z.ctypes.data, d.ctypes.data, d.ctypes.data) == \
        binding.SSA_EINVAL
    assert L.ssa_finalize_sums(5, 2, 2, None, z.ctypes.data, d.ctypes.data, d.ctypes.data) == binding.SSA_EINVAL
