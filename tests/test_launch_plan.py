"""Launch planning of the thread kernel (host logic, compiled for the CPU).

plan_thread_launch picks threads per CTA from the trajectories per SM and the
CTA count from the work, and, with the hand-off between warps, takes full
512-thread CTAs beyond 256 trajectories per SM and at least one CTA per SM so
that warps without a trajectory wait for handed-off ones from the start;
explicit shapes are kept.  The probe prints one plan per argument list."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

PROBE = r"""
#include <cstdio>
#include <cstdlib>
#include "ssa_internal.h"
int main(int argc, char** argv) {
  // S M G N sms smem_optin reduce block_threads grid_blocks handoff
  ssa_impl::LaunchPlan p{};
  const char* msg = ssa_impl::plan_thread_launch(atoi(argv[1]), atoi(argv[2]), atoi(argv[3]), atoll(argv[4]),
                                                 atoi(argv[5]), (size_t)atoll(argv[6]), atoi(argv[7]),
                                                 atoi(argv[8]), atoi(argv[9]), &p, atoi(argv[10]) != 0);
  if (msg) { printf("err %s\n", msg); return 0; }
  printf("ok %d %d %d %zu\n", p.threads, p.blocks, (int)p.shared_d, p.smem);
  return 0;
}
"""


@pytest.fixture(scope="module")
def probe():
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not found")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "plan.cpp")
    exe = os.path.join(d, "plan")
    open(src, "w").write(PROBE)
    subprocess.run(["g++", "-std=c++17", "-I", CUDA_INC, "-I", os.path.join(ROOT, "paper_1007_1768_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)

    def plan(N, S=4, M=10, G=3001, sms=152, smem=232448, reduce=0, bt=0, gb=0, handoff=True):
        out = subprocess.run([exe, str(S), str(M), str(G), str(N), str(sms), str(smem), str(reduce), str(bt), str(gb),
                              str(int(handoff))], capture_output=True, text=True, check=True).stdout.split()
        if out[0] == "err":
            return "err"
        return int(out[1]), int(out[2]), int(out[3])
    return plan


def test_bench_workload_takes_full_ctas_on_every_sm(probe):
    assert probe(65536) == (512, 152, 0)           # 384 warps start without a trajectory
    assert probe(65536, handoff=False) == (448, 147, 0)


def test_small_ensembles_spread_over_every_sm(probe):
    assert probe(1000) == (64, 152, 0)
    assert probe(1000, handoff=False) == (64, 16, 0)


def test_large_ensembles_stay_persistent(probe):
    threads, blocks, _ = probe(1 << 20)
    assert threads == 512 and blocks >= 152 and blocks * threads < (1 << 20)


def test_explicit_shapes_are_kept(probe):
    assert probe(1000, bt=128) == (128, 8, 0)      # no raise to one CTA per SM
    assert probe(4000, bt=64, gb=2000) == (64, 2000, 0)
    assert probe(65536, bt=256, gb=10) == (256, 10, 0)


@pytest.mark.parametrize("N", [1, 31, 32, 500, 9000, 38912, 38913, 77824, 300000])
def test_default_shapes_are_valid(probe, N):
    threads, blocks, _ = probe(N)
    assert threads % 32 == 0 and 64 <= threads <= 512
    assert blocks >= 152                            # hand-off: every SM has a CTA
    assert threads == 512 or N <= 256 * 152


def test_shared_reduction_that_does_not_fit_is_refused(probe):
    assert probe(1000, G=100000, reduce=1) == "err"
    threads, blocks, shared = probe(1000, G=101, reduce=1)
    assert shared == 1
