// Thread-per-trajectory kernels for networks with at most 4 species.
#include "ssa_thread_kernel.cuh"

namespace ssa_impl {

cudaError_t launch_thread_s4(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st) {
  return launch_for_s<4>(a, blocks, threads, shared_d, smem, st);
}

cudaError_t set_smem_s4(int M, bool shared_d, size_t smem) { return set_smem_for_s<4>(M, shared_d, smem); }

}  // namespace ssa_impl
