// Thread-per-trajectory kernels for networks with at most 8 species.
#include "ssa_thread_kernel.cuh"

namespace ssa_impl {

cudaError_t launch_thread_s8(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st) {
  return launch_for_s<8>(a, blocks, threads, shared_d, smem, st);
}

cudaError_t set_smem_s8(int M, bool shared_d, size_t smem) { return set_smem_for_s<8>(M, shared_d, smem); }

}  // namespace ssa_impl
