// Thread-per-trajectory kernels writing the event log, for networks with at
// most 8 species.
#define SSA_THREAD_LOG_ONLY
#include "ssa_thread_kernel.cuh"

namespace ssa_impl {

cudaError_t launch_thread_log_s8(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                  cudaStream_t st) {
  return launch_log_for_s<8>(a, lg, blocks, threads, smem, st);
}

cudaError_t set_smem_log_s8(int M, size_t smem) { return set_smem_log_for_s<8>(M, smem); }

}  // namespace ssa_impl
