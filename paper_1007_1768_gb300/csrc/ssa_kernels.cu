// Reduction and support kernels, and the dispatch of the simulation kernel
// (ssa_thread_kernel.cuh, instantiated in ssa_thread_s{4,8,16}.cu).
//
//   Selective memory (Sec. 3.2.1) is done without storing any trajectory:
//   the grid state of a trajectory is x0 plus the changes of all events with
//   time <= g_k, so the per-grid sums are
//       sum1[k] = N x0 + sum_{k' <= k} D1[k'],   sum2[k] = N x0^2 + sum_{k' <= k} D2[k'],
//   where an event at time t with change v of species s adds v to D1 and
//   (2 x + v) v to D2 at k' = first grid index with g_{k'} >= t.  Integer
//   adds make these sums exact and independent of the order of the atomics.
//   D1 / D2 sit in shared memory per CTA when 2 G S 8 bytes fit, else in
//   global memory; either way they end up summed in global memory.
//
// k_finalize (k_finalize_batch: for many networks at once): one CTA per
//   species scans D1 / D2 along the grid, adds N x0,
//   and writes sum1, sum2, mean = sum1 / N and
//   var = (N sum2 - sum1^2) / (N (N - 1)) with an exact 128-bit numerator.
#include <cstdint>

#include "ssa_device.cuh"
#include "ssa_internal.h"
#include "ssa_logtab.h"
#include "ssa_softfloat.cuh"

namespace ssa_impl {
namespace {

using ssa_dev::obits;

// Inclusive block scan of a 64-bit unsigned value (blockDim.x a multiple of
// 32, at most 1024).  `warp_tot` holds 32 words.  Returns the inclusive prefix;
// *total receives the block total.
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long* warp_tot,
                                                             unsigned long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = (lane < nw) ? warp_tot[lane] : 0ULL;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += u;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  const unsigned long long excl = (wid > 0) ? warp_tot[wid - 1] : 0ULL;
  *total = warp_tot[nw - 1];
  __syncthreads();
  return v + excl;
}

// Scans species column s of one network's difference sums (the calling CTA).
__device__ __forceinline__ void finalize_column(const unsigned long long* __restrict__ D1,
                                                const unsigned long long* __restrict__ D2, int G, int S,
                                                long long N, const int32_t* __restrict__ x0, double* mean,
                                                double* var, long long* sum1, long long* sum2, int s,
                                                unsigned long long* tot1, unsigned long long* tot2) {
  const long long xv = x0[s];
  unsigned long long carry1 = (unsigned long long)N * (unsigned long long)xv;
  unsigned long long carry2 = (unsigned long long)N * (unsigned long long)(xv * xv);
  const double dN = __ll2double_rn(N);
  const double den = __dmul_rn(dN, __ll2double_rn(N - 1));
  for (int base = 0; base < G; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const size_t q = (size_t)k * S + s;
    const unsigned long long v1 = (k < G) ? D1[q] : 0ULL;
    const unsigned long long v2 = (k < G) ? D2[q] : 0ULL;
    unsigned long long t1, t2;
    const unsigned long long p1 = block_scan_u64(v1, tot1, &t1);
    const unsigned long long p2 = block_scan_u64(v2, tot2, &t2);
    if (k < G) {
      const long long s1 = (long long)(carry1 + p1);
      const long long s2 = (long long)(carry2 + p2);
      if (sum1) sum1[q] = s1;
      if (sum2) sum2[q] = s2;
      mean[q] = __ddiv_rn(__ll2double_rn(s1), dN);
      if (N < 2) {
        var[q] = __longlong_as_double(0x7FF8000000000000LL);
      } else {
        // N * s2 - s1 * s1 in 128 bits (s2 >= 0, N > 0)
        const unsigned long long a_lo = (unsigned long long)N * (unsigned long long)s2;
        const long long a_hi = __mul64hi((long long)N, s2);
        const unsigned long long b_lo = (unsigned long long)s1 * (unsigned long long)s1;
        const long long b_hi = __mul64hi(s1, s1);
        const unsigned long long lo = a_lo - b_lo;
        const long long hi = a_hi - b_hi - ((a_lo < b_lo) ? 1LL : 0LL);
        var[q] = __ddiv_rn(ssa_dev::i128_to_double_rn(hi, lo), den);
      }
    }
    carry1 += t1;
    carry2 += t2;
  }
}

__global__ void __launch_bounds__(1024) k_finalize(const unsigned long long* __restrict__ D1,
                                                   const unsigned long long* __restrict__ D2, int G, int S,
                                                   long long N, const int32_t* __restrict__ x0, double* mean,
                                                   double* var, long long* sum1, long long* sum2) {
  __shared__ unsigned long long tot1[32], tot2[32];
  finalize_column(D1, D2, G, S, N, x0, mean, var, sum1, sum2, blockIdx.x, tot1, tot2);
}

// Batched finalisation: CTA c serves species c - cta_begin[b] of network b,
// where cta_begin[b] <= c < cta_begin[b + 1].
__global__ void __launch_bounds__(1024) k_finalize_batch(const FinalizeNet* __restrict__ nets,
                                                         const int* __restrict__ cta_begin, int n_nets) {
  __shared__ unsigned long long tot1[32], tot2[32];
  const int c = blockIdx.x;
  int lo = 0, hi = n_nets;  // last b with cta_begin[b] <= c
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cta_begin[mid] <= c) lo = mid; else hi = mid;
  }
  const FinalizeNet f = nets[lo];
  finalize_column(f.D1, f.D2, f.G, f.S, f.N, f.x0, f.mean, f.var, reinterpret_cast<long long*>(f.sum1),
                  reinterpret_cast<long long*>(f.sum2), c - cta_begin[lo], tot1, tot2);
}

__global__ void k_uniform_grid(double* grid, int G, double t_end) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G) return;
  grid[k] = (G == 1) ? t_end : __ddiv_rn(__dmul_rn(__int2double_rn(k), t_end), __int2double_rn(G - 1));
}

}  // namespace

cudaError_t launch_thread_kernel(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem,
                                 cudaStream_t stream) {
  switch (bucket_s(a.m.S)) {
    case 4: return launch_thread_s4(a, blocks, threads, shared_d, smem, stream);
    case 8: return launch_thread_s8(a, blocks, threads, shared_d, smem, stream);
    default: return launch_thread_s16(a, blocks, threads, shared_d, smem, stream);
  }
}

cudaError_t thread_kernel_set_smem(int M, int S, bool shared_d, size_t smem) {
  switch (bucket_s(S)) {
    case 4: return set_smem_s4(M, shared_d, smem);
    case 8: return set_smem_s8(M, shared_d, smem);
    default: return set_smem_s16(M, shared_d, smem);
  }
}

cudaError_t launch_thread_log_kernel(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                     cudaStream_t stream) {
  switch (bucket_s(a.m.S)) {
    case 4: return launch_thread_log_s4(a, lg, blocks, threads, smem, stream);
    case 8: return launch_thread_log_s8(a, lg, blocks, threads, smem, stream);
    default: return launch_thread_log_s16(a, lg, blocks, threads, smem, stream);
  }
}

cudaError_t thread_log_kernel_set_smem(int M, int S, size_t smem) {
  switch (bucket_s(S)) {
    case 4: return set_smem_log_s4(M, smem);
    case 8: return set_smem_log_s8(M, smem);
    default: return set_smem_log_s16(M, smem);
  }
}

cudaError_t launch_finalize(const unsigned long long* D1, const unsigned long long* D2, int G, int S, int64_t N,
                            const int32_t* x0, double* mean, double* var, int64_t* sum1, int64_t* sum2,
                            cudaStream_t stream) {
  int threads = 1024;
  if (G < 1024) threads = ((G + 31) / 32) * 32;
  k_finalize<<<S, threads, 0, stream>>>(D1, D2, G, S, (long long)N, x0, mean, var,
                                         reinterpret_cast<long long*>(sum1), reinterpret_cast<long long*>(sum2));
  return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const FinalizeNet* nets, const int* cta_begin, int n_nets, int total_ctas,
                                  int max_G, cudaStream_t stream) {
  int threads = 1024;
  if (max_G < 1024) threads = ((max_G + 31) / 32) * 32;
  k_finalize_batch<<<total_ctas, threads, 0, stream>>>(nets, cta_begin, n_nets);
  return cudaGetLastError();
}

cudaError_t launch_uniform_grid(double* grid, int G, double t_end, cudaStream_t stream) {
  k_uniform_grid<<<(G + 255) / 256, 256, 0, stream>>>(grid, G, t_end);
  return cudaGetLastError();
}

}  // namespace ssa_impl
