// The single-network simulation kernel for large networks: one trajectory
// per warp (schedule W32; the step itself is in ssa_warp_step.cuh).  Every
// CTA stages the network's tables in shared memory once: rates, packed
// reactant words, the net-change CSR, x0, the per-lane dependency bits and
// the log tables; each warp then takes trajectory ids from a global counter.
#include <cstdint>

#include "ssa_warp_step.cuh"

namespace ssa_impl {
namespace {

// Shared-memory layout of the warp kernel (bytes).
struct WarpSmem {
  size_t log_inv, log_lnf, cbits, c32, rinfo, nu_ptr, nu_idx, nu_val, x0, depw, mod, x, xrec, total;
};

// The rate-modifier tables (4 x M words) are always reserved: they are small
// and keep the layout independent of the model's contents.
__host__ __device__ inline WarpSmem warp_smem_layout(int M, int S, int nnz, int warps) {
  WarpSmem L;
  size_t o = 0;
  L.log_inv = o; o += kLogCells * 8;
  L.log_lnf = o; o += kLogCells * 8;
  L.cbits = o; o += align_up((size_t)M * 8, 16);
  L.c32 = o; o += align_up((size_t)M * 4, 16);
  L.rinfo = o; o += align_up((size_t)M * 4, 16);
  L.nu_ptr = o; o += align_up((size_t)(M + 1) * 4, 16);
  L.nu_idx = o; o += align_up((size_t)nnz * 4, 16);
  L.nu_val = o; o += align_up((size_t)nnz * 4, 16);
  L.x0 = o; o += align_up((size_t)S * 4, 16);
  L.depw = o; o += align_up((size_t)M * 32 * 2, 16);
  L.mod = o; o += align_up((size_t)M * 4, 16) + (size_t)M * 24;
  L.x = o; o += align_up((size_t)warps * S * 4, 16);
  L.xrec = o; o += (size_t)warps * 32 * kRecPerEvent * 4;  // pre-event counts of a batch, per warp
  L.total = o;
  return L;
}

// MAXCH bounds the chunk ceil(M / 32); F32 selects the FP32-propensity mode;
// LOG also writes the event log (selective memory along the time axis).
// Chunks of at most 4 reactions per lane are held to 64 registers (four
// 256-thread CTAs per SM; measured faster than 80-92 registers at three or
// two); larger chunks take the registers the compiler chooses (a 512-reaction
// FP64 network ran slower at two CTAs per SM under 128 registers than at one
// with 162).
template <int MAXCH, bool F32, bool LOG>
__global__ void __launch_bounds__(256, MAXCH <= 4 ? 4 : 1) k_ssa_warp(const RunArgs a, const EventLog lg) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long blk[4];
  __shared__ int s_nnz_max;
  const int S = a.m.S, M = a.m.M, T = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
  const int ch = (M + 31) / 32;
  const WarpSmem L = warp_smem_layout(M, S, a.m.nnz, nwarps);
  uint64_t* s_inv = reinterpret_cast<uint64_t*>(smem + L.log_inv);
  uint64_t* s_lnf = reinterpret_cast<uint64_t*>(smem + L.log_lnf);
  unsigned long long* s_cbits = reinterpret_cast<unsigned long long*>(smem + L.cbits);
  float* s_c32 = reinterpret_cast<float*>(smem + L.c32);
  int32_t* s_rinfo = reinterpret_cast<int32_t*>(smem + L.rinfo);
  int32_t* s_nuptr = reinterpret_cast<int32_t*>(smem + L.nu_ptr);
  int32_t* s_nuidx = reinterpret_cast<int32_t*>(smem + L.nu_idx);
  int32_t* s_nuval = reinterpret_cast<int32_t*>(smem + L.nu_val);
  int32_t* s_x0 = reinterpret_cast<int32_t*>(smem + L.x0);
  uint16_t* s_depw = reinterpret_cast<uint16_t*>(smem + L.depw);
  int32_t* xs = reinterpret_cast<int32_t*>(smem + L.x) + (size_t)warp * S;
  int32_t* xrec = reinterpret_cast<int32_t*>(smem + L.xrec) + (size_t)warp * 32 * kRecPerEvent;
  if (tid == 0) s_nnz_max = 0;

  for (int i = tid; i < kLogCells; i += T) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  for (int j = tid; j < M; j += T) {
    s_cbits[j] = (unsigned long long)obits(a.m.c[j]);
    s_c32[j] = __double2float_rn(a.m.c[j]);
    s_rinfo[j] = a.m.rinfo[j];
  }
  __syncthreads();
  for (int j = tid; j <= M; j += T) {
    s_nuptr[j] = a.m.nu_ptr[j];
    if (j < M) atomicMax(&s_nnz_max, a.m.nu_ptr[j + 1] - a.m.nu_ptr[j]);
  }
  for (int i = tid; i < a.m.nnz; i += T) {
    s_nuidx[i] = a.m.nu_idx[i];
    s_nuval[i] = a.m.nu_val[i];
  }
  for (int s = tid; s < S; s += T) s_x0[s] = a.m.x0[s];
  for (int i = tid; i < M * 32; i += T) s_depw[i] = depw_entry(a.m.dep_ptr, a.m.dep_idx, ch, i >> 5, i & 31);
  int32_t* s_modf = reinterpret_cast<int32_t*>(smem + L.mod);
  double* s_modk = reinterpret_cast<double*>(smem + L.mod + align_up((size_t)M * 4, 16));
  double* s_modlo = s_modk + M;
  double* s_modhi = s_modlo + M;
  const bool has_mod = a.m.mod_f != nullptr;
  if (has_mod) {
    for (int j = tid; j < M; j += T) {
      s_modf[j] = a.m.mod_f[j];
      s_modk[j] = a.m.mod_k[j];
      s_modlo[j] = a.m.mod_lo[j];
      s_modhi[j] = a.m.mod_hi[j];
    }
  }
  if (tid < 4) blk[tid] = 0ULL;
  __syncthreads();

  WarpNet net;
  net.rinfo = s_rinfo;
  net.cbits = s_cbits;
  net.c32 = s_c32;
  net.nu_ptr = s_nuptr;
  net.nu_idx = s_nuidx;
  net.nu_val = s_nuval;
  net.depw = s_depw;
  net.x0 = s_x0;
  net.grid = a.grid;
  net.D1 = a.D1;
  net.D2 = a.D2;
  net.mod_f = has_mod ? s_modf : nullptr;
  net.mod_k = has_mod ? s_modk : nullptr;
  net.mod_lo = has_mod ? s_modlo : nullptr;
  net.mod_hi = has_mod ? s_modhi : nullptr;
  net.t_end_bits = obits(a.t_end);
  net.S = S;
  net.M = M;
  net.G = a.G;
  net.nnz_max = s_nnz_max;
  net.grid_uniform = a.grid_uniform;
  net.grid_scale = a.grid_scale;
  net.grid_margin = a.grid_margin;
  net.sid = (uint32_t)a.stream_id;
  const uint32_t key0 = (uint32_t)a.seed, key1 = (uint32_t)(a.seed >> 32);
  WarpLogState lst{kLogSentinel, 0, false, 0ULL};

  for (;;) {
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(a.counter, 1ULL);
    next = __shfl_sync(kFullMask, next, 0);
    if (next >= (unsigned long long)a.N) break;
    const long long li = (long long)next;
    const WarpTraj r = warp_trajectory<MAXCH, F32, LOG>(net, xs, xrec, a.traj_offset + next, key0, key1,
                                                        a.max_events, s_inv, s_lnf, &lg, &lst);
    if (lane == 0) {
      if (a.traj_events) a.traj_events[li] = (long long)r.n;
      if (a.traj_hash) a.traj_hash[li] = r.hash;
      if (a.traj_flags) a.traj_flags[li] = r.flags;
      atomicAdd(&blk[0], (unsigned long long)r.n);
      if (r.flags & kWarpFlagTruncated) atomicAdd(&blk[1], 1ULL);
      if (r.flags & kWarpFlagOverflow) atomicAdd(&blk[2], 1ULL);
      atomicMax(&blk[3], (unsigned long long)r.maxx);
    }
    __syncwarp();
  }
  if constexpr (LOG) log_close(lg, lst);

  __syncthreads();
  if (tid == 0) {
    atomicAdd(a.stats + kStatEvents, blk[0]);
    atomicAdd(a.stats + kStatTruncated, blk[1]);
    atomicAdd(a.stats + kStatOverflowed, blk[2]);
    atomicMax(a.stats + kStatMaxX, blk[3]);
    if (a.device_totals) {
      atomicAdd(a.device_totals + 0, blk[0]);
      atomicAdd(a.device_totals + 1, blk[1]);
      atomicAdd(a.device_totals + 2, blk[2]);
      atomicMax(a.device_totals + 3, blk[3]);
    }
  }
}

template <int MAXCH, bool F32, bool LOG>
cudaError_t launch_ch(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem, cudaStream_t st) {
  k_ssa_warp<MAXCH, F32, LOG><<<blocks, threads, smem, st>>>(a, lg);
  return cudaGetLastError();
}

template <int MAXCH, bool F32, bool LOG>
cudaError_t prepare_ch(size_t smem, int threads, int* per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(k_ssa_warp<MAXCH, F32, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ssa_warp<MAXCH, F32, LOG>, threads, smem);
}

template <bool F32, bool LOG>
cudaError_t dispatch(int M, bool launch, const RunArgs* a, const EventLog* lg, int blocks, int threads, size_t smem,
                     cudaStream_t st, int* per_sm) {
  switch (warp_max_chunk(M)) {
#define SSA_CH_CASE(C)                                                                     \
  case C:                                                                                  \
    return launch ? launch_ch<C, F32, LOG>(*a, *lg, blocks, threads, smem, st)            \
                  : prepare_ch<C, F32, LOG>(smem, threads, per_sm);
    SSA_CH_CASE(1)
    SSA_CH_CASE(2)
    SSA_CH_CASE(4)
    SSA_CH_CASE(8)
    SSA_CH_CASE(16)
#undef SSA_CH_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch_all(int M, bool fp32, bool log, bool launch, const RunArgs* a, const EventLog* lg, int blocks,
                         int threads, size_t smem, cudaStream_t st, int* per_sm) {
  if (fp32) {
    return log ? dispatch<true, true>(M, launch, a, lg, blocks, threads, smem, st, per_sm)
               : dispatch<true, false>(M, launch, a, lg, blocks, threads, smem, st, per_sm);
  }
  return log ? dispatch<false, true>(M, launch, a, lg, blocks, threads, smem, st, per_sm)
             : dispatch<false, false>(M, launch, a, lg, blocks, threads, smem, st, per_sm);
}

}  // namespace

int warp_max_chunk(int M) {
  const int ch = (M + 31) / 32;
  return ch <= 1 ? 1 : (ch <= 2 ? 2 : (ch <= 4 ? 4 : (ch <= 8 ? 8 : (ch <= 16 ? 16 : 0))));
}

size_t warp_kernel_smem(int M, int S, int nnz, int threads) {
  return warp_smem_layout(M, S, nnz, threads / 32).total;
}

cudaError_t warp_kernel_prepare(int M, bool fp32, size_t smem, int threads, int* blocks_per_sm) {
  return dispatch_all(M, fp32, false, false, nullptr, nullptr, 0, threads, smem, nullptr, blocks_per_sm);
}

cudaError_t launch_warp_kernel(const RunArgs& a, bool fp32, int blocks, int threads, size_t smem,
                               cudaStream_t stream) {
  const EventLog none{};
  return dispatch_all(a.m.M, fp32, false, true, &a, &none, blocks, threads, smem, stream, nullptr);
}

cudaError_t warp_log_kernel_prepare(int M, bool fp32, size_t smem, int threads, int* blocks_per_sm) {
  return dispatch_all(M, fp32, true, false, nullptr, nullptr, 0, threads, smem, nullptr, blocks_per_sm);
}

cudaError_t launch_warp_log_kernel(const RunArgs& a, const EventLog& lg, bool fp32, int blocks, int threads,
                                   size_t smem, cudaStream_t stream) {
  return dispatch_all(a.m.M, fp32, true, true, &a, &lg, blocks, threads, smem, stream, nullptr);
}

}  // namespace ssa_impl
