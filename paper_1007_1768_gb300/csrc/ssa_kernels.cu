// Simulation and reduction kernels.
//
// k_ssa_thread: one trajectory per thread (networks with M <= 16 reactions).
//   Each lane runs Gillespie's direct method (Sec. 2) for the trajectories it
//   takes from a global work counter.  Propensities a_j and the left-to-right
//   prefix sums live in registers (M is a template constant), the state x in
//   shared memory ([S][threads], conflict-free), the model tables and the
//   logarithm cells in shared memory.  Comparisons of non-negative doubles
//   (selection, grid walk, t_end) run on their bit patterns.
//
//   Selective memory (Sec. 3.2.1) is done without storing any trajectory:
//   the grid state of a trajectory is x0 plus the changes of all events with
//   time <= g_k, so the per-grid sums are
//       sum1[k] = N x0 + sum_{k' <= k} D1[k'],   sum2[k] = N x0^2 + sum_{k' <= k} D2[k'],
//   where an event at time t with change v of species s adds v to D1 and
//   (2 x + v) v to D2 at k' = first grid index with g_{k'} >= t.  Integer
//   adds make these sums exact and independent of the order of the atomics.
//   D1 / D2 sit in shared memory per CTA when 2 G S 8 bytes fit, else in
//   global memory.
//
// k_finalize: one CTA per species scans D1 / D2 along the grid, adds N x0,
//   and writes sum1, sum2, mean = sum1 / N and
//   var = (N sum2 - sum1^2) / (N (N - 1)) with an exact 128-bit numerator.
#include <cstdint>

#include "ssa_device.cuh"
#include "ssa_internal.h"
#include "ssa_logtab.h"

namespace ssa_impl {
namespace {

using ssa_dev::obits;

__device__ const ssa_logtab::Tables d_log_tables = ssa_logtab::kTables;

constexpr unsigned long long kFnvOffset = 0xcbf29ce484222325ULL;
constexpr unsigned long long kFnvPrime = 0x100000001b3ULL;
constexpr long long kStateMax = 2147483647LL;

// h_j(x) for a packed reaction word; xs points at this lane's column of the
// state ([S][T] in shared memory).
__device__ __forceinline__ long long mass_action_h(int32_t w, const int32_t* xs, int T) {
  const int kind = rinfo_kind(w);
  if (kind == kOrder0) return 1LL;
  const long long xa = xs[rinfo_a(w) * T];
  if (kind == kUni) return xa;
  if (kind == kBi) return xa * (long long)xs[rinfo_b(w) * T];
  return xa * (xa - 1) / 2;
}

template <int M, bool SHARED_D>
__global__ void __launch_bounds__(512) k_ssa_thread(const RunArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long blk_events, blk_trunc, blk_over;
  __shared__ int blk_maxx;
  const int S = a.m.S, G = a.G, T = blockDim.x, tid = threadIdx.x;
  const ThreadSmem L = thread_smem_layout(S, M, a.m.nnz, G, T, SHARED_D);
  uint64_t* s_inv = reinterpret_cast<uint64_t*>(smem + L.log_inv);
  uint64_t* s_lnf = reinterpret_cast<uint64_t*>(smem + L.log_lnf);
  double* s_c = reinterpret_cast<double*>(smem + L.c);
  int32_t* s_rinfo = reinterpret_cast<int32_t*>(smem + L.rinfo);
  int32_t* s_nuptr = reinterpret_cast<int32_t*>(smem + L.nu_ptr);
  int32_t* s_nuidx = reinterpret_cast<int32_t*>(smem + L.nu_idx);
  int32_t* s_nuval = reinterpret_cast<int32_t*>(smem + L.nu_val);
  int32_t* s_x = reinterpret_cast<int32_t*>(smem + L.x);
  unsigned long long* d1 = SHARED_D ? reinterpret_cast<unsigned long long*>(smem + L.d1) : a.D1;
  unsigned long long* d2 = SHARED_D ? reinterpret_cast<unsigned long long*>(smem + L.d2) : a.D2;

  for (int i = tid; i < 128; i += T) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  for (int j = tid; j < M; j += T) {
    s_c[j] = a.m.c[j];
    s_rinfo[j] = a.m.rinfo[j];
  }
  for (int j = tid; j <= M; j += T) s_nuptr[j] = a.m.nu_ptr[j];
  for (int q = tid; q < a.m.nnz; q += T) {
    s_nuidx[q] = a.m.nu_idx[q];
    s_nuval[q] = a.m.nu_val[q];
  }
  if (SHARED_D) {
    for (int q = tid; q < G * S; q += T) {
      d1[q] = 0ULL;
      d2[q] = 0ULL;
    }
  }
  if (tid == 0) {
    blk_events = 0ULL;
    blk_trunc = 0ULL;
    blk_over = 0ULL;
    blk_maxx = 0;
  }
  __syncthreads();

  int32_t* xs = s_x + tid;
  const long long t_end_bits = obits(a.t_end);
  const bool want_hash = a.traj_hash != nullptr;

  double av[M];
  bool have = false;
  long long li = 0;
  unsigned long long traj_id = 0;
  double t = 0.0;
  long long n = 0;
  int k = 0;
  unsigned long long hash = kFnvOffset;
  unsigned long long w2 = 0ULL, w3 = 0ULL;
  int maxx = 0;

  for (;;) {
    if (!have) {
      const unsigned long long next = atomicAdd(a.counter, 1ULL);
      if (next >= (unsigned long long)a.N) break;
      have = true;
      li = (long long)next;
      traj_id = a.traj_offset + next;
      maxx = 0;
      for (int s = 0; s < S; ++s) {
        const int v = a.m.x0[s];
        xs[s * T] = v;
        maxx = max(maxx, v);
      }
      t = 0.0;
      n = 0;
      k = 0;
      hash = kFnvOffset;
#pragma unroll
      for (int j = 0; j < M; ++j)
        av[j] = __dmul_rn(s_c[j], __ll2double_rn(mass_action_h(s_rinfo[j], xs, T)));
    }

    // a0 and prefix sums, left to right
    double pre[M];
    pre[0] = av[0];
#pragma unroll
    for (int j = 1; j < M; ++j) pre[j] = __dadd_rn(pre[j - 1], av[j]);
    const double a0 = pre[M - 1];

    unsigned long long wa, wb;
    if ((n & 1) == 0) {
      const ssa_dev::Words4 w =
          ssa_dev::philox4x64_10((unsigned long long)(n >> 1), traj_id, 0ULL, 0ULL, a.seed, a.stream_id);
      wa = w.w0;
      wb = w.w1;
      w2 = w.w2;
      w3 = w.w3;
    } else {
      wa = w2;
      wb = w3;
    }

    double t_next;
    if (obits(a0) > 0) {
      const double E = ssa_dev::neg_log_u(ssa_dev::odd53(wa), s_inv, s_lnf);
      t_next = __dadd_rn(t, __ddiv_rn(E, a0));
    } else {
      t_next = __longlong_as_double(0x7FF0000000000000LL);  // +inf: absorbing state
    }

    // grid points before t_next keep the current state: only the index moves
    const long long tb = obits(t_next);
    while (k < G && obits(__ldg(a.grid + k)) < tb) ++k;

    int flags = 0;
    bool done = false;
    if (tb > t_end_bits) {
      done = true;
    } else {
      // first j with prefix_j > r2 * a0 (prefixes are non-decreasing)
      const long long gb = obits(__dmul_rn(ssa_dev::uniform_from_odd53(ssa_dev::odd53(wb)), a0));
      int cnt = 0, last_pos = 0;
#pragma unroll
      for (int j = 0; j < M; ++j) {
        cnt += (obits(pre[j]) <= gb) ? 1 : 0;
        if (obits(av[j]) > 0) last_pos = j;
      }
      const int jsel = (cnt < M) ? cnt : last_pos;
      const int q0 = s_nuptr[jsel], q1 = s_nuptr[jsel + 1];
      bool over = false;
      for (int q = q0; q < q1; ++q) {
        if ((long long)xs[s_nuidx[q] * T] + (long long)s_nuval[q] > kStateMax) over = true;
      }
      if (over) {
        flags |= 2;
        done = true;
      } else {
        for (int q = q0; q < q1; ++q) {
          const int s = s_nuidx[q];
          const int v = s_nuval[q];
          const int xo = xs[s * T];
          const int xn = xo + v;
          xs[s * T] = xn;
          maxx = max(maxx, xn);
          if (k < G) {
            atomicAdd(d1 + (size_t)k * S + s, (unsigned long long)(long long)v);
            atomicAdd(d2 + (size_t)k * S + s,
                      (unsigned long long)((long long)(2 * (long long)xo + v) * (long long)v));
          }
        }
        t = t_next;
        ++n;
        if (want_hash) {
          hash = (hash ^ (unsigned long long)jsel) * kFnvPrime;
          hash = (hash ^ (unsigned long long)obits(t)) * kFnvPrime;
        }
        if (n == a.max_events) {
          flags |= 1;
          done = true;
        } else {
#pragma unroll
          for (int j = 0; j < M; ++j)
            av[j] = __dmul_rn(s_c[j], __ll2double_rn(mass_action_h(s_rinfo[j], xs, T)));
        }
      }
    }

    if (done) {
      if (a.traj_events) a.traj_events[li] = n;
      if (want_hash) a.traj_hash[li] = hash;
      if (a.traj_flags) a.traj_flags[li] = flags;
      atomicAdd(&blk_events, (unsigned long long)n);
      if (flags & 1) atomicAdd(&blk_trunc, 1ULL);
      if (flags & 2) atomicAdd(&blk_over, 1ULL);
      atomicMax(&blk_maxx, maxx);
      have = false;
    }
  }

  __syncthreads();
  if (SHARED_D) {
    for (int q = tid; q < G * S; q += T) {
      const unsigned long long v1 = d1[q], v2 = d2[q];
      if (v1) atomicAdd(a.D1 + q, v1);
      if (v2) atomicAdd(a.D2 + q, v2);
    }
  }
  if (tid == 0) {
    atomicAdd(a.stats + kStatEvents, blk_events);
    atomicAdd(a.stats + kStatTruncated, blk_trunc);
    atomicAdd(a.stats + kStatOverflowed, blk_over);
    atomicMax(a.stats + kStatMaxX, (unsigned long long)blk_maxx);
    if (a.device_totals) {
      atomicAdd(a.device_totals + 0, blk_events);
      atomicAdd(a.device_totals + 1, blk_trunc);
      atomicAdd(a.device_totals + 2, blk_over);
      atomicMax(a.device_totals + 3, (unsigned long long)blk_maxx);
    }
  }
}

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

__global__ void __launch_bounds__(1024) k_finalize(const unsigned long long* __restrict__ D1,
                                                   const unsigned long long* __restrict__ D2, int G, int S,
                                                   long long N, const int32_t* __restrict__ x0, double* mean,
                                                   double* var, long long* sum1, long long* sum2) {
  __shared__ unsigned long long tot1[32], tot2[32];
  const int s = blockIdx.x;
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

__global__ void k_uniform_grid(double* grid, int G, double t_end) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G) return;
  grid[k] = (G == 1) ? t_end : __ddiv_rn(__dmul_rn(__int2double_rn(k), t_end), __int2double_rn(G - 1));
}

template <int M>
cudaError_t launch_m(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st) {
  if (shared_d)
    k_ssa_thread<M, true><<<blocks, threads, smem, st>>>(a);
  else
    k_ssa_thread<M, false><<<blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int M>
cudaError_t set_smem_m(bool shared_d, size_t smem) {
  if (shared_d)
    return cudaFuncSetAttribute(k_ssa_thread<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(k_ssa_thread<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#define SSA_FOR_EACH_M(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

}  // namespace

cudaError_t launch_thread_kernel(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem,
                                 cudaStream_t stream) {
  switch (a.m.M) {
#define SSA_CASE(MM) \
  case MM:           \
    return launch_m<MM>(a, blocks, threads, shared_d, smem, stream);
    SSA_FOR_EACH_M(SSA_CASE)
#undef SSA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t thread_kernel_set_smem(int M, bool shared_d, size_t smem) {
  switch (M) {
#define SSA_CASE(MM) \
  case MM:           \
    return set_smem_m<MM>(shared_d, smem);
    SSA_FOR_EACH_M(SSA_CASE)
#undef SSA_CASE
    default:
      return cudaErrorInvalidValue;
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

cudaError_t launch_uniform_grid(double* grid, int G, double t_end, cudaStream_t stream) {
  k_uniform_grid<<<(G + 255) / 256, 256, 0, stream>>>(grid, G, t_end);
  return cudaGetLastError();
}

}  // namespace ssa_impl
