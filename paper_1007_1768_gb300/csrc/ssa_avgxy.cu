// Selective memory along the time axis (Sec. 3.2.1, Fig. 3): Avg-Y on the
// union of every trajectory's event times, and Avg-XY, the average of k
// successive Avg-Y points in time and value (ssa_ensemble_avg_xy).
//
// Definitions (the oracle states them point by point): union points
// T_0 = 0 < T_1 < ... < T_{U-1} are 0 and the distinct event times of all
// trajectories; S1_m[s] = sum_i x_is(T_m), S2_m[s] = sum_i x_is(T_m)^2
// (right-continuous states).  Window p covers union points [p k, b_p),
// b_p = min(U, (p + 1) k), n_p = b_p - p k points:
//   t_p    = (T_{pk} + ... + T_{b_p - 1}) / n_p        (FP64, ascending order)
//   mean_p = sum_m S1_m / (N n_p),  msq_p = sum_m S2_m / (N n_p).
//
// Pipeline:
//   1. the event log is sized by the records per trajectory that an earlier
//      call on the model saw (same t_end, precision, schedule, max_events),
//      else by a pilot of up to 4,096 trajectories (its event count scaled
//      to the ensemble, a quarter to spare); the thread kernel (FP64 networks
//      of at most 16 reactions and species without rate modifiers, unless
//      the warp schedule is asked for) or the warp kernel then runs the
//      ensemble writing the log: one record per (event, species changed)
//      with the event time's bits, the species, v and (2 x_old + v) v (one
//      record with v = 0 for an event changing nothing).  Should the
//      estimate fall short, the run is repeated once with the exact record
//      count it reports;
//   2. a stable least-significant-digit radix sort of the 64-bit time keys
//      (8-bit digits; digits that are equal across all keys are skipped),
//      carrying each record's index;
//   3. head flags (first record of each distinct time) and their scan give
//      every record its union index u; the distinct times are scattered to
//      T[u];
//   4. window sums without materialising S1_m: with C_s(m) the change of
//      species s up to union point m,
//        sum_{m in window p} S1_m = n_p (N x0_s + C_s(pk - 1)) + sum_{r in p} v_r (b_p - u_r),
//      and C_s(pk - 1) is the exclusive scan over windows of W1[p] =
//      sum_{r in p} v_r; the same with x0^2 and (2 x_old + v) v for S2.
//      Records of a block accumulate in shared memory per (window, species)
//      and flush with one global integer atomic each;
//   5. one thread per window sums its times in ascending order; the final
//      kernel forms t, mean and msq.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "ssa.h"
#include "ssa_internal.h"

namespace ssa_impl {
namespace {

typedef unsigned long long u64;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// ------------------------------------------------------------ device scan
// Exclusive scan of n values (in place) with the total written to *total.
constexpr int kScanThreads = 1024;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_sums, T* block_total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = (lane < nw) ? warp_sums[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T y = __shfl_up_sync(0xFFFFFFFFu, s, off);
      if (lane >= off) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const T excl = x - v + ((w > 0) ? warp_sums[w - 1] : T(0));
  *block_total = warp_sums[nw - 1];
  __syncthreads();
  return excl;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(T* data, long long n, T* block_sums) {
  __shared__ T ws[32];
  const long long i = (long long)blockIdx.x * kScanThreads + threadIdx.x;
  const T v = (i < n) ? data[i] : T(0);
  T tot;
  const T e = block_exclusive_scan(v, ws, &tot);
  if (i < n) data[i] = e;
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_add(T* data, long long n, const T* block_offsets) {
  const long long i = (long long)blockIdx.x * kScanThreads + threadIdx.x;
  if (i < n) data[i] += block_offsets[blockIdx.x];
}

template <typename T>
__global__ void k_scan_single(T* data, long long n, T* total) {  // one block, sequential chunks
  __shared__ T ws[32];
  T carry = 0;
  for (long long base = 0; base < n; base += kScanThreads) {
    const long long i = base + threadIdx.x;
    const T v = (i < n) ? data[i] : T(0);
    T tot;
    const T e = block_exclusive_scan(v, ws, &tot);
    if (i < n) data[i] = e + carry;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Scratch of the scan for n values: the block sums of every level.
template <typename T>
size_t scan_scratch_elems(long long n) {
  size_t total = 0;
  while (n > kScanThreads) {
    n = (n + kScanThreads - 1) / kScanThreads;
    total += (size_t)n;
  }
  return total + 1;
}

template <typename T>
cudaError_t device_exclusive_scan(T* data, long long n, T* scratch, T* total, cudaStream_t st) {
  if (n <= kScanThreads * 64) {
    k_scan_single<T><<<1, kScanThreads, 0, st>>>(data, n, total);
    return cudaGetLastError();
  }
  const long long nb = (n + kScanThreads - 1) / kScanThreads;
  k_scan_blocks<T><<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = device_exclusive_scan<T>(scratch, nb, scratch + nb, total, st);
  if (e != cudaSuccess) return e;
  k_scan_add<T><<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, scratch);
  return cudaGetLastError();
}

// ------------------------------------------------------------ radix sort
// Counts of every 8-bit digit at every position (8 x 256), for pass skipping.
__global__ void k_digit_hist_all(const u64* keys, long long n, unsigned long long* hist) {
  __shared__ unsigned int h[8 * 256];
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const u64 k = keys[i];
#pragma unroll
    for (int p = 0; p < 8; ++p) atomicAdd(&h[p * 256 + (int)((k >> (8 * p)) & 255)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// Per-tile digit counts, digit-major: tile_hist[d * ntiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_tile_hist(const u64* keys, long long n, int shift,
                                                            unsigned int* tile_hist, long long ntiles) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long t0 = (long long)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = t0 + (long long)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1u);
  }
  __syncthreads();
  tile_hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Items are ranked in index order (round r
// holds indices r * 256 + tid of the tile; within a round, lanes of a warp
// with the same digit are ranked by __match_any_sync, warps in order by a
// per-round count table, rounds by running digit counts) into the tile's own
// digit order in shared memory; the tile then leaves in that order, so each
// digit's items go out as one contiguous run.
__global__ void __launch_bounds__(kSortThreads) k_tile_scatter(const u64* kin, const unsigned int* vin, u64* kout,
                                                               unsigned int* vout, long long n, int shift,
                                                               const unsigned int* offs, long long ntiles) {
  __shared__ unsigned int base[256];   // next local slot of each digit
  __shared__ unsigned int lbase[256];  // first local slot of each digit
  __shared__ unsigned int gbase[256];  // first global slot of each digit (this tile)
  __shared__ unsigned int wcnt[kSortThreads / 32][256];
  __shared__ u64 skey[kSortTile];
  __shared__ unsigned int sval[kSortTile];
  __shared__ unsigned int wsum[kSortThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // local digit offsets: exclusive scan of this tile's digit counts (a count
  // is the step of the digit-major exclusive scan to the next entry)
  {
    const long long idx = (long long)tid * ntiles + blockIdx.x;
    const unsigned c = (idx + 1 < 256 * ntiles) ? offs[idx + 1] - offs[idx] : (unsigned)n - offs[idx];
    unsigned x = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned pre = 0;
    for (int ww = 0; ww < w; ++ww) pre += wsum[ww];
    lbase[tid] = pre + x - c;
    base[tid] = pre + x - c;
    gbase[tid] = offs[(long long)tid * ntiles + blockIdx.x];
  }
  const long long t0 = (long long)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = t0 + (long long)r * kSortThreads + tid;
    const bool valid = i < n;
    const u64 key = valid ? kin[i] : 0ULL;
    const unsigned dig = valid ? (unsigned)((key >> shift) & 255) : 256u;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncthreads();  // also orders this round's base reads after the last round's update
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
    const unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned before = 0;
      for (int ww = 0; ww < w; ++ww) before += wcnt[ww][dig];
      const unsigned lpos = base[dig] + before + rank;
      skey[lpos] = key;
      sval[lpos] = vin[i];
    }
    __syncthreads();
    unsigned add = 0;
    for (int ww = 0; ww < kSortThreads / 32; ++ww) add += wcnt[ww][tid];
    base[tid] += add;
    __syncthreads();  // every thread has read this round's counts before they are cleared
  }
  // out in local order: slot j of digit d goes to gbase[d] + (j - lbase[d])
  const long long cnt = min((long long)kSortTile, n - t0);
  for (int j = tid; j < cnt; j += kSortThreads) {
    const u64 key = skey[j];
    const unsigned d = (unsigned)((key >> shift) & 255);
    const unsigned pos = gbase[d] + ((unsigned)j - lbase[d]);
    kout[pos] = key;
    vout[pos] = sval[j];
  }
}

__global__ void k_iota(unsigned int* v, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (unsigned int)i;
}

// ------------------------------------------------------------ union and windows
// head[r] = 1 for the first record of each distinct time (records [0, nv)).
__global__ void k_heads(const u64* keys, long long nv, unsigned int* head) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nv) head[r] = (r == 0 || keys[r] != keys[r - 1]) ? 1u : 0u;
}

// uidx holds the exclusive scan of head: union index u_r = uidx[r] + head[r]
// (union point 0 is t = 0).  Distinct times go to T[u].
__global__ void k_union_times(const u64* keys, long long nv, const unsigned int* head, const unsigned int* uidx,
                              double* T) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) T[0] = 0.0;
  if (r < nv && head[r]) T[uidx[r] + 1] = __longlong_as_double((long long)keys[r]);
}

// Window sums of one block's records, in shared memory per (window, species)
// when the block's windows fit (else straight to global), then one global
// integer atomic per entry.  W*[s * P + p] (species-major for the scans).
constexpr int kWinThreads = 256;
constexpr int kWinRecords = 4096;
constexpr int kWinSlots = 512;
constexpr int kWinRegS = 8;  // species summed in registers on the one-window path

__global__ void __launch_bounds__(kWinThreads) k_window_sums(
    const unsigned int* head, const unsigned int* uidx, const unsigned int* perm, const LogRec* rec,
    long long nv, long long U, long long k, int S, long long P,
    long long* W1, long long* A1, long long* W2, long long* A2) {
  __shared__ long long sW1[kWinSlots], sA1[kWinSlots], sW2[kWinSlots], sA2[kWinSlots];
  const long long r0 = (long long)blockIdx.x * kWinRecords;
  const long long r1 = min(nv, r0 + kWinRecords);
  const long long p_lo = (long long)(uidx[r0] + head[r0]) / k;
  const long long p_hi = (long long)(uidx[r1 - 1] + head[r1 - 1]) / k;
  const bool local = (p_hi - p_lo + 1) * S <= kWinSlots;
  for (int i = threadIdx.x; i < kWinSlots; i += blockDim.x) sW1[i] = sA1[i] = sW2[i] = sA2[i] = 0;
  __syncthreads();
  if (p_lo == p_hi && S <= kWinRegS) {
    // one window and few species (the usual case for wide windows): each
    // thread sums its records per species in registers, a warp adds its
    // threads' sums by shuffle, and one lane per warp adds them to the
    // block's slots -- instead of four contended shared atomics per record
    const long long b = min(U, (p_lo + 1) * k);
    long long w1[kWinRegS], a1[kWinRegS], w2[kWinRegS], a2[kWinRegS];
#pragma unroll
    for (int i = 0; i < kWinRegS; ++i) w1[i] = a1[i] = w2[i] = a2[i] = 0;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const long long u = (long long)uidx[r] + head[r];
      const LogRec rq = rec[perm[r]];
      const long long v = rq.change, dd = rq.d2, wt = b - u;
      const long long vw = v * wt, dw = dd * wt;
#pragma unroll
      for (int i = 0; i < kWinRegS; ++i) {
        const bool m = rq.species == i;
        w1[i] += m ? v : 0;
        a1[i] += m ? vw : 0;
        w2[i] += m ? dd : 0;
        a2[i] += m ? dw : 0;
      }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < kWinRegS; ++i) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        w1[i] += __shfl_xor_sync(0xFFFFFFFFu, w1[i], off);
        a1[i] += __shfl_xor_sync(0xFFFFFFFFu, a1[i], off);
        w2[i] += __shfl_xor_sync(0xFFFFFFFFu, w2[i], off);
        a2[i] += __shfl_xor_sync(0xFFFFFFFFu, a2[i], off);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kWinRegS; ++i) {
        if (i < S) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&sW1[i]), (unsigned long long)w1[i]);
          atomicAdd(reinterpret_cast<unsigned long long*>(&sA1[i]), (unsigned long long)a1[i]);
          atomicAdd(reinterpret_cast<unsigned long long*>(&sW2[i]), (unsigned long long)w2[i]);
          atomicAdd(reinterpret_cast<unsigned long long*>(&sA2[i]), (unsigned long long)a2[i]);
        }
      }
    }
  } else {
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const long long u = (long long)uidx[r] + head[r];
    const long long p = u / k;
    const long long b = min(U, (p + 1) * k);
    const unsigned int q = perm[r];
    const LogRec rq = rec[q];
    const int s = rq.species;
    const long long v = rq.change, dd = rq.d2, wt = b - u;
    if (local) {
      const int slot = (int)((p - p_lo) * S + s);
      atomicAdd(reinterpret_cast<unsigned long long*>(&sW1[slot]), (unsigned long long)v);
      atomicAdd(reinterpret_cast<unsigned long long*>(&sA1[slot]), (unsigned long long)(v * wt));
      atomicAdd(reinterpret_cast<unsigned long long*>(&sW2[slot]), (unsigned long long)dd);
      atomicAdd(reinterpret_cast<unsigned long long*>(&sA2[slot]), (unsigned long long)(dd * wt));
    } else {
      const long long g = (long long)s * P + p;
      atomicAdd(reinterpret_cast<unsigned long long*>(W1 + g), (unsigned long long)v);
      atomicAdd(reinterpret_cast<unsigned long long*>(A1 + g), (unsigned long long)(v * wt));
      atomicAdd(reinterpret_cast<unsigned long long*>(W2 + g), (unsigned long long)dd);
      atomicAdd(reinterpret_cast<unsigned long long*>(A2 + g), (unsigned long long)(dd * wt));
    }
  }
  }
  __syncthreads();
  if (local) {
    const int used = (int)((p_hi - p_lo + 1) * S);
    for (int i = threadIdx.x; i < used; i += blockDim.x) {
      const long long p = p_lo + i / S;
      const int s = i % S;
      const long long g = (long long)s * P + p;
      if (sW1[i]) atomicAdd(reinterpret_cast<unsigned long long*>(W1 + g), (unsigned long long)sW1[i]);
      if (sA1[i]) atomicAdd(reinterpret_cast<unsigned long long*>(A1 + g), (unsigned long long)sA1[i]);
      if (sW2[i]) atomicAdd(reinterpret_cast<unsigned long long*>(W2 + g), (unsigned long long)sW2[i]);
      if (sA2[i]) atomicAdd(reinterpret_cast<unsigned long long*>(A2 + g), (unsigned long long)sA2[i]);
    }
  }
}

// The times of each window's union points summed in ascending order (a
// serial chain of FP64 additions per window).  A block of 64 threads serves
// 32 consecutive windows: warp 0 (lane l for window 32 blockIdx.x + l) runs
// the chains from shared memory while warp 1 loads the next kTimeChunk times
// of every window into the other buffer, so no load latency sits on a chain.
constexpr int kTimeChunk = 64;
constexpr int kTimeStride = kTimeChunk + 1;  // odd stride: lanes hit distinct banks
__global__ void __launch_bounds__(64) k_window_times(const double* T, long long U, long long k, long long P,
                                                     double* t_out) {
  __shared__ double buf[2][32 * kTimeStride];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long p0 = (long long)blockIdx.x * 32;
  const long long p = p0 + lane;
  const long long a = p * k;
  const long long b = (p < P) ? min(U, a + k) : a;
  // the longest window of the block sets the number of chunks
  const long long span = min(U, (p0 + 32) * k) - p0 * k;
  const long long nchunk = (min(span, k) + kTimeChunk - 1) / kTimeChunk;
  // the producer fills buffer c & 1 with chunk c of all 32 windows by
  // asynchronous 8-byte copies (zero fill past a window's end), then waits
  // for them before the block's barrier
  auto load = [&](long long c) {
    double* dst = buf[c & 1];
    for (int wi = 0; wi < 32; ++wi) {
      const long long wa = (p0 + wi) * k, wb = (p0 + wi < P) ? min(U, wa + k) : wa;
      for (int i = lane; i < kTimeChunk; i += 32) {
        const long long q = wa + c * kTimeChunk + i;
        const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst + wi * kTimeStride + i);
        const double* src = (q < wb) ? T + q : T;
        const int nbytes = (q < wb) ? 8 : 0;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sdst), "l"(src), "r"(nbytes) : "memory");
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (warp == 1 && nchunk > 0) {
    load(0);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  }
  __syncthreads();
  double sum = 0.0;
  for (long long c = 0; c < nchunk; ++c) {
    if (warp == 1) {
      if (c + 1 < nchunk) {
        load(c + 1);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
    } else {
      const double* src = buf[c & 1] + lane * kTimeStride;
      const long long q0 = a + c * kTimeChunk;
      for (int i = 0; i < kTimeChunk; ++i) {
        if (q0 + i < b) sum = __dadd_rn(sum, src[i]);
      }
    }
    __syncthreads();
  }
  if (warp == 0 && p < P) t_out[p] = __ddiv_rn(sum, (double)(b - a));
}

// mean and msq per (window, species); CW* hold the exclusive scans of W* along p.
__global__ void k_window_final(const long long* CW1, const long long* A1, const long long* CW2, const long long* A2,
                               const int32_t* x0, long long N, long long U, long long k, int S, long long P,
                               double* mean, double* msq) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * S) return;
  const long long p = i / S;
  const int s = (int)(i % S);
  const long long n_p = min(U, (p + 1) * k) - p * k;
  const long long g = (long long)s * P + p;
  const long long xv = x0[s];
  const long long s1 = n_p * (N * xv + CW1[g]) + A1[g];
  const long long s2 = n_p * (N * xv * xv + CW2[g]) + A2[g];
  const double den = (double)(N * n_p);
  mean[i] = __ddiv_rn(__ll2double_rn(s1), den);
  msq[i] = __ddiv_rn(__ll2double_rn(s2), den);
}

__global__ void k_fill_f64(double* p, double v) { *p = v; }

}  // namespace
}  // namespace ssa_impl

using namespace ssa_impl;

extern "C" ssa_status ssa_ensemble_avg_xy(const ssa_model* model, int64_t n_traj, double t_end, uint64_t seed,
                                          const ssa_run_opts* opts, int64_t window, int64_t max_points,
                                          double* t_out, double* mean_out, double* msq_out, int64_t* n_points,
                                          int64_t* n_union) {
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  if (!model || !n_points) return (ssa_status)set_error(SSA_EINVAL, "model and n_points must not be NULL");
  if (n_traj < 1) return (ssa_status)set_error(SSA_EINVAL, "n_traj must be >= 1");
  if (!(t_end > 0.0) || !std::isfinite(t_end)) return (ssa_status)set_error(SSA_EINVAL, "t_end must be finite and > 0");
  if (window < 0) return (ssa_status)set_error(SSA_EINVAL, "window must be >= 0 (0: n_traj)");
  if (max_points < 0 || (max_points > 0 && (!t_out || !mean_out || !msq_out)))
    return (ssa_status)set_error(SSA_EINVAL, "outputs of max_points entries are required");
  if (o.memory != SSA_MEM_HOST && o.memory != SSA_MEM_DEVICE) return (ssa_status)set_error(SSA_EINVAL, "bad memory kind");
  {
    ModelImageView mv0;
    if (model_image_view(model, &mv0) && mv0.has_mod && o.precision == SSA_PREC_FP32)
      return (ssa_status)set_error(SSA_EUNSUPPORTED, "models with rate modifiers run FP64");
  }
  if (o.max_events <= 0) o.max_events = SSA_DEFAULT_MAX_EVENTS;
  const long long k = window ? window : n_traj;
  ModelImageView mv;
  if (!model_image_view(model, &mv)) return (ssa_status)set_error(SSA_EINVAL, "bad model");
  const int S = mv.S, M = mv.M;
  // one trajectory per thread when the network fits the thread kernel (FP64,
  // at most 16 reactions and species, no rate modifiers), else one per warp
  const bool fp32 = o.precision == SSA_PREC_FP32;
  const bool thread_ok = mv.small != nullptr && !fp32;
  if (o.schedule == SSA_SCHED_THREAD && !thread_ok)
    return (ssa_status)set_error(SSA_EUNSUPPORTED,
                                 "the thread schedule takes FP64 networks of at most 16 reactions and 16 species "
                                 "without rate modifiers");
  const bool use_thread = o.schedule == SSA_SCHED_THREAD || (o.schedule == SSA_SCHED_AUTO && thread_ok);
  const int32_t sched = use_thread ? SSA_SCHED_THREAD : SSA_SCHED_WARP;
  if (!use_thread && warp_max_chunk(M) == 0)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "the warp schedule takes at most 512 reactions");
  // the largest number of species one reaction changes (records per event)
  const int32_t* nu_ptr = reinterpret_cast<const int32_t*>(mv.image + mv.off_nu_ptr);
  int max_nnz = 1;
  for (int j = 0; j < M; ++j) max_nnz = std::max(max_nnz, nu_ptr[j + 1] - nu_ptr[j]);
  if (max_nnz > kLogChunk)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "a reaction changes more species than an event-log chunk holds");
  cudaStream_t st = static_cast<cudaStream_t>(o.cuda_stream);

  // pilot: the event count of up to 4,096 of the trajectories sizes the log
  const long long n_pilot = std::min<long long>(n_traj, 4096);
  ssa_run_opts o1 = o;
  o1.memory = SSA_MEM_DEVICE;
  o1.schedule = sched;
  o1.traj_events = nullptr;
  o1.traj_hash = nullptr;
  o1.traj_flags = nullptr;
  o1.workspace = nullptr;
  o1.workspace_bytes = 0;
  o1.device_totals = nullptr;
  o1.sim_event_begin = o1.sim_event_end = nullptr;
  if (o.log_records < 0) return (ssa_status)set_error(SSA_EINVAL, "opts->log_records must be >= 0");
  ssa_run_stats st1;
  std::memset(&st1, 0, sizeof st1);
  cudaError_t e = cudaSuccess;
  // records per trajectory of an earlier call with the same model and key
  LogSize lkey{t_end, o.precision, sched, o.max_events, 0.0};
  double seen_per_traj = 0.0;
  const bool seen = o.log_records == 0 && model_log_size_get(model, lkey, &seen_per_traj);
  if (o.log_records == 0 && !seen) {
    double* d_small = nullptr;
    e = pool_malloc(reinterpret_cast<void**>(&d_small), 16 * (size_t)S + 16, st);
    if (e != cudaSuccess) return (ssa_status)set_error(SSA_ENOMEM, cudaGetErrorString(e));
    ssa_status rs = ssa_ensemble_run(model, n_pilot, t_end, 1, nullptr, seed, &o1, d_small, d_small + S, nullptr,
                                     nullptr, &st1);
    cudaFreeAsync(d_small, st);
    if (rs != SSA_OK) return rs;
  }

  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  DevModel dm;
  int mst = model_device_tables(model, dev, &dm);
  if (mst != SSA_OK) return (ssa_status)mst;
  int threads, blocks;
  size_t smem;
  unsigned long long slack;  // room for every writer's open chunk, twice
  if (use_thread) {
    LaunchPlan plan;
    if (const char* msg = plan_thread_launch(S, M, 0, n_traj, prop.multiProcessorCount, prop.sharedMemPerBlockOptin,
                                             SSA_REDUCE_GLOBAL, o.block_threads, o.grid_blocks, &plan))
      return (ssa_status)set_error(SSA_EINVAL, msg);
    threads = plan.threads;
    blocks = plan.blocks;
    smem = plan.smem;
    if ((e = thread_log_kernel_set_smem(M, S, smem)) != cudaSuccess)
      return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
    slack = ((unsigned long long)blocks * (unsigned long long)threads + 1ULL) * (unsigned long long)kThreadLogChunk * 2ULL;
  } else {
    threads = 256;
    smem = warp_kernel_smem(M, S, dm.nnz, threads);
    if (smem > prop.sharedMemPerBlockOptin)
      return (ssa_status)set_error(SSA_EUNSUPPORTED, "network too large for shared memory");
    int per_sm = 0;
    if ((e = warp_log_kernel_prepare(M, fp32, smem, threads, &per_sm)) != cudaSuccess)
      return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
    if (per_sm < 1) return (ssa_status)set_error(SSA_EUNSUPPORTED, "the logging kernel cannot be resident");
    const long long want = (n_traj + threads / 32 - 1) / (threads / 32);
    const long long capb = (long long)prop.multiProcessorCount * per_sm;
    blocks = (int)(want < capb ? want : capb);
    slack = (unsigned long long)(blocks * (threads / 32) + 1) * (unsigned long long)kLogChunk * 2ULL;
  }
  // capacity: the caller's; else the records per trajectory an earlier call
  // saw, scaled, with a quarter plus 4 / sqrt(N) to spare; else the pilot's
  // events scaled to all trajectories, with a quarter to spare (exact when
  // the pilot is the whole ensemble)
  unsigned long long cap;
  if (o.log_records > 0) {
    cap = (unsigned long long)o.log_records;
  } else if (seen) {
    const long double margin = 1.25L + 4.0L / std::sqrt((long double)n_traj);
    cap = (unsigned long long)((long double)seen_per_traj * (long double)n_traj * margin) + slack;
  } else {
    const long double est = (long double)st1.events * (long double)n_traj / (long double)n_pilot;
    cap = (unsigned long long)(est * (n_pilot == n_traj ? 1.0L : 1.25L)) * (unsigned long long)max_nnz + slack;
  }

  unsigned char* ws = nullptr;
  unsigned char* ws2 = nullptr;  // window arrays, sized after the union is known
  auto fail = [&](int status, const char* msg) {
    if (ws) cudaFreeAsync(ws, st);
    if (ws2) cudaFreeAsync(ws2, st);
    return (ssa_status)set_error(status, msg);
  };
#define SSA_A_TRY(expr)                                           \
  do {                                                            \
    const cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return fail(SSA_ECUDA, cudaGetErrorString(e_)); \
  } while (0)
  size_t o_key = 0, o_key2 = 0, o_rec = 0, o_perm = 0, o_perm2 = 0, o_head = 0, o_uidx = 0, o_T = 0,
         o_th = 0, o_sc32 = 0, o_hist = 0, o_cnt = 0, o_grid = 0, o_d = 0, o_stats = 0, o_counter = 0;
  long long ntiles = 0;
  EventLog lg;
  unsigned long long hc[5];
  for (int attempt = 0;; ++attempt) {
    if (cap >= (1ULL << 31))
      return fail(SSA_EUNSUPPORTED, "the event log would exceed 2^31 records; use fewer trajectories");
    // device memory: one allocation
    ntiles = (long long)((cap + kSortTile - 1) / kSortTile);
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t at = off;
      off = align_up(off + bytes, 256);
      return at;
    };
    o_key = take(8 * cap); o_key2 = take(8 * cap); o_rec = take(sizeof(LogRec) * cap);
    o_perm = take(4 * cap); o_perm2 = take(4 * cap); o_head = take(4 * cap);
    o_uidx = take(4 * cap); o_T = take(8 * (cap + 1));
    o_th = take(4 * (size_t)(256 * ntiles)); o_sc32 = take(4 * scan_scratch_elems<unsigned>(256 * ntiles + cap));
    o_hist = take(8 * 8 * 256); o_cnt = take(8 * 5); o_grid = take(8); o_d = take(16 * (size_t)S);
    o_stats = take(8 * kStatCount); o_counter = take(8);
    if ((e = pool_malloc(reinterpret_cast<void**>(&ws), off, st)) != cudaSuccess)
      return fail(SSA_ENOMEM, cudaGetErrorString(e));
    SSA_A_TRY(cudaMemsetAsync(ws + o_cnt, 0, 8 * 5, st));
    SSA_A_TRY(cudaMemsetAsync(ws + o_d, 0, 16 * (size_t)S, st));
    SSA_A_TRY(cudaMemsetAsync(ws + o_stats, 0, 8 * kStatCount, st));
    SSA_A_TRY(cudaMemsetAsync(ws + o_counter, 0, 8, st));
    SSA_A_TRY(cudaMemsetAsync(ws + o_hist, 0, 8 * 8 * 256, st));
    k_fill_f64<<<1, 1, 0, st>>>(reinterpret_cast<double*>(ws + o_grid), t_end);
    SSA_A_TRY(cudaGetLastError());
    // the trajectories, writing the event log
    RunArgs a;
    std::memset(&a, 0, sizeof a);
    if (use_thread) a.sm = *mv.small;
    a.m = dm;
    a.G = 0;  // no grid: the window sums come from the log
    a.N = n_traj;
    a.traj_offset = o.traj_offset;
    a.seed = seed;
    a.seed_word = nullptr;
    a.stream_id = o.stream_id;
    a.max_events = o.max_events;
    a.t_end = t_end;
    a.grid = reinterpret_cast<const double*>(ws + o_grid);
    a.D1 = reinterpret_cast<unsigned long long*>(ws + o_d);
    a.D2 = a.D1 + S;
    a.counter = reinterpret_cast<unsigned long long*>(ws + o_counter);
    a.stats = reinterpret_cast<unsigned long long*>(ws + o_stats);
    a.grid_uniform = 0;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ws + o_cnt);  // counter, padded, overflow, -, needed
    lg.key = reinterpret_cast<u64*>(ws + o_key);
    lg.rec = reinterpret_cast<LogRec*>(ws + o_rec);
    lg.counter = cnt;
    lg.padded = cnt + 1;
    lg.overflow = cnt + 2;
    lg.needed = cnt + 4;
    lg.capacity = cap;
    if (use_thread)
      SSA_A_TRY(launch_thread_log_kernel(a, lg, blocks, threads, smem, st));
    else
      SSA_A_TRY(launch_warp_log_kernel(a, lg, fp32, blocks, threads, smem, st));
    SSA_A_TRY(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, st));
    unsigned long long hstats[kStatCount];
    SSA_A_TRY(cudaMemcpyAsync(hstats, ws + o_stats, sizeof hstats, cudaMemcpyDeviceToHost, st));
    SSA_A_TRY(cudaStreamSynchronize(st));
    if (hc[2] == 0) {
      lkey.per_traj = (double)hc[4] / (double)n_traj;
      model_log_size_put(model, lkey);
      const long double mx = (long double)hstats[kStatMaxX];
      if ((long double)n_traj * mx * mx * (long double)k >= 4.6e18L)
        return fail(SSA_EOVERFLOW, "window sums of x^2 could leave int64 (N * max_x^2 * window)");
      break;
    }
    if (attempt > 0) return fail(SSA_ECUDA, "the event log overflowed its capacity");
    // the estimate was short: again with the exact record count, plus the
    // padding bound (a chunk of C slots holds at least C - max_nnz + 1
    // records before it is closed, losing at most max_nnz - 1 slots)
    cudaFreeAsync(ws, st);
    ws = nullptr;
    const unsigned long long per = (unsigned long long)((use_thread ? kThreadLogChunk : kLogChunk) - max_nnz + 1);
    cap = hc[4] + (hc[4] / per + 1) * (unsigned long long)(max_nnz - 1) + slack;
  }
  u64* key = lg.key;
  u64* key2 = reinterpret_cast<u64*>(ws + o_key2);
  unsigned int* perm = reinterpret_cast<unsigned int*>(ws + o_perm);
  unsigned int* perm2 = reinterpret_cast<unsigned int*>(ws + o_perm2);
  const long long n_all = (long long)std::min<unsigned long long>(hc[0], cap);
  const long long nv = n_all - (long long)hc[1];  // valid records; sentinels sort last

  // sort (keys, record index) by time
  const int thr = 256;
  k_iota<<<(unsigned)((n_all + thr - 1) / thr), thr, 0, st>>>(perm, n_all);
  SSA_A_TRY(cudaGetLastError());
  k_digit_hist_all<<<std::max(1, std::min((int)((n_all + 4095) / 4096), 4 * prop.multiProcessorCount)), 256, 0, st>>>(
      key, n_all, reinterpret_cast<unsigned long long*>(ws + o_hist));
  SSA_A_TRY(cudaGetLastError());
  unsigned long long hh[8 * 256];
  SSA_A_TRY(cudaMemcpyAsync(hh, ws + o_hist, sizeof hh, cudaMemcpyDeviceToHost, st));
  SSA_A_TRY(cudaStreamSynchronize(st));
  const long long nt = (n_all + kSortTile - 1) / kSortTile;
  unsigned int* th = reinterpret_cast<unsigned int*>(ws + o_th);
  unsigned int* sc = reinterpret_cast<unsigned int*>(ws + o_sc32);
  for (int pass = 0; pass < 8; ++pass) {
    bool varies = true;
    for (int d = 0; d < 256; ++d)
      if (hh[pass * 256 + d] == (unsigned long long)n_all) varies = false;
    if (!varies || n_all == 0) continue;
    const int shift = 8 * pass;
    k_tile_hist<<<(unsigned)nt, kSortThreads, 0, st>>>(key, n_all, shift, th, nt);
    SSA_A_TRY(cudaGetLastError());
    SSA_A_TRY(device_exclusive_scan<unsigned int>(th, 256 * nt, sc, nullptr, st));
    k_tile_scatter<<<(unsigned)nt, kSortThreads, 0, st>>>(key, perm, key2, perm2, n_all, shift, th, nt);
    SSA_A_TRY(cudaGetLastError());
    std::swap(key, key2);
    std::swap(perm, perm2);
  }

  // union indices and times
  unsigned int* head = reinterpret_cast<unsigned int*>(ws + o_head);
  unsigned int* uidx = reinterpret_cast<unsigned int*>(ws + o_uidx);
  double* T = reinterpret_cast<double*>(ws + o_T);
  long long U = 1;
  if (nv > 0) {
    k_heads<<<(unsigned)((nv + thr - 1) / thr), thr, 0, st>>>(key, nv, head);
    SSA_A_TRY(cudaGetLastError());
    SSA_A_TRY(cudaMemcpyAsync(uidx, head, 4 * (size_t)nv, cudaMemcpyDeviceToDevice, st));
    unsigned int* dtot = reinterpret_cast<unsigned int*>(ws + o_cnt + 24);  // slot 3 of the counters
    SSA_A_TRY(device_exclusive_scan<unsigned int>(uidx, nv, sc, dtot, st));
    unsigned int heads = 0;
    SSA_A_TRY(cudaMemcpyAsync(&heads, dtot, 4, cudaMemcpyDeviceToHost, st));
    SSA_A_TRY(cudaStreamSynchronize(st));
    U = 1 + (long long)heads;
  }
  k_union_times<<<(unsigned)((std::max(nv, 1LL) + thr - 1) / thr), thr, 0, st>>>(key, nv, head, uidx, T);
  SSA_A_TRY(cudaGetLastError());
  const long long P = (U + k - 1) / k;
  *n_points = P;
  if (n_union) *n_union = U;
  if (max_points == 0) {
    cudaFreeAsync(ws, st);
    SSA_A_TRY(cudaStreamSynchronize(st));
    return SSA_OK;
  }
  const long long Pw = std::min<long long>(P, max_points);

  // window sums (species-major arrays of P entries), scans, outputs
  size_t off2 = 0;
  auto take2 = [&](size_t bytes) {
    const size_t at = off2;
    off2 = align_up(off2 + bytes, 256);
    return at;
  };
  const size_t PS = (size_t)P * S;
  const size_t o_W1 = take2(8 * PS), o_A1 = take2(8 * PS), o_W2 = take2(8 * PS), o_A2 = take2(8 * PS),
               o_sc64 = take2(8 * scan_scratch_elems<long long>((long long)P) + 8), o_x0 = take2(4 * (size_t)S),
               o_t = take2(8 * (size_t)P), o_mean = take2(8 * PS), o_msq = take2(8 * PS);
  if ((e = pool_malloc(reinterpret_cast<void**>(&ws2), off2, st)) != cudaSuccess)
    return fail(SSA_ENOMEM, cudaGetErrorString(e));
  long long* W1 = reinterpret_cast<long long*>(ws2 + o_W1);
  long long* A1 = reinterpret_cast<long long*>(ws2 + o_A1);
  long long* W2 = reinterpret_cast<long long*>(ws2 + o_W2);
  long long* A2 = reinterpret_cast<long long*>(ws2 + o_A2);
  SSA_A_TRY(cudaMemsetAsync(ws2, 0, o_sc64, st));
  if (nv > 0) {
    k_window_sums<<<(unsigned)((nv + kWinRecords - 1) / kWinRecords), kWinThreads, 0, st>>>(
        head, uidx, perm, lg.rec, nv, U, k, S, P, W1, A1, W2, A2);
    SSA_A_TRY(cudaGetLastError());
  }
  long long* sc64 = reinterpret_cast<long long*>(ws2 + o_sc64);
  for (int s = 0; s < S; ++s) {
    SSA_A_TRY(device_exclusive_scan<long long>(W1 + (size_t)s * P, P, sc64, nullptr, st));
    SSA_A_TRY(device_exclusive_scan<long long>(W2 + (size_t)s * P, P, sc64, nullptr, st));
  }
  int32_t* x0d = reinterpret_cast<int32_t*>(ws2 + o_x0);
  SSA_A_TRY(cudaMemcpyAsync(x0d, dm.x0, 4 * (size_t)S, cudaMemcpyDeviceToDevice, st));
  double* dt = reinterpret_cast<double*>(ws2 + o_t);
  double* dmean = reinterpret_cast<double*>(ws2 + o_mean);
  double* dmsq = reinterpret_cast<double*>(ws2 + o_msq);
  k_window_times<<<(unsigned)((P + 31) / 32), 64, 0, st>>>(T, U, k, P, dt);
  SSA_A_TRY(cudaGetLastError());
  k_window_final<<<(unsigned)((PS + 255) / 256), 256, 0, st>>>(W1, A1, W2, A2, x0d, n_traj, U, k, S, P, dmean, dmsq);
  SSA_A_TRY(cudaGetLastError());
  const cudaMemcpyKind kind = (o.memory == SSA_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  SSA_A_TRY(cudaMemcpyAsync(t_out, dt, 8 * (size_t)Pw, kind, st));
  SSA_A_TRY(cudaMemcpyAsync(mean_out, dmean, 8 * (size_t)Pw * S, kind, st));
  SSA_A_TRY(cudaMemcpyAsync(msq_out, dmsq, 8 * (size_t)Pw * S, kind, st));
  cudaFreeAsync(ws2, st);
  cudaFreeAsync(ws, st);
  SSA_A_TRY(cudaStreamSynchronize(st));
#undef SSA_A_TRY
  return SSA_OK;
}
