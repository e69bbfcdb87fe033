// The simulation kernel for large networks: one trajectory per warp.
//
// Gillespie's direct method (Sec. 2) with the reactions spread over the 32
// lanes: lane l owns the contiguous chunk of CH = ceil(M / 32) reactions
// starting at l * CH and keeps their propensities in registers.  Summation
// schedule W32 (the oracle implements the same order):
//   part_l = left-to-right sum of lane l's chunk (0 for an empty lane);
//   inclusive Kogge-Stone scan of the parts with offsets 1, 2, 4, 8, 16
//     (v_l <- v_l + v_{l - off} for l >= off, all lanes reading the
//     previous step's values);
//   prefix_j = inner_j for lane 0, v_{l-1} + inner_j otherwise, with
//     inner_j the running sum inside the chunk up to j; a0 = v_31.
// Selection: each lane finds its first reaction with a_j > 0 and
// prefix_j > r2 a0; a ballot picks the lowest such lane (the first j overall).  After an event,
// every lane reads its bits of the fired reaction's dependency mask (a
// per-reaction, per-lane table in shared memory) and recomputes only those
// propensities.  The state x lives in shared memory (S counts per warp); the
// changes of the fired reaction are applied one per lane.  The random numbers
// of 32 consecutive events are drawn at once, one per lane.  Selective memory
// (Sec. 3.2.1) is the same difference-sum scheme as the thread kernel.
#include <cstdint>

#include "ssa_thread_kernel.cuh"  // shared helpers: products, grid index, tables

namespace ssa_impl {
namespace {

constexpr int kWarpFlagTruncated = 1;  // per-trajectory flag bits
constexpr int kWarpFlagOverflow = 2;

// Exact binary32 -> binary64 widening of a non-negative value on the integer pipe.
__device__ __forceinline__ double widen(float f) {
  return __longlong_as_double((long long)ssa_sf::f32_to_f64(__float_as_uint(f)));
}

// Shared-memory layout of the warp kernel (bytes).
struct WarpSmem {
  size_t log_inv, log_lnf, cbits, c32, rinfo, nu_ptr, nu_idx, nu_val, x0, depw, x, total;
};

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
  L.x = o; o += align_up((size_t)warps * S * 4, 16);
  L.total = o;
  return L;
}

// MAXCH bounds the chunk ceil(M / 32) (registers only; the chunk itself is
// the runtime value, as the schedule defines it).  F32 selects the
// FP32-propensity mode.
template <int MAXCH, bool F32>
__global__ void __launch_bounds__(256) k_ssa_warp(const RunArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long blk[4];
  const int S = a.m.S, M = a.m.M, G = a.G, T = blockDim.x, tid = threadIdx.x;
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

  for (int i = tid; i < kLogCells; i += T) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  for (int j = tid; j < M; j += T) {
    s_cbits[j] = (unsigned long long)obits(a.m.c[j]);
    s_c32[j] = __double2float_rn(a.m.c[j]);
    s_rinfo[j] = a.m.rinfo[j];
  }
  for (int j = tid; j <= M; j += T) s_nuptr[j] = a.m.nu_ptr[j];
  for (int i = tid; i < a.m.nnz; i += T) {
    s_nuidx[i] = a.m.nu_idx[i];
    s_nuval[i] = a.m.nu_val[i];
  }
  for (int s = tid; s < S; s += T) s_x0[s] = a.m.x0[s];
  // entry (j, l): bit q set when reaction l * ch + q reads a species j changes
  for (int i = tid; i < M * 32; i += T) {
    const int j = i >> 5, l = i & 31;
    uint32_t bits = 0;
    for (int q = a.m.dep_ptr[j]; q < a.m.dep_ptr[j + 1]; ++q) {
      const int kk = a.m.dep_idx[q];
      if (kk / ch == l) bits |= 1u << (kk - l * ch);
    }
    s_depw[i] = (uint16_t)bits;
  }
  if (tid < 4) blk[tid] = 0ULL;
  __syncthreads();

  const long long t_end_bits = obits(a.t_end);
  const uint32_t key0 = (uint32_t)a.seed, key1 = (uint32_t)(a.seed >> 32), sid = (uint32_t)a.stream_id;
  const int my0 = lane * ch;                          // first reaction of this lane
  const int mine = max(0, min(ch, M - my0));          // reactions this lane owns

  for (;;) {
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(a.counter, 1ULL);
    next = __shfl_sync(kFullMask, next, 0);
    if (next >= (unsigned long long)a.N) break;
    const long long li = (long long)next;
    const unsigned long long traj_id = a.traj_offset + next;
    int maxx = 0;
    for (int s = lane; s < S; s += 32) {
      xs[s] = s_x0[s];
      maxx = max(maxx, s_x0[s]);
    }
    __syncwarp();
    double av[MAXCH];  // FP64 mode: a_j
    float af[MAXCH];   // FP32 mode: a_j in binary32
#pragma unroll
    for (int q = 0; q < MAXCH; ++q) {
      av[q] = 0.0;
      af[q] = 0.0f;
    }
    uint32_t dirty = (1u << mine) - 1u;
    double t = 0.0;
    uint32_t n = 0;
    int k = 0;
    unsigned long long hash = kFnvOffset;
    int flags = 0;
    uint32_t base = 0;
    unsigned long long cE = 0, cU = 0;
    bool filled = false;

    for (;;) {
      // propensities of this lane's reactions that the last event touched
#pragma unroll
      for (int q = 0; q < MAXCH; ++q) {
        if ((dirty >> q) & 1u) {
          const int j = my0 + q;
          const int32_t w = s_rinfo[j];
          const int kind = rinfo_kind(w);
          const long long xa = xs[rinfo_a(w)];
          const long long xb = xs[rinfo_b(w)];
          const long long bi = xa * ((kind == kBi) ? xb : (xa - 1));
          const long long h =
              (kind == kOrder0) ? 1LL : ((kind == kUni) ? xa : ((kind == kBi) ? bi : (bi >> 1)));
          if constexpr (F32)
            af[q] = __fmul_rn(s_c32[j], __ll2float_rn(h));
          else
            av[q] = __longlong_as_double((long long)propensity_fp64(s_cbits[j], h));
        }
      }
      // schedule W32: running sums inside the chunk, Kogge-Stone scan of the
      // chunk sums, prefixes excl + inner.  A past-the-end a_j is +0 and
      // x + (+0) = x, so the last running sum is the chunk sum (+0 for an
      // empty lane).
      double run[MAXCH];   // FP64 mode: running sums
      float run32[MAXCH];  // FP32 mode: binary32 running sums
      double a0, excl = 0.0, sel_total;
      float excl32 = 0.0f;
      if constexpr (F32) {
        // binary32 selection sums
#pragma unroll
        for (int q = 0; q < MAXCH; ++q) run32[q] = (q == 0) ? af[0] : __fadd_rn(run32[q - 1], af[q]);
        float v32 = run32[MAXCH - 1];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float u = __shfl_up_sync(kFullMask, v32, off);
          if (lane >= off) v32 = __fadd_rn(v32, u);
        }
        excl32 = __shfl_up_sync(kFullMask, v32, 1);
        sel_total = widen(__shfl_sync(kFullMask, v32, 31));
        // a0: FP64 sum of the widened a_j in the same schedule, formed anew each event
        double r64 = widen(af[0]);
#pragma unroll
        for (int q = 1; q < MAXCH; ++q) r64 = __dadd_rn(r64, widen(af[q]));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const double u = __shfl_up_sync(kFullMask, r64, off);
          if (lane >= off) r64 = __dadd_rn(r64, u);
        }
        a0 = __shfl_sync(kFullMask, r64, 31);
      } else {
#pragma unroll
        for (int q = 0; q < MAXCH; ++q) run[q] = (q == 0) ? av[0] : __dadd_rn(run[q - 1], av[q]);
        double v = run[MAXCH - 1];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const double u = __shfl_up_sync(kFullMask, v, off);
          if (lane >= off) v = __dadd_rn(v, u);
        }
        excl = __shfl_up_sync(kFullMask, v, 1);
        a0 = __shfl_sync(kFullMask, v, 31);
        sel_total = a0;
      }
      // random numbers of event n: 32 consecutive events drawn at once, one per lane
      if (!filled || n >= base + 32u) {
        base = n;
        const EventRandom r = event_random(base + (uint32_t)lane, traj_id, sid, key0, key1, s_inv, s_lnf);
        cE = r.E;
        cU = r.u2;
        filled = true;
      }
      const int slot = (int)(n - base);
      const unsigned long long Eb = __shfl_sync(kFullMask, cE, slot);
      const unsigned long long Ub = __shfl_sync(kFullMask, cU, slot);
      const double t_next = __dadd_rn(t, quotient(Eb, a0));  // a0 == 0: +inf
      const long long tb = obits(t_next);
      if (tb > t_end_bits) break;
      k = grid_index(a, tb, k);
      // selection: first j with a_j > 0 and prefix_j > r2 * total (FP64
      // product; FP32 mode compares the widened binary32 prefixes).  The
      // a_j > 0 test matters at lane boundaries, where the scan's exclusive
      // value can exceed the previous lane's last prefix by rounding.
      const long long gb = obits(__dmul_rn(__longlong_as_double((long long)Ub), sel_total));
      int myfirst = -1;
#pragma unroll
      for (int q = MAXCH - 1; q >= 0; --q) {
        if (q < mine) {
          long long pb;
          bool pos;
          if constexpr (F32) {
            pb = obits(widen((lane == 0) ? run32[q] : __fadd_rn(excl32, run32[q])));
            pos = __float_as_uint(af[q]) != 0u;
          } else {
            pb = obits((lane == 0) ? run[q] : __dadd_rn(excl, run[q]));
            pos = obits(av[q]) > 0;
          }
          if (pos && pb > gb) myfirst = my0 + q;
        }
      }
      const unsigned hit = __ballot_sync(kFullMask, myfirst >= 0);
      int jsel;
      if (hit) {
        jsel = __shfl_sync(kFullMask, myfirst, __ffs(hit) - 1);
      } else {  // rounding left no j: the last reaction with a_j > 0
        int mylast = -1;
#pragma unroll
        for (int q = 0; q < MAXCH; ++q) {
          const bool pos = F32 ? (__float_as_uint(af[q]) != 0u) : (obits(av[q]) > 0);
          if (q < mine && pos) mylast = my0 + q;
        }
        const unsigned pos = __ballot_sync(kFullMask, mylast >= 0);
        jsel = __shfl_sync(kFullMask, mylast, 31 - __clz(pos));
      }
      // state change of jsel, one nonzero entry per lane
      const int q0 = s_nuptr[jsel], q1 = s_nuptr[jsel + 1];
      bool over = false;
      for (int e = q0 + lane; e < q1; e += 32)
        over |= (long long)xs[s_nuidx[e]] + (long long)s_nuval[e] > kStateMax;
      if (__any_sync(kFullMask, over)) {
        flags |= kWarpFlagOverflow;
        break;
      }
      __syncwarp();
      for (int e = q0 + lane; e < q1; e += 32) {
        const int s = s_nuidx[e];
        const int vv = s_nuval[e];
        const int xo = xs[s];
        const int xn = xo + vv;
        xs[s] = xn;
        maxx = max(maxx, xn);
        if (k < G) {
          atomicAdd(a.D1 + (size_t)k * S + s, (unsigned long long)(long long)vv);
          atomicAdd(a.D2 + (size_t)k * S + s, (unsigned long long)((2 * (long long)xo + vv) * (long long)vv));
        }
      }
      __syncwarp();
      t = t_next;
      ++n;
      hash = (hash ^ (unsigned long long)jsel) * kFnvPrime;
      hash = (hash ^ (unsigned long long)tb) * kFnvPrime;
      dirty = s_depw[jsel * 32 + lane];
      if ((long long)n == a.max_events) {
        flags |= kWarpFlagTruncated;
        break;
      }
    }
    // trajectory done
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) maxx = max(maxx, __shfl_xor_sync(kFullMask, maxx, off));
    if (lane == 0) {
      if (a.traj_events) a.traj_events[li] = (long long)n;
      if (a.traj_hash) a.traj_hash[li] = hash;
      if (a.traj_flags) a.traj_flags[li] = flags;
      atomicAdd(&blk[0], (unsigned long long)n);
      if (flags & kWarpFlagTruncated) atomicAdd(&blk[1], 1ULL);
      if (flags & kWarpFlagOverflow) atomicAdd(&blk[2], 1ULL);
      atomicMax(&blk[3], (unsigned long long)maxx);
    }
    __syncwarp();
  }

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

template <int MAXCH, bool F32>
cudaError_t launch_ch(const RunArgs& a, int blocks, int threads, size_t smem, cudaStream_t st) {
  k_ssa_warp<MAXCH, F32><<<blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MAXCH, bool F32>
cudaError_t prepare_ch(size_t smem, int threads, int* per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(k_ssa_warp<MAXCH, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ssa_warp<MAXCH, F32>, threads, smem);
}

template <bool F32>
cudaError_t prepare_prec(int M, size_t smem, int threads, int* per_sm) {
  switch (warp_max_chunk(M)) {
    case 1: return prepare_ch<1, F32>(smem, threads, per_sm);
    case 2: return prepare_ch<2, F32>(smem, threads, per_sm);
    case 4: return prepare_ch<4, F32>(smem, threads, per_sm);
    case 8: return prepare_ch<8, F32>(smem, threads, per_sm);
    case 16: return prepare_ch<16, F32>(smem, threads, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

template <bool F32>
cudaError_t launch_prec(const RunArgs& a, int blocks, int threads, size_t smem, cudaStream_t stream) {
  switch (warp_max_chunk(a.m.M)) {
    case 1: return launch_ch<1, F32>(a, blocks, threads, smem, stream);
    case 2: return launch_ch<2, F32>(a, blocks, threads, smem, stream);
    case 4: return launch_ch<4, F32>(a, blocks, threads, smem, stream);
    case 8: return launch_ch<8, F32>(a, blocks, threads, smem, stream);
    case 16: return launch_ch<16, F32>(a, blocks, threads, smem, stream);
    default: return cudaErrorInvalidValue;
  }
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
  return fp32 ? prepare_prec<true>(M, smem, threads, blocks_per_sm)
              : prepare_prec<false>(M, smem, threads, blocks_per_sm);
}

cudaError_t launch_warp_kernel(const RunArgs& a, bool fp32, int blocks, int threads, size_t smem,
                               cudaStream_t stream) {
  return fp32 ? launch_prec<true>(a, blocks, threads, smem, stream)
              : launch_prec<false>(a, blocks, threads, smem, stream);
}

}  // namespace ssa_impl
