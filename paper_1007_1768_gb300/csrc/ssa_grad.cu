// Likelihood-ratio rate sensitivities (ssa_ensemble_grad): every trajectory
// of the forward ensemble is replayed from its Philox counters -- nothing of
// the forward pass is stored -- and its score is accumulated against the
// loss's weights on the grid.
//
// Estimator (the score of a mass-action CTMC path): for reaction r,
//   Z_r(t) = N_r(t) / c_r - int_0^t h_r(x(s)) ds,
// and trajectory i contributes g_ir = sum_k u_k Z_r(g_k) with
//   u_k = sum_s w[k][s] (x_s(g_k) - m[k][s])   (w = dL/dmean, m = mean).
// dL/dc_r is the mean of g_ir over trajectories; its standard error is the
// sample standard deviation over sqrt(N).
//
// Replay form.  B_r = Z_r(t) + h_r(x(t)) t is constant between events (Z_r
// falls at rate h_r); an event at time tau firing j adds 1 / c_j to B_j, and
// every h_r the event changes adds (h_r' - h_r) tau to B_r.  Between two
// events the state is fixed, so the grid points g_k1 .. g_k2-1 of the
// interval contribute
//   sum_k u_k Z_r(g_k) = B_r U - h_r UG,   U = sum_k u_k,  UG = sum_k u_k g_k,
// and U, UG come from prefix sums over the grid of w, c = sum_s w m, g w and
// g c in O(S) per interval.  U and UG are added into running sums SU, SUG;
// reaction r's gradient takes B_r (SU - SU0_r) - h_r (SUG - SUG0_r) only when
// B_r or h_r is about to change (r fired or its propensity changed) and at
// the end, SU0_r / SUG0_r being the running sums at its previous update.
// B, the gradients and SU0 / SUG0 sit in per-thread shared-memory slots.  The
// oracle states the definition point by point; the two agree up to FP64
// rounding order.
//
// The trajectory itself is the thread kernel's: FP64 propensities, schedule
// L prefix sums, the same random numbers, selection and stopping rules.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "ssa.h"
#include "ssa_internal.h"
#include "ssa_thread_kernel.cuh"

namespace ssa_impl {
namespace {

struct GradArgs {
  SmallModel sm;
  double invc[kSmallMax];   // RN(1 / c_j)
  int32_t S, M, G;
  int64_t N;
  uint64_t traj_offset, seed, stream_id;
  int64_t max_events;
  double t_end;
  const double* grid;       // [G]
  const double* Pw;         // [(G + 1) x S] prefix sums over k of w[k][s]
  const double* Pgw;        // [(G + 1) x S] ... of g_k w[k][s]
  const double* Pc;         // [G + 1] ... of c_k = sum_s w[k][s] m[k][s]
  const double* Pgc;        // [G + 1] ... of g_k c_k
  double* gtraj;            // [M x N] per-trajectory contributions (column r at r * N)
  const unsigned int* order;  // [N] trajectory taken at each work index, or null (index order)
  unsigned long long* counter;
  int32_t grid_uniform;
  float grid_scale, grid_margin;
};

// First k' >= k with g_{k'} >= t (t given by its bits; t may exceed t_end or be +inf), or G.
__device__ __forceinline__ int grad_grid_index(const GradArgs& a, long long tb, int k) {
  const int G = a.G;
  if (tb > obits(a.t_end)) return G;  // every grid point lies at or before t_end
  if (a.grid_uniform) {
    const float est = approx_float_rz(tb) * a.grid_scale;
    const float fl = floorf(est);
    const float fr = est - fl;
    int ke = min(max((int)fl + 1, k), G);
    if (fr > a.grid_margin && fr < 1.0f - a.grid_margin) return ke;
    if (ke > k && obits(__ldg(a.grid + ke - 1)) >= tb) --ke;
    if (ke > k && obits(__ldg(a.grid + ke - 1)) >= tb) --ke;
    if (ke < G && obits(__ldg(a.grid + ke)) < tb) ++ke;
    return ke;
  }
  while (k < G && obits(__ldg(a.grid + k)) < tb) ++k;
  return k;
}

constexpr int kGradThreads = 128;

// (double)v for any int64: exact integer bit assembly for |v| < 2^53 (the
// counts, propensity factors and their changes met here), the hardware
// conversion out of line otherwise.  Same bits as the conversion, without
// issuing it on the SM's FP64 unit.
__device__ __forceinline__ double int_to_f64(long long v) {
  const unsigned long long mag = (v < 0) ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  double r = __longlong_as_double((long long)(small_int_to_f64_bits(mag) | (v < 0 ? (1ULL << 63) : 0ULL)));
  if (__builtin_expect(mag >= (1ULL << 53), 0)) r = ll2double_rare(v);
  return r;
}

// Per-thread score state in shared memory, slot (j, tid) at j * 128 + tid:
// B_j, the gradient g_j, the running interval sums at g_j's last update, and
// the propensity factor h_j.
struct GradSlots {
  double* B;
  double* g;
  double* su0;
  double* sug0;
  long long* h;
};

// g_j += B_j (SU - SU0_j) - h_j (SUG - SUG0_j): the intervals since B_j or h_j
// last changed, all with the same B_j and h_j.  The score's products and
// sums are fused (one rounding per multiply-add, half the FP64 instructions
// of separate ones; the contributions agree with the oracle's association
// to rounding either way).
__device__ __forceinline__ void flush_slot(const GradSlots& sl, int idx, double hj, double SU, double SUG) {
  const double g1 = __fma_rn(sl.B[idx], __dsub_rn(SU, sl.su0[idx]), sl.g[idx]);
  sl.g[idx] = __fma_rn(-hj, __dsub_rn(SUG, sl.sug0[idx]), g1);
  sl.su0[idx] = SU;
  sl.sug0[idx] = SUG;
}

template <int MAXM, int MAXS>
__global__ void __launch_bounds__(kGradThreads) k_ssa_grad(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char gsm[];
  uint64_t* s_inv = reinterpret_cast<uint64_t*>(gsm);
  uint64_t* s_lnf = s_inv + kLogCells;
  double* slots = reinterpret_cast<double*>(s_lnf + kLogCells);
  const int T = kGradThreads, tid = threadIdx.x;
  GradSlots sl{slots, slots + MAXM * T, slots + 2 * MAXM * T, slots + 3 * MAXM * T,
               reinterpret_cast<long long*>(slots + 4 * MAXM * T)};
  // tables read with a runtime reaction index: rates (bits), net changes,
  // dependency masks and reaction words
  unsigned long long* s_cbits = reinterpret_cast<unsigned long long*>(slots + 5 * MAXM * T);  // [MAXM]
  int32_t* s_nu = reinterpret_cast<int32_t*>(s_cbits + MAXM);       // [MAXM][MAXS]
  uint32_t* s_dep = reinterpret_cast<uint32_t*>(s_nu + MAXM * MAXS);  // [MAXM]
  int32_t* s_rinfo = reinterpret_cast<int32_t*>(s_dep + MAXM);      // [MAXM]
  for (int i = tid; i < kLogCells; i += T) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  for (int i = tid; i < MAXM * MAXS; i += T) s_nu[i] = a.sm.nu[(i / MAXS) * kSmallMax + (i % MAXS)];
  for (int j = tid; j < MAXM; j += T) {
    s_dep[j] = a.sm.depmask[j];
    s_cbits[j] = a.sm.cbits[j];
    s_rinfo[j] = a.sm.rinfo[j];
  }
  __syncthreads();
  const int S = a.S, M = a.M, G = a.G;
  const uint32_t key0 = (uint32_t)a.seed, key1 = (uint32_t)(a.seed >> 32), sid = (uint32_t)a.stream_id;
  for (;;) {
    const unsigned long long wi = atomicAdd(a.counter, 1ULL);
    if (wi >= (unsigned long long)a.N) break;
    const unsigned long long li = a.order ? (unsigned long long)a.order[wi] : wi;  // trajectory index
    const unsigned long long traj_id = a.traj_offset + li;
    int x[MAXS];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) x[s] = (s < S) ? a.sm.x0[s] : 0;
    double av[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      sl.h[j * T + tid] = 0;
      av[j] = 0.0;
      sl.B[j * T + tid] = 0.0;
      sl.g[j * T + tid] = 0.0;
      sl.su0[j * T + tid] = 0.0;
      sl.sug0[j * T + tid] = 0.0;
    }
    double SU = 0.0, SUG = 0.0;  // running sums of U and UG over the intervals so far
    uint32_t dirty = (1u << M) - 1u;
    int fired = -1;
    double t = 0.0;
    uint32_t n = 0;
    int k = 0;
    bool done = false;
    for (;;) {
      // the event at t: flush the score of the fired reaction and of every
      // reaction whose propensity it changed, then update B and h -- a loop
      // over this lane's reactions (a pass per reaction any lane of the warp
      // needs would run most of the M flushes every event); the propensity is
      // placed by a select chain so that it stays in a register
      const uint32_t dmask = dirty & ((1u << M) - 1u);
      for (uint32_t dm = dmask | (fired >= 0 ? (1u << fired) : 0u); dm != 0u;) {
        const int j = __ffs((int)dm) - 1;
        dm &= dm - 1u;
        const int idx = j * T + tid;
        const long long hj = sl.h[idx];
        flush_slot(sl, idx, int_to_f64(hj), SU, SUG);
        double Bj = sl.B[idx];
        if (j == fired) Bj = __dadd_rn(Bj, a.invc[j]);
        if ((dmask >> j) & 1u) {
          const long long hn = mass_action_h<MAXS>(s_rinfo[j], x);
          Bj = __fma_rn(int_to_f64(hn - hj), t, Bj);
          sl.h[idx] = hn;
          const double v = __longlong_as_double((long long)propensity_fp64(s_cbits[j], hn));
#pragma unroll
          for (int i = 0; i < MAXM; ++i) av[i] = (i == j) ? v : av[i];
        }
        sl.B[idx] = Bj;
      }
      if (done) break;
      // schedule L prefix sums
      double pre[MAXM];
      pre[0] = av[0];
#pragma unroll
      for (int j = 1; j < MAXM; ++j) pre[j] = (j < M) ? __dadd_rn(pre[j - 1], av[j]) : pre[j - 1];
      const double a0 = pre[MAXM - 1];  // entries past M repeat the last prefix
      const EventRandom r = event_random(n, traj_id, sid, key0, key1, s_inv, s_lnf);
      const double t_next = __dadd_rn(t, quotient(r.E, a0));  // a0 == 0: +inf
      const long long tb = obits(t_next);
      // grid points g_k < t_next see the current state: U and UG of the interval
      const int k2 = grad_grid_index(a, tb, k);
      if (k2 > k) {
        double U = __dsub_rn(a.Pc[k], a.Pc[k2]), UG = __dsub_rn(a.Pgc[k], a.Pgc[k2]);
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
          if (s < S) {
            const double xd = int_to_f64(x[s]);
            U = __fma_rn(xd, __dsub_rn(a.Pw[(size_t)k2 * S + s], a.Pw[(size_t)k * S + s]), U);
            UG = __fma_rn(xd, __dsub_rn(a.Pgw[(size_t)k2 * S + s], a.Pgw[(size_t)k * S + s]), UG);
          }
        }
        SU = __dadd_rn(SU, U);
        SUG = __dadd_rn(SUG, UG);
        k = k2;
      }
      if (tb > obits(a.t_end)) break;
      // selection: first j with a_j > 0 and prefix_j > r2 a0, else the last j with a_j > 0
      const long long gb = obits(__dmul_rn(__longlong_as_double((long long)r.u2), a0));
      int jsel = -1, jlast = -1;
#pragma unroll
      for (int j = MAXM - 1; j >= 0; --j) {
        if (j < M && obits(av[j]) > 0) {
          if (obits(pre[j]) > gb) jsel = j;
          if (jlast < 0) jlast = j;
        }
      }
      if (jsel < 0) jsel = jlast;
      bool over = false;
#pragma unroll
      for (int s = 0; s < MAXS; ++s)
        if (s < S) over |= (long long)x[s] + (long long)s_nu[jsel * MAXS + s] > kStateMax;
      if (over) break;  // the state stays; later grid points see it
#pragma unroll
      for (int s = 0; s < MAXS; ++s)
        if (s < S) x[s] += s_nu[jsel * MAXS + s];
      dirty = s_dep[jsel];
      fired = jsel;
      t = t_next;
      ++n;
      if ((long long)n == a.max_events) done = true;  // flush this event, then stop
    }
    // every later grid point sees the final state
    if (k < G) {
      double U = __dsub_rn(a.Pc[k], a.Pc[G]), UG = __dsub_rn(a.Pgc[k], a.Pgc[G]);
#pragma unroll
      for (int s = 0; s < MAXS; ++s) {
        if (s < S) {
          const double xd = int_to_f64(x[s]);
          U = __fma_rn(xd, __dsub_rn(a.Pw[(size_t)G * S + s], a.Pw[(size_t)k * S + s]), U);
          UG = __fma_rn(xd, __dsub_rn(a.Pgw[(size_t)G * S + s], a.Pgw[(size_t)k * S + s]), UG);
        }
      }
      SU = __dadd_rn(SU, U);
      SUG = __dadd_rn(SUG, UG);
    }
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < M) {
        const int idx = j * T + tid;
        flush_slot(sl, idx, int_to_f64(sl.h[idx]), SU, SUG);
        a.gtraj[(size_t)j * a.N + li] = sl.g[idx];
      }
    }
  }
}

// Prefix sums over the grid (one thread per column, sequential, fixed order):
// Pw[k][s] = sum_{k' < k} w[k'][s], Pgw with g_k' w[k'][s], Pc with
// c_k' = sum_s w[k'][s] m[k'][s], Pgc with g_k' c_k'.
__global__ void k_grad_prefix(const double* grid, const double* w, const double* mu, int G, int S, double* Pw,
                              double* Pgw, double* Pc, double* Pgc) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col < S) {
    double p = 0.0, pg = 0.0;
    Pw[col] = 0.0;
    Pgw[col] = 0.0;
    for (int k = 0; k < G; ++k) {
      const double v = w[(size_t)k * S + col];
      p = __dadd_rn(p, v);
      pg = __dadd_rn(pg, __dmul_rn(grid[k], v));
      Pw[(size_t)(k + 1) * S + col] = p;
      Pgw[(size_t)(k + 1) * S + col] = pg;
    }
  } else if (col == S) {
    double p = 0.0, pg = 0.0;
    Pc[0] = 0.0;
    Pgc[0] = 0.0;
    for (int k = 0; k < G; ++k) {
      double ck = 0.0;
      for (int s = 0; s < S; ++s) ck = __dadd_rn(ck, __dmul_rn(w[(size_t)k * S + s], mu[(size_t)k * S + s]));
      p = __dadd_rn(p, ck);
      pg = __dadd_rn(pg, __dmul_rn(grid[k], ck));
      Pc[k + 1] = p;
      Pgc[k + 1] = pg;
    }
  }
}

// Column r of gtraj: mean and standard error, in a fixed order (thread t sums
// rows t, t + 1024, ...; then a fixed tree), so repeated runs agree bit for bit.
__global__ void __launch_bounds__(1024) k_grad_reduce(const double* gtraj, long long N, double* grad, double* se) {
  __shared__ double s1[1024], s2[1024];
  const int r = blockIdx.x;
  const double* col = gtraj + (size_t)r * N;
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < N; i += blockDim.x) {
    const double v = col[i];
    a = __dadd_rn(a, v);
    b = __dadd_rn(b, __dmul_rn(v, v));
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      s1[threadIdx.x] = __dadd_rn(s1[threadIdx.x], s1[threadIdx.x + off]);
      s2[threadIdx.x] = __dadd_rn(s2[threadIdx.x], s2[threadIdx.x + off]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dN = (double)N;
    const double m = s1[0] / dN;
    grad[r] = m;
    if (se) {
      const double var = (N > 1) ? fmax((s2[0] - s1[0] * m) / (dN - 1.0), 0.0) : 0.0;
      se[r] = sqrt(var / dN);
    }
  }
}

// Work order, longest trajectories first, from the forward's event counts:
// buckets of 1/12 of a doubling of the count, in descending order; within a
// bucket, any order.  Only the schedule depends on it: each trajectory's
// contribution lands at its own index and the reduction runs in index order.
__device__ __forceinline__ int order_bucket(long long ev) {
  const float l = log2f((float)(ev < 0 ? 0 : ev) + 1.0f) * 12.0f;
  return 255 - min(255, (int)l);
}

__global__ void k_order_hist(const long long* ev, long long n, unsigned int* hist) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[order_bucket(ev[i])], 1u);
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// In place: exclusive scan of the 256 bucket counts (one block of 256).
__global__ void k_order_scan(unsigned int* hist) {
  __shared__ unsigned int v[256];
  v[threadIdx.x] = hist[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int run = 0;
    for (int i = 0; i < 256; ++i) {
      const unsigned int c = v[i];
      v[i] = run;
      run += c;
    }
  }
  __syncthreads();
  hist[threadIdx.x] = v[threadIdx.x];
}

__global__ void k_order_scatter(const long long* ev, long long n, unsigned int* next, unsigned int* order) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) order[atomicAdd(&next[order_bucket(ev[i])], 1u)] = (unsigned int)i;
}

// launch = false: only set the shared-memory size and report the blocks one
// SM holds (*per_sm).
template <int MAXM, int MAXS>
cudaError_t launch_grad_t(const GradArgs& a, int blocks, cudaStream_t st, bool launch, int* per_sm) {
  const size_t smem = (size_t)kLogCells * 16 + (size_t)5 * MAXM * kGradThreads * 8 + (size_t)MAXM * 8 +
                      (size_t)MAXM * MAXS * 4 + (size_t)MAXM * 4 + (size_t)MAXM * 4;
  cudaError_t e = cudaFuncSetAttribute(k_ssa_grad<MAXM, MAXS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (!launch)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ssa_grad<MAXM, MAXS>, kGradThreads, smem);
  k_ssa_grad<MAXM, MAXS><<<blocks, kGradThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MAXM>
cudaError_t launch_grad_m(const GradArgs& a, int blocks, cudaStream_t st, bool launch, int* per_sm) {
  switch (bucket_s(a.S)) {
    case 4: return launch_grad_t<MAXM, 4>(a, blocks, st, launch, per_sm);
    case 8: return launch_grad_t<MAXM, 8>(a, blocks, st, launch, per_sm);
    default: return launch_grad_t<MAXM, 16>(a, blocks, st, launch, per_sm);
  }
}

cudaError_t launch_grad(const GradArgs& a, int blocks, cudaStream_t st, bool launch = true, int* per_sm = nullptr) {
  if (a.M <= 4) return launch_grad_m<4>(a, blocks, st, launch, per_sm);
  if (a.M <= 8) return launch_grad_m<8>(a, blocks, st, launch, per_sm);
  if (a.M <= 12) return launch_grad_m<12>(a, blocks, st, launch, per_sm);
  return launch_grad_m<16>(a, blocks, st, launch, per_sm);
}

}  // namespace
}  // namespace ssa_impl

using namespace ssa_impl;

extern "C" ssa_status ssa_ensemble_grad(const ssa_model* model, int64_t n_traj, double t_end, int32_t n_grid,
                                        const double* grid, uint64_t seed, const ssa_run_opts* opts,
                                        const double* dL_dmean, const double* mean, double* dL_drates,
                                        double* dL_drates_se) {
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  if (!model || !dL_dmean || !mean || !dL_drates)
    return (ssa_status)set_error(SSA_EINVAL, "model, dL_dmean, mean and dL_drates must not be NULL");
  if (n_traj < 1) return (ssa_status)set_error(SSA_EINVAL, "n_traj must be >= 1");
  if (!(t_end > 0.0) || !std::isfinite(t_end)) return (ssa_status)set_error(SSA_EINVAL, "t_end must be finite and > 0");
  if (n_grid < 1) return (ssa_status)set_error(SSA_EINVAL, "n_grid must be >= 1");
  if (o.memory != SSA_MEM_HOST && o.memory != SSA_MEM_DEVICE) return (ssa_status)set_error(SSA_EINVAL, "bad memory kind");
  if (o.max_events <= 0) o.max_events = SSA_DEFAULT_MAX_EVENTS;
  if (o.max_events > (int64_t)0xFFFFFFFFLL) return (ssa_status)set_error(SSA_EINVAL, "max_events must be below 2^32");
  if (o.stream_id > 0xFFFFFFFFULL) return (ssa_status)set_error(SSA_EINVAL, "stream_id must be below 2^32");
  if (o.precision != SSA_PREC_FP64)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "gradients replay FP64 trajectories (SSA_PREC_FP64)");
  if (o.schedule == SSA_SCHED_WARP)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "gradients replay the thread schedule");
  ModelImageView mv;
  if (!model_image_view(model, &mv)) return (ssa_status)set_error(SSA_EINVAL, "bad model");
  if (mv.has_mod)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "gradients take plain mass-action models (no rate modifiers)");
  if (!mv.small)
    return (ssa_status)set_error(SSA_EUNSUPPORTED, "gradients take networks of at most 16 reactions and 16 species");
  const double* c = model_rates(model);
  for (int j = 0; j < mv.M; ++j)
    if (!(c[j] > 0.0))
      return (ssa_status)set_error(SSA_EUNSUPPORTED, "the likelihood-ratio score needs every rate > 0");
  const bool host = o.memory == SSA_MEM_HOST;
  const int S = mv.S, M = mv.M, G = n_grid;
  if (grid && host) {
    if (!(grid[0] >= 0.0)) return (ssa_status)set_error(SSA_EINVAL, "grid[0] must be >= 0");
    for (int k = 1; k < G; ++k)
      if (!(grid[k] >= grid[k - 1])) return (ssa_status)set_error(SSA_EINVAL, "grid must be ascending");
    if (!(grid[G - 1] <= t_end)) return (ssa_status)set_error(SSA_EINVAL, "grid values must be <= t_end");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
    return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(o.cuda_stream);

  // workspace: counter | grid | w | mu | Pw | Pgw | Pc | Pgc | out (2M) | gtraj (M N)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  const size_t gs = (size_t)G * S;
  const size_t o_counter = take(8), o_grid = take(8 * (size_t)G), o_w = take(8 * gs), o_mu = take(8 * gs),
               o_Pw = take(8 * (gs + S)), o_Pgw = take(8 * (gs + S)), o_Pc = take(8 * ((size_t)G + 1)),
               o_Pgc = take(8 * ((size_t)G + 1)), o_out = take(16 * (size_t)M),
               o_gtraj = take(8 * (size_t)M * (size_t)n_traj);
  // optional work order from the forward's event counts (opts->traj_events)
  const bool ordered = o.traj_events != nullptr;
  if (ordered && n_traj > (int64_t)0xFFFFFFFFLL)
    return (ssa_status)set_error(SSA_EINVAL, "a work order takes at most 2^32 - 1 trajectories");
  const size_t o_order = ordered ? take(4 * (size_t)n_traj) : 0, o_hist = ordered ? take(4 * 256) : 0,
               o_ev = (ordered && host) ? take(8 * (size_t)n_traj) : 0;
  unsigned char* ws = nullptr;
  if ((e = pool_malloc(reinterpret_cast<void**>(&ws), off, st)) != cudaSuccess)
    return (ssa_status)set_error(SSA_ENOMEM, cudaGetErrorString(e));
  auto fail_cuda = [&](cudaError_t err) {
    cudaFreeAsync(ws, st);
    return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(err));
  };
#define SSA_G_TRY(expr)                       \
  do {                                        \
    const cudaError_t e_ = (expr);            \
    if (e_ != cudaSuccess) return fail_cuda(e_); \
  } while (0)
  SSA_G_TRY(cudaMemsetAsync(ws + o_counter, 0, 8, st));
  double* d_grid = reinterpret_cast<double*>(ws + o_grid);
  const double* w = dL_dmean;
  const double* mu = mean;
  if (!grid) {
    SSA_G_TRY(launch_uniform_grid(d_grid, G, t_end, st));
  } else if (host) {
    SSA_G_TRY(cudaMemcpyAsync(d_grid, grid, 8 * (size_t)G, cudaMemcpyHostToDevice, st));
  } else {
    SSA_G_TRY(cudaMemcpyAsync(d_grid, grid, 8 * (size_t)G, cudaMemcpyDeviceToDevice, st));
  }
  if (host) {
    SSA_G_TRY(cudaMemcpyAsync(ws + o_w, dL_dmean, 8 * gs, cudaMemcpyHostToDevice, st));
    SSA_G_TRY(cudaMemcpyAsync(ws + o_mu, mean, 8 * gs, cudaMemcpyHostToDevice, st));
    w = reinterpret_cast<const double*>(ws + o_w);
    mu = reinterpret_cast<const double*>(ws + o_mu);
  }
  double* Pw = reinterpret_cast<double*>(ws + o_Pw);
  double* Pgw = reinterpret_cast<double*>(ws + o_Pgw);
  double* Pc = reinterpret_cast<double*>(ws + o_Pc);
  double* Pgc = reinterpret_cast<double*>(ws + o_Pgc);
  k_grad_prefix<<<1, ((S + 1 + 31) / 32) * 32, 0, st>>>(d_grid, w, mu, G, S, Pw, Pgw, Pc, Pgc);
  SSA_G_TRY(cudaGetLastError());

  GradArgs a;
  std::memcpy(&a.sm, mv.small, sizeof(SmallModel));
  for (int j = 0; j < kSmallMax; ++j) a.invc[j] = (j < M) ? 1.0 / c[j] : 0.0;
  a.S = S;
  a.M = M;
  a.G = G;
  a.N = n_traj;
  a.traj_offset = o.traj_offset;
  a.seed = seed;
  a.stream_id = o.stream_id;
  a.max_events = o.max_events;
  a.t_end = t_end;
  a.grid = d_grid;
  a.Pw = Pw;
  a.Pgw = Pgw;
  a.Pc = Pc;
  a.Pgc = Pgc;
  a.gtraj = reinterpret_cast<double*>(ws + o_gtraj);
  a.order = nullptr;
  // Longest first pays when lanes take several trajectories each; when every
  // trajectory has a lane from the start it would only crowd the longest into
  // the first blocks (and SMs), so the natural order stays.
  int per_sm = 0;
  a.M = M;
  a.S = S;
  SSA_G_TRY(launch_grad(a, 0, st, false, &per_sm));
  const long long resident = (long long)std::max(per_sm, 1) * prop.multiProcessorCount * kGradThreads;
  if (ordered && n_traj >= 4 * resident) {
    const long long* ev = reinterpret_cast<const long long*>(o.traj_events);
    if (host) {
      SSA_G_TRY(cudaMemcpyAsync(ws + o_ev, o.traj_events, 8 * (size_t)n_traj, cudaMemcpyHostToDevice, st));
      ev = reinterpret_cast<const long long*>(ws + o_ev);
    }
    unsigned int* hist = reinterpret_cast<unsigned int*>(ws + o_hist);
    unsigned int* order = reinterpret_cast<unsigned int*>(ws + o_order);
    SSA_G_TRY(cudaMemsetAsync(hist, 0, 4 * 256, st));
    const int hb = (int)std::min<long long>((n_traj + 255) / 256, 4LL * prop.multiProcessorCount);
    k_order_hist<<<hb, 256, 0, st>>>(ev, n_traj, hist);
    SSA_G_TRY(cudaGetLastError());
    k_order_scan<<<1, 256, 0, st>>>(hist);
    SSA_G_TRY(cudaGetLastError());
    k_order_scatter<<<(unsigned)((n_traj + 255) / 256), 256, 0, st>>>(ev, n_traj, hist, order);
    SSA_G_TRY(cudaGetLastError());
    a.order = order;
  }
  a.counter = reinterpret_cast<unsigned long long*>(ws + o_counter);
  const bool uniform = !grid || (host && host_grid_is_uniform(grid, G, t_end));
  a.grid_uniform = (uniform && G >= 2 && G <= (1 << 20) && t_end < 1e30) ? 1 : 0;
  a.grid_scale = (float)((double)(G - 1) / t_end);
  a.grid_margin = (float)((double)G * 0x1p-21);
  const long long want = (n_traj + 127) / 128;
  const long long cap = (long long)prop.multiProcessorCount * 8;
  const int blocks = (int)(want < cap ? want : cap);
  if (o.sim_event_begin) SSA_G_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_begin), st));
  SSA_G_TRY(launch_grad(a, blocks, st));
  if (o.sim_event_end) SSA_G_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_end), st));
  double* d_out = reinterpret_cast<double*>(ws + o_out);
  k_grad_reduce<<<M, 1024, 0, st>>>(a.gtraj, (long long)n_traj, host ? d_out : dL_drates,
                                     host ? d_out + M : dL_drates_se);
  SSA_G_TRY(cudaGetLastError());
  if (host) {
    SSA_G_TRY(cudaMemcpyAsync(dL_drates, d_out, 8 * (size_t)M, cudaMemcpyDeviceToHost, st));
    if (dL_drates_se) SSA_G_TRY(cudaMemcpyAsync(dL_drates_se, d_out + M, 8 * (size_t)M, cudaMemcpyDeviceToHost, st));
  }
  if (o.workspace != nullptr) {  // per-trajectory contributions requested
    if (o.workspace_bytes < 8 * (size_t)M * (size_t)n_traj) {
      cudaFreeAsync(ws, st);
      return (ssa_status)set_error(SSA_EINVAL, "opts->workspace must hold 8 * n_reactions * n_traj bytes");
    }
    SSA_G_TRY(cudaMemcpyAsync(o.workspace, a.gtraj, 8 * (size_t)M * (size_t)n_traj,
                              host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  }
  SSA_G_TRY(cudaFreeAsync(ws, st));
  if (host) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  }
#undef SSA_G_TRY
  return SSA_OK;
}
