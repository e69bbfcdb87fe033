// One trajectory of the direct method on one warp (schedule W32), shared by
// the single-network warp kernel (tables in shared memory) and the batched
// kernel (tables of many networks in global memory).
//
// Gillespie's direct method (Sec. 2) with the reactions spread over the 32
// lanes: lane l owns the contiguous chunk of ch = ceil(M / 32) reactions
// starting at l * ch and keeps their propensities in registers.  Summation
// schedule W32 (the oracle implements the same order):
//   part_l = left-to-right sum of lane l's chunk (0 for an empty lane);
//   inclusive Kogge-Stone scan of the parts with offsets 1, 2, 4, 8, 16
//     (v_l <- v_l + v_{l - off} for l >= off, all lanes reading the
//     previous step's values);
//   prefix_j = inner_j for lane 0, v_{l-1} + inner_j otherwise, with
//     inner_j the running sum inside the chunk up to j; a0 = v_31.
// Selection: each lane finds its first reaction with a_j > 0 and
// prefix_j > r2 a0; a ballot picks the lowest such lane (the first j
// overall).  After an event every lane reads its bits of the fired
// reaction's dependency mask (a per-reaction, per-lane table) and recomputes
// only those propensities.  The state x lives in shared memory (S counts per
// warp); the changes of the fired reaction are applied one per lane.  Events
// run in batches of 32: the random numbers of the batch are drawn at once,
// one per lane; the draws (selection and state update) run back to back, and
// the waiting times, event times, end of the trajectory and the bookkeeping
// of the kept events follow once per batch.
// Selective memory (Sec. 3.2.1) is the difference-sum scheme of the thread
// kernel: an event at time t changing x_s by v adds v and (2 x_s + v) v at
// the first grid index k with g_k >= t.
//
// FP32-propensity mode (F32): a_j = (float)c_j * (float)h_j in binary32,
// binary32 selection sums; a0 formed anew at every event from each lane's
// error-compensated binary32 chunk sum (Ogita-Rump-Oishi Sum2) kept as a
// binary32 pair, the lanes' pairs scanned in pair arithmetic (TwoSum heads,
// binary32 error sums) and lane 31's pair widened once to FP64 (lane b keeps
// event b's pair and widens it when the batch is settled); FP64 time;
// selection compares the binary32 prefixes with r2 times the binary32 total
// (an FP64 product) rounded down to binary32.
#ifndef SSA_WARP_STEP_CUH_
#define SSA_WARP_STEP_CUH_

#include <cstdint>

#include "ssa_thread_kernel.cuh"  // shared helpers: products, random numbers, tables

namespace ssa_impl {
namespace {

constexpr int kWarpFlagTruncated = 1;  // per-trajectory flag bits
constexpr int kWarpFlagOverflow = 2;
// Pre-event counts recorded per event of a batch (per-warp scratch of
// 32 x kRecPerEvent words): networks whose reactions change at most this
// many species each book their kept events lane-parallel.
constexpr int kRecPerEvent = 4;

// Exact binary32 -> binary64 widening of a non-negative value on the integer pipe.
__device__ __forceinline__ double widen(float f) {
  return __longlong_as_double((long long)ssa_sf::f32_to_f64(__float_as_uint(f)));
}

// Exact widening of any finite binary32 value (sign applied to the widened magnitude).
__device__ __forceinline__ double widen_signed(float f) {
  const uint32_t fb = __float_as_uint(f);
  const unsigned long long mag = ssa_sf::f32_to_f64(fb & 0x7FFFFFFFu);
  return __longlong_as_double((long long)(mag | ((unsigned long long)(fb >> 31) << 63)));
}

// Everything a warp needs to run trajectories of one network.
struct WarpNet {
  const int32_t* rinfo;               // [M] packed reactant words
  const unsigned long long* cbits;    // [M] rates (double bits)
  const float* c32;                   // [M] rates rounded to binary32 (FP32 mode)
  const int32_t* nu_ptr;              // [M + 1] CSR of nonzero net changes
  const int32_t* nu_idx;
  const int32_t* nu_val;
  const uint16_t* depw;               // [M * 32] per-lane dependency bits
  const int32_t* x0;                  // [S]
  const double* grid;                 // [G]
  unsigned long long* D1;             // [G * S] difference sums
  unsigned long long* D2;
  const int32_t* mod_f;               // [M] rate modifiers, or null (see DevModel)
  const double* mod_k;
  const double* mod_lo;
  const double* mod_hi;
  long long t_end_bits;
  int S, M, G;
  int nnz_max;                        // most species any reaction changes
  int grid_uniform;
  float grid_scale, grid_margin;
  uint32_t sid;                       // fourth Philox counter word
};

// Outcome of one trajectory (the same on every lane).
struct WarpTraj {
  uint32_t n;
  unsigned long long hash;
  int flags;
  int maxx;
};

// First index k' >= k with g_{k'} >= t (t given by its bits tb <= t_end), or
// G; the uniform-grid estimate is checked against the grid near cell edges.
__device__ __forceinline__ int grid_index_net(const WarpNet& net, long long tb, int k) {
  const int G = net.G;
  if (net.grid_uniform) {
    const float est = approx_float_rz(tb) * net.grid_scale;
    const float fl = floorf(est);
    const float fr = est - fl;
    int ke = min(max((int)fl + 1, k), G);
    if (fr > net.grid_margin && fr < 1.0f - net.grid_margin) return ke;
    if (ke > k && obits(__ldg(net.grid + ke - 1)) >= tb) --ke;
    if (ke > k && obits(__ldg(net.grid + ke - 1)) >= tb) --ke;
    if (ke < G && obits(__ldg(net.grid + ke)) < tb) ++ke;
    return ke;
  }
  while (k < G && obits(__ldg(net.grid + k)) < tb) ++k;
  return k;
}

// Dependency-bit table entry (j, l): bit q set when reaction l * ch + q
// reads a species that reaction j changes.
__host__ __device__ inline uint16_t depw_entry(const int32_t* dep_ptr, const int32_t* dep_idx, int ch, int j,
                                               int l) {
  uint32_t bits = 0;
  for (int q = dep_ptr[j]; q < dep_ptr[j + 1]; ++q) {
    const int kk = dep_idx[q];
    if (kk / ch == l) bits |= 1u << (kk - l * ch);
  }
  return (uint16_t)bits;
}

// Optional event log (selective memory along the time axis): every kept
// event writes one record per species it changes -- key = bits of the event
// time, species, change v and (2 x_old + v) v -- or one record with v = 0
// when it changes none.  A warp fills chunks of
// kLogChunk records taken from a global counter; the unused tail of a chunk
// holds the sentinel key kLogSentinel (sorted after every time).
// (EventLog, kLogChunk and kLogSentinel are declared in ssa_internal.h.)

// Per-warp position in the current chunk (identical on every lane).
struct WarpLogState {
  unsigned long long base;   // first slot of the chunk, or kLogSentinel when none
  int fill;
  bool failed;               // the capacity ran out: nothing more is written
  unsigned long long total;  // records of this warp's events (written or not)
};

// Makes room for `cnt` (<= kLogChunk) records in this warp's chunk: pads the
// old chunk's tail with sentinels and takes a new chunk when it is full.
// Returns false (every lane) when the capacity is exhausted.
__device__ __forceinline__ bool log_reserve(const EventLog& lg, WarpLogState& st, int cnt) {
  const int lane = threadIdx.x & 31;
  st.total += (unsigned long long)cnt;
  if (st.failed) return false;
  if (st.base != kLogSentinel && st.fill + cnt <= kLogChunk) return true;
  if (st.base != kLogSentinel) {
    for (int q = st.fill + lane; q < kLogChunk; q += 32) lg.key[st.base + q] = kLogSentinel;
    if (lane == 0) atomicAdd(lg.padded, (unsigned long long)(kLogChunk - st.fill));
  }
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(lg.counter, (unsigned long long)kLogChunk);
  b = __shfl_sync(kFullMask, b, 0);
  if (b + kLogChunk > lg.capacity) {
    if (lane == 0) atomicExch(lg.overflow, 1ULL);
    st.base = kLogSentinel;
    st.failed = true;
    return false;
  }
  st.base = b;
  st.fill = 0;
  return true;
}

// Pads the tail of the warp's last chunk (call once, when the warp is done).
__device__ __forceinline__ void log_close(const EventLog& lg, WarpLogState& st) {
  const int lane = threadIdx.x & 31;
  if (lane == 0 && st.total) atomicAdd(lg.needed, st.total);
  if (st.base == kLogSentinel) return;
  for (int q = st.fill + lane; q < kLogChunk; q += 32) lg.key[st.base + q] = kLogSentinel;
  if (lane == 0) atomicAdd(lg.padded, (unsigned long long)(kLogChunk - st.fill));
  st.base = kLogSentinel;
}

// Runs trajectory traj_id of `net` on the calling warp (all 32 lanes), with
// the state in xs[0..S) (shared memory, this warp's own).  MAXCH bounds the
// chunk ceil(M / 32) (registers only; the chunk itself is the runtime value).
// LOG: also write the event log (lg, lst).
// xrec: the warp's own scratch of 32 x kRecPerEvent words (pre-event counts).
template <int MAXCH, bool F32, bool LOG = false>
__device__ __forceinline__ WarpTraj warp_trajectory(const WarpNet& net, int32_t* xs, int32_t* xrec,
                                                    unsigned long long traj_id, uint32_t key0, uint32_t key1,
                                                    long long max_events, const uint64_t* s_inv,
                                                    const uint64_t* s_lnf, const EventLog* lg = nullptr,
                                                    WarpLogState* lst = nullptr) {
  const int lane = threadIdx.x & 31;
  const int S = net.S, M = net.M;
  // kept events booked lane-parallel from recorded pre-event counts (else the
  // serial walk back through the batch; the event log takes that path too)
  const bool fast = !LOG && net.nnz_max <= kRecPerEvent;
  const int ch = (M + 31) / 32;
  const int my0 = lane * ch;                          // first reaction of this lane
  const int mine = max(0, min(ch, M - my0));          // reactions this lane owns
  int maxx = 0;
  for (int s = lane; s < S; s += 32) {
    const int v = net.x0[s];
    xs[s] = v;
    maxx = max(maxx, v);
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

  // Batches of 32 events (lane b holds event base + b's random numbers).  The
  // draws run back to back: propensities, sums, selection and state update
  // only.  Then lane b forms event b's waiting time, the warp forms the event
  // times in order and finds where the trajectory ends (past t_end, overflow,
  // max_events, an absorbing state), undoes the later applied events, and
  // books the kept ones: grid indices, hash, and -- walking back through the
  // batch to recover each event's pre-event counts -- difference sums, log
  // records and the largest count.
  for (;;) {
    const uint32_t base = n;
    const EventRandom rr = event_random(base + (uint32_t)lane, traj_id, net.sid, key0, key1, s_inv, s_lnf);
    double my_a0 = 0.0;  // lane b: a0 of event b (FP64 mode)
    float my_s = 0.0f, my_e = 0.0f;  // lane b: a0 of event b as a binary32 pair (FP32 mode)
    int my_j = 0;        // lane b: reaction of event b
    int nb = 32;         // events applied (base .. base + nb - 1)
    int nrec = 32;       // events whose time is formed: the applied ones and the one that stopped the draws
#pragma unroll 1
    for (int b = 0; b < 32; ++b) {
      // propensities of this lane's reactions that the last event touched: a
      // loop over the lane's dirty slots, as many passes as the busiest lane
      // needs (an unrolled pass per slot would run every slot that any lane
      // needs), the value placed by a select chain so that the propensities
      // stay in registers
      for (uint32_t dm = dirty; __any_sync(kFullMask, dm != 0u);) {
        if (dm != 0u) {
          const int q = __ffs((int)dm) - 1;
          dm &= dm - 1u;
          const int j = my0 + q;
          const int32_t w = net.rinfo[j];
          const int kind = rinfo_kind(w);
          const long long xa = xs[rinfo_a(w)];
          const long long xb = xs[rinfo_b(w)];
          const long long bi = xa * ((kind == kBi) ? xb : (xa - 1));
          const long long h =
              (kind == kOrder0) ? 1LL : ((kind == kUni) ? xa : ((kind == kBi) ? bi : (bi >> 1)));
          // products on the FP32 pipe (FP32 mode) or as exact integer
          // arithmetic (FP64 mode: the SM's FP64 unit binds the warp kernel)
          if constexpr (F32) {
            const float v = __fmul_rn(net.c32[j], __ll2float_rn(h));
#pragma unroll
            for (int i = 0; i < MAXCH; ++i) af[i] = (i == q) ? v : af[i];
          } else {
            unsigned long long cb = net.cbits[j];
            if (net.mod_f != nullptr) {  // state-dependent rate: clamp(c + k x_f, lo, hi), FP64
              const int f = net.mod_f[j];
              if (f >= 0) {
                const double v = __dadd_rn(__longlong_as_double((long long)cb),
                                           __dmul_rn(net.mod_k[j], (double)xs[f]));
                cb = (unsigned long long)obits(fmin(fmax(v, net.mod_lo[j]), net.mod_hi[j]));
              }
            }
            unsigned long long ab;
            if (!propensity_int(cb, h, ab)) ab = propensity_fp64(cb, h);
            const double v = __longlong_as_double((long long)ab);
#pragma unroll
            for (int i = 0; i < MAXCH; ++i) av[i] = (i == q) ? v : av[i];
          }
        }
      }
      // schedule W32: running sums inside the chunk, Kogge-Stone scan of the
      // chunk sums, prefixes excl + inner.  A past-the-end a_j (lanes owning
      // fewer than ch reactions) is +0 and x + (+0) = x, so the last running
      // sum is the chunk sum (+0 for an empty lane).
      double run[MAXCH];   // FP64 mode: running sums
      float run32[MAXCH];  // FP32 mode: binary32 running sums
      double a0 = 0.0, excl = 0.0, sel_total;
      bool absorbing;  // every a_j is 0
      float excl32 = 0.0f;
      // loops over the chunk stop at ch (warp-uniform), the runtime chunk size
      if constexpr (F32) {
        // a0, formed anew each event: the lane's chunk summed left to right in
        // binary32 with its rounding errors carried (cascaded TwoSum), kept as
        // the pair (cs, cerr); the lanes' pairs scanned in pair arithmetic
        // (the Kogge-Stone pattern; heads by TwoSum, error parts added in
        // binary32).  A past-the-end a_j = +0 leaves both parts unchanged.
        // The head of TwoSum(a, b) is RN(a + b), so the heads are the binary32
        // selection sums of schedule W32 (running sums in the chunk, the
        // scan across lanes): one pass gives both.  Every value here is a
        // non-negative binary32, so the error of a sum is formed by Fast2Sum
        // on (max, min) -- exact when the first operand is the larger, and
        // the error of a rounded sum is unique, so the same bits as TwoSum's
        // with one operation fewer.
        float cs = af[0], cerr = 0.0f;
        run32[0] = cs;
#pragma unroll
        for (int q = 1; q < MAXCH; ++q) {
          if (q >= ch) break;
          const float x = af[q];
          const float hi = fmaxf(cs, x), lo = fminf(cs, x);
          const float tt = __fadd_rn(hi, lo);
          const float d = __fsub_rn(lo, __fsub_rn(tt, hi));
          cerr = __fadd_rn(cerr, d);
          cs = tt;
          run32[q] = tt;
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float us = __shfl_up_sync(kFullMask, cs, off);
          const float ue = __shfl_up_sync(kFullMask, cerr, off);
          if (lane >= off) {
            const float hi = fmaxf(cs, us), lo = fminf(cs, us);
            const float tt = __fadd_rn(hi, lo);
            const float d = __fsub_rn(lo, __fsub_rn(tt, hi));
            cerr = __fadd_rn(__fadd_rn(cerr, ue), d);
            cs = tt;
          }
        }
        excl32 = __shfl_up_sync(kFullMask, cs, 1);
        const float a0s = __shfl_sync(kFullMask, cs, 31);
        const float a0e = __shfl_sync(kFullMask, cerr, 31);
        sel_total = widen(a0s);
        if (lane == b) {
          my_s = a0s;
          my_e = a0e;
        }
        absorbing = __float_as_uint(a0s) == 0u;  // the head is +0 exactly when every a_j is 0
      } else {
        double v = av[0];
        run[0] = v;
#pragma unroll
        for (int q = 1; q < MAXCH; ++q) {
          if (q >= ch) break;
          v = __dadd_rn(v, av[q]);
          run[q] = v;
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const double u = __shfl_up_sync(kFullMask, v, off);
          if (lane >= off) v = __dadd_rn(v, u);
        }
        excl = __shfl_up_sync(kFullMask, v, 1);
        a0 = __shfl_sync(kFullMask, v, 31);
        sel_total = a0;
        absorbing = obits(a0) == 0;
      }
      if (!F32 && lane == b) my_a0 = a0;
      if (absorbing) {  // the event's time is +inf
        nb = b;
        nrec = b + 1;
        break;
      }
      // selection: first j with a_j > 0 and prefix_j > r2 * total (FP64
      // product).  The a_j > 0 test matters at lane boundaries, where the
      // scan's exclusive value can exceed the previous lane's last prefix by
      // rounding.  FP32 mode: for a binary32 p and a double T >= 0,
      // (double)p > T exactly when p > RD32(T), T rounded down to binary32, so
      // the widened comparison runs on the binary32 bit patterns.
      const unsigned long long Ub = __shfl_sync(kFullMask, rr.u2, b);
      const double target = __dmul_rn(__longlong_as_double((long long)Ub), sel_total);
      const long long gb = obits(target);
      unsigned gf = 0;
      if constexpr (F32) gf = __float_as_uint(__double2float_rd(target));
      int jsel = -1;
      if constexpr (!F32 && MAXCH >= 4) {
        // FP64 mode, chunks of 3 or more: a lane's prefixes do not decrease
        // along its chunk, so only a lane whose last prefix exceeds the
        // target can hold the first hit.  One addition per lane finds the
        // first such lane; lanes q < ch then form that lane's prefix q, one
        // each.  If that lane has no a_j > 0 past the target (rounding at a
        // lane boundary) every lane's prefixes are formed below.  Two FP64
        // additions per event instead of ch.
        if (ch >= 3) {
          double rl = run[0];
#pragma unroll
          for (int q = 1; q < MAXCH; ++q) {
            if (q >= ch) break;
            rl = run[q];
          }
          const double pl = (lane == 0) ? rl : __dadd_rn(excl, rl);
          const unsigned cand = __ballot_sync(kFullMask, mine > 0 && obits(pl) > gb);
          if (cand) {
            const int h = __ffs(cand) - 1;
            double rq = 0.0, aq = 0.0;
#pragma unroll
            for (int q = 0; q < MAXCH; ++q) {
              if (q >= ch) break;
              const double r_ = __shfl_sync(kFullMask, run[q], h);
              const double a_ = __shfl_sync(kFullMask, av[q], h);
              if (lane == q) {
                rq = r_;
                aq = a_;
              }
            }
            const double ex = __shfl_sync(kFullMask, excl, h);
            const int mine_h = max(0, min(ch, M - h * ch));
            bool hq = false;
            if (lane < mine_h) {
              const double pre = (h == 0) ? rq : __dadd_rn(ex, rq);
              hq = (obits(aq) > 0) && (obits(pre) > gb);
            }
            const unsigned hb = __ballot_sync(kFullMask, hq);
            if (hb) jsel = h * ch + __ffs(hb) - 1;
          }
        }
      }
      int myfirst = -1;
#pragma unroll
      for (int q = 0; q < MAXCH; ++q) {
        if (jsel >= 0 || q >= ch) break;
        bool hitq;
        if constexpr (F32) {
          const float pre = (lane == 0) ? run32[q] : __fadd_rn(excl32, run32[q]);
          hitq = (__float_as_uint(af[q]) != 0u) && (__float_as_uint(pre) > gf);
        } else {
          const double pre = (lane == 0) ? run[q] : __dadd_rn(excl, run[q]);
          hitq = (obits(av[q]) > 0) && (obits(pre) > gb);
        }
        if (hitq && myfirst < 0 && q < mine) myfirst = my0 + q;
      }
      const unsigned hit = (jsel >= 0) ? 0u : __ballot_sync(kFullMask, myfirst >= 0);
      if (jsel >= 0) {
        // found by the candidate lane above
      } else if (hit) {
        jsel = __shfl_sync(kFullMask, myfirst, __ffs(hit) - 1);
      } else {  // rounding left no j: the last reaction with a_j > 0
        int mylast = -1;
#pragma unroll
        for (int q = 0; q < MAXCH; ++q) {
          if (q >= ch) break;
          const bool pos = F32 ? (__float_as_uint(af[q]) != 0u) : (obits(av[q]) > 0);
          if (q < mine && pos) mylast = my0 + q;
        }
        const unsigned pos = __ballot_sync(kFullMask, mylast >= 0);
        jsel = __shfl_sync(kFullMask, mylast, 31 - __clz(pos));
      }
      if (lane == b) my_j = jsel;
      // state change of jsel, one nonzero entry per lane (the fast path
      // records the pre-event count of entry e in xrec[b][e])
      const int q0 = net.nu_ptr[jsel], q1 = net.nu_ptr[jsel + 1];
      bool over = false;
      for (int e = q0 + lane; e < q1; e += 32) {
        const int xo = xs[net.nu_idx[e]];
        over |= (long long)xo + (long long)net.nu_val[e] > kStateMax;
        if (fast) xrec[b * kRecPerEvent + (e - q0)] = xo;
      }
      if (__any_sync(kFullMask, over)) {  // not applied: the trajectory ends here unless past t_end
        nb = b;
        nrec = b + 1;
        break;
      }
      __syncwarp();
      for (int e = q0 + lane; e < q1; e += 32) xs[net.nu_idx[e]] += net.nu_val[e];
      __syncwarp();
      dirty = net.depw[jsel * 32 + lane];
    }

    // the event times in order (lane b: event b's waiting time; FP32 mode
    // widens its event's a0 pair here, once per batch)
    if constexpr (F32) my_a0 = __dadd_rn(widen(my_s), widen_signed(my_e));
    const double my_tau = quotient(rr.E, lane < nrec ? my_a0 : 1.0);  // a0 == 0: +inf
    double tt = t;
    long long my_tb = 0;
    int K = 0;      // events kept
    int endf = -1;  // the trajectory ends: 0 past t_end, 1 max_events, 2 overflow
    for (int b = 0; b < nrec && endf < 0; ++b) {
      const double t_b = __dadd_rn(tt, __shfl_sync(kFullMask, my_tau, b));
      const int j_b = __shfl_sync(kFullMask, my_j, b);
      const long long tb_b = obits(t_b);
      if (lane == b) my_tb = tb_b;
      if (tb_b > net.t_end_bits) {
        endf = 0;
      } else if (b == nb) {
        endf = 2;
      } else {
        K = b + 1;
        tt = t_b;
        hash = (hash ^ (unsigned long long)j_b) * kFnvPrime;  // the sequence hash, in order
        hash = (hash ^ (unsigned long long)tb_b) * kFnvPrime;
        if ((long long)base + K == max_events) endf = 1;
      }
    }
    // the applied events that were not kept, last first
    for (int b = nb - 1; b >= K; --b) {
      const int j = __shfl_sync(kFullMask, my_j, b);
      const int q0 = net.nu_ptr[j], q1 = net.nu_ptr[j + 1];
      for (int e = q0 + lane; e < q1; e += 32) xs[net.nu_idx[e]] -= net.nu_val[e];
      __syncwarp();
    }
    int kk = k;
    if (fast) {
      // lane b books kept event b: its grid index (searched from the batch's
      // starting index), difference sums from the recorded pre-event counts,
      // and the largest count; xs already holds the state after the kept events
      int my_k = k;
      if (lane < K) {
        my_k = grid_index_net(net, my_tb, k);
        const int q0 = net.nu_ptr[my_j], q1 = net.nu_ptr[my_j + 1];
        for (int e = q0; e < q1; ++e) {
          const int sp = net.nu_idx[e];
          const int vv = net.nu_val[e];
          const int xo = xrec[lane * kRecPerEvent + (e - q0)];
          maxx = max(maxx, xo + vv);
          if (my_k < net.G) {
            atomicAdd(net.D1 + (size_t)my_k * S + sp, (unsigned long long)(long long)vv);
            atomicAdd(net.D2 + (size_t)my_k * S + sp,
                      (unsigned long long)((2 * (long long)xo + vv) * (long long)vv));
          }
        }
      }
      kk = __shfl_sync(kFullMask, my_k, max(K - 1, 0));
      __syncwarp();
    } else {
      // grid indices (lane b: event b's), in order
      int my_k = k;
      for (int b = 0; b < K; ++b) {
        const long long tb_b = __shfl_sync(kFullMask, my_tb, b);
        kk = grid_index_net(net, tb_b, kk);
        if (lane == b) my_k = kk;
      }
      // kept events, last first: the counts before each one (walking the state
      // back), its difference sums and log records, the largest count
      for (int b = K - 1; b >= 0; --b) {
        const int j = __shfl_sync(kFullMask, my_j, b);
        const long long tb_b = __shfl_sync(kFullMask, my_tb, b);
        const int kb = __shfl_sync(kFullMask, my_k, b);
        const int q0 = net.nu_ptr[j], q1 = net.nu_ptr[j + 1];
        bool logged = false;
        // an event with no net change still adds its time to the union: one
        // record with v = 0 (species 0, no effect on the sums)
        const int nrc = (q1 > q0) ? (q1 - q0) : 1;
        if constexpr (LOG) {
          logged = log_reserve(*lg, *lst, nrc);
          if (logged && q1 == q0 && lane == 0) {
            const unsigned long long slot = lst->base + (unsigned long long)lst->fill;
            lg->key[slot] = (unsigned long long)tb_b;
            lg->rec[slot] = LogRec{0, 0, 0};
          }
        }
        for (int e = q0 + lane; e < q1; e += 32) {
          const int sp = net.nu_idx[e];
          const int vv = net.nu_val[e];
          const int xn = xs[sp];
          const int xo = xn - vv;
          xs[sp] = xo;
          maxx = max(maxx, xn);
          const long long d2 = (2 * (long long)xo + vv) * (long long)vv;
          if (kb < net.G) {
            atomicAdd(net.D1 + (size_t)kb * S + sp, (unsigned long long)(long long)vv);
            atomicAdd(net.D2 + (size_t)kb * S + sp, (unsigned long long)d2);
          }
          if constexpr (LOG) {
            if (logged) {
              const unsigned long long slot = lst->base + (unsigned long long)(lst->fill + (e - q0));
              lg->key[slot] = (unsigned long long)tb_b;
              lg->rec[slot] = LogRec{sp, vv, d2};
            }
          }
        }
        if constexpr (LOG) {
          if (logged) lst->fill += nrc;
        }
        __syncwarp();
      }
      // and forward again to the state after the kept events
      for (int b = 0; b < K; ++b) {
        const int j = __shfl_sync(kFullMask, my_j, b);
        const int q0 = net.nu_ptr[j], q1 = net.nu_ptr[j + 1];
        for (int e = q0 + lane; e < q1; e += 32) xs[net.nu_idx[e]] += net.nu_val[e];
        __syncwarp();
      }
    }
    if (K > 0) {
      t = tt;
      k = kk;
    }
    n += (uint32_t)K;
    if (endf >= 0) {
      flags |= (endf == 1) ? kWarpFlagTruncated : ((endf == 2) ? kWarpFlagOverflow : 0);
      break;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) maxx = max(maxx, __shfl_xor_sync(kFullMask, maxx, off));
  __syncwarp();
  return WarpTraj{n, hash, flags, maxx};
}

}  // namespace
}  // namespace ssa_impl

#endif  // SSA_WARP_STEP_CUH_
