// The simulation kernel for small networks (at most 16 reactions and 16
// species).  Included by ssa_thread_s{4,8,16}.cu and, for the logging
// variants, ssa_thread_log_s{4,8,16}.cu, each of which instantiates it for one
// species bucket so the builds run in parallel; the warp kernel, the batch
// kernel and the gradient replay include it for its helpers (propensity
// products, random numbers, quotient, grid index).
//
// Gillespie's direct method (Sec. 2), one trajectory per lane; lanes take
// trajectory ids from a global work counter.
//   * The state x, the propensities a_j (double bit patterns) and the
//     left-to-right prefix sums are registers (MAXS / MAXM are template
//     bounds).  Per-reaction tables read with a constant index come from the
//     kernel parameters; those read with the fired reaction's index (net
//     change rows, dependency masks) from shared memory.
//   * After an event only the propensities it touched are recomputed (mask
//     from the dependency graph).
//   * a0 and the prefix sums are left-to-right FP64 sums; comparisons run on
//     double bit patterns.
//   * The loop is software-pipelined by one event: the event drawn in one
//     iteration is applied to x at once, and kept or undone in the next
//     iteration, once its time (E / a0 resolves meanwhile) is compared with
//     t_end.  The kept sequence is exactly the plain loop's.
//   * Selective memory (Sec. 3.2.1): a kept event at time t adds v and
//     (2 x_old + v) v to the difference sums D1 / D2 at the first grid index
//     with g_k >= t, for every species it changes by v; the finalize kernel
//     scans them along the grid.
//   * LOG (the Avg-Y / Avg-XY pipeline): a kept event also writes one record
//     (time bits, species, v, (2 x_old + v) v) per species it changes -- one
//     record with v = 0 when it changes none -- into the lane's current
//     chunk of kThreadLogChunk slots of the event log.
//
// The products c_j h_j run on the FP64 unit, only for the reactions the last
// event touched; the quotient E / a0 runs as exact integer arithmetic
// (ssa_softfloat.cuh).  (Integer products for every reaction in full warps
// were measured slower: with them the integer ALU pipe, not the FP64 unit,
// bounds a full GPU.)  Two per-warp regimes give the same bits:
//   * one trajectory per lane;
//   * cooperative (at most 16 trajectories left and no new work): groups of
//     2, 4, 8, 16 or 32 lanes run one trajectory each in batches of speculative
//     rounds -- every lane evaluates the next selection from the state a
//     path of likely reactions would reach, so one prefix chain fires
//     several events -- then settle the batch's times, grid sums and records
//     lane-parallel (described at coop_run below).  This cuts the latency per
//     event of the long trajectories that end the run.
#ifndef SSA_THREAD_KERNEL_CUH_
#define SSA_THREAD_KERNEL_CUH_

#include <cstdint>

#include "ssa_device.cuh"
#include "ssa_internal.h"
#include "ssa_logtab.h"
#include "ssa_softfloat.cuh"

namespace ssa_impl {
namespace {

using ssa_dev::obits;

__device__ const ssa_logtab::Tables d_log_tables = ssa_logtab::kTables;

constexpr unsigned long long kFnvOffset = 0xcbf29ce484222325ULL;
constexpr unsigned long long kFnvPrime = 0x100000001b3ULL;
constexpr long long kStateMax = 2147483647LL;
constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kCoopMaxTraj = 16;   // at most this many trajectories left: cooperative mode

// x[s] for a runtime species index s < MAXS (select chain over registers).
template <int MAXS>
__device__ __forceinline__ int xget(const int (&x)[MAXS], int s) {
  int v = x[0];
#pragma unroll
  for (int i = 1; i < MAXS; ++i) v = (s == i) ? x[i] : v;
  return v;
}

// h_j(x) for a packed reaction word (branch-free: every form is formed and
// the reaction's kind selects one).
template <int MAXS>
__device__ __forceinline__ long long mass_action_h(int32_t w, const int (&x)[MAXS]) {
  const int kind = rinfo_kind(w);
  const long long xa = xget<MAXS>(x, rinfo_a(w));
  const long long xb = xget<MAXS>(x, rinfo_b(w));
  const long long bi = xa * ((kind == kBi) ? xb : (xa - 1));  // x_a x_b, or x_a (x_a - 1)
  const long long two = (kind == kBi) ? bi : (bi >> 1);
  return (kind == kOrder0) ? 1LL : ((kind == kUni) ? xa : two);
}

// Exact (double)v for 0 <= v < 2^53, integer ops only.
__device__ __forceinline__ unsigned long long small_int_to_f64_bits(unsigned long long v) {
  const int lz = __clzll((long long)(v | 1ULL));
  const unsigned long long r = ((unsigned long long)(1086 - lz) << 52) + ((v << lz) >> 11) - (1ULL << 52);
  return (v == 0ULL) ? 0ULL : r;
}

// a_j = RN(c_j * h) as bits, exact integer product.  Returns false when the
// product needs the hardware path (h >= 2^53, subnormal or overflowing cases).
__device__ __forceinline__ bool propensity_int(unsigned long long cbits, long long h, unsigned long long& out) {
  bool ok;
  const unsigned long long r = ssa_sf::mul_u53(cbits, (unsigned long long)h & ((1ULL << 53) - 1), ok);
  out = r;
  return ok && (unsigned long long)h < (1ULL << 53);
}

// (double)h for h outside [0, 2^53) (counts far beyond any seen in practice).
// Kept out of line: as a select operand the conversion would be issued for
// every product.
__device__ __noinline__ double ll2double_rare(long long h) { return __ll2double_rn(h); }

// a_j = RN(c_j * h) as bits with the hardware multiply.
__device__ __forceinline__ unsigned long long propensity_fp64(unsigned long long cbits, long long h) {
  double hd = __longlong_as_double((long long)small_int_to_f64_bits((unsigned long long)h));
  if (__builtin_expect((unsigned long long)h >= (1ULL << 53), 0)) hd = ll2double_rare(h);
  return (unsigned long long)obits(__dmul_rn(__longlong_as_double((long long)cbits), hd));
}

// A float at or below the non-negative double with bits `b`, within 2^-23
// relative (integer ops only; 0 below float's normal range).  Only used for
// the grid index estimate, which is checked against the grid when close to
// a cell boundary.
__device__ __forceinline__ float approx_float_rz(long long b) {
  const int e = (int)(b >> 52) - 1023 + 127;
  const int f = (e << 23) | (int)((b >> 29) & 0x7FFFFF);
  return __int_as_float(e <= 0 ? 0 : (e >= 255 ? 0x7F800000 : f));
}

// First index k' >= k with g_{k'} >= t (t given by its bits tb <= t_end), or G.
__device__ __forceinline__ int grid_index(const RunArgs& a, long long tb, int k) {
  const int G = a.G;
  if (a.grid_uniform) {
    // x = t (G - 1) / t_end; the estimate is within (G - 1) 2^-22 of x and
    // the grid points within G 2^-50 (in index units) of k t_end / (G - 1):
    // away from integers by more than grid_margin, ceil(estimate) is exact.
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

// Per-lane position in the event log.
struct ThreadLog {
  unsigned long long base;    // first slot of the lane's chunk, or kLogSentinel when none
  int fill;
  bool failed;                // the capacity ran out: nothing more is written
  unsigned long long total;   // records of this lane's events (written or not)
  unsigned long long padded;  // sentinel slots this lane wrote
};

// Makes room for `cnt` (<= kThreadLogChunk) records: pads the old chunk's
// tail with sentinels and takes a new chunk when it is full.  Returns false
// when the capacity is exhausted.
__device__ __forceinline__ bool thread_log_reserve(const EventLog& lg, ThreadLog& tl, int cnt) {
  tl.total += (unsigned long long)cnt;
  if (tl.failed) return false;
  if (tl.base != kLogSentinel && tl.fill + cnt <= kThreadLogChunk) return true;
  if (tl.base != kLogSentinel) {
    for (int q = tl.fill; q < kThreadLogChunk; ++q) lg.key[tl.base + q] = kLogSentinel;
    tl.padded += (unsigned long long)(kThreadLogChunk - tl.fill);
  }
  const unsigned long long b = atomicAdd(lg.counter, (unsigned long long)kThreadLogChunk);
  if (b + kThreadLogChunk > lg.capacity) {
    atomicExch(lg.overflow, 1ULL);
    tl.base = kLogSentinel;
    tl.failed = true;
    return false;
  }
  tl.base = b;
  tl.fill = 0;
  return true;
}

// The records of a kept event at time bits tb; x is the state after it and
// pv its change.
template <int MAXS>
__device__ __forceinline__ void thread_log_event(const EventLog& lg, ThreadLog& tl, long long tb,
                                                 const int (&x)[MAXS], const int (&pv)[MAXS]) {
  int nrec = 0;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) nrec += (pv[s] != 0) ? 1 : 0;
  const bool none = nrec == 0;
  nrec = none ? 1 : nrec;
  if (!thread_log_reserve(lg, tl, nrec)) return;
  unsigned long long slot = tl.base + (unsigned long long)tl.fill;
  if (none) {
    lg.key[slot] = (unsigned long long)tb;
    lg.rec[slot] = LogRec{0, 0, 0};
  }
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    if (pv[s] != 0) {
      const long long xo = (long long)x[s] - pv[s];
      lg.key[slot] = (unsigned long long)tb;
      lg.rec[slot] = LogRec{s, pv[s], (2 * xo + pv[s]) * (long long)pv[s]};
      ++slot;
    }
  }
  tl.fill += nrec;
}

// Pads the tail of the lane's last chunk (once, when the lane is done).
__device__ __forceinline__ void thread_log_close(const EventLog& lg, ThreadLog& tl) {
  if (tl.base == kLogSentinel) return;
  for (int q = tl.fill; q < kThreadLogChunk; ++q) lg.key[tl.base + q] = kLogSentinel;
  tl.padded += (unsigned long long)(kThreadLogChunk - tl.fill);
  tl.base = kLogSentinel;
}

// Random numbers of event n of a trajectory: E = -ln(r1) and r2 = q2 2^-53,
// both as double bit patterns.
struct EventRandom {
  unsigned long long E;
  unsigned long long u2;
};

__device__ __forceinline__ EventRandom event_random(uint32_t n, unsigned long long traj_id, uint32_t stream,
                                                    uint32_t k0, uint32_t k1, const uint64_t* s_inv,
                                                    const uint64_t* s_lnf) {
  const ssa_dev::Words4 w =
      ssa_dev::philox4x32_10(n, (uint32_t)traj_id, (uint32_t)(traj_id >> 32), stream, k0, k1);
  EventRandom r;
  r.E = ssa_dev::neg_log_u_bits(ssa_dev::odd53(w.w0, w.w1), s_inv, s_lnf);
  r.u2 = small_int_to_f64_bits(ssa_dev::odd53(w.w2, w.w3)) - (53ULL << 52);
  return r;
}

// Everything one trajectory carries between iterations.
template <int MAXM, int MAXS>
struct Traj {
  int x[MAXS];
  int pv[MAXS];                 // state change of the pending event
  unsigned long long av[MAXM];  // propensities (bits)
  double pre[MAXM];             // prefix sums
  uint32_t dirty;               // propensities to recompute
  bool have;
  long long li;                 // index in this launch
  unsigned long long traj_id;   // global id (Philox counter)
  double t;
  uint32_t n;                   // events kept so far
  int k;                        // grid index of the last kept event
  unsigned long long hash;
  int maxx;
  int flags;
  EventRandom rnd;              // random numbers of the event to draw next (thread mode)
  bool pend;                    // an event was drawn and applied, not yet settled
  bool pend_over;               // it would leave the int32 range: not applied
  int pend_j;
  unsigned long long pend_E;    // its -ln(r1) (bits); its time is t + pend_E / pend_a0
  double pend_a0;
};

// Per-launch constants of the step.
struct StepEnv {
  int M, S, G;
  long long t_end_bits;
  uint32_t key0, key1, sid;
  const uint64_t* s_inv;
  const uint64_t* s_lnf;
  const int32_t* s_nu;
  const uint32_t* s_depmask;
  const uint32_t* s_rmask;      // per species: the reactions whose propensity reads it
  const int32_t* s_rinfo;       // reaction words (read with a runtime reaction index)
  const unsigned long long* s_cbits;  // rates as double bit patterns (same)
  unsigned long long* d1;
  unsigned long long* d2;
};

template <int MAXM, int MAXS>
__device__ __forceinline__ void start_trajectory(const RunArgs& a, const StepEnv& e, Traj<MAXM, MAXS>& q,
                                                 unsigned long long next) {
  q.have = true;
  q.li = (long long)next;
  q.traj_id = a.traj_offset + next;
  q.maxx = 0;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    q.x[s] = (s < e.S) ? a.sm.x0[s] : 0;
    q.maxx = max(q.maxx, q.x[s]);
  }
  q.t = 0.0;
  q.n = 0;
  q.k = 0;
  q.hash = kFnvOffset;
  q.flags = 0;
  q.dirty = (1u << MAXM) - 1u;
  q.pend = false;
  q.pend_over = false;
  q.pend_j = 0;
  q.pend_E = 0ULL;
  q.pend_a0 = 0.0;
}

// The hardware division, for the rare operands the integer quotient does not
// cover (a0 == 0 gives +inf: the state is absorbing).  Out of line and behind
// a branch: as a select operand it would be issued (hundreds of cycles) for
// every quotient.
__device__ __noinline__ double quotient_rare(unsigned long long Eb, double a0) {
  return __ddiv_rn(__longlong_as_double((long long)Eb), a0);
}

// tau = RN(E / a0) as a double: the exact integer quotient (branch-free, so
// its instructions fill the stalls of the prefix chain it is issued with).
__device__ __forceinline__ double quotient(unsigned long long Eb, double a0) {
  bool ok;
  const unsigned long long qb = ssa_sf::div_pos(Eb, (unsigned long long)obits(a0), ok);
  double q = __longlong_as_double((long long)qb);
  if (__builtin_expect(!ok, 0)) q = quotient_rare(Eb, a0);
  return q;
}

// Prefix sums and a0 from the propensities, left to right.
template <int MAXM, int MAXS>
__device__ __forceinline__ double prefix_sums(int M, Traj<MAXM, MAXS>& q) {
  q.pre[0] = __longlong_as_double((long long)q.av[0]);
  if (M == MAXM) {  // the bucket's own size: a plain chain
#pragma unroll
    for (int j = 1; j < MAXM; ++j) q.pre[j] = __dadd_rn(q.pre[j - 1], __longlong_as_double((long long)q.av[j]));
  } else {
#pragma unroll
    for (int j = 1; j < MAXM; ++j) {
      if (j < M) q.pre[j] = __dadd_rn(q.pre[j - 1], __longlong_as_double((long long)q.av[j]));
      else q.pre[j] = q.pre[j - 1];
    }
  }
  return q.pre[MAXM - 1];
}

// Settle the pending event, whose waiting time is tau: keep it (grid index,
// difference sums and, LOG, the event-log records when `emit`, time, count,
// hash) or, past t_end, undo it.
// Returns true when the trajectory ends (flags set).
template <bool LOG, int MAXM, int MAXS>
__device__ __forceinline__ bool settle(const RunArgs& a, const StepEnv& e, Traj<MAXM, MAXS>& q, double tau,
                                       bool emit, const EventLog& lg, ThreadLog& tl) {
  const double t_next = __dadd_rn(q.t, tau);
  const long long tb = obits(t_next);
  const bool beyond = q.pend && tb > e.t_end_bits;  // not fired: undo
  const bool keep = q.pend && !beyond && !q.pend_over;
  const bool undo = beyond && !q.pend_over;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) q.x[s] -= undo ? q.pv[s] : 0;
  if (keep) q.k = grid_index(a, tb, q.k);
  const bool in_grid = emit && keep && q.k < e.G;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    const bool ch = keep && q.pv[s] != 0;
    q.maxx = ch ? max(q.maxx, q.x[s]) : q.maxx;
    if (in_grid && q.pv[s] != 0) {
      const long long xo = (long long)q.x[s] - q.pv[s];
      atomicAdd(e.d1 + (size_t)q.k * e.S + s, (unsigned long long)(long long)q.pv[s]);
      atomicAdd(e.d2 + (size_t)q.k * e.S + s, (unsigned long long)((2 * xo + q.pv[s]) * (long long)q.pv[s]));
    }
  }
  if constexpr (LOG) {
    if (emit && keep) thread_log_event<MAXS>(lg, tl, tb, q.x, q.pv);
  }
  q.t = keep ? t_next : q.t;
  q.n += keep ? 1u : 0u;
  const unsigned long long h1 = (q.hash ^ (unsigned long long)q.pend_j) * kFnvPrime;
  const unsigned long long h2 = (h1 ^ (unsigned long long)tb) * kFnvPrime;
  q.hash = keep ? h2 : q.hash;
  const bool trunc = keep && (long long)q.n == a.max_events;
  const bool over_end = q.pend && !beyond && q.pend_over;
  q.flags = (trunc ? 1 : 0) | (over_end ? 2 : 0);
  q.pend = false;
  return beyond || over_end || trunc;
}

// Draw the next event with random numbers r: target r2 a0, selection, and
// the state update applied at once.  Its time t + E / a0 is formed and
// checked against t_end in the next iteration.
template <int MAXM, int MAXS>
__device__ __forceinline__ void draw(const StepEnv& e, Traj<MAXM, MAXS>& q, double a0, const EventRandom& r,
                                     bool done) {
  const long long gb = obits(__dmul_rn(__longlong_as_double((long long)r.u2), a0));
  // first j with prefix_j > target (prefixes are non-decreasing)
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < MAXM; ++j) {
    if (j < e.M) cnt += (obits(q.pre[j]) <= gb) ? 1 : 0;
  }
  int jsel = cnt;
  if (cnt >= e.M) {  // rounding left no j (or a0 == 0): the last reaction with a_j > 0
    jsel = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < e.M && q.av[j] != 0ULL) jsel = j;
    }
  }
  const int* row = e.s_nu + jsel * MAXS;
  bool over = false;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    q.pv[s] = row[s];
    over |= (long long)q.x[s] + (long long)q.pv[s] > kStateMax;
  }
  const bool apply = !done && !over;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) q.x[s] += apply ? q.pv[s] : 0;
  q.pend = !done;
  q.pend_over = over;
  q.pend_j = jsel;
  q.pend_E = r.E;
  q.pend_a0 = a0;
  q.dirty = apply ? e.s_depmask[jsel] : 0u;
}

// Thread mode: the propensities the last event touched, for every lane of
// the warp together (lanes without a trajectory have none): a loop over each
// lane's dirty reactions, as many passes as the busiest lane needs (a pass
// per reaction that any lane needs would run most of the M products every
// event), the value placed by a select chain so that the propensities stay
// in registers.
template <int MAXM, int MAXS>
__device__ __forceinline__ void thread_propensities(const StepEnv& e, Traj<MAXM, MAXS>& q) {
  for (uint32_t dm = q.have ? (q.dirty & ((1u << e.M) - 1u)) : 0u; __any_sync(kFullMask, dm != 0u);) {
    if (dm != 0u) {
      const int j = __ffs((int)dm) - 1;
      dm &= dm - 1u;
      const unsigned long long v = propensity_fp64(e.s_cbits[j], mass_action_h<MAXS>(e.s_rinfo[j], q.x));
#pragma unroll
      for (int i = 0; i < MAXM; ++i) q.av[i] = (i == j) ? v : q.av[i];
    }
  }
}

// One thread-mode iteration (after thread_propensities).  Returns true when
// the trajectory has ended.
template <bool LOG, int MAXM, int MAXS>
__device__ __forceinline__ bool thread_step(const RunArgs& a, const StepEnv& e, Traj<MAXM, MAXS>& q,
                                            const EventLog& lg, ThreadLog& tl) {
  // one straight-line block of independent chains: the pending event's
  // quotient, the prefix sums of the new state, and the random numbers of
  // the event after the one drawn below (index n + 2 once the pending event
  // is kept; n + 1 when there is none)
  const double tau = quotient(q.pend_E, q.pend_a0);
  const double a0 = prefix_sums(e.M, q);
  const EventRandom r_after = event_random(q.n + (q.pend ? 2u : 1u), q.traj_id, e.sid, e.key0, e.key1, e.s_inv,
                                           e.s_lnf);
  const bool done = settle<LOG>(a, e, q, tau, true, lg, tl);
  const EventRandom r = q.rnd;
  q.rnd = r_after;
  draw(e, q, a0, r, done);
  return done;
}

template <int MAXM, int MAXS>
__device__ __forceinline__ void finish_trajectory(const RunArgs& a, const Traj<MAXM, MAXS>& q,
                                                  unsigned long long* blk) {
  if (a.traj_events) a.traj_events[q.li] = (long long)q.n;
  if (a.traj_hash) a.traj_hash[q.li] = q.hash;
  if (a.traj_flags) a.traj_flags[q.li] = q.flags;
  atomicAdd(&blk[0], (unsigned long long)q.n);
  if (q.flags & 1) atomicAdd(&blk[1], 1ULL);
  if (q.flags & 2) atomicAdd(&blk[2], 1ULL);
  atomicMax(&blk[3], (unsigned long long)q.maxx);
}

template <typename T>
__device__ __forceinline__ T shfl_all(T v, int src, int width = 32) {
  return __shfl_sync(kFullMask, v, src, width);
}

// ---------------------------------------------------------------------------
// Hand-off between warps (the pool is described in ssa_internal.h).
//
// A waiting warp registers on `avail`; a producer claims one registration
// before it writes a state, so the states claimed and not yet taken never
// outnumber the warps still waiting: no state is left without a taker.  A
// waiting warp leaves only by taking back an unclaimed registration, once no
// warp can hand off any more (multi == 0: every warp counts there from its
// start until it runs at most one trajectory) or after a long idle wait.
// Every wait is bounded; a wait that runs out counts an error in the run's
// stats.

constexpr int kPoolClaimTries = 64;              // CAS attempts on a contended counter
constexpr int kPoolIdlePolls = 1 << 17;          // polls without work (about 1 s) before a waiting warp may leave
constexpr int kPoolMaxPolls = 1 << 18;           // bound on any wait, about 2 s at most (an error beyond it)
constexpr unsigned long long kPoolRead = 1ULL << 62;  // sequence mark: the state was read

__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Takes one unit from a counter if it is positive.
__device__ __forceinline__ bool pool_take_one(unsigned long long* c) {
  unsigned long long v = vload(c);
  for (int i = 0; i < kPoolClaimTries && v > 0ULL; ++i) {
    const unsigned long long o = atomicCAS(c, v, v - 1ULL);
    if (o == v) return true;
    v = o;
  }
  return false;
}

// Writes trajectory q (between batches: nothing pending) to the next slot.
// One lane.  Returns false (error counted) if the slot's previous state was
// never read.
template <int MAXM, int MAXS>
__device__ __forceinline__ bool pool_put(const RunArgs& a, const Traj<MAXM, MAXS>& q) {
  unsigned long long* P = a.pool;
  const unsigned long long p = atomicAdd(P + kPoolTail, 1ULL);
  const int slot = (int)(p % (unsigned long long)kPoolSlots);
  unsigned long long* seq = P + kPoolSeq + slot;
  const unsigned long long prev = (p >= (unsigned long long)kPoolSlots) ? (p - kPoolSlots + 1ULL + kPoolRead) : 0ULL;
  int i = 0;
  while (vload(seq) != prev && i < kPoolMaxPolls) {
    __nanosleep(256);
    ++i;
  }
  if (i == kPoolMaxPolls) {
    atomicAdd(a.stats + kStatPoolError, 1ULL);
    return false;
  }
  __threadfence();  // the previous state's reader is done before this state is written
  volatile unsigned long long* w = a.pool_slots + (size_t)slot * kPoolSlotWords;
  w[0] = (unsigned long long)obits(q.t);
  w[1] = q.hash;
  w[2] = q.traj_id;
  w[3] = (unsigned long long)q.li;
  w[4] = (unsigned long long)q.n | ((unsigned long long)(uint32_t)q.k << 32);
  w[5] = (unsigned long long)(uint32_t)q.maxx;
#pragma unroll
  for (int s = 0; s < MAXS; s += 2) {
    const unsigned long long hi = (s + 1 < MAXS) ? (unsigned long long)(uint32_t)q.x[s + 1] : 0ULL;
    w[6 + s / 2] = (unsigned long long)(uint32_t)q.x[s] | (hi << 32);
  }
  __threadfence();
  atomicExch(seq, p + 1ULL);
  atomicAdd(a.stats + kStatHandoffs, 1ULL);
  return true;
}

// Reads state p (claimed by this warp) into q.  One lane.  Returns false
// (error counted) if it never appears.
template <int MAXM, int MAXS>
__device__ __forceinline__ bool pool_get(const RunArgs& a, unsigned long long p, Traj<MAXM, MAXS>& q) {
  const int slot = (int)(p % (unsigned long long)kPoolSlots);
  unsigned long long* seq = a.pool + kPoolSeq + slot;
  int i = 0;
  while (vload(seq) != p + 1ULL && i < kPoolMaxPolls) {
    __nanosleep(128);
    ++i;
  }
  if (i == kPoolMaxPolls) {
    atomicAdd(a.stats + kStatPoolError, 1ULL);
    return false;
  }
  __threadfence();
  const volatile unsigned long long* w = a.pool_slots + (size_t)slot * kPoolSlotWords;
  q.t = __longlong_as_double((long long)w[0]);
  q.hash = w[1];
  q.traj_id = w[2];
  q.li = (long long)w[3];
  const unsigned long long nk = w[4];
  q.n = (uint32_t)nk;
  q.k = (int)(uint32_t)(nk >> 32);
  q.maxx = (int)(uint32_t)w[5];
#pragma unroll
  for (int s = 0; s < MAXS; s += 2) {
    const unsigned long long v = w[6 + s / 2];
    q.x[s] = (int)(uint32_t)v;
    if (s + 1 < MAXS) q.x[s + 1] = (int)(uint32_t)(v >> 32);
  }
  __threadfence();
  atomicExch(seq, p + 1ULL + kPoolRead);
  return true;
}

// ---------------------------------------------------------------------------
// Cooperative mode: speculative batches.
//
// When at most 16 trajectories are left in a warp and no new work remains,
// the warp splits into groups of L lanes (L = 32 / n rounded down to a power
// of two for n trajectories: 2 lanes each for 9 to 16, ..., 32 for one; the
// warp regroups as trajectories end), one trajectory per group.  A group runs its trajectory in batches of L events; lane b holds
// the random numbers of event base + b of the batch.
//
// The events of a batch are selected in rounds.  In a round every lane of the
// group takes one node of a heap-ordered tree: node 0 is the trajectory's
// current state X; the children of node v are 2v + 1 and 2v + 2, reached by
// firing H1 and H2, the two reactions with the largest propensities at the
// start of the batch; the state of node v is X plus the net changes of the
// reactions on its path.  Each lane recomputes, for its node's state, the
// propensities the previous round changed, the left-to-right prefix sums and
// the direct method's selection with the random number of the event at its
// node's depth -- the same instructions in every lane, so a round costs one
// prefix chain whatever the number of nodes.  A node is verified when its
// parent selected the node's reaction and every ancestor is verified; the
// deepest verified node w closes a path of depth(w) + 1 events, which the
// round fires: each node on it made exactly the selection the plain loop
// makes from the same state with the same random number.  Hypotheses decide
// how many events a round fires, never which events.
//
// When the window is full (or an event would leave the int32 range) the batch
// is settled: lane b forms event b's waiting time, the group forms the event
// times in order and finds where the trajectory ends (past t_end, at
// max_events or at an overflow: the later events are undone), and lane b does
// event b's grid index, difference sums and log records, from the states
// given by a scan of the batch's net changes.
constexpr int kSpecMaxDepth = 5;  // node 31 of a 32-lane tree

__device__ __forceinline__ int node_depth(int v) { return 31 - __clz(v + 1); }

// The ancestor of node v at depth d (0 <= d <= depth(v)).
__device__ __forceinline__ int node_ancestor(int v, int d) { return ((v + 1) >> (node_depth(v) - d)) - 1; }

// Lanes per trajectory for n (1 <= n <= 16) trajectories in a warp: 32 / n
// rounded down to a power of two.
__device__ __forceinline__ int spec_group_size(int n) { return 32 >> (32 - __clz(n - 1)); }

// The bits of a warp ballot that belong to the group starting at lane gbase.
__device__ __forceinline__ unsigned group_bits(unsigned ballot, int gbase, int L) {
  return L == 32 ? ballot : (ballot >> gbase) & ((1u << L) - 1u);
}

// Prefix sum j (left to right) from the propensities, given prefix j - 1.
// Propensities of the bucket's padding reactions (j >= M) are +0, so the
// padding prefixes equal prefix M - 1 and the last one is a0.
template <int J, int MAXM, int MAXS>
__device__ __forceinline__ void prefix_at(Traj<MAXM, MAXS>& q) {
  if constexpr (J == 0) {
    q.pre[0] = __longlong_as_double((long long)q.av[0]);
  } else if constexpr (J < MAXM) {
    q.pre[J] = __dadd_rn(q.pre[J - 1], __longlong_as_double((long long)q.av[J]));
  }
}

// Prefix sums and a0 when the propensities below `lo` (warp-uniform) are
// unchanged: the prefixes below lo are reused bit for bit and the chain
// restarts at lo (a jump into the unrolled chain).
template <int MAXM, int MAXS>
__device__ __forceinline__ double prefix_sums_from(Traj<MAXM, MAXS>& q, int lo) {
  switch (lo) {
    case 0: prefix_at<0>(q); [[fallthrough]];
    case 1: prefix_at<1>(q); [[fallthrough]];
    case 2: prefix_at<2>(q); [[fallthrough]];
    case 3: prefix_at<3>(q); [[fallthrough]];
    case 4: prefix_at<4>(q); [[fallthrough]];
    case 5: prefix_at<5>(q); [[fallthrough]];
    case 6: prefix_at<6>(q); [[fallthrough]];
    case 7: prefix_at<7>(q); [[fallthrough]];
    case 8: prefix_at<8>(q); [[fallthrough]];
    case 9: prefix_at<9>(q); [[fallthrough]];
    case 10: prefix_at<10>(q); [[fallthrough]];
    case 11: prefix_at<11>(q); [[fallthrough]];
    case 12: prefix_at<12>(q); [[fallthrough]];
    case 13: prefix_at<13>(q); [[fallthrough]];
    case 14: prefix_at<14>(q); [[fallthrough]];
    case 15: prefix_at<15>(q); [[fallthrough]];
    default: break;
  }
  return q.pre[MAXM - 1];
}

// Direct-method selection: the first j with prefix_j > target (prefixes are
// non-decreasing), else the last j with a_j > 0.
template <int MAXM, int MAXS>
__device__ __forceinline__ int select_reaction(int M, const Traj<MAXM, MAXS>& q, long long gb) {
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < MAXM; ++j) {
    if (j < M) cnt += (obits(q.pre[j]) <= gb) ? 1 : 0;
  }
  int jsel = cnt;
  if (cnt >= M) {
    jsel = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
      if (j < M && q.av[j] != 0ULL) jsel = j;
    }
  }
  return jsel;
}

// Settles a batch of the cooperative mode for groups of L lanes: lane b <
// nres holds event base + b (its a0, reaction and random numbers), event nb
// (if < L) would have left the int32 range and was not applied.  Lane b forms
// event b's waiting time; the group forms the event times in order (one
// unconditional FP64 chain, replicated in every lane: times only grow, so it
// is right up to the first event that ends the trajectory) and the sequence
// hash after every event; the first event past t_end or at the overflow, or
// the max_events limit, ends the trajectory (later events are undone); lane b
// does the grid index, difference sums and log records of its kept event from
// the states given by a scan of the batch's net changes.
template <int L, bool LOG, int MAXM, int MAXS>
__device__ __forceinline__ void settle_batch(const RunArgs& a, const StepEnv& e, Traj<MAXM, MAXS>& q, int gl, int gbase,
                                             uint32_t base, int nres, int nb, double my_a0, int my_j,
                                             const EventRandom& rr, unsigned long long* blk, const EventLog& lg,
                                             ThreadLog& tl) {
  const bool mine = gl < nres;
  const double my_tau = quotient(rr.E, mine ? my_a0 : 1.0);
  const int* myrow = e.s_nu + my_j * MAXS;
  int cum[MAXS];  // net change of the batch's applied events up to this lane's (inclusive scan)
#pragma unroll
  for (int s = 0; s < MAXS; ++s) cum[s] = (mine && gl != nb) ? myrow[s] : 0;
#pragma unroll
  for (int off = 1; off < L; off <<= 1) {
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
      const int u = __shfl_up_sync(kFullMask, cum[s], off, L);
      cum[s] += (gl >= off) ? u : 0;
    }
  }
  // event times and prefix hashes in order; lane b keeps those after event b
  double tt = q.t, my_t = q.t;
  unsigned long long h = q.hash, my_h = q.hash;
#pragma unroll 8
  for (int b = 0; b < L; ++b) {
    const double tau_b = __shfl_sync(kFullMask, my_tau, b, L);
    const int j_b = __shfl_sync(kFullMask, my_j, b, L);
    tt = __dadd_rn(tt, tau_b);
    const unsigned long long h1 = (h ^ (unsigned long long)j_b) * kFnvPrime;
    h = (h1 ^ (unsigned long long)obits(tt)) * kFnvPrime;
    my_t = (gl == b) ? tt : my_t;
    my_h = (gl == b) ? h : my_h;
  }
  const long long my_tb = obits(my_t);
  // the first drawn event that is not kept: past t_end, or the overflowing one
  const bool stop = mine && (my_tb > e.t_end_bits || gl == nb);
  const unsigned stops = group_bits(__ballot_sync(kFullMask, stop), gbase, L);
  const int K0 = stops ? (__ffs((int)stops) - 1) : nres;
  const bool past_K0 = __shfl_sync(kFullMask, (int)(my_tb > e.t_end_bits), min(K0, L - 1), L) != 0;
  const long long kmax = a.max_events - (long long)base;  // >= 1 for a live trajectory
  int K;          // events kept
  int endf = -1;  // the trajectory ends: 0 past t_end, 1 max_events, 2 overflow
  if (kmax <= (long long)K0) {
    K = (int)max(kmax, 0LL);
    endf = 1;
  } else {
    K = K0;
    if (K0 < nres) endf = past_K0 ? 0 : 2;
  }
  const int last = max(K - 1, 0);
  const double t_last = __shfl_sync(kFullMask, my_t, last, L);
  const unsigned long long h_last = __shfl_sync(kFullMask, my_h, last, L);
  // states: at the start of the batch, and after the kept events
  int xs[MAXS], xk[MAXS];
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    const int tot = __shfl_sync(kFullMask, cum[s], L - 1, L);
    const int ck = __shfl_sync(kFullMask, cum[s], last, L);
    xs[s] = q.x[s] - tot;
    xk[s] = xs[s] + (K > 0 ? ck : 0);
  }
  // bookkeeping of the kept events, lane b for event base + b
  const bool mine_kept = q.have && gl < K;
  int my_k = q.k;
  int mx = 0;
  if (mine_kept) {
    my_k = grid_index(a, my_tb, q.k);
    int xa[MAXS], pv[MAXS];  // the state after this lane's event, and its change
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
      xa[s] = xs[s] + cum[s];
      pv[s] = myrow[s];
      if (pv[s] != 0) mx = max(mx, xa[s]);
      if (pv[s] != 0 && my_k >= 0 && my_k < e.G) {
        const long long xo = (long long)xa[s] - pv[s];
        atomicAdd(e.d1 + (size_t)my_k * e.S + s, (unsigned long long)(long long)pv[s]);
        atomicAdd(e.d2 + (size_t)my_k * e.S + s, (unsigned long long)((2 * xo + pv[s]) * (long long)pv[s]));
      }
    }
    if constexpr (LOG) thread_log_event<MAXS>(lg, tl, my_tb, xa, pv);
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(kFullMask, mx, off, L));
  const int k_last = __shfl_sync(kFullMask, my_k, last, L);
  if (q.have) {
    q.maxx = max(q.maxx, mx);
    if (K > 0) {
      q.k = k_last;
      q.t = t_last;
      q.hash = h_last;
    }
    q.n = base + (uint32_t)K;
#pragma unroll
    for (int s = 0; s < MAXS; ++s) q.x[s] = xk[s];
    if (endf >= 0) {
      q.flags = (endf == 1) ? 1 : ((endf == 2) ? 2 : 0);
      if (gl == 0) finish_trajectory(a, q, blk);
      q.have = false;
    }
  }
}

template <bool LOG, int MAXM, int MAXS>
__device__ __forceinline__ void coop_run(const RunArgs& a, const StepEnv& e, Traj<MAXM, MAXS>& q, unsigned act,
                                         bool& in_multi, unsigned long long* blk, const EventLog& lg, ThreadLog& tl) {
  const int lane = threadIdx.x & 31;
  int L = 0, gl = 0;
  int gbase = 0;
  unsigned anc_mask = 0u;  // the nodes on this lane's path below the root (heap order)
  unsigned long long avail_seen = 0ULL;  // waiting warps seen at the start of the batch (lane 0)
  double root_a0 = 0.0;            // a0 of this lane's node in the last round (the root's on group lane 0)
  int P[MAXS], up[MAXS];  // net change along this lane's path and its largest rise, per species
  bool path_ok = false;   // every reaction on the path exists
  int H1 = -2, H2 = -2;   // hypotheses (-2: not chosen since the last regrouping)
  uint32_t dirty = 0u;    // propensities this lane must recompute
  bool entry = true;
  unsigned owners = act;  // one lane per live trajectory
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    P[s] = 0;
    up[s] = 0;
  }

  for (;;) {
    const int nlive = __popc(owners);
    if (nlive == 0) break;
    if constexpr (!LOG) {
      if (a.pool) {
        const bool want = nlive >= 2;
        if (want != in_multi) {
          if (lane == 0) atomicAdd(a.pool + kPoolMulti, want ? 1ULL : ~0ULL);
          in_multi = want;
        }
      }
    }
    // (re)grouping: at entry, and when the live trajectories fit larger groups
    const int Lw = spec_group_size(nlive);
    if (Lw != L) {
      L = Lw;
      gl = lane & (L - 1);
      gbase = lane & ~(L - 1);
      anc_mask = 0u;
      for (int v = gl; v > 0; v = (v - 1) >> 1) anc_mask |= 1u << v;
      const int grp = lane / L;
      unsigned m = owners;
      int owner = -1;  // the grp-th live trajectory's lane
#pragma unroll
      for (int r = 0; r < kCoopMaxTraj; ++r) {
        const int b = __ffs((int)m) - 1;
        if (r == grp) owner = b;
        if (b >= 0) m &= m - 1;
      }
      const bool gactive = owner >= 0;
      const int src = gactive ? owner : lane;
#pragma unroll
      for (int s = 0; s < MAXS; ++s) q.x[s] = shfl_all(q.x[s], src);
      q.li = shfl_all(q.li, src);
      q.traj_id = shfl_all(q.traj_id, src);
      q.t = shfl_all(q.t, src);
      q.n = shfl_all(q.n, src);
      q.k = shfl_all(q.k, src);
      q.hash = shfl_all(q.hash, src);
      q.maxx = shfl_all(q.maxx, src);
      q.have = gactive;
      H1 = H2 = -2;
      if (entry) {
        // the event drawn and applied in thread mode, not yet settled: a
        // group without a trajectory carries none
#pragma unroll
        for (int s = 0; s < MAXS; ++s) q.pv[s] = shfl_all(q.pv[s], src);
        q.pend = (shfl_all((int)q.pend, src) != 0) && gactive;
        q.pend_over = shfl_all((int)q.pend_over, src) != 0;
        q.pend_j = shfl_all(q.pend_j, src);
        q.pend_E = shfl_all(q.pend_E, src);
        q.pend_a0 = shfl_all(q.pend_a0, src);
        const double tau = quotient(q.pend_E, q.pend_a0);
        const bool done = settle<LOG>(a, e, q, tau, gl == 0, lg, tl) && q.have;
        if (done) {
          if (gl == 0) finish_trajectory(a, q, blk);
          q.have = false;
        }
        q.pend = false;
        entry = false;
      }
    }
    if (!__any_sync(kFullMask, q.have)) break;
    if constexpr (!LOG) {
      if (in_multi && lane == 0) avail_seen = vload(a.pool + kPoolAvail);
    }

    const uint32_t base = q.n;
    const EventRandom rr = event_random(base + (uint32_t)gl, q.traj_id, e.sid, e.key0, e.key1, e.s_inv, e.s_lnf);
    const int dep = node_depth(gl);
    // hypotheses: the two largest propensities of the root lane (as left by
    // the last round), as an unordered pair so that swaps keep the tree
    {
      unsigned long long b1 = 0ULL, b2 = 0ULL;
      int i1 = -1, i2 = -1;
#pragma unroll
      for (int j = 0; j < MAXM; ++j) {
        if (j < e.M) {
          const unsigned long long v = q.av[j];
          const bool top = v > b1;
          const bool second = !top && v > b2;
          b2 = top ? b1 : (second ? v : b2);
          i2 = top ? i1 : (second ? j : i2);
          b1 = top ? v : b1;
          i1 = top ? j : i1;
        }
      }
      int h1 = (i2 < 0) ? i1 : min(i1, i2);
      int h2 = (i2 < 0) ? -1 : max(i1, i2);
      h1 = __shfl_sync(kFullMask, h1, 0, L);
      h2 = __shfl_sync(kFullMask, h2, 0, L);
      if (h1 != H1 || h2 != H2) {
        H1 = h1;
        H2 = h2;
        int cum[MAXS];
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
          cum[s] = 0;
          up[s] = 0;
        }
        path_ok = true;
#pragma unroll
        for (int d = 1; d <= kSpecMaxDepth; ++d) {
          if (d <= dep) {
            const int anc = node_ancestor(gl, d);
            const int hyp = (anc & 1) ? H1 : H2;
            path_ok = path_ok && hyp >= 0;
            const int* row = e.s_nu + max(hyp, 0) * MAXS;
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
              cum[s] += row[s];
              up[s] = max(up[s], cum[s]);
            }
          }
        }
#pragma unroll
        for (int s = 0; s < MAXS; ++s) P[s] = cum[s];
        dirty = (1u << MAXM) - 1u;
      }
    }

    // ---- rounds until the window of L events is full
    int nres = 0;  // events of the batch drawn so far (group-uniform)
    int nb = L;    // index of an event that would overflow (not applied), else L
    double my_a0 = 0.0;
    int my_j = 0;
    bool run = q.have;
    const int par = max((gl - 1) >> 1, 0);
    const int hyp_me = (gl & 1) ? H1 : H2;
    while (__any_sync(kFullMask, run)) {
      int xl[MAXS];
      bool safe = path_ok;
#pragma unroll
      for (int s = 0; s < MAXS; ++s) {
        xl[s] = q.x[s] + P[s];
        safe = safe && (long long)q.x[s] + up[s] <= kStateMax;
      }
      // products of the reactions any running lane must recompute (a
      // warp-uniform set), unrolled so that each reaction's word and rate
      // are launch constants and no index is dynamic
      const uint32_t dany = __reduce_or_sync(kFullMask, run ? dirty : 0u) & ((1u << MAXM) - 1u);
#pragma unroll
      for (int j = 0; j < MAXM; ++j) {
        if ((dany >> j) & 1u) {
          const unsigned long long pj = propensity_fp64(a.sm.cbits[j], mass_action_h<MAXS>(a.sm.rinfo[j], xl));
          if (run && ((dirty >> j) & 1u)) q.av[j] = pj;
        }
      }
      // the lowest changed reaction of any running lane: the lowest bit of
      // the union
      const int lo = (dany != 0u) ? (__ffs((int)dany) - 1) : MAXM;
      const double a0 = prefix_sums_from(q, lo);
      root_a0 = a0;
      if (run) dirty = 0u;
      const int ei = nres + dep;  // this node's event within the batch
      const bool inwin = ei < L;
      const unsigned long long u2 = __shfl_sync(kFullMask, rr.u2, min(ei, L - 1), L);
      const long long gb = obits(__dmul_rn(__longlong_as_double((long long)u2), a0));
      const int jsel = select_reaction(e.M, q, gb);
      // this node's state after its own selection (taken as the new state if
      // the node closes the round's path); not applied if it would leave the
      // int32 range
      int xpost[MAXS];
      bool over_me = false;
      {
        const int* rowj = e.s_nu + jsel * MAXS;
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
          xpost[s] = xl[s] + rowj[s];
          over_me = over_me || (long long)xl[s] + rowj[s] > kStateMax;
        }
      }
      // verification: a node is verified when it and every ancestor below
      // the root made their parent's hypothesis
      const int jp = __shfl_sync(kFullMask, jsel, par, L);
      const bool cons = (gl == 0) || (jp == hyp_me && safe && inwin);
      const unsigned C = group_bits(__ballot_sync(kFullMask, cons), gbase, L);
      const bool ver = run && (C & anc_mask) == anc_mask;
      const unsigned V = group_bits(__ballot_sync(kFullMask, ver), gbase, L);
      const int w = 31 - __clz((int)(V | 1u));  // deepest verified node
      const int dw = node_depth(w);
      // lane nres + d records the event of the path's node at depth d
      const int d = gl - nres;
      const bool rec = run && d >= 0 && d <= dw;
      const int src = rec ? node_ancestor(w, d) : gl;
      const double a0_s = __shfl_sync(kFullMask, a0, src, L);
      const int j_s = __shfl_sync(kFullMask, jsel, src, L);
      if (rec) {
        my_a0 = a0_s;
        my_j = j_s;
      }
      // the new state: node w's state after its selection, or before it
      // when that would leave the int32 range
      const bool over = __shfl_sync(kFullMask, (int)over_me, w, L) != 0;
      int xn_w[MAXS];
#pragma unroll
      for (int s = 0; s < MAXS; ++s) {
        const int xb = __shfl_sync(kFullMask, xl[s], w, L);
        const int xa = __shfl_sync(kFullMask, xpost[s], w, L);
        xn_w[s] = over ? xb : xa;
      }
      if (run) {
        uint32_t dm = 0u;
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
          const int xn = xn_w[s];
          dm |= (xn != q.x[s]) ? e.s_rmask[s] : 0u;
          q.x[s] = xn;
        }
        dirty = dm;
        if (over) nb = nres + dw;
        nres += dw + 1;
        run = !over && nres < L;
      }
    }

    // ---- settle the batch (loops unrolled for the group size)
    switch (L) {
      case 32: settle_batch<32, LOG>(a, e, q, gl, gbase, base, nres, nb, my_a0, my_j, rr, blk, lg, tl); break;
      case 16: settle_batch<16, LOG>(a, e, q, gl, gbase, base, nres, nb, my_a0, my_j, rr, blk, lg, tl); break;
      case 8: settle_batch<8, LOG>(a, e, q, gl, gbase, base, nres, nb, my_a0, my_j, rr, blk, lg, tl); break;
      case 4: settle_batch<4, LOG>(a, e, q, gl, gbase, base, nres, nb, my_a0, my_j, rr, blk, lg, tl); break;
      default: settle_batch<2, LOG>(a, e, q, gl, gbase, base, nres, nb, my_a0, my_j, rr, blk, lg, tl); break;
    }
    owners = __ballot_sync(kFullMask, q.have && gl == 0);

    // hand off one trajectory to a waiting warp: the one with the most
    // expected remaining events, a0 (t_end - t)
    if constexpr (!LOG) {
      if (in_multi && __popc(owners) >= 2) {
        bool claimed = false;
        if (lane == 0 && avail_seen > 0ULL) claimed = pool_take_one(a.pool + kPoolAvail);
        if (__shfl_sync(kFullMask, (int)claimed, 0) != 0) {
          const bool cand = gl == 0 && q.have;
          const float est = fmaxf((float)root_a0 * (float)(a.t_end - q.t), 0.f);
          const unsigned key = cand ? (0x80000000u | (__float_as_uint(est) & 0x7FFFFFE0u) | (unsigned)lane) : 0u;
          const int c = (int)(__reduce_max_sync(kFullMask, key) & 31u);
          bool put = false;
          if (lane == c) put = pool_put(a, q);
          if (__shfl_sync(kFullMask, (int)put, c) != 0 && gbase == c) q.have = false;
          owners = __ballot_sync(kFullMask, q.have && gl == 0);
        }
      }
    }
  }
  if constexpr (!LOG) {
    if (in_multi && lane == 0) atomicAdd(a.pool + kPoolMulti, ~0ULL);
  }
  in_multi = false;
}

// For a warp with no trajectory left: waits for a handed-off trajectory and
// puts it in lane 0 (returns 1, the owner mask) or returns 0 when the pool
// closes for this warp (see the hand-off description above).
template <int MAXM, int MAXS>
__device__ __forceinline__ unsigned pool_take(const RunArgs& a, Traj<MAXM, MAXS>& q) {
  const int lane = threadIdx.x & 31;
  unsigned long long* P = a.pool;
  long long got = -1;  // the state taken; -2: leave
  if (lane == 0) {
    atomicAdd(P + kPoolAvail, 1ULL);  // register as waiting
    unsigned ns = 256;
    int idle = 0;
    for (int it = 0; it < kPoolMaxPolls; ++it) {
      const unsigned long long h = vload(P + kPoolHead);
      if (h < vload(P + kPoolTail)) {
        if (atomicCAS(P + kPoolHead, h, h + 1ULL) == h) {
          got = (long long)h;
          break;
        }
        continue;
      }
      if ((vload(P + kPoolMulti) == 0ULL || ++idle >= kPoolIdlePolls) && pool_take_one(P + kPoolAvail)) {
        got = -2;
        break;
      }
      __nanosleep(ns);
      ns = min(ns * 2u, 8192u);
    }
    if (got == -1) atomicAdd(a.stats + kStatPoolError, 1ULL);
    if (got >= 0 && !pool_get(a, (unsigned long long)got, q)) got = -1;
  }
  got = __shfl_sync(kFullMask, got, 0);
  if (got < 0) return 0u;
  q.have = lane == 0;
  q.pend = false;
  q.pend_over = false;
  q.pend_j = 0;
  q.pend_E = 0ULL;
  q.pend_a0 = 1.0;
  q.flags = 0;
  return 1u;
}

template <int MAXM, int MAXS, bool SHARED_D, bool LOG>
__global__ void __launch_bounds__(512, 1) k_ssa_thread(const RunArgs a, const EventLog lg) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long blk[6];  // events, truncated, overflowed, max x, log records, log padding
  const int S = a.m.S, M = a.m.M, G = a.G, T = blockDim.x, tid = threadIdx.x;
  const ThreadSmem L = thread_smem_layout(MAXM, MAXS, S, G, SHARED_D);
  uint64_t* s_inv = reinterpret_cast<uint64_t*>(smem + L.log_inv);
  uint64_t* s_lnf = reinterpret_cast<uint64_t*>(smem + L.log_lnf);
  int32_t* s_nu = reinterpret_cast<int32_t*>(smem + L.nu);
  uint32_t* s_depmask = reinterpret_cast<uint32_t*>(smem + L.depmask);
  uint32_t* s_rmask = reinterpret_cast<uint32_t*>(smem + L.rmask);
  int32_t* s_rinfo = reinterpret_cast<int32_t*>(smem + L.rinfo);
  unsigned long long* s_cbits = reinterpret_cast<unsigned long long*>(smem + L.cbits);
  unsigned long long* d1 = SHARED_D ? reinterpret_cast<unsigned long long*>(smem + L.d1) : a.D1;
  unsigned long long* d2 = SHARED_D ? reinterpret_cast<unsigned long long*>(smem + L.d2) : a.D2;

  for (int i = tid; i < kLogCells; i += T) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  for (int i = tid; i < MAXM * MAXS; i += T) {
    const int j = i / MAXS, s = i % MAXS;
    s_nu[i] = (j < M && s < S) ? a.sm.nu[j * kSmallMax + s] : 0;
  }
  for (int j = tid; j < MAXM; j += T) {
    s_depmask[j] = (j < M) ? a.sm.depmask[j] : 0u;
    s_rinfo[j] = (j < M) ? a.sm.rinfo[j] : 0;
    s_cbits[j] = (j < M) ? a.sm.cbits[j] : 0ULL;
  }
  for (int s = tid; s < MAXS; s += T) {
    uint32_t m = 0u;
    for (int j = 0; j < M; ++j) {
      const int32_t w = a.sm.rinfo[j];
      const int kind = rinfo_kind(w);
      const bool reads = (kind != kOrder0 && rinfo_a(w) == s) || (kind == kBi && rinfo_b(w) == s);
      m |= reads ? (1u << j) : 0u;
    }
    s_rmask[s] = m;
  }
  if (SHARED_D) {
    for (int i = tid; i < G * S; i += T) {
      d1[i] = 0ULL;
      d2[i] = 0ULL;
    }
  }
  if (tid < 6) blk[tid] = 0ULL;
  __syncthreads();

  StepEnv e;
  e.M = M;
  e.S = S;
  e.G = G;
  e.t_end_bits = obits(a.t_end);
  const uint64_t seed = a.seed_word ? (uint64_t)*a.seed_word : a.seed;
  e.key0 = (uint32_t)seed;
  e.key1 = (uint32_t)(seed >> 32);
  e.sid = (uint32_t)a.stream_id;
  e.s_inv = s_inv;
  e.s_lnf = s_lnf;
  e.s_nu = s_nu;
  e.s_depmask = s_depmask;
  e.s_rmask = s_rmask;
  e.s_rinfo = s_rinfo;
  e.s_cbits = s_cbits;
  e.d1 = d1;
  e.d2 = d2;

  Traj<MAXM, MAXS> q;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    q.x[s] = 0;
    q.pv[s] = 0;
  }
#pragma unroll
  for (int j = 0; j < MAXM; ++j) {
    q.av[j] = 0ULL;
    q.pre[j] = 0.0;
  }
  q.have = false;
  q.pend = false;
  q.pend_over = false;
  q.dirty = 0;
  q.li = 0;
  q.traj_id = 0;
  q.t = 0.0;
  q.n = 0;
  q.k = 0;
  q.hash = kFnvOffset;
  q.maxx = 0;
  q.flags = 0;
  q.pend_j = 0;
  q.pend_E = 0ULL;
  q.pend_a0 = 0.0;
  q.rnd = EventRandom{0ULL, 0ULL};
  bool exhausted = false;  // this lane saw the work counter run out
  // a warp may hand off trajectories from its start until it runs at most one
  bool in_multi = false;
  if constexpr (!LOG) {
    if (a.pool) {
      if ((threadIdx.x & 31) == 0) atomicAdd(a.pool + kPoolMulti, 1ULL);
      in_multi = true;
    }
  }
  ThreadLog tl{kLogSentinel, 0, false, 0ULL, 0ULL};

  // Every lane of the warp stays in this loop until the warp has no work, so
  // warp-wide votes see all 32 lanes.
  for (;;) {
    if (!q.have && !exhausted) {
      const unsigned long long next = atomicAdd(a.counter, 1ULL);
      if (next < (unsigned long long)a.N) {
        start_trajectory(a, e, q, next);
        q.rnd = event_random(0u, q.traj_id, e.sid, e.key0, e.key1, e.s_inv, e.s_lnf);
      } else {
        exhausted = true;
      }
    }
    const unsigned act = __ballot_sync(kFullMask, q.have);
    if (act == 0u) break;
    const int nact = __popc(act);
    if (nact <= kCoopMaxTraj && __any_sync(kFullMask, exhausted)) break;  // cooperative mode
    thread_propensities(e, q);
    if (q.have) {
      const bool done = thread_step<LOG>(a, e, q, lg, tl);
      if (done) {
        finish_trajectory(a, q, blk);
        q.have = false;
      }
    }
  }
  // the cooperative tail of this warp's trajectories, then (with a pool)
  // trajectories handed off by other warps
  for (unsigned act = __ballot_sync(kFullMask, q.have);;) {
    if (act != 0u) coop_run<LOG>(a, e, q, act, in_multi, blk, lg, tl);
    if constexpr (!LOG) {
      if (in_multi && (threadIdx.x & 31) == 0) atomicAdd(a.pool + kPoolMulti, ~0ULL);  // no trajectory to hand off
    }
    in_multi = false;
    act = 0u;
    if constexpr (!LOG) {
      if (a.pool) act = pool_take(a, q);
    }
    if (act == 0u) break;
  }

  if constexpr (LOG) {
    thread_log_close(lg, tl);
    if (tl.total) atomicAdd(&blk[4], tl.total);
    if (tl.padded) atomicAdd(&blk[5], tl.padded);
  }
  __syncthreads();
  if (SHARED_D) {
    for (int i = tid; i < G * S; i += T) {
      const unsigned long long v1 = d1[i], v2 = d2[i];
      if (v1) atomicAdd(a.D1 + i, v1);
      if (v2) atomicAdd(a.D2 + i, v2);
    }
  }
  if (tid == 0) {
    atomicAdd(a.stats + kStatEvents, blk[0]);
    atomicAdd(a.stats + kStatTruncated, blk[1]);
    atomicAdd(a.stats + kStatOverflowed, blk[2]);
    atomicMax(a.stats + kStatMaxX, blk[3]);
    if constexpr (LOG) {
      if (blk[4]) atomicAdd(lg.needed, blk[4]);
      if (blk[5]) atomicAdd(lg.padded, blk[5]);
    }
    if (a.device_totals) {
      atomicAdd(a.device_totals + 0, blk[0]);
      atomicAdd(a.device_totals + 1, blk[1]);
      atomicAdd(a.device_totals + 2, blk[2]);
      atomicMax(a.device_totals + 3, blk[3]);
    }
  }
}

#ifndef SSA_THREAD_LOG_ONLY
template <int MAXM, int MAXS>
cudaError_t launch_bucket(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st) {
  const EventLog none{};
  if (shared_d)
    k_ssa_thread<MAXM, MAXS, true, false><<<blocks, threads, smem, st>>>(a, none);
  else
    k_ssa_thread<MAXM, MAXS, false, false><<<blocks, threads, smem, st>>>(a, none);
  return cudaGetLastError();
}

template <int MAXM, int MAXS>
cudaError_t set_smem_bucket(bool shared_d, size_t smem) {
  if (shared_d)
    return cudaFuncSetAttribute(k_ssa_thread<MAXM, MAXS, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return cudaFuncSetAttribute(k_ssa_thread<MAXM, MAXS, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}
#else
// The logging variants (difference sums in global memory; the Avg-XY
// pipeline runs them with G = 0, so none are formed).
template <int MAXM, int MAXS>
cudaError_t launch_bucket(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                          cudaStream_t st) {
  k_ssa_thread<MAXM, MAXS, false, true><<<blocks, threads, smem, st>>>(a, lg);
  return cudaGetLastError();
}

template <int MAXM, int MAXS>
cudaError_t set_smem_bucket(size_t smem) {
  return cudaFuncSetAttribute(k_ssa_thread<MAXM, MAXS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}
#endif

// Dispatch on the M bucket for one S bucket (ARGS: the launch arguments).
#define SSA_M_BUCKETS(FN, ...)                    \
  switch (bucket_m(M)) {                          \
    case 2: return FN<2, MAXS>(__VA_ARGS__);      \
    case 4: return FN<4, MAXS>(__VA_ARGS__);      \
    case 6: return FN<6, MAXS>(__VA_ARGS__);      \
    case 8: return FN<8, MAXS>(__VA_ARGS__);      \
    case 10: return FN<10, MAXS>(__VA_ARGS__);    \
    case 12: return FN<12, MAXS>(__VA_ARGS__);    \
    case 14: return FN<14, MAXS>(__VA_ARGS__);    \
    case 16: return FN<16, MAXS>(__VA_ARGS__);    \
    default: return cudaErrorInvalidValue;        \
  }

#ifndef SSA_THREAD_LOG_ONLY
template <int MAXS>
cudaError_t launch_for_s(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st) {
  const int M = a.m.M;
  SSA_M_BUCKETS(launch_bucket, a, blocks, threads, shared_d, smem, st)
}

template <int MAXS>
cudaError_t set_smem_for_s(int M, bool shared_d, size_t smem) {
  SSA_M_BUCKETS(set_smem_bucket, shared_d, smem)
}
#else
template <int MAXS>
cudaError_t launch_log_for_s(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                             cudaStream_t st) {
  const int M = a.m.M;
  SSA_M_BUCKETS(launch_bucket, a, lg, blocks, threads, smem, st)
}

template <int MAXS>
cudaError_t set_smem_log_for_s(int M, size_t smem) {
  SSA_M_BUCKETS(set_smem_bucket, smem)
}
#endif
#undef SSA_M_BUCKETS

}  // namespace
}  // namespace ssa_impl

#endif  // SSA_THREAD_KERNEL_CUH_
