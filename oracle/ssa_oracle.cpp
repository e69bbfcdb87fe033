// Oracle: a plain, slow, single-threaded CPU statement of the ensemble SSA with
// time-aligned mean / variance reduction.
//
// TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
// CPU-baseline leg load this file's library.  It shares no code, header, table
// or constant generator with the CUDA library; the constants of its fixed-point
// logarithm are computed by oracle/__init__.py with Python integers and handed
// in through oracle_init_log().
//
// What it computes, per trajectory id i in [traj_begin, traj_end):
//   * Gillespie's direct method (Sec. 2: the next transition and its time are
//     drawn exactly from the CTMC's law; "a single transition amongst the
//     possible ones is selected, and the state updated accordingly").
//   * Mass-action propensities over an integer state and integer
//     stoichiometry (Sec. 3.2, model files: state vector, stoichiometric
//     matrix, propensity vector; "the more the reactants (and the rate) the
//     highest the probability").
//   * Selective memory with average as combining function (Sec. 3.2.1 and
//     Fig. 3): every trajectory's state is aligned on common simulation-time
//     points and reduced across trajectories by associative, commutative sums
//     (sum of x and of x^2, from which mean and variance follow; Sec. 4 reports
//     average and variance).
//
// Readings where the paper is silent (each also listed in the design notes):
//   * the random source is Philox4x32-10 (Salmon et al., SC'11), one block
//     per event: key = (seed low word, seed high word), counter = (event
//     index n, trajectory id low word, trajectory id high word, stream id);
//   * r1 = u(w0, w1), r2 = u(w2, w3) with u(a, b) = (2 m + 1) 2^-53,
//     m = (a << 20) | (b >> 12), exactly representable, in (0, 1);
//   * -ln(r1) is a fixed-point table-driven logarithm (Tang, ACM TOMS 16(4),
//     1990: 512-cell table of ln F_i and 1/F_i, short series for ln(1+r));
//   * h_j = prod_s C(x_s, R_js); a_j = c_j * (double)h_j;
//     a0 and the selection prefix sums are left-to-right FP64 sums (schedule
//     L) or the 32-lane chunked scan described at w32_prefix() (schedule W32);
//   * selection: smallest j with a_j > 0 and prefix_j > r2 * a0; if rounding
//     leaves none, the last j with a_j > 0 (zero-propensity transitions are
//     never chosen);
//   * grid value at g_k is the state after all events with time <= g_k
//     (right-continuous); an event whose time exceeds t_end is not fired;
//   * a0 == 0 makes the state absorbing (t_next = +inf).
//
// FP32-propensity mode (the precision variant; time stays FP64):
//   * a_j = (float)c_j * (float)h_j in binary32, each step rounded to nearest;
//   * the selection prefix sums are binary32 sums of these a_j in the
//     run's schedule (L or W32), with total A32 (the last prefix or the
//     scan's lane-31 value);
//   * a0 in FP64, formed again at every event (no incremental drift): under
//     W32 each lane's chunk is summed left to right in binary32 with error
//     compensation and kept as a binary32 pair (head, error sum)
//     (compensated_pair); the 32 pairs are combined by the W32 Kogge-Stone
//     scan in pair arithmetic (heads by TwoSum, errors added in binary32:
//     pair_add), and lane 31's pair is widened and added once in FP64; under
//     L the whole list is one compensated pair, widened and added the same
//     way; t_next = t + (-ln r1) / a0;
//   * selection: smallest j with a_j > 0 and (double)prefix_j > r2 *
//     (double)A32 (FP64 product); if none, the last j with a_j > 0.
// When every product and sum is exact in binary32, this mode reproduces the
// FP64 mode's trajectories bit for bit.
//
// Build: g++ -O2 -ffp-contract=off (no FMA contraction), no -ffast-math.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

// ---------------------------------------------------------------- Philox4x32-10
// Round function and key schedule as published by Salmon, Moraes, Dror and
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11 (Philox-4x32:
// multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
// 0xBB67AE85, ten rounds).
const uint32_t kPhiloxM0 = 0xD2511F53u;
const uint32_t kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u;
const uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ------------------------------------------------------- fixed-point -ln(u)
// Constants handed in by the Python side (integers, see oracle/__init__.py):
//   inv[i] = round(2^64 / F_i), lnf[i] = round(2^64 ln F_i), F_i = 1 + (2i+1)/1024,
//   i = 0..511; ln2 = round(2^64 ln 2); k3 = round(2^31 / 3), k5 = round(2^31 / 5).
struct LogTables {
  uint64_t inv[512];
  uint64_t lnf[512];
  uint64_t ln2;
  int64_t k3, k5;
  bool ready;
};
LogTables g_log = {};

// E = -ln(q * 2^-53) for odd q in [1, 2^53).
//   q = 2^e (1 + f), f in [0, 1) held as Q0.64;
//   1 + f = F_i (1 + r), F_i the centre of f's cell (top 9 bits of f),
//   r = (f - c_i) / F_i, |r| < 2^-10, formed as floor(d * inv_i / 2^64);
//   -ln(u) = (53 - e) ln 2 - ln F_i - ln(1 + r);
//   ln(1 + r) = r - r^2/2 + r^3 w,  w = 1/3 - r/4 + r^2/5 (series of ln(1 + r);
//   the omitted terms are below 2^-62), with r^2 and r^3 in Q.64 and w in
//   Q1.31 (32-bit; its error times |r^3| < 2^-30 stays below 2^-61).
// Every floor below is an arithmetic shift of a two's-complement value.  The
// sum is formed in Q.64 (units of 2^-64) and rounded once to double.
double neg_log_u(uint64_t q) {
  const int e = 63 - __builtin_clzll(q);                 // floor(log2 q), 0..52
  const uint64_t f = (q << (63 - e)) << 1;               // fraction bits of q / 2^e
  const int i = (int)(f >> 55);                          // cell index, top 9 bits
  const uint64_t center = ((uint64_t)(2 * i + 1)) << 54; // (2i+1)/1024 in Q.64
  const int64_t d = (int64_t)(f - center);               // f - c_i, |d| <= 2^-10
  const int64_t r = (int64_t)(((i128)d * (i128)(u128)g_log.inv[i]) >> 64);
  const int64_t r2 = (int64_t)(((i128)r * (i128)r) >> 64);
  const int64_t r3 = (int64_t)(((i128)r2 * (i128)r) >> 64);
  // w = 1/3 - r/4 + r^2/5 in Q1.31
  const int32_t rq = (int32_t)(r >> 33);                 // r in Q.31
  const int32_t r2q = (int32_t)(r2 >> 33);               // r^2 in Q.31
  const int32_t w = (int32_t)g_log.k3 - (rq >> 2) + (int32_t)(((int64_t)r2q * g_log.k5) >> 31);
  // r^3 w in Q.64: (r3 >> 4) * w >> 27
  const int64_t t3 = ((r3 >> 4) * (int64_t)w) >> 27;
  const int64_t ln1p = r - (r2 >> 1) + t3;
  const i128 E = (i128)(53 - e) * (i128)(u128)g_log.ln2 - (i128)(u128)g_log.lnf[i] - (i128)ln1p;
  const u128 Eu = (u128)E;
  if ((Eu >> 64) == 0) return (double)(uint64_t)Eu * 0x1p-64;
  return (double)(uint64_t)(Eu >> 6) * 0x1p-58;
}

// u(a, b) = (2 * ((a << 20) | (b >> 12)) + 1) * 2^-53 from two 32-bit words:
// 52 random bits, exact in double, strictly inside (0, 1).
inline uint64_t odd53(uint32_t a, uint32_t b) {
  return ((((uint64_t)a << 20) | (uint64_t)(b >> 12)) << 1) | 1ULL;
}

// --------------------------------------------------------------- model
struct Model {
  int S = 0, M = 0;
  std::vector<int32_t> R, P, nu;  // M x S
  std::vector<double> c;          // M
  std::vector<int32_t> x0;        // S
  // rate modifiers (state-dependent rates): reaction j with mod_f[j] >= 0
  // uses min(max(c_j + mod_k[j] * x_{mod_f[j]}, mod_lo[j]), mod_hi[j])
  std::vector<int32_t> mod_f;
  std::vector<double> mod_k, mod_lo, mod_hi;
};

// Modifiers for the models the calling thread builds next (set by
// oracle_set_modifiers; empty = plain mass action).
thread_local std::vector<int32_t> t_mod_f;
thread_local std::vector<double> t_mod_k, t_mod_lo, t_mod_hi;

// The rate of reaction j in state x: c_j, or for a modified reaction the
// clamped linear function of its modifier species' count (FP64: one product,
// one sum, then the clamp).
double rate(const Model& m, int j, const std::vector<int64_t>& x) {
  if (m.mod_f.empty() || m.mod_f[j] < 0) return m.c[j];
  const double v = m.c[j] + m.mod_k[j] * (double)x[m.mod_f[j]];
  return std::fmin(std::fmax(v, m.mod_lo[j]), m.mod_hi[j]);
}

// Mass-action combinatorial factor: h_j(x) = prod_s C(x_s, R_js)  (R_js in 0..2).
int64_t mass_action_h(const Model& m, int j, const std::vector<int64_t>& x) {
  int64_t h = 1;
  for (int s = 0; s < m.S; ++s) {
    int r = m.R[(size_t)j * m.S + s];
    if (r == 1) h *= x[s];
    else if (r == 2) h *= x[s] * (x[s] - 1) / 2;
  }
  return h;
}

// Schedule W32: 32 lanes; lane l owns the contiguous chunk of ceil(M/32)
// reactions starting at l * ceil(M/32); each lane sums its chunk left to right;
// lane partials are combined by an inclusive Kogge-Stone scan with offsets
// 1, 2, 4, 8, 16 (v[l] = v[l] + v[l - off] for l >= off, all lanes reading the
// previous step's values).  The prefix of reaction j is (scan of lanes before
// j's lane) + (left-to-right sum inside j's chunk up to j), formed as
// excl + inner with excl = 0 for lane 0.  a0 is lane 31's inclusive value.
template <typename T>
void w32_prefix(const std::vector<T>& a, int M, std::vector<T>& prefix, T* a0) {
  const int chunk = (M + 31) / 32;
  T part[32];
  for (int l = 0; l < 32; ++l) {
    T s = 0;
    for (int q = 0; q < chunk; ++q) {
      int j = l * chunk + q;
      if (j < M) s = (q == 0) ? a[j] : s + a[j];
    }
    part[l] = s;
  }
  T scan[32];
  for (int l = 0; l < 32; ++l) scan[l] = part[l];
  for (int off = 1; off < 32; off <<= 1) {
    T prev[32];
    for (int l = 0; l < 32; ++l) prev[l] = scan[l];
    for (int l = off; l < 32; ++l) scan[l] = prev[l] + prev[l - off];
  }
  for (int l = 0; l < 32; ++l) {
    T excl = (l == 0) ? 0 : scan[l - 1];
    T inner = 0;
    for (int q = 0; q < chunk; ++q) {
      int j = l * chunk + q;
      if (j >= M) break;
      inner = (q == 0) ? a[j] : inner + a[j];
      prefix[j] = (l == 0) ? inner : excl + inner;
    }
  }
  *a0 = scan[31];
}

// FP32 mode: the binary32 pair (head, error) of an unevaluated sum.
struct Pair32 {
  float s, e;
};

// FP32 mode: a[b..e) (binary32 values) summed left to right with error
// compensation in binary32 -- the cascaded TwoSum of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005,
// Algorithm Sum2): s_j = s_{j-1} + a_j rounded, its exact rounding error by
// Knuth's TwoSum, the errors added up in binary32 -- kept as the pair (s, err).
Pair32 compensated_pair(const std::vector<float>& a, int b, int e) {
  float s = a[b], err = 0.0f;
  for (int j = b + 1; j < e; ++j) {
    const float x = a[j];
    const float t = s + x;
    const float bp = t - s;
    const float d = (s - (t - bp)) + (x - bp);  // TwoSum: s + x = t + d exactly
    err = err + d;
    s = t;
  }
  return Pair32{s, err};
}

// The sum of two pairs in the same spirit: the heads added with their exact
// rounding error (TwoSum), the two error parts and that error added in
// binary32.  (TwoSum's error is the exact residual, so the result does not
// depend on the order of the operands.)
Pair32 pair_add(Pair32 p, Pair32 q) {
  const float t = p.s + q.s;
  const float bp = t - p.s;
  const float d = (p.s - (t - bp)) + (q.s - bp);
  return Pair32{t, (p.e + q.e) + d};
}

// A pair widened exactly to FP64 and its two parts added once (rounded).
double pair_value(Pair32 p) { return (double)p.s + (double)p.e; }

// FP32 mode, schedule L: a0 from one compensated pair over the whole list.
double compensated_sum(const std::vector<float>& a, int b, int e) { return pair_value(compensated_pair(a, b, e)); }

// FP32 mode, schedule W32: each lane's chunk as a compensated pair, the 32
// pairs combined by the inclusive Kogge-Stone scan of w32_prefix (offsets 1,
// 2, 4, 8, 16, every lane reading the previous step's values) with pair_add,
// and lane 31's pair widened.
double w32_pair_a0(const std::vector<float>& a32, int M) {
  const int chunk = (M + 31) / 32;
  Pair32 scan[32];
  for (int l = 0; l < 32; ++l) {
    const int b = l * chunk, e = std::min(M, b + chunk);
    scan[l] = (b < e) ? compensated_pair(a32, b, e) : Pair32{0.0f, 0.0f};
  }
  for (int off = 1; off < 32; off <<= 1) {
    Pair32 prev[32];
    for (int l = 0; l < 32; ++l) prev[l] = scan[l];
    for (int l = off; l < 32; ++l) scan[l] = pair_add(prev[l], prev[l - off]);
  }
  return pair_value(scan[31]);
}

// Selection (Sec. 2: one of the possible transitions is chosen): the
// smallest j with a_j > 0 and prefix_j > target; if rounding leaves none,
// the last j with a_j > 0.  A transition whose propensity is zero is not
// possible and is never chosen.  Under schedule L the prefixes never
// decrease, so a_j = 0 already rules j out; under W32 a lane's exclusive
// scan value can exceed the previous lane's last prefix by rounding, and
// without the a_j > 0 condition a zero-propensity reaction at the start of a
// lane could be chosen.
int select_reaction(const std::vector<double>& a, const std::vector<double>& prefix, int M, double target) {
  for (int j = 0; j < M; ++j)
    if (a[j] > 0.0 && prefix[j] > target) return j;
  for (int j = M - 1; j >= 0; --j)
    if (a[j] > 0.0) return j;
  return -1;
}

const int kFlagTruncated = 1;
const int kFlagOverflow = 2;
const int64_t kStateLimit = 2147483647LL;  // int32 state
const uint64_t kFnvOffset = 0xcbf29ce484222325ULL;
const uint64_t kFnvPrime = 0x100000001b3ULL;

inline uint64_t dbits(double v) { uint64_t b; std::memcpy(&b, &v, 8); return b; }

struct TrajResult {
  int64_t events = 0;
  uint64_t hash = kFnvOffset;
  int flags = 0;
  int64_t max_x = 0;
};

// One trajectory of the direct method with grid alignment (emission into
// S1 / S2 of x and x^2 at every grid point, right-continuous).
TrajResult run_one(const Model& m, uint64_t traj_id, double t_end, int G, const double* grid,
                   uint64_t seed, uint64_t stream, int64_t max_events, int schedule, int precision,
                   uint64_t* S1, uint64_t* S2, double* S3, double* S4,
                   int record_max, double* rec_t, int32_t* rec_j) {
  TrajResult res;
  std::vector<int64_t> x(m.S);
  for (int s = 0; s < m.S; ++s) { x[s] = m.x0[s]; if (x[s] > res.max_x) res.max_x = x[s]; }
  std::vector<double> a(m.M), prefix(m.M), a_wide(m.M);
  std::vector<float> a32(m.M), prefix32(m.M);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t words[4] = {0, 0, 0, 0};
  double t = 0.0;
  int64_t n = 0;
  int k = 0;
  auto emit_until = [&](double t_next) {  // grid points with g_k < t_next see the current x
    while (k < G && grid[k] < t_next) {
      for (int s = 0; s < m.S; ++s) {
        S1[(size_t)k * m.S + s] += (uint64_t)x[s];
        S2[(size_t)k * m.S + s] += (uint64_t)(x[s] * x[s]);
        if (S3) {
          const double xd = (double)x[s];
          S3[(size_t)k * m.S + s] += xd * xd * xd;
          S4[(size_t)k * m.S + s] += (xd * xd) * (xd * xd);
        }
      }
      ++k;
    }
  };
  for (;;) {
    // propensities (Sec. 3.2: mass action), a0 and selection prefix sums
    double a0 = 0.0;
    float a0_32 = 0.0f;
    if (precision == 0) {
      for (int j = 0; j < m.M; ++j) a[j] = rate(m, j, x) * (double)mass_action_h(m, j, x);
      if (schedule == 0) {
        for (int j = 0; j < m.M; ++j) { a0 = (j == 0) ? a[0] : a0 + a[j]; prefix[j] = a0; }
      } else {
        w32_prefix(a, m.M, prefix, &a0);
      }
    } else {
      for (int j = 0; j < m.M; ++j) {
        a32[j] = (float)m.c[j] * (float)mass_action_h(m, j, x);  // FP32 mode has no modifiers
        a_wide[j] = (double)a32[j];
        a[j] = a_wide[j];
      }
      if (schedule == 0) {
        for (int j = 0; j < m.M; ++j) {
          a0_32 = (j == 0) ? a32[0] : a0_32 + a32[j];
          prefix32[j] = a0_32;
        }
        a0 = compensated_sum(a32, 0, m.M);
      } else {
        w32_prefix(a32, m.M, prefix32, &a0_32);
        a0 = w32_pair_a0(a32, m.M);
      }
      for (int j = 0; j < m.M; ++j) prefix[j] = (double)prefix32[j];
    }
    // random numbers for event n
    const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)traj_id, (uint32_t)(traj_id >> 32), (uint32_t)stream};
    philox4x32_10(ctr, key, words);
    // next event time (Sec. 2: the time at which the next transition occurs)
    double t_next;
    if (a0 > 0.0) {
      double E = neg_log_u(odd53(words[0], words[1]));
      t_next = t + E / a0;
    } else {
      t_next = std::numeric_limits<double>::infinity();
    }
    emit_until(t_next);
    if (t_next > t_end) break;
    // select the transition: smallest j with a_j > 0 and prefix_j > r2 * a0
    // (FP32 mode: r2 times the binary32 total of the prefix sums)
    const double sel_total = (precision == 0) ? a0 : (double)a0_32;
    const double target = ((double)odd53(words[2], words[3]) * 0x1p-53) * sel_total;
    const int jsel = select_reaction(a, prefix, m.M, target);
    // state update, refusing to leave the int32 range
    bool over = false;
    for (int s = 0; s < m.S; ++s) {
      int64_t v = x[s] + m.nu[(size_t)jsel * m.S + s];
      if (v > kStateLimit) over = true;
    }
    if (over) { res.flags |= kFlagOverflow; break; }
    for (int s = 0; s < m.S; ++s) {
      x[s] += m.nu[(size_t)jsel * m.S + s];
      if (x[s] > res.max_x) res.max_x = x[s];
    }
    t = t_next;
    if (n < record_max) { rec_t[n] = t; rec_j[n] = jsel; }
    res.hash = (res.hash ^ (uint64_t)jsel) * kFnvPrime;
    res.hash = (res.hash ^ dbits(t)) * kFnvPrime;
    ++n;
    if (n == max_events) { res.flags |= kFlagTruncated; break; }
  }
  // points not yet emitted keep the last state (truncation, overflow, t_end)
  emit_until(std::numeric_limits<double>::infinity());
  res.events = n;
  return res;
}

// Likelihood-ratio sensitivities of one FP64 trajectory (the reading of the
// score of a CTMC path under mass action): for reaction r with rate c_r,
//   Z_r(t) = N_r(t) / c_r - I_r(t),  I_r(t) = integral_0^t h_r(x(s)) ds,
// N_r(t) the firings of r up to t.  The path's contribution to dL/dc_r is
//   g_r = sum_k u_k Z_r(g_k),  u_k = sum_s w[k][s] (x_s(g_k) - m[k][s]),
// with w = dL/dmean and m the ensemble mean (centering).  The trajectory is
// the same as run_one's (same draws, schedule L or W32, FP64 propensities).
// I_r accumulates h_r (t_next - t) over each inter-event interval; at a grid
// point inside the current interval, I_r(g_k) = I_r(t) + h_r (g_k - t).
void run_one_grad(const Model& m, uint64_t traj_id, double t_end, int G, const double* grid, uint64_t seed,
                  uint64_t stream, int64_t max_events, int schedule, const double* w, const double* mu,
                  double* g_out) {
  std::vector<int64_t> x(m.S), nfire(m.M, 0), h(m.M);
  for (int s = 0; s < m.S; ++s) x[s] = m.x0[s];
  std::vector<double> a(m.M), prefix(m.M), I(m.M, 0.0), g(m.M, 0.0);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t words[4] = {0, 0, 0, 0};
  double t = 0.0;
  int64_t n = 0;
  int k = 0;
  auto emit_until = [&](double t_next) {
    while (k < G && grid[k] < t_next) {
      double u = 0.0;
      for (int s = 0; s < m.S; ++s) u += w[(size_t)k * m.S + s] * ((double)x[s] - mu[(size_t)k * m.S + s]);
      for (int r = 0; r < m.M; ++r) {
        const double Z = (double)nfire[r] / m.c[r] - (I[r] + (double)h[r] * (grid[k] - t));
        g[r] += u * Z;
      }
      ++k;
    }
  };
  for (;;) {
    for (int j = 0; j < m.M; ++j) {
      h[j] = mass_action_h(m, j, x);
      a[j] = rate(m, j, x) * (double)h[j];
    }
    double a0 = 0.0;
    if (schedule == 0) {
      for (int j = 0; j < m.M; ++j) { a0 = (j == 0) ? a[0] : a0 + a[j]; prefix[j] = a0; }
    } else {
      w32_prefix(a, m.M, prefix, &a0);
    }
    const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)traj_id, (uint32_t)(traj_id >> 32), (uint32_t)stream};
    philox4x32_10(ctr, key, words);
    double t_next;
    if (a0 > 0.0) {
      double E = neg_log_u(odd53(words[0], words[1]));
      t_next = t + E / a0;
    } else {
      t_next = std::numeric_limits<double>::infinity();
    }
    emit_until(t_next);
    if (t_next > t_end) break;
    const double target = ((double)odd53(words[2], words[3]) * 0x1p-53) * a0;
    const int jsel = select_reaction(a, prefix, m.M, target);
    bool over = false;
    for (int s = 0; s < m.S; ++s)
      if (x[s] + m.nu[(size_t)jsel * m.S + s] > kStateLimit) over = true;
    if (over) break;
    for (int r = 0; r < m.M; ++r) I[r] += (double)h[r] * (t_next - t);
    for (int s = 0; s < m.S; ++s) x[s] += m.nu[(size_t)jsel * m.S + s];
    nfire[jsel] += 1;
    t = t_next;
    ++n;
    if (n == max_events) break;
  }
  for (int j = 0; j < m.M; ++j) h[j] = mass_action_h(m, j, x);
  emit_until(std::numeric_limits<double>::infinity());
  for (int r = 0; r < m.M; ++r) g_out[r] = g[r];
}

bool build_model(int S, int M, const int32_t* R, const int32_t* P, const double* c,
                 const int32_t* x0, Model* m) {
  if (S <= 0 || M <= 0) return false;
  if (!t_mod_f.empty()) {
    if ((int)t_mod_f.size() != M) return false;
    m->mod_f = t_mod_f;
    m->mod_k = t_mod_k;
    m->mod_lo = t_mod_lo;
    m->mod_hi = t_mod_hi;
  }
  m->S = S; m->M = M;
  m->R.assign(R, R + (size_t)M * S);
  m->P.assign(P, P + (size_t)M * S);
  m->nu.resize((size_t)M * S);
  for (size_t q = 0; q < (size_t)M * S; ++q) m->nu[q] = P[q] - R[q];
  m->c.assign(c, c + M);
  m->x0.assign(x0, x0 + S);
  return true;
}

}  // namespace

extern "C" {

int oracle_init_log(const uint64_t* inv, const uint64_t* lnf, uint64_t ln2, int64_t k3, int64_t k5) {
  for (int i = 0; i < 512; ++i) { g_log.inv[i] = inv[i]; g_log.lnf[i] = lnf[i]; }
  g_log.ln2 = ln2;
  g_log.k3 = k3;
  g_log.k5 = k5;
  g_log.ready = true;
  return 0;
}

void oracle_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

double oracle_neg_log_u(uint64_t q) { return neg_log_u(q); }

void oracle_neg_log_u_many(int64_t n, const uint64_t* q, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = neg_log_u(q[i]);
}

// Uniform grid reading: g_k = ((double)k * t_end) / (double)(G - 1).
void oracle_uniform_grid(int G, double t_end, double* grid) {
  if (G == 1) { grid[0] = t_end; return; }
  for (int k = 0; k < G; ++k) grid[k] = ((double)k * t_end) / (double)(G - 1);
}

// Runs trajectories [traj_begin, traj_end) and ADDS their x and x^2 grid sums
// into S1 / S2 (int64, wrapping, G x S row-major), and, when S3 / S4 are
// given, x^3 and x^4 as FP64 sums (for standard errors of the variance).
// schedule: 0 = L, 1 = W32; precision: 0 = FP64, 1 = FP32 propensities.
// Per-trajectory outputs are indexed by id - traj_begin and may be null.  totals[0..3] receive (added):
// events, truncated trajectories, overflowed trajectories, max state seen.
// Returns 0, or -1 on bad arguments / uninitialised tables.
int oracle_run(int S, int M, const int32_t* R, const int32_t* P, const double* c, const int32_t* x0,
               int64_t traj_begin, int64_t traj_end, double t_end, int G, const double* grid,
               uint64_t seed, uint64_t stream, int64_t max_events, int schedule, int precision,
               int64_t* S1, int64_t* S2, double* S3, double* S4,
               int64_t* traj_events, uint64_t* traj_hash, int32_t* traj_flags, int64_t* totals) {
  if (!g_log.ready || traj_end < traj_begin || G < 1 || (schedule != 0 && schedule != 1) ||
      (precision != 0 && precision != 1) || ((S3 == nullptr) != (S4 == nullptr)))
    return -1;
  Model m;
  if (!build_model(S, M, R, P, c, x0, &m)) return -1;
  if (precision == 1 && !m.mod_f.empty()) return -1;
  for (int64_t id = traj_begin; id < traj_end; ++id) {
    TrajResult r = run_one(m, (uint64_t)id, t_end, G, grid, seed, stream, max_events, schedule, precision,
                           (uint64_t*)S1, (uint64_t*)S2, S3, S4, 0, nullptr, nullptr);
    const int64_t o = id - traj_begin;
    if (traj_events) traj_events[o] = r.events;
    if (traj_hash) traj_hash[o] = r.hash;
    if (traj_flags) traj_flags[o] = r.flags;
    if (totals) {
      totals[0] += r.events;
      totals[1] += (r.flags & kFlagTruncated) ? 1 : 0;
      totals[2] += (r.flags & kFlagOverflow) ? 1 : 0;
      if (r.max_x > totals[3]) totals[3] = r.max_x;
    }
  }
  return 0;
}

// Records the event times and reaction indices of one trajectory (first
// record_max events) and its per-grid states into xs (G x S).
int oracle_trace(int S, int M, const int32_t* R, const int32_t* P, const double* c, const int32_t* x0,
                 int64_t traj_id, double t_end, int G, const double* grid, uint64_t seed,
                 uint64_t stream, int64_t max_events, int schedule, int precision, int record_max,
                 double* rec_t, int32_t* rec_j, int64_t* xs, int64_t* n_events) {
  if (!g_log.ready) return -1;
  Model m;
  if (!build_model(S, M, R, P, c, x0, &m)) return -1;
  std::vector<uint64_t> s1((size_t)G * S, 0), s2((size_t)G * S, 0);
  if ((schedule != 0 && schedule != 1) || (precision != 0 && precision != 1)) return -1;
  TrajResult r = run_one(m, (uint64_t)traj_id, t_end, G, grid, seed, stream, max_events, schedule, precision,
                         s1.data(), s2.data(), nullptr, nullptr, record_max, rec_t, rec_j);
  for (size_t q = 0; q < (size_t)G * S; ++q) xs[q] = (int64_t)s1[q];
  *n_events = r.events;
  return r.flags;
}

// Selective memory along the time axis (Sec. 3.2.1, Fig. 3), for
// trajectories [traj_begin, traj_begin + N):
//   Avg-Y: the union of every trajectory's event times, with t = 0, gives
//     points T_0 = 0 < T_1 < ... < T_{U-1}; at each, S1_m[s] = sum_i x_is(T_m)
//     and S2_m[s] = sum_i x_is(T_m)^2 (right-continuous states; int64);
//   Avg-XY: window p covers union points [p k, min(U, (p + 1) k)) of size n_p;
//     t_p = (T_a + ... + T_{b-1}) / n_p (FP64, ascending order), and
//     mean_p[s] = (double)(sum_m S1_m[s]) / (double)(N n_p),
//     msq_p[s]  = (double)(sum_m S2_m[s]) / (double)(N n_p).
// Writes min(P, max_points) points (P = ceil(U / k)); *n_points = P and
// *n_union = U.  Returns 0, or -1 on bad arguments.
int oracle_avg_xy(int S, int M, const int32_t* R, const int32_t* P, const double* c, const int32_t* x0,
                  int64_t traj_begin, int64_t N, double t_end, uint64_t seed, uint64_t stream, int64_t max_events,
                  int schedule, int precision, int64_t window, int64_t max_points, double* t_out, double* mean_out,
                  double* msq_out, int64_t* n_points, int64_t* n_union) {
  if (!g_log.ready || N < 1 || window < 1 || (schedule != 0 && schedule != 1) || (precision != 0 && precision != 1))
    return -1;
  Model m;
  if (!build_model(S, M, R, P, c, x0, &m)) return -1;
  // every trajectory's event list (a grid beyond t_end: no grid point is emitted)
  const double no_grid[1] = {std::numeric_limits<double>::infinity()};
  std::vector<std::vector<double>> times(N);
  std::vector<std::vector<int32_t>> rxn(N);
  std::vector<uint64_t> d1(S, 0), d2(S, 0);
  std::vector<double> all;
  for (int64_t i = 0; i < N; ++i) {
    const uint64_t id = (uint64_t)(traj_begin + i);
    TrajResult r = run_one(m, id, t_end, 1, no_grid, seed, stream, max_events, schedule, precision, d1.data(),
                           d2.data(), nullptr, nullptr, 0, nullptr, nullptr);
    times[i].resize(r.events);
    rxn[i].resize(r.events);
    run_one(m, id, t_end, 1, no_grid, seed, stream, max_events, schedule, precision, d1.data(), d2.data(),
            nullptr, nullptr, (int)r.events, times[i].data(), rxn[i].data());
    all.insert(all.end(), times[i].begin(), times[i].end());
  }
  std::sort(all.begin(), all.end());
  std::vector<double> T(1, 0.0);
  for (double v : all)
    if (v != T.back()) T.push_back(v);
  const int64_t U = (int64_t)T.size();
  std::vector<int64_t> S1((size_t)U * S, 0), S2((size_t)U * S, 0);
  for (int64_t i = 0; i < N; ++i) {
    std::vector<int64_t> x(m.x0.begin(), m.x0.end());
    size_t e = 0;
    for (int64_t q = 0; q < U; ++q) {
      while (e < times[i].size() && times[i][e] <= T[q]) {
        for (int s = 0; s < S; ++s) x[s] += m.nu[(size_t)rxn[i][e] * S + s];
        ++e;
      }
      for (int s = 0; s < S; ++s) {
        S1[(size_t)q * S + s] += x[s];
        S2[(size_t)q * S + s] += x[s] * x[s];
      }
    }
  }
  const int64_t Pn = (U + window - 1) / window;
  for (int64_t p = 0; p < Pn && p < max_points; ++p) {
    const int64_t a = p * window, b = std::min(U, a + window), n_p = b - a;
    double tsum = 0.0;
    for (int64_t q = a; q < b; ++q) tsum += T[q];
    t_out[p] = tsum / (double)n_p;
    for (int s = 0; s < S; ++s) {
      int64_t w1 = 0, w2 = 0;
      for (int64_t q = a; q < b; ++q) {
        w1 += S1[(size_t)q * S + s];
        w2 += S2[(size_t)q * S + s];
      }
      mean_out[(size_t)p * S + s] = (double)w1 / (double)(N * n_p);
      msq_out[(size_t)p * S + s] = (double)w2 / (double)(N * n_p);
    }
  }
  *n_points = Pn;
  *n_union = U;
  return 0;
}

// Sets (M > 0) or clears (M == 0) the rate modifiers of the models the
// calling thread builds next: for reaction j with f[j] >= 0 the rate is
// min(max(c_j + k[j] * x_{f[j]}, lo[j]), hi[j]) (the paper's TNF-dependent
// infectivities, Sec. 2.1).  Returns 0.
int oracle_set_modifiers(int M, const int32_t* f, const double* k, const double* lo, const double* hi) {
  if (M <= 0) {
    t_mod_f.clear();
    t_mod_k.clear();
    t_mod_lo.clear();
    t_mod_hi.clear();
    return 0;
  }
  t_mod_f.assign(f, f + M);
  t_mod_k.assign(k, k + M);
  t_mod_lo.assign(lo, lo + M);
  t_mod_hi.assign(hi, hi + M);
  return 0;
}

// Prefix sums of a[0..M) in the given schedule (0 = L, 1 = W32); for tests.
void oracle_prefix(int M, const double* a, int schedule, double* prefix, double* a0) {
  std::vector<double> av(a, a + M), pv(M);
  if (schedule == 0) {
    double s = 0.0;
    for (int j = 0; j < M; ++j) { s = (j == 0) ? av[0] : s + av[j]; pv[j] = s; }
    *a0 = s;
  } else {
    w32_prefix(av, M, pv, a0);
  }
  for (int j = 0; j < M; ++j) prefix[j] = pv[j];
}

// FP32 mode's a0 for binary32 propensities a[0..M) in the given schedule
// (L: one compensated pair; W32: the lanes' pairs scanned).  For tests.
double oracle_fp32_a0(int M, const float* a, int schedule) {
  std::vector<float> av(a, a + M);
  return (schedule == 0) ? compensated_sum(av, 0, M) : w32_pair_a0(av, M);
}

// The reaction the direct method picks for propensities a[0..M) (FP64
// values; FP32-mode callers pass the widened binary32 values and prefixes)
// and a target r2 * total; prefixes in the given schedule.  For tests.
int oracle_select(int M, const double* a, int schedule, double target) {
  std::vector<double> av(a, a + M), pv(M);
  double a0 = 0.0;
  if (schedule == 0) {
    for (int j = 0; j < M; ++j) { a0 = (j == 0) ? av[0] : a0 + av[j]; pv[j] = a0; }
  } else {
    w32_prefix(av, M, pv, &a0);
  }
  return select_reaction(av, pv, M, target);
}

// Per-trajectory likelihood-ratio contributions g[i][r] (run_one_grad) of
// trajectories [traj_begin, traj_end), FP64 mode; w, mu are G x S.  The
// gradient of L is the mean of g over trajectories.  Returns 0, or -1 on bad
// arguments (including a zero rate: the score needs c_r > 0).
int oracle_grad(int S, int M, const int32_t* R, const int32_t* P, const double* c, const int32_t* x0,
                int64_t traj_begin, int64_t traj_end, double t_end, int G, const double* grid, uint64_t seed,
                uint64_t stream, int64_t max_events, int schedule, const double* w, const double* mu, double* g) {
  if (!g_log.ready || traj_end < traj_begin || G < 1 || (schedule != 0 && schedule != 1)) return -1;
  Model m;
  if (!build_model(S, M, R, P, c, x0, &m)) return -1;
  if (!m.mod_f.empty()) return -1;  // the score below is for plain mass action
  for (int r = 0; r < M; ++r)
    if (!(c[r] > 0.0)) return -1;
  for (int64_t id = traj_begin; id < traj_end; ++id)
    run_one_grad(m, (uint64_t)id, t_end, G, grid, seed, stream, max_events, schedule, w, mu,
                 g + (size_t)(id - traj_begin) * M);
  return 0;
}

// mean = S1 / N; var = (N S2 - S1^2) / (N (N - 1)), numerator exact in int128
// and rounded once to double (var is NaN for N < 2).
void oracle_finalize(int64_t N, int G, int S, const int64_t* S1, const int64_t* S2,
                     double* mean, double* var) {
  for (size_t q = 0; q < (size_t)G * S; ++q) {
    mean[q] = (double)S1[q] / (double)N;
    if (N < 2) { var[q] = std::numeric_limits<double>::quiet_NaN(); continue; }
    i128 num = (i128)N * (i128)S2[q] - (i128)S1[q] * (i128)S1[q];
    var[q] = (double)num / ((double)N * (double)(N - 1));
  }
}

}  // extern "C"
