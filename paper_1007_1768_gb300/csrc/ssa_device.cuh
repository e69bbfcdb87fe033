// Device primitives of the SSA step: counter-based random numbers, the
// fixed-point -ln(u), integer-pattern comparisons of non-negative doubles and
// an exactly rounded int128 -> double conversion.
//
// Everything here is compiled with -fmad=false and uses the _rn intrinsics,
// so each FP64 operation is one IEEE operation in round-to-nearest-even.
#ifndef SSA_DEVICE_CUH_
#define SSA_DEVICE_CUH_

#include <cstdint>

#include "ssa_logtab.h"

namespace ssa_dev {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): 10 rounds of two 64x64->128 multiplies and a
// key-dependent xor, key bumped by two Weyl increments between rounds.
struct Words4 {
  uint64_t w0, w1, w2, w3;
};

__device__ __forceinline__ Words4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1) {
  constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ULL;
  constexpr uint64_t kM1 = 0xCA5A826395121157ULL;
  constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ULL;
  constexpr uint64_t kW1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
    const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0;
    const uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return Words4{c0, c1, c2, c3};
}

// Odd 53-bit integer q = 2 (w >> 12) + 1; the uniform variate is q * 2^-53.
__device__ __forceinline__ uint64_t odd53(uint64_t w) { return ((w >> 12) << 1) | 1ULL; }

// Exact q * 2^-53 for q < 2^53.
__device__ __forceinline__ double uniform_from_odd53(uint64_t q) {
  return __dmul_rn(__ull2double_rn(q), 0x1p-53);
}

// floor(d * v / 2^64) for signed d and unsigned v.
__device__ __forceinline__ int64_t mulhi_su(int64_t d, uint64_t v) {
  uint64_t h = __umul64hi((uint64_t)d, v);
  if (d < 0) h -= v;
  return (int64_t)h;
}

// E = -ln(q * 2^-53) for odd q in [1, 2^53), formed in units of 2^-64 and
// rounded once to double.  q = 2^e (1 + f); the top 7 bits of f pick the cell
// centre c_i and F_i = 1 + c_i; r = (f - c_i) / F_i with |r| < 2^-8;
// E = (53 - e) ln 2 - ln F_i - ln(1 + r), ln(1 + r) by its series to r^7.
// inv / lnf are the cell tables (kLogInv, kLogLnF), staged in shared memory.
__device__ __forceinline__ double neg_log_u(uint64_t q, const uint64_t* __restrict__ inv,
                                            const uint64_t* __restrict__ lnf) {
  const int e = 63 - __clzll((long long)q);
  const uint64_t f = (q << (63 - e)) << 1;
  const int i = (int)(f >> 57);
  const uint64_t center = ((uint64_t)(2 * i + 1)) << 56;
  const int64_t d = (int64_t)(f - center);
  const int64_t r = mulhi_su(d, inv[i]);
  constexpr int64_t K1 = ssa_logtab::kTables.horner[1];
  constexpr int64_t K2 = ssa_logtab::kTables.horner[2];
  constexpr int64_t K3 = ssa_logtab::kTables.horner[3];
  constexpr int64_t K4 = ssa_logtab::kTables.horner[4];
  constexpr int64_t K5 = ssa_logtab::kTables.horner[5];
  constexpr int64_t K6 = ssa_logtab::kTables.horner[6];
  constexpr int64_t K7 = ssa_logtab::kTables.horner[7];
  int64_t acc = K7;
  acc = K6 + __mul64hi(acc, r);
  acc = K5 + __mul64hi(acc, r);
  acc = K4 + __mul64hi(acc, r);
  acc = K3 + __mul64hi(acc, r);
  acc = K2 + __mul64hi(acc, r);
  acc = K1 + __mul64hi(acc, r);
  // ln(1 + r) = (acc * r) >> 62 as a signed 128-bit product, fits in 64 bits
  const uint64_t plo = (uint64_t)acc * (uint64_t)r;
  const int64_t phi = __mul64hi(acc, r);
  const int64_t ln1p = (int64_t)(((uint64_t)phi << 2) | (plo >> 62));
  // E = n ln2 - lnF_i - ln1p in 128 bits
  constexpr uint64_t LN2 = ssa_logtab::kTables.ln2;
  const uint64_t n = (uint64_t)(53 - e);
  uint64_t lo = n * LN2;
  uint64_t hi = __umul64hi(n, LN2);
  const uint64_t lf = lnf[i];
  hi -= (lo < lf) ? 1ULL : 0ULL;
  lo -= lf;
  const uint64_t l1 = (uint64_t)ln1p;
  hi = hi - ((lo < l1) ? 1ULL : 0ULL) + ((ln1p < 0) ? 1ULL : 0ULL);
  lo -= l1;
  if (hi == 0) return __dmul_rn(__ull2double_rn(lo), 0x1p-64);
  return __dmul_rn(__ull2double_rn((hi << 58) | (lo >> 6)), 0x1p-58);
}

// Bit pattern of a double as a signed integer; for non-negative doubles (and
// +inf) the integer order equals the numeric order, so comparisons of
// propensity sums, targets and times run on the integer pipe.
__device__ __forceinline__ long long obits(double v) { return __double_as_longlong(v); }

// Exactly rounded (nearest-even) conversion of a signed 128-bit value given
// as (hi, lo) to double: values below 2^64 convert directly; larger values
// keep their top 64 bits with a sticky bit for everything below, which
// cannot change a rounding made 11 bits higher up, and are rescaled by an
// exact power of two.
__device__ __forceinline__ double i128_to_double_rn(int64_t hi_s, uint64_t lo) {
  const bool neg = hi_s < 0;
  uint64_t hi = (uint64_t)hi_s;
  if (neg) {  // magnitude of the two's complement value
    lo = ~lo + 1ULL;
    hi = ~hi + ((lo == 0) ? 1ULL : 0ULL);
  }
  double mag;
  if (hi == 0) {
    mag = __ull2double_rn(lo);
  } else {
    const int lz = __clzll((long long)hi);
    const uint64_t top = (lz == 0) ? hi : ((hi << lz) | (lo >> (64 - lz)));
    const uint64_t rest = lo << lz;
    const uint64_t jam = top | ((rest != 0) ? 1ULL : 0ULL);
    mag = __dmul_rn(__ull2double_rn(jam), __longlong_as_double((long long)(1023 + 64 - lz) << 52));
  }
  return neg ? -mag : mag;
}

}  // namespace ssa_dev

#endif  // SSA_DEVICE_CUH_
