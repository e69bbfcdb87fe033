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
#include "ssa_softfloat.cuh"

namespace ssa_dev {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies and a
// key-dependent xor, the key bumped by two Weyl increments between rounds.
struct Words4 {
  uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                uint32_t k1) {
  constexpr uint32_t kM0 = 0xD2511F53u;
  constexpr uint32_t kM1 = 0xCD9E8D57u;
  constexpr uint32_t kW0 = 0x9E3779B9u;
  constexpr uint32_t kW1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kM0, c0), lo0 = kM0 * c0;
    const uint32_t hi1 = __umulhi(kM1, c2), lo1 = kM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return Words4{c0, c1, c2, c3};
}

// q = 2 ((a << 20) | (b >> 12)) + 1: an odd 53-bit integer; the uniform
// variate is q * 2^-53, exactly representable and strictly inside (0, 1).
__device__ __forceinline__ uint64_t odd53(uint32_t a, uint32_t b) {
  return ((((uint64_t)a << 20) | (uint64_t)(b >> 12)) << 1) | 1ULL;
}

// floor(d * v / 2^64) for signed d and unsigned v.
__device__ __forceinline__ int64_t mulhi_su(int64_t d, uint64_t v) {
  return (int64_t)(__umul64hi((uint64_t)d, v) - ((d < 0) ? v : 0ULL));
}

// E = -ln(q * 2^-53) for odd q in [1, 2^53), formed in units of 2^-64 and
// rounded once to double; returned as the double's bit pattern.
//   q = 2^e (1 + f); the top 9 bits of f pick the cell centre c_i, F_i = 1 + c_i;
//   r = (f - c_i) / F_i with |r| < 2^-10 (floor(d * inv_i / 2^64));
//   E = (53 - e) ln 2 - ln F_i - ln(1 + r),
//   ln(1 + r) = r - r^2/2 + r^3 w, w = 1/3 - r/4 + r^2/5 kept in 32-bit Q1.31
//   (w only needs ~2^-31 since |r^3| < 2^-30), r^2 and r^3 in Q.64.
// inv / lnf are the 512-cell tables of ssa_logtab.h, staged in shared memory.
__device__ __forceinline__ uint64_t neg_log_u_bits(uint64_t q, const uint64_t* __restrict__ inv,
                                                   const uint64_t* __restrict__ lnf) {
  const int e = 63 - __clzll((long long)q);
  const uint64_t f = (q << (63 - e)) << 1;
  const int i = (int)(f >> 55);
  const uint64_t center = ((uint64_t)(2 * i + 1)) << 54;
  const int64_t d = (int64_t)(f - center);
  const int64_t r = mulhi_su(d, inv[i]);
  const int64_t r2 = __mul64hi(r, r);
  const int64_t r3 = __mul64hi(r2, r);
  constexpr int32_t K3 = ssa_logtab::kTables.k3;
  constexpr int32_t K5 = ssa_logtab::kTables.k5;
  const int32_t rq = (int32_t)(r >> 33);
  const int32_t r2q = (int32_t)(r2 >> 33);
  const int32_t w = K3 - (rq >> 2) + (int32_t)(((long long)r2q * K5) >> 31);
  const int64_t t3 = ((r3 >> 4) * (int64_t)w) >> 27;
  const int64_t ln1p = r - (r2 >> 1) + t3;
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
  // the integer is >= 2^11 and its double >= 2^11, so scaling by 2^-64 or
  // 2^-58 keeps it normal: subtract from the exponent field
  const bool small = hi == 0;
  const uint64_t v = small ? lo : ((hi << 58) | (lo >> 6));
  return ssa_sf::u64_to_f64(v) - ((small ? 64ULL : 58ULL) << 52);
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
