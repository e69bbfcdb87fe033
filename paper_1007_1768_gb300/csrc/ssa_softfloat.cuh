// IEEE binary64 round-to-nearest-even results computed with integer
// instructions.
//
// On this GPU one FP64 warp instruction occupies the SM's FP64 unit for about
// 19 cycles (a division for about 143), whether 1 or 32 lanes are active,
// while the integer pipes issue several warp instructions per cycle.  The
// step therefore moves the FP64 products, the quotient and the
// integer-to-double conversions of the direct method to these routines.  Each
// returns exactly the bit pattern of the corresponding IEEE operation in
// round-to-nearest-even (so results stay bit-identical to plain FP64
// arithmetic), for the operand ranges stated at each function; outside them it
// reports `ok = false` and the caller uses the hardware operation instead.
//
// Methods: products are exact 128-bit integer products of the significands,
// normalised by a leading-zero count and rounded with guard and sticky bits.
// The quotient uses a reciprocal of the normalised divisor from a float seed
// refined by two Newton-Raphson steps in 64-bit fixed point, a quotient
// estimate, and an exact remainder correction before rounding.
//
// The routines avoid data-dependent branches (both sides of a choice are
// formed and selected), so independent calls overlap and lanes of a warp do
// not diverge.  They compile for the host as well (for exhaustive checks
// against the CPU's own IEEE arithmetic).
#ifndef SSA_SOFTFLOAT_CUH_
#define SSA_SOFTFLOAT_CUH_

#include <cstdint>

#if defined(__CUDACC__)
#define SF_HD __host__ __device__ __forceinline__
#else
#define SF_HD inline
#endif

namespace ssa_sf {

constexpr uint64_t kFracMask = 0x000FFFFFFFFFFFFFULL;
constexpr uint64_t kImplicit = 0x0010000000000000ULL;

SF_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

SF_HD int64_t mulhi64(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

SF_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

SF_HD float rcp_f32(float x) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}

// Round the 64-bit significand `top` (leading one at bit 63), with `sticky`
// telling whether anything nonzero lies below it, to 53 bits and pack it with
// biased exponent `e` (the exponent of the leading one).  Carries from the
// rounding move into the exponent field as they should.
SF_HD uint64_t round_pack(uint64_t top, bool sticky, int e) {
  uint64_t mant = top >> 11;
  const uint64_t rbit = (top >> 10) & 1ULL;
  const uint64_t st = (((top & 0x3FFULL) != 0) || sticky) ? 1ULL : 0ULL;
  mant += rbit & (st | (mant & 1ULL));
  return ((uint64_t)(e - 1) << 52) + mant;
}

// x << s for 0 <= s <= 63 and (x >> 1) >> (63 - s), i.e. x >> (64 - s) with
// x >> 64 taken as 0: the pieces of a 128-bit left shift.
SF_HD uint64_t shl_hi_part(uint64_t lo, int s) { return (lo >> 1) >> (63 - s); }

// (double)v for v > 0 (any uint64), round to nearest even.
SF_HD uint64_t u64_to_f64(uint64_t v) {
  const int lz = clz64(v);
  return round_pack(v << lz, false, 1086 - lz);
}

// RN(x * h) for x a non-negative double given by its bits and an integer
// 0 <= h < 2^53 (so (double)h is exact).  ok = false when x is subnormal,
// infinite or NaN, h >= 2^53, or the product overflows.  No data-dependent
// branches: both normalisations are formed and selected.
SF_HD uint64_t mul_u53(uint64_t xb, uint64_t h, bool& ok) {
  const int ex = (int)(xb >> 52);
  const uint64_t mx = (xb & kFracMask) | kImplicit;
  const uint64_t lo = mx * h;
  const uint64_t hi = umulhi64(mx, h);
  const bool big = hi != 0;
  const int lzh = clz64(hi | 1ULL);                  // valid when big
  const int lzl = clz64(lo | 1ULL);                  // valid when !big (lo != 0 then)
  const uint64_t top = big ? ((hi << lzh) | shl_hi_part(lo, lzh)) : (lo << lzl);
  const bool sticky = big && ((lo << lzh) != 0);
  const int lz = big ? lzh : 64 + lzl;
  // product = mx * h; value = product * 2^(ex - 1075); leading one of the
  // product at bit 127 - lz, so the result's biased exponent is ex + 75 - lz
  const uint64_t r = round_pack(top, sticky, ex + 75 - lz);
  const bool zero = (xb == 0) || (h == 0);
  ok = zero || (ex != 0 && ex < 2047 && (h >> 53) == 0 && (r >> 52) < 2047);
  return zero ? 0ULL : r;
}

// Scale a positive normal double by 2^-s (s > 0) when the result stays
// normal; ok = false otherwise.
SF_HD uint64_t scale_down(uint64_t xb, int s, bool& ok) {
  const int ex = (int)(xb >> 52);
  ok = ex > s;
  return xb - ((uint64_t)s << 52);
}

// Reciprocal estimate V ~ (2^127 - 1) / D for a normalised 64-bit D in
// [2^63, 2^64): float seed (about 22 good bits) and two Newton-Raphson steps
// V <- V + V (2^127 - D V) / 2^127 in fixed point.  |V - 2^127/D| stays below
// a few units, which the caller's exact remainder step absorbs.
SF_HD uint64_t recip_norm64(uint64_t D) {
  const float f = (float)(uint32_t)(D >> 40);            // exact: 24 bits
  const float r = rcp_f32(f) * 0x1p87f;                   // ~ 2^127 / D
  uint64_t V = (r >= 0x1p64f) ? ~0ULL : (uint64_t)r;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // E = 2^127 - D V as a signed 128-bit value (|E| << 2^127)
    const uint64_t plo = D * V;
    const uint64_t phi = umulhi64(D, V);
    const uint64_t elo = 0ULL - plo;
    const uint64_t ehi = 0x8000000000000000ULL - phi - ((plo != 0) ? 1ULL : 0ULL);
    // C = V * E / 2^127 ~ mulhi(V, E >> 63), E >> 63 signed
    const uint64_t e63 = (ehi << 1) | (elo >> 63);
    const uint64_t c = umulhi64(V, e63) - (((int64_t)e63 < 0) ? V : 0ULL);
    V += c;
  }
  return V;
}

// RN(n / d) for positive normal doubles n, d given by their bits.  ok = false
// when an operand is not a positive normal double or the quotient would be
// subnormal or overflow.  No data-dependent branches.
SF_HD uint64_t div_pos(uint64_t nb, uint64_t db, bool& ok) {
  const int en = (int)(nb >> 52), ed = (int)(db >> 52);
  const uint64_t mn = (nb & kFracMask) | kImplicit;
  const uint64_t md = (db & kFracMask) | kImplicit;
  // Q = floor(mn 2^54 / md) = floor(mn 2^65 / D), D = md 2^11; Q in (2^53, 2^55)
  const uint64_t V = recip_norm64(md << 11);
  // estimate: mn * V / 2^62
  const uint64_t plo = mn * V;
  const uint64_t phi = umulhi64(mn, V);
  uint64_t q = (phi << 2) | (plo >> 62);
  // exact remainder mn 2^54 - q md, small, computed modulo 2^64
  int64_t rem = (int64_t)((mn << 54) - q * md);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const bool low = rem < 0;
    q -= low ? 1ULL : 0ULL;
    rem += low ? (int64_t)md : 0;
    const bool high = rem >= (int64_t)md;
    q += high ? 1ULL : 0ULL;
    rem -= high ? (int64_t)md : 0;
  }
  const bool wide = (q >> 54) != 0;  // q in [2^54, 2^55) versus [2^53, 2^54)
  const int e = en - ed + (wide ? 1023 : 1022);
  const uint64_t top = wide ? (q << 9) : (q << 10);
  const uint64_t r = round_pack(top, rem != 0, e);
  ok = en != 0 && en < 2047 && ed != 0 && ed < 2047 && rem >= 0 && rem < (int64_t)md && e > 0 && e < 2047 &&
       (r >> 52) < 2047;
  return r;
}

// Exact widening of a non-negative binary32 value (zero, subnormal, normal
// or +inf, given by its bits) to binary64, returned as bits.  Normal values
// rebias the exponent (127 -> 1023) and move the significand up 29 bits;
// subnormal ones m 2^-149 are normalised by the leading-zero count of m.
SF_HD uint64_t f32_to_f64(uint32_t fb) {
  const uint32_t e = fb >> 23;
  const uint64_t m = fb & 0x7FFFFFu;
  const uint64_t normal = ((uint64_t)(e + 896u) << 52) | (m << 29);
  const uint64_t inf = 0x7FF0000000000000ULL | (m << 29);
  // subnormal: leading one of m at bit 22 - (lz - 41) with lz = clz64(m)
  const int lz = clz64(m | 1ULL);
  const int sh = lz - 40;                                  // moves the leading one to bit 23
  const uint64_t sub = ((uint64_t)(897 - sh) << 52) | (((m << sh) & 0x7FFFFFULL) << 29);
  return (e == 255u) ? inf : (e != 0u ? normal : (m != 0 ? sub : 0ULL));
}

}  // namespace ssa_sf

#endif  // SSA_SOFTFLOAT_CUH_
