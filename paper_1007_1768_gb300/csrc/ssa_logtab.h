// Compile-time constants of the fixed-point -ln(u) used by the device step.
//
// Method: Tang's table-driven logarithm (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic",
// ACM TOMS 16(4), 1990), carried out in 64-bit fixed point:
//   F_i = 1 + (2i + 1) / 256, i = 0..127  (centres of 128 cells of [1, 2))
//   kLogInv[i] = round(2^64 / F_i)
//   kLogLnF[i] = round(2^64 ln F_i)
//   kLogLn2    = round(2^64 ln 2)
//   kLogHorner[m] = round((-1)^(m+1) 2^62 / m), m = 1..7 (Taylor coefficients
//   of ln(1 + r) in Q1.62).
// ln F = 2 atanh(a / b) with a = 2i + 1, b = 513 + 2i (and ln 2 = 2 atanh(1/3))
// is summed here in Q.100 fixed point with unsigned 128-bit integers: the
// powers (a/b)^(2k+1) follow p_{k+1} = floor(p_k a^2 / b^2), each term is
// floor(p_k / (2k + 1)); the accumulated floor error stays below 2^-92, far
// under the final rounding to 2^-64.
#ifndef SSA_LOGTAB_H_
#define SSA_LOGTAB_H_

#include <cstdint>

namespace ssa_logtab {

typedef unsigned __int128 u128;

constexpr int kFracBits = 100;

// 2 * atanh(a / b) * 2^kFracBits (floor-accumulated), a / b < 1/2.
constexpr u128 two_atanh_q100(uint64_t a, uint64_t b) {
  u128 p = ((u128)a << kFracBits) / b;
  u128 sum = 0;
  const u128 a2 = (u128)a * a, b2 = (u128)b * b;
  for (uint64_t k = 0; p != 0; ++k) {
    sum += p / (2 * k + 1);
    p = p * a2 / b2;
  }
  return 2 * sum;
}

// round(v / 2^(kFracBits - 64)) as a 64-bit word.
constexpr uint64_t to_q64(u128 v) {
  return (uint64_t)((v + ((u128)1 << (kFracBits - 65))) >> (kFracBits - 64));
}

struct Tables {
  uint64_t inv[128];
  uint64_t lnf[128];
  uint64_t ln2;
  int64_t horner[8];
};

constexpr Tables make_tables() {
  Tables t{};
  for (int i = 0; i < 128; ++i) {
    const uint64_t den = 257 + 2 * (uint64_t)i;            // 256 F_i
    const u128 q = ((u128)1 << 73) / den;                  // 2 * 2^72 / den, floored
    t.inv[i] = (uint64_t)((q + 1) >> 1);                   // round(2^72 / den)
    t.lnf[i] = to_q64(two_atanh_q100(2 * (uint64_t)i + 1, 513 + 2 * (uint64_t)i));
  }
  t.ln2 = to_q64(two_atanh_q100(1, 3));
  t.horner[0] = 0;
  for (int m = 1; m <= 7; ++m) {
    const uint64_t num = (uint64_t)1 << 62;
    const uint64_t mag = (num + (uint64_t)m / 2) / (uint64_t)m;  // round(2^62 / m)
    t.horner[m] = (m % 2 == 1) ? (int64_t)mag : -(int64_t)mag;
  }
  return t;
}

constexpr Tables kTables = make_tables();

}  // namespace ssa_logtab

#endif  // SSA_LOGTAB_H_
