// Compile-time constants of the fixed-point -ln(u) used by the device step.
//
// Method: Tang's table-driven logarithm (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic",
// ACM TOMS 16(4), 1990), carried out in 64-bit fixed point:
//   F_i = 1 + (2i + 1) / 1024, i = 0..511  (centres of 512 cells of [1, 2))
//   inv[i] = round(2^64 / F_i)
//   lnf[i] = round(2^64 ln F_i)
//   ln2    = round(2^64 ln 2)
//   k3, k5 = round(2^31 / 3), round(2^31 / 5)  (series coefficients in Q1.31)
// ln F = 2 atanh(a / b) with a = 2i + 1, b = 2049 + 2i (and ln 2 = 2 atanh(1/3))
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

constexpr int kCells = 512;

struct Tables {
  uint64_t inv[kCells];
  uint64_t lnf[kCells];
  uint64_t ln2;
  int32_t k3, k5;
};

constexpr Tables make_tables() {
  Tables t{};
  for (int i = 0; i < kCells; ++i) {
    const uint64_t den = 1025 + 2 * (uint64_t)i;           // 1024 F_i
    const u128 q = ((u128)1 << 75) / den;                  // 2 * 2^74 / den, floored
    t.inv[i] = (uint64_t)((q + 1) >> 1);                   // round(2^74 / den)
    t.lnf[i] = to_q64(two_atanh_q100(2 * (uint64_t)i + 1, 2049 + 2 * (uint64_t)i));
  }
  t.ln2 = to_q64(two_atanh_q100(1, 3));
  t.k3 = (int32_t)((((uint64_t)1 << 32) / 3 + 1) >> 1);   // round(2^31 / 3)
  t.k5 = (int32_t)((((uint64_t)1 << 32) / 5 + 1) >> 1);   // round(2^31 / 5)
  return t;
}

constexpr Tables kTables = make_tables();

}  // namespace ssa_logtab

#endif  // SSA_LOGTAB_H_
