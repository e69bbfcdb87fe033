// Host-side check of libssa's integer FP64 routines (csrc/ssa_softfloat.cuh)
// against the CPU's IEEE round-to-nearest-even double arithmetic.
// Usage: softfloat_check <cases> <seed>; prints "<op> <tested> <mismatches> <fallbacks>" lines.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ssa_softfloat.cuh"

static uint64_t s_state;
static uint64_t next64() {  // splitmix64
  uint64_t z = (s_state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t bits(double v) { uint64_t b; std::memcpy(&b, &v, 8); return b; }
static double dbl(uint64_t b) { double v; std::memcpy(&v, &b, 8); return v; }

// positive normal double with exponent in [lo, hi] (biased)
static uint64_t rand_pos(int lo, int hi) {
  const uint64_t e = (uint64_t)(lo + (int)(next64() % (uint64_t)(hi - lo + 1)));
  uint64_t frac = next64() & ssa_sf::kFracMask;
  switch (next64() % 8) {  // edge mantissas
    case 0: frac = 0; break;
    case 1: frac = ssa_sf::kFracMask; break;
    case 2: frac = 1; break;
    default: break;
  }
  return (e << 52) | frac;
}

int main(int argc, char** argv) {
  const long cases = argc > 1 ? atol(argv[1]) : 1000000;
  s_state = argc > 2 ? strtoull(argv[2], nullptr, 10) : 1;
  long bad_mul = 0, fb_mul = 0, bad_div = 0, fb_div = 0, bad_cvt = 0, bad_scale = 0;
  for (long i = 0; i < cases; ++i) {
    // products c * h with h an integer below 2^53
    const uint64_t c = (next64() % 16 == 0) ? 0 : rand_pos(1, 2046);
    uint64_t h;
    switch (next64() % 4) {
      case 0: h = next64() % 1000; break;
      case 1: h = next64() & 0xFFFFFFFFULL; break;
      case 2: h = next64() >> 11; break;  // up to 2^53 - 1
      default: h = (next64() >> 11) | 1; break;
    }
    bool ok;
    const uint64_t got = ssa_sf::mul_u53(c, h, ok);
    const uint64_t want = bits(dbl(c) * (double)h);
    const bool in_range = (want >> 52) < 2047;
    if (!ok) {
      if (in_range) ++fb_mul;
    } else if (got != want) {
      ++bad_mul;
      if (bad_mul < 5) printf("MUL %016llx * %llu got %016llx want %016llx\n", (unsigned long long)c,
                              (unsigned long long)h, (unsigned long long)got, (unsigned long long)want);
    }
    // quotients n / d, exponents chosen so most results stay normal
    const uint64_t n = rand_pos(900, 1150), d = rand_pos(900, 1150);
    const uint64_t q = ssa_sf::div_pos(n, d, ok);
    const uint64_t qw = bits(dbl(n) / dbl(d));
    if (!ok) {
      ++fb_div;
    } else if (q != qw) {
      ++bad_div;
      if (bad_div < 5) printf("DIV %016llx / %016llx got %016llx want %016llx\n", (unsigned long long)n,
                              (unsigned long long)d, (unsigned long long)q, (unsigned long long)qw);
    }
    // conversions
    const uint64_t v = (next64() >> (next64() % 64)) | 1;
    if (ssa_sf::u64_to_f64(v) != bits((double)v)) ++bad_cvt;
    // scaling by 2^-53
    const uint64_t sx = rand_pos(60, 2046);
    const uint64_t sg = ssa_sf::scale_down(sx, 53, ok);
    if (!ok || sg != bits(dbl(sx) * 0x1p-53)) ++bad_scale;
  }
  // widening binary32 -> binary64: every non-negative finite value and +inf
  long bad_widen = 0, widened = 0;
  for (uint64_t fb = 0; fb <= 0x7F800000ULL; ++fb) {
    float f;
    const uint32_t fb32 = (uint32_t)fb;
    std::memcpy(&f, &fb32, 4);
    if (ssa_sf::f32_to_f64(fb32) != bits((double)f)) {
      ++bad_widen;
      if (bad_widen < 5) printf("WIDEN %08x\n", fb32);
    }
    ++widened;
  }
  printf("widen %ld %ld 0\n", widened, bad_widen);
  printf("mul %ld %ld %ld\n", cases, bad_mul, fb_mul);
  printf("div %ld %ld %ld\n", cases, bad_div, fb_div);
  printf("cvt %ld %ld 0\n", cases, bad_cvt);
  printf("scale %ld %ld 0\n", cases, bad_scale);
  return (bad_mul || bad_div || bad_cvt || bad_scale || bad_widen) ? 1 : 0;
}
