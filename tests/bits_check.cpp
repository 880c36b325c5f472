// Host check of the bit-level helpers of the CUDA path (hs_bits.cuh) against
// independent references: integer division, and splits computed with frexp /
// ldexp / round / nearbyint in double arithmetic. Prints "ok" or the first
// mismatch and exits non-zero.
#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "hs_bits.cuh"

using namespace hs;

static uint32_t fbits(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

// x rounded to `bits` significant bits: ties away (away) or ties to even
static double round_sig(double x, int bits, bool away) {
  int e;
  std::frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  const double s = std::ldexp(x, bits - e);
  const double r = away ? std::round(s) : std::nearbyint(s);
  return std::ldexp(r, e - bits);
}

int main() {
  std::fesetround(FE_TONEAREST);
  // 1. division by invariant integers
  std::mt19937_64 rng(12345);
  const unsigned ds[] = {1, 2, 3, 5, 6, 7, 10, 15, 21, 36, 144, 666, 1023, 1024, 1025, 2592, 65535, 65536,
                         65537, 1000003, 2147483647u, 2147483648u, 4294967295u};
  const unsigned ns[] = {0, 1, 2, 3, 1023, 1024, 65535, 65536, 2147483647u, 2147483648u, 4294967294u,
                         4294967295u};
  for (unsigned d : ds) {
    unsigned mag;
    unsigned char s1, s2;
    fast_div_magic(d, &mag, &s1, &s2);
    for (unsigned n : ns)
      if (fast_div(n, mag, s1, s2) != n / d) {
        std::printf("div %u / %u\n", n, d);
        return 1;
      }
    for (int i = 0; i < 200000; ++i) {
      const unsigned n = (unsigned)rng();
      if (fast_div(n, mag, s1, s2) != n / d) {
        std::printf("div %u / %u\n", n, d);
        return 1;
      }
    }
  }
  for (int i = 0; i < 200000; ++i) {
    const unsigned d = (unsigned)(rng() % 100000) + 1, n = (unsigned)rng();
    unsigned mag;
    unsigned char s1, s2;
    fast_div_magic(d, &mag, &s1, &s2);
    if (fast_div(n, mag, s1, s2) != n / d) {
      std::printf("div %u / %u\n", n, d);
      return 1;
    }
  }
  // 2. splits: TF32 (11 bits, ties away) + FP32 remainder; BF16 (8, even) + BF16
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-120, 120);
  for (int i = 0; i < 2000000; ++i) {
    double x = std::ldexp(u(rng), ex(rng));
    if (i % 97 == 0) x = std::ldexp(std::nearbyint(std::ldexp(u(rng), 12)) + 0.5, -12 + ex(rng));  // ties
    if (x == 0.0) continue;
    uint32_t h, l;
    split_f64(x, 11, 24, true, h, l);
    if (std::fabs(x) < 1.17549435e-38) {  // below the single normal range: zeros (documented)
      if ((h & 0x7FFFFFFFu) != 0u || (l & 0x7FFFFFFFu) != 0u) return std::printf("flush %.17g\n", x), 1;
      continue;
    }
    const double hr = round_sig(x, 11, true);
    const float lr = (float)(x - hr);
    // below the single normal range the split returns zero (documented)
    const bool lr_tiny = std::fabs(lr) < 1.17549435e-38f;
    if (h != fbits((float)hr) || (l != fbits(lr) && !(lr_tiny && (l & 0x7FFFFFFFu) == 0u))) {
      std::printf("tf32 split of %.17g: %08x %08x vs %08x %08x\n", x, h, l, fbits((float)hr), fbits(lr));
      return 1;
    }
    split_f64(x, 8, 8, false, h, l);
    const double hb = round_sig(x, 8, false);
    const double rb = x - hb;
    const double lb = rb == 0.0 ? 0.0 : round_sig(rb, 8, false);
    const bool lb_tiny = std::fabs(lb) < 1.17549435e-38;
    if (h != fbits((float)hb) || (l != fbits((float)lb) && !(lb_tiny && (l & 0x7FFFFFFFu) == 0u))) {
      std::printf("bf16 split of %.17g: %08x %08x vs %08x %08x\n", x, h, l, fbits((float)hb), fbits((float)lb));
      return 1;
    }
  }
  // 2b. the 32-bit TF32 split is bit-identical to the general one, over
  // random significands at every exponent (both ends of the single range
  // included) and on ties
  std::uniform_int_distribution<unsigned long long> um(0, (1ull << 52) - 1);
  for (int e = 0; e < 2047; ++e)
    for (int i = 0; i < 600; ++i) {
      unsigned long long m = um(rng);
      if (i % 5 == 1) m = (m >> 42) << 42 | (1ull << 41);        // exact tie of hi
      if (i % 5 == 2) m &= ~((1ull << 41) - 1);                  // zero remainder
      if (i % 5 == 3) m = (m >> 42) << 42 | (m & 0xFFFull);      // tiny remainder
      const unsigned long long bb = (unsigned long long)(i & 1) << 63 | (unsigned long long)e << 52 | m;
      const double x = f64_from_bits(bb);
      uint32_t h1, l1, h2, l2;
      split_f64(x, 11, 24, true, h1, l1);
      split_tf32x3(x, h2, l2);
      if (h1 != h2 || l1 != l2) {
        std::printf("tf32x3 split of %.17g: %08x %08x vs %08x %08x\n", x, h2, l2, h1, l1);
        return 1;
      }
    }
  // 2c. the split of an FP32 value through one FP32 subtraction equals the
  // general split of the same value, at every single exponent
  std::uniform_int_distribution<uint32_t> u23(0, (1u << 23) - 1);
  for (uint32_t e = 1; e < 255; ++e)
    for (int i = 0; i < 4000; ++i) {
      uint32_t m = u23(rng);
      if (i % 7 == 1) m = (m & ~0x1FFFu) | 0x1000u;  // exact tie of hi
      if (i % 7 == 2) m &= ~0x1FFFu;                 // zero remainder
      if (i % 7 == 3) m = 0x7FFFFFu;                  // carry into the exponent
      const uint32_t uu = (uint32_t)(i & 1) << 31 | e << 23 | m;
      float fv;
      std::memcpy(&fv, &uu, 4);
      uint32_t h1, l1, h2, l2;
      split_f64((double)fv, 11, 24, true, h1, l1);
      split_f32_tf32x3(uu, h2, l2);
      if (h1 != h2 || l1 != l2) {
        std::printf("f32 tf32x3 split of %08x: %08x %08x vs %08x %08x\n", uu, h2, l2, h1, l1);
        return 1;
      }
    }
  // 2d. the select form of that split gives the same bits for every pattern
  // (all exponents, zeros, subnormals, infinities, NaNs)
  for (uint64_t k = 0; k < (1ull << 32); k += 4093) {
    const uint32_t uu = (uint32_t)k;
    for (uint32_t v : {uu, uu | 0x7F800000u, uu & 0x807FFFFFu, uu | 0x7FFFF000u, uu & 0x80000000u}) {
      uint32_t h2, l2, h3, l3;
      split_f32_tf32x3(v, h2, l2);
      split_f32_tf32x3_sel(v, h3, l3);
      if (h2 != h3 || l2 != l3) {
        std::printf("select split of %08x: %08x %08x vs %08x %08x\n", v, h3, l3, h2, l2);
        return 1;
      }
    }
  }
  // 2e. the epilogue's form: the same bits except where the general split
  // rounds up to 2^128 or the input is NaN / infinity; non-finite there
  for (uint64_t k = 0; k < (1ull << 32); k += 4093) {
    const uint32_t uu = (uint32_t)k;
    for (uint32_t v : {uu, uu | 0x7F800000u, uu & 0x807FFFFFu, uu | 0x7FFFF000u, uu & 0x80000000u,
                       (uu & 0x80FFFFFFu) | 0x7E800000u}) {
      uint32_t h2, l2, h4, l4;
      split_f32_tf32x3(v, h2, l2);
      split_f32_tf32x3_fin(v, h4, l4);
      const bool top = (v & 0x7F800000u) == 0x7F800000u || ((h2 & 0x7F800000u) == 0x7F800000u);
      if (top) {
        if ((h4 & 0x7F800000u) != 0x7F800000u && (l4 & 0x7F800000u) != 0x7F800000u) {
          std::printf("fin split of %08x is finite: %08x %08x\n", v, h4, l4);
          return 1;
        }
      } else if (h2 != h4 || l2 != l4) {
        std::printf("fin split of %08x: %08x %08x vs %08x %08x\n", v, h4, l4, h2, l2);
        return 1;
      }
    }
  }
  // zero, tiny, NaN
  uint32_t h, l;
  split_f64(0.0, 11, 24, true, h, l);
  if (h != 0u || l != 0u) return std::printf("zero\n"), 1;
  split_f64(-1e-300, 11, 24, true, h, l);
  if (h != 0x80000000u || l != 0x80000000u) return std::printf("tiny\n"), 1;
  split_f64(std::nan(""), 11, 24, true, h, l);
  if (h != 0x7FC00000u) return std::printf("nan\n"), 1;
  // 3. FP32 -> FP64 widening
  std::uniform_int_distribution<uint32_t> ub;
  for (int i = 0; i < 2000000; ++i) {
    uint32_t f = ub(rng);
    if (i < 4) f = (uint32_t[]){0u, 0x80000000u, 0x7F800000u, 0xFF800000u}[i];
    float fv;
    std::memcpy(&fv, &f, 4);
    unsigned long long o;
    if (!f32_widen_fast(f, o)) {
      if ((f & 0x7F800000u) != 0u) return std::printf("widen refused %08x\n", f), 1;
      continue;
    }
    const double d = f64_from_bits(o);
    if (std::isnan(fv) ? !std::isnan(d) : (f64_bits(d) != f64_bits((double)fv))) {
      std::printf("widen %08x\n", f);
      return 1;
    }
  }
  std::printf("ok\n");
  return 0;
}
