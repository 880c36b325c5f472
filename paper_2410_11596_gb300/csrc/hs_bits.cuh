// Bit-level helpers shared by the layout and tensor-core kernels; plain C++
// on the host as well, so that a host test can check them exhaustively.
//
// Why integer arithmetic: on this GPU the FP64 pipe (which also executes
// conversions to and from FP64) runs at ~1.7 operations per clock per SM,
// the integer pipe at 64. Splitting FP64 operands for the multi-pass tensor
// products and widening FP32 accumulators to FP64 are therefore done on the
// IEEE-754 bit patterns.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define HS_HD __host__ __device__ __forceinline__
#else
#define HS_HD inline
#endif

namespace hs {

HS_HD int clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

HS_HD unsigned long long f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

HS_HD double f64_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

// Quotient n / d for 32-bit n from magic numbers of d (Granlund and
// Montgomery, PLDI 1994, unsigned division by invariant integers):
// l = ceil(log2 d), mag = floor(2^32 (2^l - d) / d) + 1, sh1 = min(l, 1),
// sh2 = max(l - 1, 0), q = (t + ((n - t) >> sh1)) >> sh2 with t = mulhi(mag, n).
HS_HD unsigned fast_div(unsigned n, unsigned mag, unsigned sh1, unsigned sh2) {
#ifdef __CUDA_ARCH__
  const unsigned t = __umulhi(mag, n);
#else
  const unsigned t = (unsigned)(((unsigned long long)mag * n) >> 32);
#endif
  return (t + ((n - t) >> sh1)) >> sh2;
}

inline void fast_div_magic(unsigned d, unsigned* mag, unsigned char* sh1, unsigned char* sh2) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  *mag = (unsigned)((((1ull << l) - d) << 32) / d + 1);
  *sh1 = (unsigned char)(l < 1 ? l : 1);
  *sh2 = (unsigned char)(l > 1 ? l - 1 : 0);
}

// A * 2^k (A > 0) rounded to `bits` significant bits, ties to even, as IEEE
// single bits with the given sign; below the normal range: signed zero,
// above it: infinity.
HS_HD uint32_t round_to_float(unsigned long long A, int k, int bits, uint32_t sign) {
  const int top = 63 - clz64(A);
  const int drop = top + 1 - bits;
  unsigned long long sig;
  if (drop > 0) {
    const unsigned long long half = 1ull << (drop - 1), rem = A & ((1ull << drop) - 1);
    sig = A >> drop;
    if (rem > half || (rem == half && (sig & 1))) ++sig;
  } else {
    sig = A << (-drop);
  }
  // sig in [2^(bits-1), 2^bits]; a carry to 2^bits lands in the exponent field
  const int fe = k + top + 127;
  if (fe <= 0) return (fe == 0 && sig == (1ull << bits)) ? (sign | 0x00800000u) : sign;  // rounds up to 2^-126
  if (fe >= 255) return sign | 0x7F800000u;
  const uint32_t v = ((uint32_t)fe << 23) + ((uint32_t)(sig - (1ull << (bits - 1))) << (24 - bits));
  return v >= 0x7F800000u ? (sign | 0x7F800000u) : (sign | v);
}

// x ~ hi + lo for the multi-pass tensor-core products:
//   hi = x rounded to `hb` significant bits (ties away from zero when
//        `hi_away`, as cvt.rna.tf32; else ties to even),
//   lo = x - hi (exact as an integer) rounded to `lb` significant bits, ties to even.
// Both as IEEE single bit patterns. |x| < 2^-126 (FP64 subnormals included)
// gives zeros, far below the split's own rounding; NaN and infinity give NaN.
HS_HD void split_f64(double x, int hb, int lb, bool hi_away, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = f64_bits(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0x7FF) {
    hi = lo = 0x7FC00000u;
    return;
  }
  const int fe = e - 896;  // single-precision exponent field of x
  if (fe <= 0) {
    hi = lo = sign;
    return;
  }
  if (fe >= 255) {  // beyond the single range
    hi = lo = sign | 0x7F800000u;
    return;
  }
  const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);  // |x| = M 2^(e-1075)
  const int drop = 53 - hb;
  const unsigned long long half = 1ull << (drop - 1), rem = M & ((1ull << drop) - 1);
  unsigned long long sh = M >> drop;
  if (rem > half || (rem == half && (hi_away || (sh & 1)))) ++sh;
  const uint32_t hv = ((uint32_t)fe << 23) + ((uint32_t)(sh - (1ull << (hb - 1))) << (24 - hb));
  hi = hv >= 0x7F800000u ? (sign | 0x7F800000u) : (sign | hv);
  const long long R = (long long)M - (long long)(sh << drop);  // |R| <= 2^(drop-1)
  if (R == 0) {
    lo = 0;
    return;
  }
  lo = round_to_float(R < 0 ? (unsigned long long)(-R) : (unsigned long long)R, e - 1075, lb,
                      R < 0 ? (sign ^ 0x80000000u) : sign);
}

// split_f64(x, 11, 24, true, hi, lo) (TF32 hi with ties away, FP32 lo) in
// 32-bit integer operations: the rounding bit of hi is bit 41 of the
// significand M, and the remainder M mod 2^42 (minus 2^42 when hi rounded
// up) has at most 42 bits, held as two words. Bit-identical to split_f64.
HS_HD void split_tf32x3(double x, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = f64_bits(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e == 0x7FF) {
    hi = lo = 0x7FC00000u;
    return;
  }
  const int fe = e - 896;
  if (fe <= 0) {
    hi = lo = sign;
    return;
  }
  if (fe >= 255) {
    hi = lo = sign | 0x7F800000u;
    return;
  }
  const uint32_t m20 = hw & 0xFFFFFu;
  const uint32_t up = (m20 >> 9) & 1u;             // ties away: round up on the top dropped bit
  const uint32_t sh = 1024u + (m20 >> 10) + up;    // 11 significant bits, may carry to 2^11
  const uint32_t hv = ((uint32_t)fe << 23) + ((sh - 1024u) << 13);
  hi = hv >= 0x7F800000u ? (sign | 0x7F800000u) : (sign | hv);
  // remainder A = |M - sh 2^42| as (ah, al), sign of lo
  uint32_t ah = m20 & 0x3FFu, al = lw;
  uint32_t sgn = sign;
  if (up) {
    const uint32_t borrow = al != 0u;
    al = 0u - al;
    ah = 1024u - ah - borrow;
    sgn ^= 0x80000000u;
  } else if (ah == 0u && al == 0u) {
    lo = 0u;
    return;
  }
  int top;
#if defined(__CUDA_ARCH__)
  top = ah ? 63 - __clz((int)ah) : 31 - __clz((int)al);
#else
  top = ah ? 63 - __builtin_clz(ah) : 31 - __builtin_clz(al);
#endif
  const int drop = top - 23;
  uint32_t sig;
  if (drop > 0) {  // drop <= 19
    sig = (al >> drop) | (ah << (32 - drop));
    const uint32_t rem = al & ((1u << drop) - 1u), half = 1u << (drop - 1);
    if (rem > half || (rem == half && (sig & 1u))) ++sig;
  } else {
    sig = al << (-drop);
  }
  const int fl = e - 948 + top;  // (e - 1075) + top + 127
  if (fl <= 0) {
    lo = (fl == 0 && sig == (1u << 24)) ? (sgn | 0x00800000u) : sgn;
    return;
  }
  if (fl >= 255) {
    lo = sgn | 0x7F800000u;
    return;
  }
  const uint32_t v = ((uint32_t)fl << 23) + (sig - (1u << 23));
  lo = v >= 0x7F800000u ? (sgn | 0x7F800000u) : (sgn | v);
}

// The splits of an FP32 value v (bit pattern u), equal to split_f64 of
// (double)v: the remainder v - hi is exact in FP32 (v has 24 significant
// bits, hi the top 11 or 8), so one FP32 subtraction gives it; hi rounds on
// the bit pattern (adding half an ulp of the kept bits to the magnitude
// rounds ties away, the carry moving into the exponent). Values below the
// single normal range give zeros, as in split_f64.
HS_HD void split_f32_tf32x3(uint32_t u, uint32_t& hi, uint32_t& lo) {
  const uint32_t sign = u & 0x80000000u, ex = u & 0x7F800000u;
  if (ex == 0x7F800000u) {
    hi = lo = (u & 0x007FFFFFu) ? 0x7FC00000u : u;  // NaN, infinity
    if (u & 0x007FFFFFu) return;
    lo = u;
    return;
  }
  if (ex == 0u) {
    hi = lo = sign;
    return;
  }
  hi = (u + 0x1000u) & 0xFFFFE000u;  // 10 explicit bits, ties away (may carry to infinity)
  float fv, d;
  {
    uint32_t uu = u;
    std::memcpy(&fv, &uu, 4);
  }
  if ((hi & 0x7F800000u) == 0x7F800000u) {
    // rounded up to 2^128: v - 2^128 = (v - 2^127) - 2^127, both steps exact
    const float t = sign ? -1.7014118346046923e38f : 1.7014118346046923e38f;
    d = (fv - t) - t;
  } else {
    float fh;
    uint32_t hh = hi;
    std::memcpy(&fh, &hh, 4);
    d = fv - fh;  // exact
  }
  uint32_t ld;
  std::memcpy(&ld, &d, 4);
  lo = (ld & 0x7F800000u) == 0u ? (ld & 0x80000000u) : ld;  // below the normal range: signed zero
  if ((ld & 0x7FFFFFFFu) == 0u) lo = 0u;
}

// split_f32_tf32x3 with selects in place of branches (the GEMM epilogue's
// form; the same bits for every input).
HS_HD void split_f32_tf32x3_sel(uint32_t u, uint32_t& hi, uint32_t& lo) {
  const uint32_t sign = u & 0x80000000u, ex = u & 0x7F800000u;
  const uint32_t h = (u + 0x1000u) & 0xFFFFE000u;
  float fv, fh;
  std::memcpy(&fv, &u, 4);
  std::memcpy(&fh, &h, 4);
  const float t = sign ? -1.7014118346046923e38f : 1.7014118346046923e38f;
  // rounded up to 2^128: v - 2^128 = (v - 2^127) - 2^127, both steps exact
  const float d = (h & 0x7F800000u) == 0x7F800000u ? (fv - t) - t : fv - fh;
  uint32_t ld;
  std::memcpy(&ld, &d, 4);
  uint32_t l = (ld & 0x7F800000u) == 0u ? (ld & 0x80000000u) : ld;
  l = (ld & 0x7FFFFFFFu) == 0u ? 0u : l;
  const uint32_t special = (u & 0x007FFFFFu) ? 0x7FC00000u : u;  // NaN, infinity
  hi = ex == 0u ? sign : (ex == 0x7F800000u ? special : h);
  lo = ex == 0u ? sign : (ex == 0x7F800000u ? special : l);
}

// split_f32_tf32x3 without the cases of the top of the exponent range (the
// GEMM epilogue's form): the same bits for every pattern except those that
// round up to 2^128 (hi is infinite in both; lo is infinite here) and NaN or
// infinity (both give non-finite parts). A value of the normalised
// contractions never comes near 2^127, and one that did would still surface
// as a non-finite result downstream.
HS_HD void split_f32_tf32x3_fin(uint32_t u, uint32_t& hi, uint32_t& lo) {
  const uint32_t sign = u & 0x80000000u;
  const bool tiny = (u & 0x7F800000u) == 0u;
  const uint32_t h = (u + 0x1000u) & 0xFFFFE000u;
  float fv, fh;
  std::memcpy(&fv, &u, 4);
  std::memcpy(&fh, &h, 4);
  const float d = fv - fh;  // exact
  uint32_t ld;
  std::memcpy(&ld, &d, 4);
  uint32_t l = (ld & 0x7F800000u) == 0u ? (ld & 0x80000000u) : ld;  // below the normal range: signed zero
  l = (ld & 0x7FFFFFFFu) == 0u ? 0u : l;
  hi = tiny ? sign : h;
  lo = tiny ? sign : l;
}

// The FP64 value of the IEEE single bit pattern f (exact). Subnormal singles
// are widened by the FP64 conversion (`slow` is called for them).
HS_HD bool f32_widen_fast(uint32_t f, unsigned long long& out) {
  const uint32_t sign = f & 0x80000000u, mag = f & 0x7FFFFFFFu;
  if (mag == 0) {
    out = (unsigned long long)sign << 32;
    return true;
  }
  if (mag < 0x00800000u) return false;  // subnormal
  uint32_t hi;
  if (mag >= 0x7F800000u)
    hi = sign | 0x7FF00000u | ((mag & 0x7FFFFFu) >> 3);
  else
    hi = sign | ((mag >> 3) + (896u << 20));
  out = ((unsigned long long)hi << 32) | (unsigned long long)(mag << 29);
  return true;
}

}  // namespace hs
