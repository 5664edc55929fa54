// fp_bits.h -- IEEE-754 operations computed on bit patterns with integer
// arithmetic.  On GB300 a conversion between double and float occupies the
// FP64 pipe as long as an FMA does (about 64 cycles per warp instruction per
// sub-partition), while the integer pipes are otherwise idle in the FP64-bound
// kernels; these functions give the same result as the hardware instruction
// (bit for bit, save for which NaN a NaN becomes).
// Plain C as well as CUDA, so that a host unit test checks them against the
// host's own IEEE conversion.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FPB_FN __host__ __device__ __forceinline__
#else
#define FPB_FN static inline
#endif

FPB_FN uint64_t fpb_bits_of_double(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
}

FPB_FN float fpb_float_of_bits(uint32_t b) {
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}

// x rounded to the nearest float, ties to even (cvt.rn.f32.f64): overflow
// gives an infinity, results below the smallest normal float are the
// correctly rounded subnormals (no flush to zero), a NaN gives a quiet NaN
// with the sign and the leading payload bits of x
FPB_FN float fpb_double_to_float_rn(double x) {
  const uint64_t b = fpb_bits_of_double(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0x000fffffffffffffull;
  if (e == 0x7ff)  // infinity, or NaN made quiet
    return fpb_float_of_bits(sign | 0x7f800000u | (m ? 0x00400000u | (uint32_t)(m >> 29) : 0u));
  const int fe = e - 1023 + 127;  // biased float exponent of a normal result
  if (fe >= 0xff) return fpb_float_of_bits(sign | 0x7f800000u);
  if (fe > 0) {
    // 52 -> 23 fraction bits; a carry out of the fraction steps the
    // exponent, up to infinity, which is the right result
    uint32_t r = (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r += 1u;
    return fpb_float_of_bits(sign | (((uint32_t)fe << 23) + r));
  }
  if (e == 0) return fpb_float_of_bits(sign);  // zero or a double subnormal
  // a float subnormal: k = round(M 2^-s) units of 2^-149, M the 53-bit
  // significand; s >= 30, and beyond 54 the result is zero
  const int s = 926 - e;
  if (s > 54) return fpb_float_of_bits(sign);
  const uint64_t M = m | 0x0010000000000000ull;
  uint64_t k = M >> s;
  const uint64_t rem = M & ((1ull << s) - 1ull), half = 1ull << (s - 1);
  if (rem > half || (rem == half && (k & 1ull))) k += 1ull;
  return fpb_float_of_bits(sign | (uint32_t)k);
}

// comparisons of doubles on integer arithmetic.  The IEEE order of doubles
// that are not NaN is the order of the keys b ^ ((b >> 63) & 0x7fff...) of
// their bit patterns b, read as signed integers, save that -0 and +0 compare
// equal.  Each function gives exactly the IEEE answer for the inputs its
// name allows ("num": neither is NaN; "ieee": any input, false with a NaN).
FPB_FN int64_t fpb_order_key(double x) {
  const int64_t b = (int64_t)fpb_bits_of_double(x);
  return b ^ ((b >> 63) & INT64_MAX);
}
FPB_FN int fpb_is_nan(double x) {
  return (int64_t)(fpb_bits_of_double(x) & 0x7fffffffffffffffull) > 0x7ff0000000000000ll;
}
// a < b
FPB_FN int fpb_lt_num(double a, double b) {
  const uint64_t both = fpb_bits_of_double(a) | fpb_bits_of_double(b);
  return fpb_order_key(a) < fpb_order_key(b) && (both << 1) != 0;
}
FPB_FN int fpb_lt_ieee(double a, double b) {
  return !fpb_is_nan(a) && !fpb_is_nan(b) && fpb_lt_num(a, b);
}
// a <= b
FPB_FN int fpb_le_ieee(double a, double b) {
  return !fpb_is_nan(a) && !fpb_is_nan(b) && !fpb_lt_num(b, a);
}
// x >= 0 and x > 0
FPB_FN int fpb_ge0_num(double x) {
  const int64_t b = (int64_t)fpb_bits_of_double(x);
  return b >= 0 || b == INT64_MIN;
}
FPB_FN int fpb_gt0_num(double x) { return (int64_t)fpb_bits_of_double(x) > 0; }
