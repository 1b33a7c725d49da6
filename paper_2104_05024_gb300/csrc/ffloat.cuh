// Float-float arithmetic for the pointwise reaction kernels.  On this part
// every float64 instruction, conversions between float64 and float32
// included, issues at 2 per SM per clock, 64x below the float32 rate, so the
// backward-Euler reaction evaluates its Newton residual on unevaluated float
// pairs (hi + lo, about 48 significant bits) and meets float64 only to read
// and write the state.  Doubles are split into float pairs, and floats widened
// to doubles, on the bit patterns with integer and float32 instructions.
//
// Error-free transformations: Knuth's TwoSum (s + e = a + b exactly) and the
// product error by a fused multiply-add (p + e = a b exactly).
//
// Everything here is plain host/device code so that the same source runs on
// the host against exact rational arithmetic.
#pragma once

#include <stdint.h>

#include <cmath>
#include <cstring>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace kfbi {
namespace ffl {

FF_HD uint64_t bits64(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
FF_HD double from_bits64(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}
FF_HD uint32_t bits32(float x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
FF_HD float from_bits32(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}
FF_HD float fmaf_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
// an unsigned integer below 2^29 to the nearest float
FF_HD float u29_to_float(uint32_t r) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(r);
#else
  return (float)r;
#endif
}

struct ff {
  float h, l;
};

// x = h + l + r exactly with h the top 24 significant bits of x (truncated),
// l the remaining 29 bits rounded to 24 significant bits, |r| <= 2^-48 |x|.
// For |x| < 2^-60 h = l = 0 (absolute error below 8.7e-19).  Returns false
// for |x| >= 2^128 (beyond the float range), infinities and NaN.
FF_HD bool split(double x, ff& out) {
  const uint64_t b = bits64(x);
  const int E = (int)((b >> 52) & 0x7ff);  // biased exponent
  if (E < 1023 - 60) {
    out.h = 0.0f;
    out.l = 0.0f;
    return true;
  }
  if (E >= 1023 + 128) return false;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
  // float exponent field E - 1023 + 127; the top 23 fraction bits
  out.h = from_bits32(sign | ((uint32_t)(E - 896) << 23) | (uint32_t)(m >> 29));
  // the low 29 fraction bits r weigh 2^(E - 1075): float field E - 948 >= 15
  const float scale = from_bits32(sign | ((uint32_t)(E - 948) << 23));
  out.l = u29_to_float((uint32_t)(m & 0x1FFFFFFFu)) * scale;
  return true;
}

// the float nearest to x (from its pair: off by one unit only within 2^-48
// |x| of a rounding tie; 0 below 2^-60; infinities beyond the float range
// and for infinite x; NaN for NaN)
FF_HD float narrow(double x) {
  ff p;
  if (split(x, p)) return p.h + p.l;
  const uint64_t b = bits64(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const bool nan = ((b >> 52) & 0x7ff) == 0x7ff && (b & 0xFFFFFFFFFFFFFull) != 0;
  return from_bits32(sign | (nan ? 0x7fc00000u : 0x7f800000u));
}

// the double equal to the float f (subnormal floats, below 2^-126, to zero)
FF_HD double widen(float f) {
  const uint32_t u = bits32(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t s = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t frac = (uint64_t)(u & 0x7fffffu) << 29;
  if (e == 0) return from_bits64(s);
  if (e == 0xffu) return from_bits64(s | 0x7ff0000000000000ull | frac);
  return from_bits64(s | ((uint64_t)(e + 896) << 52) | frac);
}

FF_HD void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
FF_HD void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf_(a, b, -p);
}
FF_HD ff renorm(float s, float e) {
  ff r;
  r.h = s + e;
  r.l = e - (r.h - s);
  return r;
}
FF_HD ff add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return renorm(s, e);
}
FF_HD ff neg(ff a) { return ff{-a.h, -a.l}; }
FF_HD ff mul(ff a, float b) {
  float p, e;
  two_prod(a.h, b, p, e);
  e = fmaf_(a.l, b, e);
  return renorm(p, e);
}
FF_HD ff mul(ff a, ff b) {
  float p, e;
  two_prod(a.h, b.h, p, e);
  e = fmaf_(a.h, b.l, fmaf_(a.l, b.h, e));
  return renorm(p, e);
}

}  // namespace ffl
}  // namespace kfbi
