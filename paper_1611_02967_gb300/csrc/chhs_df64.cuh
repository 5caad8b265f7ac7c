// chhs_df64.cuh -- double-single ("df64") arithmetic: a value carried as an
// unevaluated sum hi + lo of two single-precision numbers, about 48
// significant bits, computed on the single-precision pipes.
//
// GB300 runs double precision at 1/64 of the single-precision rate, and the
// mixed-precision form's one double-precision kernel per iteration -- the
// defect-correction residual f - N(u) -- was bound by that pipe.  The
// residual only has to be accurate to far below the stopping tolerance
// (1e-10 against values of order one), which 48 bits give.  The operations
// are the error-free transformations of Knuth (two-sum) and of Dekker and
// Kahan (the exact product error through a fused multiply-add), combined as
// in the double-single libraries of the GPU literature (for instance
// Thall, "Extended-precision floating-point numbers for GPU computation",
// 2006): a sum or product is formed in single precision together with its
// rounding error, then renormalised.  Every step uses the round-to-nearest
// intrinsics so that the compiler never contracts a product into a
// following sum, which would break the error terms.
//
// Usable from host code too (plain single-precision operations with
// std::fmaf; build with -ffp-contract=off), so the host tests can check
// the arithmetic against long double references.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define DF_HD inline
#endif

namespace chhs_dev {

struct df64 {
  float hi, lo;
};

DF_HD float df_fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_HD float df_fsub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_HD float df_fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_HD float df_ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

DF_HD uint64_t df_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
DF_HD float df_from_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// x split into hi + lo with integer and single-precision operations only (a
// conversion instruction runs at the double-precision rate on this GPU): hi
// is x with its significand cut to 24 bits, lo the next 23 bits (the last 6
// of the 53 are dropped), so |x - (hi + lo)| < 2^-46 |x|.  Magnitudes below 2^-126 give 0
// (an absolute error far below anything the residual resolves), magnitudes
// beyond the float range and non-finite values give +-infinity in hi, so a
// non-finite state still yields a non-finite residual.
DF_HD df64 df_split(double x) {
  const uint64_t b = df_bits(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e < 897) return df64{df_from_bits(sign), 0.f};
  if (e > 1150) return df64{df_from_bits(sign | 0x7F800000u), 0.f};
  const float hi = df_from_bits(sign | ((uint32_t)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // the next 23 significand bits as an exact float integer m (the bits of
  // 2^23 + m, minus 2^23), scaled by 2^(e - 1069): their place value
  const uint32_t m = (lw & 0x1FFFFFFFu) >> 6;
  const float mf = df_fsub(df_from_bits(0x4B000000u | m), 8388608.0f);
  const int se = e - 942;
  const float scale = se > 0 ? df_from_bits((uint32_t)se << 23) : 0.f;
  const float lo_mag = df_fmul(mf, scale);
  const float lo = sign ? -lo_mag : lo_mag;
  return df64{hi, lo};
}

// Knuth's two-sum: s + err = a + b exactly.
DF_HD df64 df_two_sum(float a, float b) {
  const float s = df_fadd(a, b);
  const float bb = df_fsub(s, a);
  const float err = df_fadd(df_fsub(a, df_fsub(s, bb)), df_fsub(b, bb));
  return df64{s, err};
}

// Renormalisation for |a| >= |b| (or a = 0): s + err = a + b exactly.
DF_HD df64 df_quick_sum(float a, float b) {
  const float s = df_fadd(a, b);
  return df64{s, df_fsub(b, df_fsub(s, a))};
}

DF_HD df64 df_add(df64 x, df64 y) {
  const df64 s = df_two_sum(x.hi, y.hi);
  return df_quick_sum(s.hi, df_fadd(s.lo, df_fadd(x.lo, y.lo)));
}

DF_HD df64 df_neg(df64 x) { return df64{-x.hi, -x.lo}; }

DF_HD df64 df_sub(df64 x, df64 y) { return df_add(x, df_neg(y)); }

// Product: p + e = x.hi * y.hi exactly through the fused multiply-add; the
// cross terms are added to the error before the renormalisation.
DF_HD df64 df_mul(df64 x, df64 y) {
  const float p = df_fmul(x.hi, y.hi);
  float e = df_ffma(x.hi, y.hi, -p);
  e = df_ffma(x.hi, y.lo, e);
  e = df_ffma(x.lo, y.hi, e);
  return df_quick_sum(p, e);
}

DF_HD float df_to_float(df64 x) { return df_fadd(x.hi, x.lo); }

DF_HD double df_to_double(df64 x) { return (double)x.hi + (double)x.lo; }

// A host double as an exact-as-possible df64 (kernel arguments).
inline df64 df_from_double_host(double x) {
  const float hi = (float)x;
  return df64{hi, (float)(x - (double)hi)};
}

}  // namespace chhs_dev
