// Double-float arithmetic: a value is a pair of FP32 numbers (hi, lo) with
// hi + lo the represented number (about 48 significant bits).  Sums use an
// error-free two-sum and products an FMA-based two-product, so the work runs
// on the FP32 pipes, tens of times the FP64 rate on this GPU; conversions
// from and to FP64 use integer operations and at most one FP64 addition.
#pragma once

#include <cstdint>

namespace isdf {
namespace {

struct DF {
  float hi, lo;
};

// Error-free transformations with explicitly rounded operations (the
// compiler must not contract them into FMAs or reassociate them).
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  DF s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact error of the product
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ DF df_half(DF x) { return {__fmul_rn(0.5f, x.hi), __fmul_rn(0.5f, x.lo)}; }


// Conversions between FP64 and double-float with integer operations, so that
// they stay off the narrow FP64 unit.  hi is x's significand rounded to 24
// bits (the round bit added into the exponent|significand field carries
// correctly); lo = x - hi is the signed remainder of the low 29 bits, exact in
// FP64 and rounded once to FP32.  Values whose hi or lo would leave FP32's
// normal range (|x| < 2^-73 or > 2^126, zeros) take the FP64 route.
__device__ __forceinline__ DF df_from_double(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int E = int((b >> 52) & 0x7FF);
  if (E < 950 || E > 1148) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - double(hi))};
  }
  const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
  const uint32_t m29 = uint32_t(b) & 0x1FFFFFFFu;
  const uint32_t up = m29 >> 28;
  const uint32_t hb = ((uint32_t(E - 896) << 23) | (uint32_t(b >> 29) & 0x7FFFFFu)) + up;
  const float scale = __uint_as_float(uint32_t(E - 948) << 23);  // 2^(E - 1075)
  const float lo = __int2float_rn(int(m29) - int(up << 29)) * scale;
  return {__uint_as_float(hb | sign), sign ? -lo : lo};
}

// FP32 value as FP64 bits (exact; zeros, subnormals and non-finite values
// take the conversion instruction)
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ef = (b >> 23) & 0xFFu;
  if (ef == 0u || ef == 0xFFu) return double(f);
  const uint64_t bits = (uint64_t(b & 0x80000000u) << 32) | (uint64_t(ef + 896u) << 52) | (uint64_t(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double df_to_double(DF x) { return f32_to_f64(x.hi) + f32_to_f64(x.lo); }

}  // namespace
}  // namespace isdf
