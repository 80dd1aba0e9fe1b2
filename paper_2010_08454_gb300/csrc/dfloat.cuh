// Double-float arithmetic: a value carried as the unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  Sums by
// Knuth's TwoSum (TAOCP vol. 2, 4.2.2), products by the FMA-exact TwoProduct
// (after Dekker 1971).  Reductions that need more than FP32 precision use
// these instead of FP64, whose pipe is narrow and slow on GB300: a chain of a
// few hundred dependent FP64 operations (one thread's exp, log and
// divisions) took tens of microseconds there.
#pragma once

#include <stdint.h>

namespace ppl {

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(s, t);
  return make_float2(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float2 p = df_prod(a.x, b.x);
  p.y = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, p.y));
  const float hi = __fadd_rn(p.x, p.y);
  return make_float2(hi, __fsub_rn(p.y, __fsub_rn(hi, p.x)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float b) {
  return df_mul(a, make_float2(b, 0.0f));
}
__device__ __forceinline__ float2 df_shfl_xor(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 df_warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// a / b in FP32 (b > 0): the FP32 quotient of the high parts, corrected by the
// residual (a - q b) / b, so the result is within a few FP32 ulps of the exact
// quotient of the double-float values.
__device__ __forceinline__ float df_div(float2 a, float2 b) {
  const float q = __fdiv_rn(a.x, b.x);
  const float r = __fadd_rn(__fmaf_rn(-q, b.x, a.x), __fmaf_rn(-q, b.y, a.y));
  return __fmaf_rn(r, __frcp_rn(b.x), q);
}

// An integer count as a double-float (exact below 2^48).
__device__ __forceinline__ float2 df_from_i64(int64_t n) {
  const float hi = (float)n;
  return make_float2(hi, (float)(n - (int64_t)hi));
}

// Natural logarithm of a positive normal double-float x, as a double-float
// with an absolute error of a few 1e-8: with x.hi = m 2^e, m in
// [sqrt(1/2), sqrt(2)),
//   log x = e ln2 + log m + log1p(x.lo / x.hi),  log1p(t) = t to 2^-48.
// ln 2 is split as hi + lo with hi = 0x1.62e4p-1 (15 significant bits, so
// e hi is exact for |e| < 512) and lo the FP32 rounding of ln 2 - hi; log m
// is FP32 logf (within an ulp of |log m| <= 0.35).
__device__ __forceinline__ float2 df_log(float2 x) {
  const uint32_t b = __float_as_uint(x.x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);  // [1, 2)
  if (m >= 1.41421356f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float ef = (float)e;
  const float lo = __fmaf_rn(ef, 0x1.7f7d1cp-20f, __fadd_rn(logf(m), __fdiv_rn(x.y, x.x)));
  const float hi = __fmul_rn(ef, 0x1.62e4p-1f);
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

// e^d for an FP32 d <= 0 as 2^n m, with n an integer and m = e^r, r in
// [-ln2/2, ln2/2] (Cody and Waite's reduction r = d - n ln2, ln 2 split as
// above so n hi is exact for |n| < 512): m keeps FP32's relative precision
// where e^d itself lies far below FP32's range.  d < -1000 (below FP64's
// range too) gives m = 0.
struct ExpSplit {
  int n;
  float m;
};
__device__ __forceinline__ ExpSplit exp_split(float d) {
  if (!(d >= -1000.0f)) return ExpSplit{0, 0.0f};
  const float n = rintf(__fmul_rn(d, 1.44269504f));
  const float r = __fmaf_rn(-n, 0x1.7f7d1cp-20f, __fmaf_rn(-n, 0x1.62e4p-1f, d));
  return ExpSplit{(int)n, expf(r)};
}

// 2^n as an FP32 value, for n in [-126, 127].
__device__ __forceinline__ float exp2i(int n) { return __int_as_float((127 + n) << 23); }

}  // namespace ppl
