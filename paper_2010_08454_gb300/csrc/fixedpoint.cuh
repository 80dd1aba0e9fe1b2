// Fixed-point resampling weights shared by the resampling kernels: the FP32
// exponential E32 that decides them and the saturating u64 arithmetic of the
// prefix sums (see resample.cu for the definition).
#pragma once

#include "common.cuh"

namespace ppl {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint64_t kLimit = (1ull << 61) + 1;  // saturation: any value above 2^61 is an error
constexpr int kMaxSpin = 1 << 22;               // bounded wait of the look-back

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
  const uint64_t s = a + b;  // a, b <= kLimit, so no wrap-around
  return s > kLimit ? kLimit : s;
}

__device__ __forceinline__ float exp32(float d) {
  const float kLog2e = 0x1.715476p+0f;   // log2(e), FP32
  const float kLn2Hi = 0x1.62e4p-1f;     // ln 2 to 16 significant bits
  const float kLn2Lo = 0x1.7f7d1cp-20f;  // ln 2 - kLn2Hi, FP32
  const float k = rintf(__fmul_rn(d, kLog2e));
  float r = __fmaf_rn(-k, kLn2Hi, d);
  r = __fmaf_rn(-k, kLn2Lo, r);
  float p = 0x1.a01a02p-13f;             // 1/7!
  p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);  // 1/6!
  p = __fmaf_rn(p, r, 0x1.111112p-7f);   // 1/5!
  p = __fmaf_rn(p, r, 0x1.555556p-5f);   // 1/4!
  p = __fmaf_rn(p, r, 0x1.555556p-3f);   // 1/3!
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  return __fmul_rn(p, __int_as_float((127 + (int)k) << 23));  // exact: 2^k is normal for k >= -64
}

// floor(v) for finite 0 <= v < 2^64, from the bits of v (the same value as a
// truncating conversion; integer operations only, which keeps the 64-bit
// conversion off this GPU's narrow FP64 pipe).
__device__ __forceinline__ uint64_t floor_u64(float v) {
  const uint32_t b = __float_as_uint(v);
  const int ex = (int)(b >> 23) - 150;  // v = mant * 2^ex for normal v
  if ((b >> 23) == 0 || ex < -24) return 0;
  if (ex > 40) return ~0ull;  // v >= 2^64 (never for the weights here)
  const uint64_t mant = (uint64_t)((b & 0x7fffffu) | 0x800000u);
  return ex >= 0 ? mant << ex : mant >> -ex;
}

__device__ __forceinline__ uint64_t quantize(float lw, float m, float scale) {
  const float d = __fsub_rn(lw, m);
  if (!(d >= -44.5f)) return 0;
  return floor_u64(__fmul_rn(exp32(d), scale));
}

// First index j in [lo, hi) with C[j] > p (hi if none), by one warp: each
// round the 32 lanes probe 32 evenly spaced positions, so 2^24 entries take
// five dependent loads.
__device__ __forceinline__ int64_t warp_upper_bound(const uint64_t* C, int64_t lo, int64_t hi,
                                                    uint64_t p, int lane) {
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t q = lo + (int64_t)(lane + 1) * step - 1;
    const bool gt = (q >= hi) || (C[q] > p);
    const unsigned m = __ballot_sync(0xffffffffu, gt);
    const int f = __ffs(m) - 1;  // m != 0: lane 31 probes at or past hi - 1
    const int64_t new_lo = (f == 0) ? lo : lo + (int64_t)f * step;
    hi = (lo + (int64_t)(f + 1) * step - 1) + 1 < hi ? lo + (int64_t)(f + 1) * step : hi;
    lo = new_lo;
  }
  const int64_t q = lo + lane;
  const bool gt = (q >= hi) || (C[q] > p);
  const unsigned m = __ballot_sync(0xffffffffu, gt);
  return m ? lo + (__ffs(m) - 1) : hi;
}

}  // namespace ppl
