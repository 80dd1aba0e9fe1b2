/*
 * Oracle systematic resampling with 64-bit fixed-point weights, and the gather
 * of resampled particle state.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper names particle methods as future work (§6); the resampling step is
 * the standard systematic scheme (Kitagawa 1996; Douc, Cappé and Moulines
 * 2005) stated over integers so that ancestors are exact:
 *   m   = max_i lw_i                           (FP32 log-weights)
 *   S   = 61 - ceil(log2 N)
 *   q_i = floor(E32(lw_i - m) * 2^S)           (u64; 0 when lw_i - m < -44.5)
 *   T   = sum_i q_i  (<= 2^61),  step = floor(T / M)
 *   u'  = floor(w * step / 2^32)               (w: word 0 of purpose RESAMPLE)
 *   a_k = min { j : C_j > u' + k * step },  C_j = q_0 + ... + q_j,  k = 0..M-1
 * E32 is the fixed FP32 exponential below.  It is part of the definition
 * because the integers q_i are decided in FP32 and must be the same on every
 * implementation: Cody-Waite reduction by ln 2 (Cody and Waite 1980), then the
 * degree-7 Taylor polynomial of exp on |r| <= ln(2)/2 in Horner form, every
 * step a correctly rounded FP32 multiply or fused multiply-add.  The scale
 * 2^S keeps T below 2^61, so any prefix sum fits in 62 bits.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

float orc_exp32(float d) {
  const float log2e = 0x1.715476p+0f;    /* log2(e) rounded to FP32 */
  const float ln2_hi = 0x1.62e4p-1f;     /* ln 2 cut to 16 significant bits */
  const float ln2_lo = 0x1.7f7d1cp-20f;  /* ln 2 - ln2_hi, rounded to FP32 */
  float t = d * log2e;
  float k = rintf(t);
  float r = fmaf(-k, ln2_hi, d);
  r = fmaf(-k, ln2_lo, r);
  float p = 0x1.a01a02p-13f;          /* 1/5040 */
  p = fmaf(p, r, 0x1.6c16c2p-10f);    /* 1/720 */
  p = fmaf(p, r, 0x1.111112p-7f);     /* 1/120 */
  p = fmaf(p, r, 0x1.555556p-5f);     /* 1/24 */
  p = fmaf(p, r, 0x1.555556p-3f);     /* 1/6 */
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  return ldexpf(p, (int)k);
}

int orc_fixed_shift(int64_t N) {
  int s = 0;
  while (((int64_t)1 << s) < N) s++;
  return 61 - s;
}

void orc_quantize_weights(const float* lw, int64_t N, uint64_t* q) {
  float m = -INFINITY;
  for (int64_t i = 0; i < N; i++)
    if (lw[i] > m) m = lw[i];
  float scale = ldexpf(1.0f, orc_fixed_shift(N));
  for (int64_t i = 0; i < N; i++) {
    float d = lw[i] - m;
    if (!(d >= -44.5f)) {
      q[i] = 0;
      continue;
    }
    float w = orc_exp32(d);
    q[i] = (uint64_t)(w * scale);
  }
}

int orc_resample_systematic(const uint64_t* q, int64_t N, int64_t M, uint64_t seed,
                            uint32_t instance, uint32_t step, int32_t* ancestors) {
  uint64_t T = 0;
  for (int64_t i = 0; i < N; i++) T += q[i];
  if (T == 0) return 5; /* every weight is zero */
  if (T < (uint64_t)M) return 1;
  uint64_t stride = T / (uint64_t)M;
  uint32_t w[4];
  orc_philox_block(seed, 0, instance, step, ORC_PURPOSE_RESAMPLE, 0, w);
  uint64_t u = (uint64_t)(((unsigned __int128)w[0] * stride) >> 32);

  /* search form: walk the inclusive prefix sums C_j alongside the positions */
  int64_t j = 0;
  uint64_t C = q[0];
  for (int64_t k = 0; k < M; k++) {
    uint64_t p = u + (uint64_t)k * stride;
    while (C <= p) { /* first j with C_j > p */
      j++;
      C += q[j];
    }
    ancestors[k] = (int32_t)j;
  }
  return 0;
}

int orc_resample_from_lw(const float* lw, int64_t N, int64_t M, uint64_t seed,
                         uint32_t instance, uint32_t step, int32_t* ancestors) {
  for (int64_t i = 0; i < N; i++)
    if (isnan(lw[i])) return 4;
  uint64_t* q = (uint64_t*)malloc((size_t)N * sizeof(uint64_t));
  if (!q) return 2;
  orc_quantize_weights(lw, N, q);
  int st = orc_resample_systematic(q, N, M, seed, instance, step, ancestors);
  free(q);
  return st;
}

/* out[k] = in[a_k], records of stride_bytes bytes. */
void orc_gather(const void* in, int64_t stride_bytes, const int32_t* anc, int64_t M, void* out) {
  const char* src = (const char*)in;
  char* dst = (char*)out;
  for (int64_t k = 0; k < M; k++)
    memcpy(dst + k * stride_bytes, src + (int64_t)anc[k] * stride_bytes, (size_t)stride_bytes);
}
