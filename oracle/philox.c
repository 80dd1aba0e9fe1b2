/*
 * Oracle random numbers: Philox4x32-10 and the transforms that turn its words
 * into the draws made by `sample` (§3.2 built-in distributions, §3.4 sample).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3" (SC'11): a 4x32-bit counter, a 2x32-bit key,
 * ten rounds of two 32x32->64 multiplications, and a Weyl key schedule.
 *
 * Counter layout (the written specification both sides implement):
 *   key = (seed mod 2^32, seed div 2^32)
 *   ctr = (particle, instance, step, purpose << 16 | block)
 */
#include "oracle.h"

#include <math.h>
#include <omp.h>
#include <string.h>

/* Multipliers and key increments as published by Salmon et al. (SC'11). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) { /* the key advances by the Weyl constants before every round but the first */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_philox_block(uint64_t seed, uint32_t particle, uint32_t instance, uint32_t step,
                      uint32_t purpose, uint32_t block, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {particle, instance, step, (purpose << 16) | block};
  orc_philox4x32_10(ctr, key, out);
}

/* Uniform on the open interval (0, 1): the top 23 bits of a word, centred in
 * their cell: u = (floor(w / 2^9) + 1/2) / 2^23.  Every value is exact in FP32. */
double orc_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) / 8388608.0; }

/* Box and Muller (1958): two independent standard normals from two uniforms. */
void orc_box_muller(uint32_t wa, uint32_t wb, double* z0, double* z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double ua = orc_u01(wa), ub = orc_u01(wb);
  double rho = sqrt(-2.0 * log(ua));
  *z0 = rho * cos(two_pi * ub);
  *z1 = rho * sin(two_pi * ub);
}

/* uniform-discrete(lo, hi), both ends included: lo + floor(w * (hi - lo + 1) / 2^32). */
int orc_uniform_discrete(uint32_t w, int lo, int hi) {
  uint64_t range = (uint64_t)(hi - lo + 1);
  return lo + (int)(((uint64_t)w * range) >> 32);
}

/*
 * FP32 standard normal with a fixed, reproducible result: the Box-Muller
 * cosine branch z = sqrt(-2 ln u_a) cos(2 pi u_b), where every step is one
 * correctly rounded FP32 operation (+, -, *, /, fma, sqrt, rint) in the order
 * written, so any implementation of this definition returns the same bits.
 *  ln u: u = m 2^e with m in [sqrt(1/2), sqrt(2)]; ln m = 2 atanh(s),
 *        s = (m - 1)/(m + 1), atanh(s)/s = 1 + s^2/3 + s^4/5 + s^6/7 + s^8/9
 *        (truncation < 3e-9 relative); ln u = e ln2_hi + (e ln2_lo + ln m).
 *  cos(2 pi u): v = 4u = k + r exactly (k = rint(v), |r| <= 1/2); cos and sin
 *        of (pi/2) r by their Taylor series to degree 10 and 9 (truncation
 *        < 2e-9); the quadrant k mod 4 picks cos, -sin, -cos or sin.
 * Coefficients are the FP32 roundings of the exact series coefficients.
 */
static float ln32(float u) {
  uint32_t b;
  memcpy(&b, &u, sizeof b);
  int e = (int)((b >> 23) & 0xffu) - 127;
  uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, sizeof m);
  if (m > 0x1.6a09e6p+0f) { /* above sqrt(2) */
    m = m * 0.5f;
    e += 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  float p = 0x1.c71c72p-4f;        /* 1/9 */
  p = fmaf(p, s2, 0x1.24924ap-3f); /* 1/7 */
  p = fmaf(p, s2, 0x1.99999ap-3f); /* 1/5 */
  p = fmaf(p, s2, 0x1.555556p-2f); /* 1/3 */
  float t = s2 * p;
  float two_s = s + s;
  float lnm = fmaf(two_s, t, two_s);
  float ef = (float)e;
  return fmaf(ef, 0x1.62e4p-1f, fmaf(ef, 0x1.7f7d1cp-20f, lnm)); /* ln2 = hi + lo */
}

static float cos2pi32(float u) {
  float v = 4.0f * u;
  float k = rintf(v);
  float r = v - k;
  float r2 = r * r;
  float sp = 0x1.507834p-13f;          /* (pi/2)^9 / 9! */
  sp = fmaf(sp, r2, -0x1.32d2ccp-8f);  /* -(pi/2)^7 / 7! */
  sp = fmaf(sp, r2, 0x1.466bc6p-4f);   /* (pi/2)^5 / 5! */
  sp = fmaf(sp, r2, -0x1.4abbcep-1f);  /* -(pi/2)^3 / 3! */
  sp = fmaf(sp, r2, 0x1.921fb6p+0f);   /* pi/2 */
  sp = sp * r;
  float cp = -0x1.a6d1f2p-16f;         /* -(pi/2)^10 / 10! */
  cp = fmaf(cp, r2, 0x1.e1f506p-11f);  /* (pi/2)^8 / 8! */
  cp = fmaf(cp, r2, -0x1.55d3c8p-6f);  /* -(pi/2)^6 / 6! */
  cp = fmaf(cp, r2, 0x1.03c1f0p-2f);   /* (pi/2)^4 / 4! */
  cp = fmaf(cp, r2, -0x1.3bd3ccp+0f);  /* -(pi/2)^2 / 2! */
  cp = fmaf(cp, r2, 1.0f);
  switch (((int)k) & 3) {
    case 0: return cp;
    case 1: return -sp;
    case 2: return -cp;
    default: return sp;
  }
}

float orc_ln32(float u) { return ln32(u); }
float orc_cos2pi32(float u) { return cos2pi32(u); }

float orc_normal32(uint32_t wa, uint32_t wb) {
  float ua = (float)orc_u01(wa), ub = (float)orc_u01(wb); /* exact */
  float rho = sqrtf(-2.0f * ln32(ua));
  return rho * cos2pi32(ub);
}

void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_get_threads(void) { return omp_get_max_threads(); }
