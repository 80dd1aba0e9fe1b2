/*
 * Oracle sequential Monte Carlo and Kalman filter for the one-dimensional
 * linear-Gaussian state-space model
 *   x_0 = 0,  x_t = phi x_{t-1} + q_sigma e_t,  y_t = x_t + r_sigma v_t,  e_t, v_t ~ N(0, 1).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Each particle runs the model forward; the observation enters through
 * `observe(dist, y) = factor(dist-score(dist, y))` (§3.4, Fig. 2), i.e. the
 * normalised log-density of y_t under N(x_t, r_sigma^2) is added to the
 * log-weight.  Particle methods are the paper's stated future work (§6).
 * This is the bootstrap filter with adaptive resampling:
 *   for t = 1..T: propagate, add the observe term, ESS = (sum e)^2 / sum e^2;
 *     if ESS < N/2: logZ_acc += LSE(lw) - log N; resample (resample.c); lw = 0
 *   log Z = logZ_acc + LSE(lw) - log N
 * Draws: word 0 and 1 of block 0 of (particle i, instance 0, step t, purpose
 * LGSSM_PROPAGATE) -> the cosine Box-Muller normal e_t.
 *
 * Precision: with state_f32 = 0 everything is FP64.  With state_f32 = 1 the
 * particle state and log-weights are held in FP32, as the method's precision
 * policy fixes (FP32 state and log-weights, FP64 normalisation and evidence
 * accumulator): the normal is the reproducible FP32 Box-Muller draw
 * orc_normal32 of the same two words, and every update below is FP32
 * arithmetic, one rounding per operation, in the order written:
 *   x = phi * x + q * e;   d = y - x;   lw = lw + (c + (h * d) * d)
 * with c = -log(2 pi r^2) / 2 and h = -1 / (2 r^2) rounded to FP32.  The
 * resampling decisions (integers) then come from the same FP32 values a
 * particle filter in that precision holds.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double log_normal_pdf(double y, double mean, double var) {
  const double two_pi = 6.283185307179586476925286766559;
  double d = y - mean;
  return -0.5 * log(two_pi * var) - d * d / (2.0 * var);
}

/* Kalman (1960) filter: the exact log-evidence log p(y_1..y_T). */
double orc_kalman_logz(const orc_lgssm* m, const double* y, int64_t T) {
  double mean = 0.0, var = 0.0, logz = 0.0;
  double q2 = m->q_sigma * m->q_sigma, r2 = m->r_sigma * m->r_sigma;
  for (int64_t t = 0; t < T; t++) {
    double mp = m->phi * mean;
    double vp = m->phi * m->phi * var + q2;
    double s = vp + r2;
    logz += log_normal_pdf(y[t], mp, s);
    double gain = vp / s;
    mean = mp + gain * (y[t] - mp);
    var = (1.0 - gain) * vp;
  }
  return logz;
}

double orc_smc_lgssm(const orc_lgssm* m, const double* y, int64_t T, int64_t N, uint64_t seed,
                     int state_f32, double* ess_t, int32_t* resampled_t, double* x_out,
                     double* lw_out) {
  const double two_pi = 6.283185307179586476925286766559;
  const float phi_f = (float)m->phi, q_f = (float)m->q_sigma;
  const float c_f = (float)(-0.5 * log(two_pi * m->r_sigma * m->r_sigma));
  const float h_f = (float)(-1.0 / (2.0 * m->r_sigma * m->r_sigma));
  double* x = (double*)calloc((size_t)N, sizeof(double));
  double* xn = (double*)calloc((size_t)N, sizeof(double));
  double* lw = (double*)calloc((size_t)N, sizeof(double));
  float* lw32 = (float*)calloc((size_t)N, sizeof(float));
  int32_t* anc = (int32_t*)calloc((size_t)N, sizeof(int32_t));
  double r2 = m->r_sigma * m->r_sigma;
  double logz_acc = 0.0;
  for (int64_t t = 1; t <= T; t++) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
      uint32_t w[4];
      double z0, z1;
      orc_philox_block(seed, (uint32_t)i, 0, (uint32_t)t, ORC_PURPOSE_LGSSM_PROPAGATE, 0, w);
      orc_box_muller(w[0], w[1], &z0, &z1);
      if (state_f32) {
        float xf = (float)x[i], lf = (float)lw[i], zf = orc_normal32(w[0], w[1]);
        float yf = (float)y[t - 1];
        xf = phi_f * xf + q_f * zf;
        float d = yf - xf;
        lf = lf + (c_f + (h_f * d) * d);
        x[i] = xf;
        lw[i] = lf;
      } else {
        x[i] = m->phi * x[i] + m->q_sigma * z0;
        lw[i] += log_normal_pdf(y[t - 1], x[i], r2);
      }
    }
    double lse, ess;
    orc_lse_ess(lw, N, &lse, &ess, NULL, NULL);
    if (ess_t) ess_t[t - 1] = ess;
    int resample = ess < 0.5 * (double)N;
    if (resampled_t) resampled_t[t - 1] = resample;
    if (resample) {
      logz_acc += lse - log((double)N);
      /* the fixed-point weights are decided from FP32 log-weights */
      for (int64_t i = 0; i < N; i++) lw32[i] = (float)lw[i];
      orc_resample_from_lw(lw32, N, N, seed, 0, (uint32_t)t, anc);
      for (int64_t k = 0; k < N; k++) xn[k] = x[anc[k]];
      double* tmp = x;
      x = xn;
      xn = tmp;
      for (int64_t i = 0; i < N; i++) lw[i] = 0.0;
    }
  }
  double lse;
  orc_lse_ess(lw, N, &lse, NULL, NULL, NULL);
  double logz = logz_acc + lse - log((double)N);
  if (x_out) memcpy(x_out, x, (size_t)N * sizeof(double));
  if (lw_out) memcpy(lw_out, lw, (size_t)N * sizeof(double));
  free(x);
  free(xn);
  free(lw);
  free(lw32);
  free(anc);
  return logz;
}
