/*
 * Oracle traces of the polynomial line-fitting model (Fig. 1, §1.1) under the
 * prior proposal, i.e. likelihood weighting (§3.6.2).  TEST INFRASTRUCTURE ONLY.
 *
 * One trace, following the model's statements in order:
 *   n  <- sample(uniform-discrete(min_deg, max_deg))
 *   c  <- repeat(sample(normal(0, prior_sigma)), n + coef_offset)
 *   factor(-distance(c, data)),  distance = sum_l (y_l - f(x_l))^2 / (2 obs_sigma^2)
 *   f(x) = sum_k c_k x^k
 * `sample` draws (§3.4) are fixed by the counter layout:
 *   block 0 (purpose POLY_TRACE) -> words w0..w3, block 1 -> w4..w7
 *   (z0, z1) = BoxMuller(w0, w1), (z2, z3) = BoxMuller(w2, w3), (z4, z5) = BoxMuller(w4, w5)
 *   n = uniform-discrete(w6), c_k = prior_sigma * z_k; w7 is unused.
 * The log-weight is the sum of the `factor` terms (§3.4): the prior draws are
 * the proposal, so they contribute nothing.
 */
#include "oracle.h"

#include <math.h>

double orc_poly_trace(const orc_poly* m, const double* x, const double* y, int64_t L,
                      uint64_t seed, uint32_t instance, uint32_t particle, int* n_out,
                      double c_out[6]) {
  uint32_t w[8];
  orc_philox_block(seed, particle, instance, 0, ORC_PURPOSE_POLY_TRACE, 0, w);
  orc_philox_block(seed, particle, instance, 0, ORC_PURPOSE_POLY_TRACE, 1, w + 4);
  double z[6];
  orc_box_muller(w[0], w[1], &z[0], &z[1]);
  orc_box_muller(w[2], w[3], &z[2], &z[3]);
  orc_box_muller(w[4], w[5], &z[4], &z[5]);
  int n = orc_uniform_discrete(w[6], m->min_deg, m->max_deg);
  int ncoef = n + m->coef_offset;
  double c[6];
  for (int k = 0; k < 6; k++) c[k] = (k < ncoef) ? m->prior_sigma * z[k] : 0.0;

  double sum_sq = 0.0;
  for (int64_t l = 0; l < L; l++) {
    double f = 0.0, xp = 1.0;
    for (int k = 0; k < ncoef; k++) {
      f += c[k] * xp;
      xp *= x[l];
    }
    double r = y[l] - f;
    sum_sq += r * r;
  }
  double lw = -sum_sq / (2.0 * m->obs_sigma * m->obs_sigma);
  if (n_out) *n_out = n;
  if (c_out)
    for (int k = 0; k < 6; k++) c_out[k] = c[k];
  return lw;
}

/* Likelihood weighting over particles 0..N-1 of one instance (§3.6.2): run the
 * model N times and keep each trace's log-weight and returned coefficients. */
void orc_is_poly(const orc_poly* m, const double* x, const double* y, int64_t L, int64_t N,
                 uint64_t seed, uint32_t instance, double* lw, int32_t* n, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    int ni;
    double ci[6];
    lw[i] = orc_poly_trace(m, x, y, L, seed, instance, (uint32_t)i, &ni, ci);
    if (n) n[i] = ni;
    if (c)
      for (int k = 0; k < 6; k++) c[6 * i + k] = ci[k];
  }
}

/* The same traces for a chosen set of particle indices (sampled checks). */
void orc_is_poly_indices(const orc_poly* m, const double* x, const double* y, int64_t L,
                         const int64_t* idx, int64_t K, uint64_t seed, uint32_t instance,
                         double* lw, int32_t* n, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < K; j++) {
    int ni;
    double ci[6];
    lw[j] = orc_poly_trace(m, x, y, L, seed, instance, (uint32_t)idx[j], &ni, ci);
    if (n) n[j] = ni;
    if (c)
      for (int k = 0; k < 6; k++) c[6 * j + k] = ci[k];
  }
}
