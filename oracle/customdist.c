/*
 * The `customdist` benchmark (Table 1 of §5.1): importance sampling from a
 * user-defined distribution whose density is the sum of two weighted Gaussian
 * densities, conditioned here on observations of the drawn value.
 * TEST INFRASTRUCTURE ONLY.
 *
 *   x <- sample(custom: w1 N(mu1, s1^2) + (1 - w1) N(mu2, s2^2))
 *   observe(normal(x, obs_sigma), y_j)   for every data point y_j   (§3.4)
 *   return x
 *
 * Likelihood weighting (§3.6.2) draws x from the custom distribution:
 * component 1 when u01(w0) < w1, then mu + s z with z the first Box-Muller
 * normal of (w1, w2), the words of block 0 of (particle, 0, 0, POLY_TRACE);
 * the log-weight is the sum of the observations' log-densities.
 *
 * The exact answer is closed-form: each component times the Gaussian
 * likelihood integrates to a Gaussian in the sample mean, so
 *   Z = sum_k w_k (2 pi r^2)^(-n/2) exp(-(S2 - n ybar^2) / (2 r^2))
 *         * N(ybar; mu_k, s_k^2 + r^2 / n)
 * and x | y is a two-component mixture of the per-component Gaussian
 * posteriors (precision 1/s_k^2 + n/r^2).
 */
#include "oracle.h"

#include <math.h>

static const double kPi = 3.14159265358979323846;

void orc_customdist_is(const double* prm, const float* y, int64_t n, int64_t N, uint64_t seed,
                       double* x_out, double* lw_out) {
  const double w1 = prm[0], mu1 = prm[1], s1 = prm[2], mu2 = prm[3], s2 = prm[4], r = prm[5];
  const double c = -0.5 * log(2.0 * kPi * r * r);
  for (int64_t i = 0; i < N; i++) {
    uint32_t w[4];
    orc_philox_block(seed, (uint32_t)i, 0, 0, ORC_PURPOSE_POLY_TRACE, 0, w);
    double z0, z1;
    orc_box_muller(w[1], w[2], &z0, &z1);
    const double x = (orc_u01(w[0]) < w1) ? mu1 + s1 * z0 : mu2 + s2 * z0;
    double l = 0.0;
    for (int64_t j = 0; j < n; j++) {
      const double d = (double)y[j] - x;
      l += c - d * d / (2.0 * r * r);
    }
    x_out[i] = x;
    lw_out[i] = l;
  }
}

/* out: log Z, posterior mean and variance of x. */
void orc_customdist_exact(const double* prm, const float* y, int64_t n, double* out) {
  const double w[2] = {prm[0], 1.0 - prm[0]};
  const double mu[2] = {prm[1], prm[3]}, s[2] = {prm[2], prm[4]}, r = prm[5];
  double S1 = 0.0, S2 = 0.0;
  for (int64_t j = 0; j < n; j++) {
    S1 += y[j];
    S2 += (double)y[j] * y[j];
  }
  double lz[2], pm[2], pv[2];
  for (int k = 0; k < 2; k++) {
    if (n == 0) {
      lz[k] = log(w[k]);
      pm[k] = mu[k];
      pv[k] = s[k] * s[k];
      continue;
    }
    const double ybar = S1 / n, v = s[k] * s[k] + r * r / n;
    lz[k] = log(w[k]) - 0.5 * n * log(2.0 * kPi * r * r) - (S2 - n * ybar * ybar) / (2.0 * r * r)
            + 0.5 * log(2.0 * kPi * r * r / n)  /* the sample-mean density's normaliser */
            - 0.5 * log(2.0 * kPi * v) - (ybar - mu[k]) * (ybar - mu[k]) / (2.0 * v);
    const double prec = 1.0 / (s[k] * s[k]) + n / (r * r);
    pv[k] = 1.0 / prec;
    pm[k] = pv[k] * (mu[k] / (s[k] * s[k]) + S1 / (r * r));
  }
  const double m = lz[0] > lz[1] ? lz[0] : lz[1];
  const double e0 = exp(lz[0] - m), e1 = exp(lz[1] - m);
  const double p0 = e0 / (e0 + e1), p1 = 1.0 - p0;
  out[0] = m + log(e0 + e1);
  out[1] = p0 * pm[0] + p1 * pm[1];
  out[2] = p0 * (pv[0] + pm[0] * pm[0]) + p1 * (pv[1] + pm[1] * pm[1]) - out[1] * out[1];
}
