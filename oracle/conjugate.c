/*
 * Closed-form evidence of the line-fitting model for a fixed degree, used to
 * pin the importance-sampling estimates.  TEST INFRASTRUCTURE ONLY.
 *
 * For a fixed coefficient count d the model of Fig. 1 is Bayesian linear
 * regression with the unnormalised factor exp(-||y - Phi c||^2 / (2 sigma^2)),
 * Phi_lk = x_l^k, and the prior c ~ N(0, s^2 I).  Completing the square:
 *   A = I / s^2 + Phi^T Phi / sigma^2,   b = Phi^T y / sigma^2,   m = A^{-1} b
 *   log Z_d = -(d/2) log s^2 - (1/2) log|A| + (1/2) b^T m - y^T y / (2 sigma^2)
 * (no (2 pi sigma^2)^{-L/2} term: `factor` adds the distance, not a density).
 * The posterior of c given the degree is N(m, A^{-1}).  Over degrees,
 *   Z = sum_n p(n) Z_n,  p(n | y) = p(n) Z_n / Z,  p(n) = 1 / (max_deg - min_deg + 1).
 * A is factorised by Cholesky in FP64.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

/* Cholesky A = R R^T (lower triangular R) of a d x d matrix, d <= 6; returns 0 on success. */
static int cholesky(int d, const double* A, double* R) {
  memset(R, 0, sizeof(double) * (size_t)(d * d));
  for (int i = 0; i < d; i++) {
    for (int j = 0; j <= i; j++) {
      double s = A[i * d + j];
      for (int k = 0; k < j; k++) s -= R[i * d + k] * R[j * d + k];
      if (i == j) {
        if (s <= 0.0) return 1;
        R[i * d + i] = sqrt(s);
      } else {
        R[i * d + j] = s / R[j * d + j];
      }
    }
  }
  return 0;
}

double orc_blr_evidence(const double* x, const double* y, int64_t L, int ncoef, double sigma,
                        double prior_sigma, double* mean, double* var) {
  int d = ncoef;
  double A[36], b[6], R[36];
  double s2 = prior_sigma * prior_sigma, sg2 = sigma * sigma;
  for (int i = 0; i < d; i++) {
    b[i] = 0.0;
    for (int j = 0; j < d; j++) A[i * d + j] = (i == j) ? 1.0 / s2 : 0.0;
  }
  double yy = 0.0;
  for (int64_t l = 0; l < L; l++) {
    double phi[6];
    double xp = 1.0;
    for (int k = 0; k < d; k++) {
      phi[k] = xp;
      xp *= x[l];
    }
    for (int i = 0; i < d; i++) {
      b[i] += phi[i] * y[l] / sg2;
      for (int j = 0; j < d; j++) A[i * d + j] += phi[i] * phi[j] / sg2;
    }
    yy += y[l] * y[l];
  }
  if (cholesky(d, A, R)) return NAN;
  /* m = A^{-1} b by forward then back substitution */
  double z[6], m[6];
  for (int i = 0; i < d; i++) {
    double s = b[i];
    for (int k = 0; k < i; k++) s -= R[i * d + k] * z[k];
    z[i] = s / R[i * d + i];
  }
  for (int i = d - 1; i >= 0; i--) {
    double s = z[i];
    for (int k = i + 1; k < d; k++) s -= R[k * d + i] * m[k];
    m[i] = s / R[i * d + i];
  }
  double logdet = 0.0, bm = 0.0;
  for (int i = 0; i < d; i++) {
    logdet += 2.0 * log(R[i * d + i]);
    bm += b[i] * m[i];
  }
  if (mean)
    for (int i = 0; i < d; i++) mean[i] = m[i];
  if (var) {
    /* diag(A^{-1}): solve A v = e_i for each unit vector */
    for (int i = 0; i < d; i++) {
      double e[6], zz[6], v[6];
      for (int k = 0; k < d; k++) e[k] = (k == i) ? 1.0 : 0.0;
      for (int r = 0; r < d; r++) {
        double s = e[r];
        for (int k = 0; k < r; k++) s -= R[r * d + k] * zz[k];
        zz[r] = s / R[r * d + r];
      }
      for (int r = d - 1; r >= 0; r--) {
        double s = zz[r];
        for (int k = r + 1; k < d; k++) s -= R[k * d + r] * v[k];
        v[r] = s / R[r * d + r];
      }
      var[i] = v[i];
    }
  }
  return -0.5 * d * log(s2) - 0.5 * logdet + 0.5 * bm - yy / (2.0 * sg2);
}

/* Exact log Z over the degree prior, p(n | y), and per-degree posterior moments
 * (deg_mean, deg_var are [4][6], zero beyond each degree's coefficient count). */
double orc_poly_exact(const orc_poly* m, const double* x, const double* y, int64_t L,
                      double* p_n, double* deg_mean, double* deg_var) {
  int n_deg = m->max_deg - m->min_deg + 1;
  double logzn[4], mx = -INFINITY;
  for (int d = 0; d < n_deg; d++) {
    int ncoef = m->min_deg + d + m->coef_offset;
    double mean[6] = {0}, var[6] = {0};
    logzn[d] = orc_blr_evidence(x, y, L, ncoef, m->obs_sigma, m->prior_sigma, mean, var);
    if (deg_mean)
      for (int k = 0; k < 6; k++) deg_mean[d * 6 + k] = (k < ncoef) ? mean[k] : 0.0;
    if (deg_var)
      for (int k = 0; k < 6; k++) deg_var[d * 6 + k] = (k < ncoef) ? var[k] : 0.0;
    if (logzn[d] > mx) mx = logzn[d];
  }
  double s = 0.0;
  for (int d = 0; d < n_deg; d++) s += exp(logzn[d] - mx);
  if (p_n)
    for (int d = 0; d < n_deg; d++) p_n[d] = exp(logzn[d] - mx) / s;
  return mx + log(s) - log((double)n_deg);
}
