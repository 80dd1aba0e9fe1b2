/*
 * Oracle normalisation of log-weights and the weighted posterior summary.
 * TEST INFRASTRUCTURE ONLY.
 *
 * §3.6.2: importance sampling repeats the model N times and obtains the
 * posterior by normalising the log-probabilities of the returned values.  With
 * log-weights lw_i:
 *   LSE   = log sum_i exp(lw_i)
 *   log Z = LSE - log N            (the estimate of the evidence E_prior[exp(factor)])
 *   W_i   = exp(lw_i - LSE)        (normalised weights)
 *   ESS   = (sum_i exp lw_i)^2 / sum_i exp(2 lw_i)
 * Sums are formed after subtracting the maximum, which leaves every ratio
 * unchanged and keeps exp() finite.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

void orc_lse_ess(const double* lw, int64_t N, double* lse, double* ess, double* max_lw,
                 int64_t* argmax) {
  double m = -INFINITY;
  int64_t am = -1;
  for (int64_t i = 0; i < N; i++)
    if (lw[i] > m) { /* strict: the lowest index wins ties */
      m = lw[i];
      am = i;
    }
  double s = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < N; i++) {
    double e = exp(lw[i] - m);
    s += e;
    s2 += e * e;
  }
  if (lse) *lse = m + log(s);
  if (ess) *ess = s * s / s2;
  if (max_lw) *max_lw = m;
  if (argmax) *argmax = am;
}

/*
 * Posterior summary of a weighted population of line-fitting traces.  The
 * model returns the coefficient vector (Fig. 1); the paper takes the mode of
 * the empirical distribution as the line of best fit (§1.1).  Reported:
 *   p_n[d]        posterior mass of degree min_deg + d
 *   mean_c[k]     weighted mean of c_k, coefficients beyond a trace's count taken as 0
 *   deg_mean/var  weighted mean and variance of c_k among traces of one degree
 *   argmax        the mode: the highest-weight trace (lowest index on ties)
 *   map_deg       the degree with the largest p_n (lowest degree on ties)
 * A per-degree ratio of weighted sums does not depend on the constant the
 * weights are scaled by, so each degree uses exp(lw - max over that degree).
 */
void orc_posterior_poly(const orc_poly* m, const double* lw, const int32_t* n, const double* c,
                        int64_t N, orc_is_result* out) {
  memset(out, 0, sizeof(*out));
  int n_deg = m->max_deg - m->min_deg + 1;
  out->n_deg = n_deg;
  out->n_particles = N;
  orc_lse_ess(lw, N, &out->lse, &out->ess, &out->max_lw, &out->argmax);
  out->log_z = out->lse - log((double)N);

  for (int d = 0; d < n_deg; d++) {
    out->deg_max_lw[d] = -INFINITY;
    out->deg_argmax[d] = -1;
  }
  for (int64_t i = 0; i < N; i++) {
    int d = n[i] - m->min_deg;
    if (lw[i] > out->deg_max_lw[d]) {
      out->deg_max_lw[d] = lw[i];
      out->deg_argmax[d] = i;
    }
  }

  double total = 0.0;
  double mass[4] = {0, 0, 0, 0};
  for (int d = 0; d < n_deg; d++) {
    if (out->deg_argmax[d] < 0) continue; /* no trace of this degree */
    int ncoef = m->min_deg + d + m->coef_offset;
    double sw = 0.0, swc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < N; i++) {
      if (n[i] - m->min_deg != d) continue;
      double w = exp(lw[i] - out->deg_max_lw[d]);
      sw += w;
      for (int k = 0; k < ncoef; k++) swc[k] += w * c[6 * i + k];
    }
    for (int k = 0; k < ncoef; k++) out->deg_mean[d][k] = swc[k] / sw;
    double swv[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < N; i++) {
      if (n[i] - m->min_deg != d) continue;
      double w = exp(lw[i] - out->deg_max_lw[d]);
      for (int k = 0; k < ncoef; k++) {
        double dev = c[6 * i + k] - out->deg_mean[d][k];
        swv[k] += w * dev * dev;
      }
    }
    for (int k = 0; k < ncoef; k++) out->deg_var[d][k] = swv[k] / sw;
    /* mass of degree d relative to the global maximum: exp(max_d - max) * sum_d */
    mass[d] = exp(out->deg_max_lw[d] - out->max_lw) * sw;
    total += mass[d];
  }
  out->map_deg = m->min_deg;
  double best = -1.0;
  for (int d = 0; d < n_deg; d++) {
    out->p_n[d] = mass[d] / total;
    if (out->p_n[d] > best) {
      best = out->p_n[d];
      out->map_deg = m->min_deg + d;
    }
  }
  for (int d = 0; d < n_deg; d++)
    for (int k = 0; k < 6; k++) out->mean_c[k] += out->p_n[d] * out->deg_mean[d][k];
}
