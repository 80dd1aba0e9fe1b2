/*
 * Oracle for the learned proposal: a small network maps a data set to a
 * proposal over the line-fitting trace's random choices (degree n and the
 * coefficients), importance weights correct it to the posterior (§3.6.2: any
 * proposal, weighted by p/q, targets the same posterior as the prior run of
 * Fig. 1).  Training minimises -log q(n, c | data) over (data, trace) pairs
 * the model generates forward (inference compilation, Le, Baydin and Wood,
 * AISTATS 2017).  TEST INFRASTRUCTURE ONLY.
 *
 * Network (precision fixed by the method: BF16 weights and GEMM inputs, FP32
 * accumulation; the oracle accumulates in FP64):
 *   in[64]  = the 32 points sorted by x:  in[2l] = x_(l),  in[2l+1] = y_(l) / 10
 *             (y / 10 in FP32), each rounded to BF16
 *   h1      = relu(W1 in + b1)            W1 [256 x 64]
 *   h2      = relu(W2 bf16(h1) + b2)      W2 [256 x 256]
 *   out     = W3 bf16(h2) + b3            W3 [48 x 256] (rows 40..47 unused)
 * Proposal for degree slot k = n - min_deg with ncoef_k = min_deg + k +
 * coef_offset coefficients, base_k = ncoef_0 + ... + ncoef_{k-1}:
 *   q(k)      = softmax(out[0..n_deg))_k
 *   mu_kj     = prior_sigma * out[4 + 2 (base_k + j)]
 *   s_kj      = prior_sigma * exp(t),  t = clamp(out[5 + 2 (base_k + j)], -9, 1)
 *   log s_kj  = log(prior_sigma) + t
 *   c_j | k   ~ N(mu_kj, s_kj^2),  j < ncoef_k
 * Draws reuse the prior trace's words (purpose POLY_TRACE): the degree by the
 * inverse CDF of q at u = u01(w6), c_j = mu + s z_j with the Box-Muller z_j, so
 * a proposal equal to the prior reproduces the prior trace exactly.
 *   log w = log p(n) + sum_j log N(c_j; 0, prior_sigma) + factor(c)
 *           - log q(k) - sum_j log N(c_j; mu_kj, s_kj)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

float orc_bf16(float v);
void orc_mlp_set_bf16(int on);

#define IN 64
#define H 256
#define OUT 48
#define NPTS 32

/* Round to the nearest BF16 value (ties to even) from FP32 bits. */
float orc_bf16(float v) {
  uint32_t b;
  memcpy(&b, &v, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) return v; /* inf / nan */
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7fffu + lsb;
  b &= 0xffff0000u;
  float r;
  memcpy(&r, &b, 4);
  return r;
}

static double log_normal(double x, double mu, double s, double log_s) {
  const double half_log_2pi = 0.91893853320467274178032973640562;
  double z = (x - mu) / s;
  return -half_log_2pi - log_s - 0.5 * z * z;
}

/* With rounding off, activations keep full precision (for derivative checks). */
static int g_round_bf16 = 1;
void orc_mlp_set_bf16(int on) { g_round_bf16 = on; }
static double act(double v) {
  double r = v > 0.0 ? v : 0.0;
  return g_round_bf16 ? (double)orc_bf16((float)r) : r;
}

/* Features of one data set of NPTS points: sorted by x (ties keep input order). */
void orc_mlp_features(const float* x, const float* y, float* feat) {
  int order[NPTS];
  for (int i = 0; i < NPTS; i++) order[i] = i;
  for (int i = 1; i < NPTS; i++) { /* insertion sort: stable */
    int v = order[i], j = i - 1;
    while (j >= 0 && x[order[j]] > x[v]) {
      order[j + 1] = order[j];
      j--;
    }
    order[j + 1] = v;
  }
  for (int l = 0; l < NPTS; l++) {
    float yd = y[order[l]] / 10.0f;
    feat[2 * l] = orc_bf16(x[order[l]]);
    feat[2 * l + 1] = orc_bf16(yd);
  }
}

/* Forward pass; h1, h2 (BF16-rounded activations) and out are outputs. */
void orc_mlp_forward(const float* W1, const float* b1, const float* W2, const float* b2,
                     const float* W3, const float* b3, const float* feat, double* h1,
                     double* h2, double* out) {
  for (int o = 0; o < H; o++) {
    double s = b1[o];
    for (int i = 0; i < IN; i++) s += (double)W1[o * IN + i] * (double)feat[i];
    h1[o] = act(s);
  }
  for (int o = 0; o < H; o++) {
    double s = b2[o];
    for (int i = 0; i < H; i++) s += (double)W2[o * H + i] * h1[i];
    h2[o] = act(s);
  }
  for (int o = 0; o < OUT; o++) {
    double s = b3[o];
    for (int i = 0; i < H; i++) s += (double)W3[o * H + i] * h2[i];
    out[o] = s;
  }
}

static int coef_base(const orc_poly* m, int k) {
  int b = 0;
  for (int kk = 0; kk < k; kk++) b += m->min_deg + kk + m->coef_offset;
  return b;
}

/* log q(n, c | out) and, optionally, d(-log q)/d out (zero outside the used slots). */
double orc_proposal_logq(const orc_poly* m, const double* out, int n, const double* c,
                         double* grad) {
  int n_deg = m->max_deg - m->min_deg + 1, k = n - m->min_deg;
  double mx = -INFINITY;
  for (int i = 0; i < n_deg; i++)
    if (out[i] > mx) mx = out[i];
  double se = 0.0;
  for (int i = 0; i < n_deg; i++) se += exp(out[i] - mx);
  double logq = out[k] - mx - log(se);
  if (grad) {
    for (int i = 0; i < OUT; i++) grad[i] = 0.0;
    for (int i = 0; i < n_deg; i++) grad[i] = exp(out[i] - mx) / se - (i == k ? 1.0 : 0.0);
  }
  int ncoef = n + m->coef_offset, base = coef_base(m, k);
  double ls0 = log(m->prior_sigma);
  for (int j = 0; j < ncoef; j++) {
    double om = out[4 + 2 * (base + j)], os = out[5 + 2 * (base + j)];
    double cl = os < -9.0 ? -9.0 : (os > 1.0 ? 1.0 : os);
    double mu = m->prior_sigma * om, s = m->prior_sigma * exp(cl), ls = ls0 + cl;
    logq += log_normal(c[j], mu, s, ls);
    if (grad) {
      double z = (c[j] - mu) / s;
      grad[4 + 2 * (base + j)] = -z / s * m->prior_sigma;
      grad[5 + 2 * (base + j)] = (os > -9.0 && os < 1.0) ? (1.0 - z * z) : 0.0;
    }
  }
  return logq;
}

/* One trace under the learned proposal (see the header): returns log w. */
double orc_learned_trace(const orc_poly* m, const double* out, const double* x, const double* y,
                         int64_t L, uint64_t seed, uint32_t instance, uint32_t particle,
                         int* n_out, double* c_out) {
  uint32_t w[8];
  orc_philox_block(seed, particle, instance, 0, ORC_PURPOSE_POLY_TRACE, 0, w);
  orc_philox_block(seed, particle, instance, 0, ORC_PURPOSE_POLY_TRACE, 1, w + 4);
  double z[6];
  orc_box_muller(w[0], w[1], &z[0], &z[1]);
  orc_box_muller(w[2], w[3], &z[2], &z[3]);
  orc_box_muller(w[4], w[5], &z[4], &z[5]);
  int n_deg = m->max_deg - m->min_deg + 1;
  double mx = -INFINITY, se = 0.0, p[4];
  for (int i = 0; i < n_deg; i++)
    if (out[i] > mx) mx = out[i];
  for (int i = 0; i < n_deg; i++) se += exp(out[i] - mx);
  for (int i = 0; i < n_deg; i++) p[i] = exp(out[i] - mx) / se;
  double u = orc_u01(w[6]), cum = 0.0;
  int k = n_deg - 1;
  for (int i = 0; i < n_deg; i++) { /* inverse CDF: first k with u < p_0 + ... + p_k */
    cum += p[i];
    if (u < cum) {
      k = i;
      break;
    }
  }
  int n = m->min_deg + k, ncoef = n + m->coef_offset, base = coef_base(m, k);
  double c[6] = {0, 0, 0, 0, 0, 0}, ls0 = log(m->prior_sigma), lw = 0.0;
  for (int j = 0; j < ncoef; j++) {
    double os = out[5 + 2 * (base + j)];
    double cl = os < -9.0 ? -9.0 : (os > 1.0 ? 1.0 : os);
    double mu = m->prior_sigma * out[4 + 2 * (base + j)];
    double s = m->prior_sigma * exp(cl), ls = ls0 + cl;
    c[j] = mu + s * z[j];
    lw += log_normal(c[j], 0.0, m->prior_sigma, ls0) - log_normal(c[j], mu, s, ls);
  }
  lw += -log((double)n_deg) - log(p[k]);
  double sum_sq = 0.0;
  for (int64_t l = 0; l < L; l++) {
    double f = 0.0, xp = 1.0;
    for (int j = 0; j < ncoef; j++) {
      f += c[j] * xp;
      xp *= x[l];
    }
    double r = y[l] - f;
    sum_sq += r * r;
  }
  lw += -sum_sq / (2.0 * m->obs_sigma * m->obs_sigma);
  if (n_out) *n_out = n;
  if (c_out)
    for (int j = 0; j < 6; j++) c_out[j] = c[j];
  return lw;
}

void orc_learned_is(const orc_poly* m, const double* out, const double* x, const double* y,
                    int64_t L, int64_t N, uint64_t seed, uint32_t instance, double* lw,
                    int32_t* n, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    int ni;
    double ci[6];
    lw[i] = orc_learned_trace(m, out, x, y, L, seed, instance, (uint32_t)i, &ni, ci);
    if (n) n[i] = ni;
    if (c)
      for (int j = 0; j < 6; j++) c[6 * i + j] = ci[j];
  }
}

/*
 * Forward simulation of a training pair p (purpose FORWARD_SIM, instance 0):
 *   blocks 0, 1 of (p, 0, 0): the trace exactly as a prior trace (degree from
 *   w6, coefficients prior_sigma * z_j);  block 2 + l: point l, x = 2 u01(w0)
 *   - 1, y = f(x) + obs_sigma * BoxMuller(w1, w2).z0.
 * FP64 here; x, y are returned rounded to FP32 as the features take them.
 */
void orc_forward_sim(const orc_poly* m, uint64_t seed, uint32_t pair, float* x, float* y,
                     int* n_out, double* c_out) {
  uint32_t w[8];
  orc_philox_block(seed, pair, 0, 0, ORC_PURPOSE_FORWARD_SIM, 0, w);
  orc_philox_block(seed, pair, 0, 0, ORC_PURPOSE_FORWARD_SIM, 1, w + 4);
  double z[6];
  orc_box_muller(w[0], w[1], &z[0], &z[1]);
  orc_box_muller(w[2], w[3], &z[2], &z[3]);
  orc_box_muller(w[4], w[5], &z[4], &z[5]);
  int n = orc_uniform_discrete(w[6], m->min_deg, m->max_deg), ncoef = n + m->coef_offset;
  double c[6] = {0, 0, 0, 0, 0, 0};
  for (int j = 0; j < ncoef; j++) c[j] = m->prior_sigma * z[j];
  for (int l = 0; l < NPTS; l++) {
    uint32_t v[4];
    orc_philox_block(seed, pair, 0, 0, ORC_PURPOSE_FORWARD_SIM, 2 + (uint32_t)l, v);
    double xl = 2.0 * orc_u01(v[0]) - 1.0, e0, e1;
    orc_box_muller(v[1], v[2], &e0, &e1);
    double f = 0.0, xp = 1.0;
    for (int j = 0; j < ncoef; j++) {
      f += c[j] * xp;
      xp *= xl;
    }
    x[l] = (float)xl;
    y[l] = (float)(f + m->obs_sigma * e0);
  }
  *n_out = n;
  for (int j = 0; j < 6; j++) c_out[j] = c[j];
}

/*
 * Mean training loss -log q over B pairs and its gradient with respect to all
 * parameters (FP64 backpropagation through the network above; the BF16
 * rounding of activations is treated as the identity for the gradient).
 */
double orc_mlp_loss_grad(const orc_poly* m, const float* W1, const float* b1, const float* W2,
                         const float* b2, const float* W3, const float* b3, const float* feats,
                         const int32_t* n, const double* c, int64_t B, double* gW1, double* gb1,
                         double* gW2, double* gb2, double* gW3, double* gb3) {
  if (gW1) {
    memset(gW1, 0, sizeof(double) * H * IN);
    memset(gb1, 0, sizeof(double) * H);
    memset(gW2, 0, sizeof(double) * H * H);
    memset(gb2, 0, sizeof(double) * H);
    memset(gW3, 0, sizeof(double) * OUT * H);
    memset(gb3, 0, sizeof(double) * OUT);
  }
  double loss = 0.0;
  double h1[H], h2[H], out[OUT], d3[OUT], d2[H], d1[H];
  for (int64_t b = 0; b < B; b++) {
    const float* f = feats + b * IN;
    orc_mlp_forward(W1, b1, W2, b2, W3, b3, f, h1, h2, out);
    loss -= orc_proposal_logq(m, out, n[b], c + 6 * b, d3);
    if (!gW1) continue;
    for (int o = 0; o < OUT; o++) d3[o] /= (double)B;
    for (int i = 0; i < H; i++) {
      double s = 0.0;
      for (int o = 0; o < OUT; o++) s += d3[o] * W3[o * H + i];
      d2[i] = h2[i] > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < OUT; o++) {
      gb3[o] += d3[o];
      for (int i = 0; i < H; i++) gW3[o * H + i] += d3[o] * h2[i];
    }
    for (int i = 0; i < H; i++) {
      double s = 0.0;
      for (int o = 0; o < H; o++) s += d2[o] * W2[o * H + i];
      d1[i] = h1[i] > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < H; o++) {
      gb2[o] += d2[o];
      for (int i = 0; i < H; i++) gW2[o * H + i] += d2[o] * h1[i];
    }
    for (int o = 0; o < H; o++) {
      gb1[o] += d1[o];
      for (int i = 0; i < IN; i++) gW1[o * IN + i] += d1[o] * (double)f[i];
    }
  }
  return loss / (double)B;
}
