/*
 * Exact enumeration (§3.6.1) and likelihood weighting (§3.6.2) on tiny
 * discrete models, used to pin the importance-sampling definition against an
 * exact posterior.  TEST INFRASTRUCTURE ONLY.
 *
 * Enumeration runs the model down every path through its `sample` calls,
 * one branch per value in the support of each distribution, multiplying the
 * branch probabilities and the exp(factor) terms; it stops at a depth limit.
 * The result is the normalised distribution of return values.
 *
 * Models (the names follow the benchmark table, Table 1 of §5.1):
 *   0 biasedcoin: theta ~ uniform-discrete over {1..9}/10; observe each flip in
 *                 `data` (0/1) as bernoulli(theta); return theta.
 *   1 binomial:   k = sum of data[0] flips of bernoulli(0.3), each a `sample`;
 *                 return k (no conditioning).
 *   2 geometric:  count bernoulli(0.5) failures before the first success, at
 *                 most data[0] draws deep; return the count.
 * Likelihood weighting draws every `sample` from its distribution with the
 * counter layout (particle i, instance 0, step 0, purpose POLY_TRACE, block j)
 * word (j*4 + slot), one word per draw in program order, and sums the factors.
 */
#include "oracle.h"

#include <math.h>

#define MODEL_BIASEDCOIN 0
#define MODEL_BINOMIAL 1
#define MODEL_GEOMETRIC 2

static int add_outcome(double v, double p, double* values, double* probs, int* n, int max_out) {
  for (int i = 0; i < *n; i++)
    if (values[i] == v) {
      probs[i] += p;
      return 0;
    }
  if (*n >= max_out) return 1;
  values[*n] = v;
  probs[*n] = p;
  (*n)++;
  return 0;
}

/* Returns the number of distinct return values, or -1 if max_out is too small. */
int orc_enumerate(int model, const int32_t* data, int64_t n_data, int max_depth, double* values,
                  double* probs, int max_out) {
  int n = 0;
  if (model == MODEL_BIASEDCOIN) {
    for (int a = 1; a <= 9; a++) { /* branch on every value of theta */
      double theta = a / 10.0;
      double p = 1.0 / 9.0;
      for (int64_t f = 0; f < n_data; f++) p *= data[f] ? theta : 1.0 - theta;
      if (add_outcome(theta, p, values, probs, &n, max_out)) return -1;
    }
  } else if (model == MODEL_BINOMIAL) {
    int trials = data[0];
    if (trials > 20) return -1;
    for (uint32_t path = 0; path < (1u << trials); path++) { /* every branch sequence */
      double p = 1.0;
      int k = 0;
      for (int t = 0; t < trials; t++) {
        int success = (path >> t) & 1;
        p *= success ? 0.3 : 0.7;
        k += success;
      }
      if (add_outcome((double)k, p, values, probs, &n, max_out)) return -1;
    }
  } else if (model == MODEL_GEOMETRIC) {
    int depth = data[0] < max_depth ? data[0] : max_depth;
    double reach = 1.0; /* probability of the path of `c` failures so far */
    for (int c = 0; c < depth; c++) {
      if (add_outcome((double)c, reach * 0.5, values, probs, &n, max_out)) return -1;
      reach *= 0.5;
    }
  } else {
    return -1;
  }
  double s = 0.0;
  for (int i = 0; i < n; i++) s += probs[i];
  for (int i = 0; i < n; i++) probs[i] /= s;
  return n;
}

static uint32_t draw_word(uint64_t seed, uint32_t i, int idx) {
  uint32_t w[4];
  orc_philox_block(seed, i, 0, 0, ORC_PURPOSE_POLY_TRACE, (uint32_t)(idx / 4), w);
  return w[idx % 4];
}

static int bernoulli(uint32_t w, double p) { return orc_u01(w) < p; }

void orc_is_discrete(int model, const int32_t* data, int64_t n_data, int64_t N, uint64_t seed,
                     double* values, double* lw) {
  for (int64_t i = 0; i < N; i++) {
    double v = 0.0, l = 0.0;
    if (model == MODEL_BIASEDCOIN) {
      int a = orc_uniform_discrete(draw_word(seed, (uint32_t)i, 0), 1, 9);
      double theta = a / 10.0;
      for (int64_t f = 0; f < n_data; f++) l += log(data[f] ? theta : 1.0 - theta);
      v = theta;
    } else if (model == MODEL_BINOMIAL) {
      int k = 0;
      for (int t = 0; t < data[0]; t++) k += bernoulli(draw_word(seed, (uint32_t)i, t), 0.3);
      v = k;
    } else if (model == MODEL_GEOMETRIC) {
      int c = 0;
      while (c < data[0] && !bernoulli(draw_word(seed, (uint32_t)i, c), 0.5)) c++;
      /* a path that reaches the depth limit is outside the truncated support */
      l = (c >= data[0]) ? -INFINITY : 0.0;
      v = c;
    }
    values[i] = v;
    lw[i] = l;
  }
}
