// Draw policy of a learned proposal: the trace's random choices come from
// q(n, c | data) computed by the network (mlp.cu); the log-weight gains
// log p(n, c) - log q(n, c), so importance weighting (§3.6.2) still targets the
// posterior of the model of Fig. 1.  The draw reuses the prior trace's words
// (purpose POLY_TRACE): the degree by the inverse CDF of q at u = u01(w6), and
// c_j = mu + s z_j with the prior's Box-Muller normals.  A proposal equal to the
// prior therefore gives the prior trace bit for bit (correction exactly 0).
#pragma once

#include "trace.cuh"

namespace ppl {

constexpr int kMaxSlots = 22;  // coefficient slots the 48 network outputs can describe

struct ProposalSmem {
  float cum[kMaxDegrees];
  float logq[kMaxDegrees];
  int base[kMaxDegrees];
  float mu[kMaxSlots], s[kMaxSlots], logs[kMaxSlots], inv_s[kMaxSlots];
  float log_p, log_sigma, sigma, inv_sigma;
};

// Proposal of one data set from its 48 network outputs (one thread).
__device__ __forceinline__ void load_proposal(const PolyParams& p, const float* o,
                                              ProposalSmem& ps) {
  float mx = -INFINITY;
  for (int k = 0; k < p.n_deg; ++k) mx = fmaxf(mx, o[k]);
  float se = 0.0f;
  for (int k = 0; k < p.n_deg; ++k) se += expf(o[k] - mx);
  const float lse = logf(se);
  float cum = 0.0f;
  int base = 0;
  for (int k = 0; k < kMaxDegrees; ++k) {
    if (k < p.n_deg) {
      cum += expf(o[k] - mx) / se;
      ps.cum[k] = cum;
      ps.logq[k] = (o[k] - mx) - lse;
      ps.base[k] = base;
      base += p.min_deg + k + p.coef_offset;
    } else {
      ps.cum[k] = 2.0f;
      ps.logq[k] = 0.0f;
      ps.base[k] = 0;
    }
  }
  ps.sigma = p.prior_sigma;
  ps.inv_sigma = 1.0f / p.prior_sigma;
  ps.log_sigma = logf(p.prior_sigma);
  ps.log_p = -logf((float)p.n_deg);
  for (int i = 0; i < kMaxSlots && i < base; ++i) {
    const float t = fminf(fmaxf(o[5 + 2 * i], -9.0f), 1.0f);
    ps.mu[i] = p.prior_sigma * o[4 + 2 * i];
    ps.s[i] = p.prior_sigma * expf(t);
    ps.inv_s[i] = 1.0f / ps.s[i];  // (the prior's reciprocal when s equals sigma)
    ps.logs[i] = ps.log_sigma + t;
  }
}

// log N(x; mu, s^2) with 1/s given (one multiply instead of a division, in
// the same form for the prior and the proposal, so a proposal equal to the
// prior cancels exactly)
__device__ __forceinline__ float log_normal32(float x, float mu, float inv_s, float logs) {
  const float z = (x - mu) * inv_s;
  return -0.918938533f - logs - 0.5f * z * z;
}

struct LearnedDraw {
  PolyParams p;
  uint64_t seed;
  uint32_t instance;
  const ProposalSmem* ps;
  __device__ __forceinline__ int operator()(uint32_t i, float (&c)[kMaxCoef], float& corr) const {
    const uint4 a = philox_block(seed, i, instance, 0, kPolyTrace, 0);
    const uint4 b = philox_block(seed, i, instance, 0, kPolyTrace, 1);
    float z[kMaxCoef];
    box_muller(a.x, a.y, z[0], z[1]);
    box_muller(a.z, a.w, z[2], z[3]);
    box_muller(b.x, b.y, z[4], z[5]);
    // the inverse CDF of q at u: the first degree whose cumulative mass
    // exceeds u (the last one when rounding leaves u above every mass)
    const float u = u01(b.z);
    int k = 0;
#pragma unroll
    for (int kk = 0; kk < kMaxDegrees - 1; ++kk) k += (kk < p.n_deg - 1 && u >= ps->cum[kk]);
    const int n = p.min_deg + k, ncoef = n + p.coef_offset, base = ps->base[k];
    float cr = ps->log_p - ps->logq[k];
#pragma unroll
    for (int j = 0; j < kMaxCoef; ++j) {
      if (j < ncoef) {
        const float mu = ps->mu[base + j], s = ps->s[base + j];
        c[j] = fmaf(s, z[j], mu);
        cr += log_normal32(c[j], 0.0f, ps->inv_sigma, ps->log_sigma) -
              log_normal32(c[j], mu, ps->inv_s[base + j], ps->logs[base + j]);
      } else {
        c[j] = 0.0f;
      }
    }
    corr = cr;
    return n;
  }
};

}  // namespace ppl
