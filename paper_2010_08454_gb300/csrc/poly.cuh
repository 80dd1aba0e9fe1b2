// The polynomial line-fitting model of Fig. 1 (§1.1) as a device function of
// the model registry, and the per-thread accumulators of the normalisation
// (§3.6.2) and posterior passes.
#pragma once

#include "common.cuh"
#include "rng.cuh"

namespace ppl {

struct PolyParams {
  int min_deg, n_deg, coef_offset;
  float prior_sigma;
  float neg_half_inv_var;  // -1 / (2 obs_sigma^2)
};

// One trace's `sample` statements (§3.4):
//   n <- sample(uniform-discrete(min_deg, max_deg))
//   c_k <- sample(normal(0, prior_sigma)), k < n + coef_offset
// Draw addresses: blocks 0 and 1 of purpose POLY_TRACE give words w0..w7;
// (z0,z1), (z2,z3), (z4,z5) are Box-Muller pairs of (w0,w1), (w2,w3), (w4,w5),
// and n comes from w6.  Coefficients past the trace's count are 0, so a
// Horner evaluation padded to six coefficients gives the same value exactly.
__device__ __forceinline__ int poly_draw(const PolyParams& p, uint64_t seed, uint32_t instance,
                                         uint32_t particle, float c[kMaxCoef]) {
  const uint4 a = philox_block(seed, particle, instance, 0, kPolyTrace, 0);
  const uint4 b = philox_block(seed, particle, instance, 0, kPolyTrace, 1);
  float z[kMaxCoef];
  box_muller(a.x, a.y, z[0], z[1]);
  box_muller(a.z, a.w, z[2], z[3]);
  box_muller(b.x, b.y, z[4], z[5]);
  const int n = uniform_discrete(b.z, p.min_deg, p.min_deg + p.n_deg - 1);
  const int ncoef = n + p.coef_offset;
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) c[k] = (k < ncoef) ? p.prior_sigma * z[k] : 0.0f;
  return n;
}

// Compensated (Kahan) addition: the factor sums of the trace kernels add their
// 16-point inner sums this way, which keeps the FP32 accumulation error at a
// few ulps.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
  const float y = __fsub_rn(v, comp);
  const float t = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

// Running log-sum-exp statistics of one thread / block: maximum and its
// (lowest) index, sums of exp(lw - m) and exp(2 (lw - m)), and the best trace
// of each degree.  Merging rescales by exp(m_a - m), which is exact in real
// arithmetic; -inf log-weights contribute nothing.
struct StatAcc {
  float m, s, s2;
  int arg;
  float dm[kMaxDegrees];
  int darg[kMaxDegrees];
  int nan;

  __device__ __forceinline__ void init() {
    m = -INFINITY;
    s = 0.0f;
    s2 = 0.0f;
    arg = 0x7fffffff;
    nan = 0;
#pragma unroll
    for (int d = 0; d < kMaxDegrees; ++d) {
      dm[d] = -INFINITY;
      darg[d] = 0x7fffffff;
    }
  }
  // Indices passed to add() by one thread must increase, so `>` keeps the lowest.
  __device__ __forceinline__ void add(float lw, int i, int d) {
    if (lw > m) {
      const float e = (m == -INFINITY) ? 0.0f : expf(m - lw);
      s = fmaf(s, e, 1.0f);
      s2 = fmaf(s2, e * e, 1.0f);
      m = lw;
      arg = i;
    } else if (lw > -INFINITY) {
      const float e = expf(lw - m);
      s += e;
      s2 = fmaf(e, e, s2);
    } else if (lw != lw) {
      nan = 1;
    }
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k)
      if (k == d && lw > dm[k]) {
        dm[k] = lw;
        darg[k] = i;
      }
  }
  __device__ __forceinline__ void merge(const StatAcc& o) {
    const float M = fmaxf(m, o.m);
    if (M > -INFINITY) {
      const float ea = (m == -INFINITY) ? 0.0f : expf(m - M);
      const float eb = (o.m == -INFINITY) ? 0.0f : expf(o.m - M);
      s = s * ea + o.s * eb;
      s2 = s2 * ea * ea + o.s2 * eb * eb;
    }
    if (o.m > m || (o.m == m && o.arg < arg)) arg = o.arg;
    m = M;
    nan |= o.nan;
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k)
      if (o.dm[k] > dm[k] || (o.dm[k] == dm[k] && o.darg[k] < darg[k])) {
        dm[k] = o.dm[k];
        darg[k] = o.darg[k];
      }
  }
  __device__ __forceinline__ StatAcc shfl_xor(int lane_mask) const {
    StatAcc o;
    o.m = __shfl_xor_sync(0xffffffffu, m, lane_mask);
    o.s = __shfl_xor_sync(0xffffffffu, s, lane_mask);
    o.s2 = __shfl_xor_sync(0xffffffffu, s2, lane_mask);
    o.arg = __shfl_xor_sync(0xffffffffu, arg, lane_mask);
    o.nan = __shfl_xor_sync(0xffffffffu, nan, lane_mask);
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      o.dm[k] = __shfl_xor_sync(0xffffffffu, dm[k], lane_mask);
      o.darg[k] = __shfl_xor_sync(0xffffffffu, darg[k], lane_mask);
    }
    return o;
  }
};

// Per-block result of the statistics pass, written to the workspace.
struct StatPartial {
  float m, s, s2;
  int arg;
  float dm[kMaxDegrees];
  int darg[kMaxDegrees];
  int nan, pad[3];
};

}  // namespace ppl
