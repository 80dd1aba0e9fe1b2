// Sufficient statistics of the line-fitting factor (Fig. 1): a second way to
// evaluate  sum_l (y_l - f(x_l))^2,  f(x) = sum_{j<d} c_j x^j,  that is exact in
// real arithmetic and costs O(d^2) per trace instead of O(L d).
//
// With Phi the L x 6 matrix of powers x_l^j, G = Phi^T Phi = R^T R (Cholesky,
// R upper triangular) and w = R^-T Phi^T y, for the first d coefficients
//   sum_l (y_l - f(x_l))^2 = (y^T y - sum_{i<d} w_i^2) + sum_{i<d} z_i^2,
//   z_i = sum_{i<=j<d} R_ij c_j - w_i.
// (Cholesky factors and forward substitution are nested, so the leading d x d
// blocks serve degree d.)  The first term is the squared distance from y to
// the span of the first d powers: non-negative, formed once in FP64; the
// second is a sum of squares, so nothing cancels in FP32.
#pragma once

#include "common.cuh"

namespace ppl {

struct SuffStat {
  float R[kMaxCoef][kMaxCoef];  // upper triangle used
  float w[kMaxCoef];
  float base[kMaxCoef + 1];     // base[d] = y^T y - sum_{i<d} w_i^2
  int ok;                       // 0: G is singular to working precision (use the direct sum)
  int pad[2];
};

// The sum of squared residuals of a trace with d coefficients (c_j = 0 for j >= d).
__device__ __forceinline__ float suff_residual(const SuffStat& s, const float (&c)[kMaxCoef],
                                               int d) {
  float ss = s.base[d];
#pragma unroll
  for (int i = 0; i < kMaxCoef; ++i) {
    if (i < d) {
      float z = -s.w[i];
#pragma unroll
      for (int j = i; j < kMaxCoef; ++j) z = fmaf(s.R[i][j], c[j], z);
      ss = fmaf(z, z, ss);
    }
  }
  return ss;
}

}  // namespace ppl
