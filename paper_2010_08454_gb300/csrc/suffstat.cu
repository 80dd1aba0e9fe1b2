// The sufficient statistics of a data set for the line-fitting factor (see
// suffstat.cuh): power sums in FP64 over the points, then the Cholesky factor
// of the 6 x 6 Gram matrix, the forward substitution and the per-degree
// distances, by one thread.  One block; the data are read once.
#include "kernels.h"
#include "suffstat.cuh"

namespace ppl {

constexpr int kSsPow = 2 * kMaxCoef - 1;  // x^0 .. x^10

__global__ void __launch_bounds__(kTpb) suffstat_kernel(const float* __restrict__ xs,
                                                        const float* __restrict__ ys, int64_t L,
                                                        int d_max, SuffStat* out) {
  __shared__ double red[kTpb / 32][kSsPow + kMaxCoef + 1];
  constexpr int V = kSsPow + kMaxCoef + 1;  // sum x^k, sum x^k y, sum y^2
  double acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.0;
  for (int64_t l = threadIdx.x; l < L; l += kTpb) {
    const double x = xs[l], y = ys[l];
    double pw = 1.0;
#pragma unroll
    for (int k = 0; k < kSsPow; ++k) {
      acc[k] += pw;
      if (k < kMaxCoef) acc[kSsPow + k] += pw * y;
      pw *= x;
    }
    acc[V - 1] += y * y;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double a = acc[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[warp][v] = a;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double S[V];
  for (int v = 0; v < V; ++v) {
    S[v] = 0.0;
    for (int w = 0; w < kTpb / 32; ++w) S[v] += red[w][v];
  }
  // Cholesky G = R^T R of the leading d_max x d_max block (G_ij = sum x^(i+j))
  double R[kMaxCoef][kMaxCoef] = {};
  int ok = 1;
  for (int i = 0; i < d_max && ok; ++i) {
    double dsum = S[2 * i];
    for (int k = 0; k < i; ++k) dsum -= R[k][i] * R[k][i];
    // a pivot that lost all but ~8 digits of the diagonal marks G singular for FP32 use
    if (!(dsum > 1e-8 * S[2 * i])) {
      ok = 0;
      break;
    }
    R[i][i] = sqrt(dsum);
    for (int j = i + 1; j < d_max; ++j) {
      double v = S[i + j];
      for (int k = 0; k < i; ++k) v -= R[k][i] * R[k][j];
      R[i][j] = v / R[i][i];
    }
  }
  double w[kMaxCoef] = {};
  if (ok)
    for (int i = 0; i < d_max; ++i) {  // R^T w = Phi^T y
      double v = S[kSsPow + i];
      for (int k = 0; k < i; ++k) v -= R[k][i] * w[k];
      w[i] = v / R[i][i];
    }
  SuffStat o;
  double base = S[V - 1];
  o.base[0] = (float)base;
  for (int i = 0; i < kMaxCoef; ++i) {
    for (int j = 0; j < kMaxCoef; ++j) o.R[i][j] = (float)R[i][j];
    o.w[i] = (float)w[i];
    base -= w[i] * w[i];
    o.base[i + 1] = (float)(base > 0.0 ? base : 0.0);
  }
  o.ok = ok;
  o.pad[0] = o.pad[1] = 0;
  *out = o;
}

size_t suffstat_bytes() { return sizeof(SuffStat); }

cudaError_t launch_suffstat(const float* x, const float* y, int64_t L, int d_max, void* out,
                            cudaStream_t s) {
  if (d_max < 1 || d_max > kMaxCoef) return cudaErrorInvalidValue;
  suffstat_kernel<<<1, kTpb, 0, s>>>(x, y, L, d_max, reinterpret_cast<SuffStat*>(out));
  return cudaGetLastError();
}

}  // namespace ppl
