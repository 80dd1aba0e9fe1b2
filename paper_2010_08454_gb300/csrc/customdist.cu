// The customdist benchmark (Table 1 of §5.1): likelihood weighting (§3.6.2)
// from a user-defined distribution whose density is the sum of two weighted
// Gaussian densities, with every data point observed as normal(x, obs_sigma)
// (§3.4):
//   x <- sample(custom: w1 N(mu1, s1^2) + (1 - w1) N(mu2, s2^2));
//   observe(normal(x, obs_sigma), y_j) for all j;  return x.
// The custom distribution's sampler picks the component from word 0 of block 0
// of (particle, 0, 0, POLY_TRACE) -- component 1 when u01(w0) < w1, decided
// exactly on the word's top 23 bits -- and takes the first Box-Muller normal
// of words 1 and 2.  Counter-based draws make both branches cost the same, so
// the component choice does not diverge a warp.
//
// One fused kernel: per particle the draw and the log-likelihood sum, per
// thread running sums (max m, sum e, sum e^2, sum e (x - ybar), sum e (x -
// ybar)^2 with e = exp(lw - m), rescaled when m grows), per block a merge,
// and the last block's FP64 summary.
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

constexpr int kCdData = 4096;  // observations staged in shared memory

struct CdAcc {
  float m, s, s2, sx, sxx;
  __device__ __forceinline__ void init() {
    m = -INFINITY;
    s = s2 = sx = sxx = 0.0f;
  }
  __device__ __forceinline__ void add(float l, float dx) {
    if (l > m) {
      const float r = (m == -INFINITY) ? 0.0f : expf(m - l);
      s = fmaf(s, r, 1.0f);
      s2 = fmaf(s2, r * r, 1.0f);
      sx = fmaf(sx, r, dx);
      sxx = fmaf(sxx, r, dx * dx);
      m = l;
    } else if (l > -INFINITY) {
      const float e = expf(l - m);
      s += e;
      s2 = fmaf(e, e, s2);
      sx = fmaf(e, dx, sx);
      sxx = fmaf(e * dx, dx, sxx);
    }
  }
  __device__ __forceinline__ void merge(const CdAcc& o) {
    const float M = fmaxf(m, o.m);
    if (!(M > -INFINITY)) return;
    const float a = (m == -INFINITY) ? 0.0f : expf(m - M);
    const float b = (o.m == -INFINITY) ? 0.0f : expf(o.m - M);
    s = s * a + o.s * b;
    s2 = s2 * a * a + o.s2 * b * b;
    sx = sx * a + o.sx * b;
    sxx = sxx * a + o.sxx * b;
    m = M;
  }
};

struct __align__(16) CdPartial {
  float m, s, s2, sx, sxx;
  int nan, pad[2];
};

struct CdArgs {
  float w1, mu1, s1, mu2, s2, neg_half_inv_r2, log_norm;  // log_norm = -log(2 pi r^2) / 2
  uint32_t comp_threshold;
  const float* y;
  int64_t n, N;
  uint64_t seed;
  float* x_out;
  float* lw_out;
  CdPartial* parts;
  WsHeader* hdr;
  ppl_customdist_result* res;
};

__global__ void __launch_bounds__(kTpb) customdist_kernel(CdArgs a) {
  __shared__ float sy[kCdData];
  __shared__ float red[kTpb / 32];
  __shared__ CdAcc wacc[kTpb / 32];
  __shared__ int nan_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_sm = a.n < kCdData ? a.n : kCdData;
  float ysum = 0.0f;
  for (int64_t j = tid; j < a.n; j += kTpb) {
    const float v = a.y[j];
    if (j < n_sm) sy[j] = v;
    ysum += v;
  }
  ysum = warp_sum(ysum);
  if (lane == 0) red[warp] = ysum;
  if (tid == 0) nan_sh = 0;
  __syncthreads();
  float ybar = 0.0f;
  if (a.n > 0) {
    float t = 0.0f;
    for (int w = 0; w < kTpb / 32; ++w) t += red[w];
    ybar = t / (float)a.n;  // only a shift of the moments: any value is exact in the end
  }
  CdAcc acc;
  acc.init();
  int nan = 0;
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + tid; i < a.N; i += stride) {
    const uint4 w = philox_block(a.seed, (uint32_t)i, 0, 0, kPolyTrace, 0);
    float z0, z1;
    box_muller(w.y, w.z, z0, z1);
    const bool first = (w.x >> 9) < a.comp_threshold;
    const float x = first ? fmaf(a.s1, z0, a.mu1) : fmaf(a.s2, z0, a.mu2);
    float ss = 0.0f;
    for (int64_t j = 0; j < a.n; ++j) {
      const float d = (j < n_sm ? sy[j] : a.y[j]) - x;
      ss = fmaf(d, d, ss);
    }
    const float lw = fmaf(ss, a.neg_half_inv_r2, (float)a.n * a.log_norm);
    if (a.x_out) a.x_out[i] = x;
    if (a.lw_out) a.lw_out[i] = lw;
    nan |= lw != lw;
    acc.add(lw, x - ybar);
  }
  // block merge: warps by shuffles, then warp 0 over the warps
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    CdAcc b;
    b.m = __shfl_xor_sync(0xffffffffu, acc.m, o);
    b.s = __shfl_xor_sync(0xffffffffu, acc.s, o);
    b.s2 = __shfl_xor_sync(0xffffffffu, acc.s2, o);
    b.sx = __shfl_xor_sync(0xffffffffu, acc.sx, o);
    b.sxx = __shfl_xor_sync(0xffffffffu, acc.sxx, o);
    acc.merge(b);
  }
  nan = __any_sync(0xffffffffu, nan);
  if (lane == 0) {
    wacc[warp] = acc;
    if (nan) nan_sh = 1;
  }
  __syncthreads();
  if (tid == 0) {
    CdAcc t = wacc[0];
    for (int w = 1; w < kTpb / 32; ++w) t.merge(wacc[w]);
    CdPartial p;
    p.m = t.m;
    p.s = t.s;
    p.s2 = t.s2;
    p.sx = t.sx;
    p.sxx = t.sxx;
    p.nan = nan_sh;
    p.pad[0] = p.pad[1] = 0;
    a.parts[blockIdx.x] = p;
  }
  if (!elect_last_block(&a.hdr->ticket[0])) return;
  if (tid != 0) return;
  double M = -INFINITY;
  int any_nan = 0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    const CdPartial p = a.parts[b];
    if (p.m > M) M = p.m;
    any_nan |= p.nan;
  }
  double S = 0.0, S2 = 0.0, SX = 0.0, SXX = 0.0;
  if (M > -INFINITY)
    for (unsigned b = 0; b < gridDim.x; ++b) {
      const CdPartial p = a.parts[b];
      if (p.m == -INFINITY) continue;
      const double e = exp((double)p.m - M);
      S += p.s * e;
      S2 += p.s2 * e * e;
      SX += p.sx * e;
      SXX += p.sxx * e;
    }
  ppl_customdist_result r;
  r.n_particles = a.N;
  r.max_lw = M;
  r.status = 0;
  r.pad = 0;
  if (any_nan) {
    record_status(&a.hdr->status, PPL_ENAN);
    r.status = PPL_ENAN;
  } else if (!(S > 0.0)) {
    record_status(&a.hdr->status, PPL_EEMPTY);
    r.status = PPL_EEMPTY;
  }
  r.lse = M + log(S);
  r.log_z = r.lse - log((double)a.N);
  r.ess = S * S / S2;
  const double mx = SX / S;
  r.mean_x = (double)ybar + mx;
  r.var_x = SXX / S - mx * mx;
  *a.res = r;
}

cudaError_t launch_customdist(const ppl_customdist_model& m, uint32_t comp_threshold,
                              const float* y, int64_t n, int64_t N, uint64_t seed, float* x_out,
                              float* lw_out, void* parts, WsHeader* hdr,
                              ppl_customdist_result* res, cudaStream_t s) {
  CdArgs a;
  a.w1 = m.w1;
  a.mu1 = m.mu1;
  a.s1 = m.sigma1;
  a.mu2 = m.mu2;
  a.s2 = m.sigma2;
  const double r2 = (double)m.obs_sigma * (double)m.obs_sigma;
  a.neg_half_inv_r2 = (float)(-1.0 / (2.0 * r2));
  a.log_norm = (float)(-0.5 * log(2.0 * 3.14159265358979323846 * r2));
  a.comp_threshold = comp_threshold;
  a.y = y;
  a.n = n;
  a.N = N;
  a.seed = seed;
  a.x_out = x_out;
  a.lw_out = lw_out;
  a.parts = reinterpret_cast<CdPartial*>(parts);
  a.hdr = hdr;
  a.res = res;
  customdist_kernel<<<stream_grid(N), kTpb, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ppl
