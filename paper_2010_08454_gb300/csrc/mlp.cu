// The learned proposal's network: forward simulation of training pairs from
// the line-fitting model (Fig. 1), the features of a data set, the BF16
// tensor-core MLP (FP32 accumulation), the loss -log q(n, c | data) and its
// gradient, backpropagation and Adam (FP32 master weights).  The proposal is
// the inference-compilation construction (Le, Baydin and Wood, AISTATS 2017);
// importance weights correct it to the posterior (§3.6.2).
//
// Network and proposal (identical to the definitions the oracle restates):
//   in[64]  = the 32 points sorted by x (ties by position): (x, y / 10), BF16
//   h1 = relu(W1 in + b1), h2 = relu(W2 h1 + b2) (BF16), out = W3 h2 + b3 (FP32)
//   q(k) = softmax(out[0..n_deg))_k; for coefficient j of degree slot k:
//   mu = prior_sigma out[4 + 2 (base_k + j)], s = prior_sigma exp(t),
//   t = clamp(out[5 + 2 (base_k + j)], -9, 1).
#include <cuda_bf16.h>

#include "kernels.h"
#include "poly.cuh"
#include "rng.cuh"

namespace ppl {

constexpr int kIn = 64, kHid = 256, kOut = 48, kPts = 32;
// parameter buffer layout (FP32): W1 | b1 | W2 | b2 | W3 | b3
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
                 kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid,
                 kOffB3 = kOffW3 + kOut * kHid, kNumParams = kOffB3 + kOut;

// ---------------------------------------------------------------------------
// Features: one warp per data set; lane l holds point l; bitonic sort by
// (x, original position) with shuffles; lane l writes features 2l, 2l + 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_features(float x, float y, int lane, __nv_bfloat16* feat) {
  int idx = lane;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const float ox = __shfl_xor_sync(0xffffffffu, x, j);
      const float oy = __shfl_xor_sync(0xffffffffu, y, j);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, j);
      const bool other_smaller = (ox < x) || (ox == x && oi < idx);
      const bool ascending = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool take = (lower == ascending) ? other_smaller : !other_smaller;
      if (take) {
        x = ox;
        y = oy;
        idx = oi;
      }
    }
  }
  feat[2 * lane] = __float2bfloat16_rn(x);
  feat[2 * lane + 1] = __float2bfloat16_rn(__fdiv_rn(y, 10.0f));
}

__global__ void __launch_bounds__(kTpb) features_kernel(const float* __restrict__ x,
                                                        const float* __restrict__ y,
                                                        int32_t n_sets,
                                                        __nv_bfloat16* __restrict__ feat) {
  const int warp = (blockIdx.x * kTpb + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_sets) return;
  warp_features(x[(int64_t)warp * kPts + lane], y[(int64_t)warp * kPts + lane], lane,
                feat + (int64_t)warp * kIn);
}

// Training pair p (purpose FORWARD_SIM, instance 0): blocks 0, 1 draw the trace
// as a prior trace; block 2 + l draws point l: x = 2 u01(w0) - 1 and
// y = f(x) + obs_sigma BoxMuller(w1, w2).z0.
// With `step` (a training run's device step counter, steps done so far) the
// batch is pairs [(step mod steps_per_epoch) B, + B) instead of [pair0, + B),
// so a run of training steps needs no value from the host.
__global__ void __launch_bounds__(kTpb) forward_sim_kernel(PolyParams p, float obs_sigma,
                                                           uint64_t seed, int64_t pair0,
                                                           int32_t B,
                                                           __nv_bfloat16* __restrict__ feat,
                                                           int32_t* __restrict__ n_out,
                                                           float* __restrict__ c_out,
                                                           const int32_t* step = nullptr,
                                                           int64_t steps_per_epoch = 1) {
  const int warp = (blockIdx.x * kTpb + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  if (step) pair0 = ((int64_t)*step % steps_per_epoch) * B;
  const uint32_t pair = (uint32_t)(pair0 + warp);
  const uint4 a = philox_block(seed, pair, 0, 0, kForwardSim, 0);
  const uint4 b = philox_block(seed, pair, 0, 0, kForwardSim, 1);
  float z[kMaxCoef], c[kMaxCoef];
  box_muller(a.x, a.y, z[0], z[1]);
  box_muller(a.z, a.w, z[2], z[3]);
  box_muller(b.x, b.y, z[4], z[5]);
  const int n = uniform_discrete(b.z, p.min_deg, p.min_deg + p.n_deg - 1);
  const int ncoef = n + p.coef_offset;
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) c[k] = (k < ncoef) ? p.prior_sigma * z[k] : 0.0f;
  const uint4 v = philox_block(seed, pair, 0, 0, kForwardSim, 2 + (uint32_t)lane);
  const float xl = __fsub_rn(__fmul_rn(2.0f, u01(v.x)), 1.0f);
  float e0, e1;
  box_muller(v.y, v.z, e0, e1);
  float f = c[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) f = fmaf(f, xl, c[k]);
  const float yl = fmaf(obs_sigma, e0, f);
  warp_features(xl, yl, lane, feat + (int64_t)warp * kIn);
  if (lane == 0) n_out[warp] = n;
  if (lane < kMaxCoef) c_out[(int64_t)warp * kMaxCoef + lane] = c[lane];
}

// ---------------------------------------------------------------------------
// BF16 GEMM on the fifth-generation tensor cores (umma_gemm.cu):
//   C[m, n] = sum_k A(m, k) B(n, k)  (+ bias[n]) (relu) (* [mask(m, n) > 0])
// A(m, k) = A[m * sam + k * sak], B(n, k) = B[n * sbn + k * sbk]: any layout,
// so the backward products read transposed operands in place.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const __nv_bfloat16* A;
  int64_t sam, sak;
  const __nv_bfloat16* B;
  int64_t sbn, sbk;
  int M, N, K;
  const float* bias;
  const __nv_bfloat16* mask;  // [M x N] row-major, multiply by (mask > 0)
  int relu;
  float* Cf;           // FP32 output [M x N] (ldc = N), optional
  __nv_bfloat16* Cb;   // BF16 output [M x N], optional
};

// Split-K scratch of the network's products: the largest product (256 x
// 256) in up to 16 K slices.
constexpr size_t kSplitFloats = (size_t)16 * 256 * 256;

static cudaError_t gemm(const GemmArgs& g, int32_t* status, cudaStream_t s, float* split = nullptr) {
  return launch_umma_gemm(g.A, g.sam, g.sak, g.B, g.sbn, g.sbk, g.M, g.N, g.K, g.bias, g.mask,
                          g.relu, g.Cf, g.Cb, status, s, split, split ? kSplitFloats : 0);
}

// ---------------------------------------------------------------------------
// Loss -log q per pair and its gradient with respect to the outputs (divided
// by the batch size), one thread per pair; per-block loss sums.
// ---------------------------------------------------------------------------
struct ProposalShape {
  int min_deg, n_deg, coef_offset;
  float prior_sigma, log_prior_sigma;
};

__device__ __forceinline__ int slot_base(const ProposalShape& q, int k) {
  int b = 0;
  for (int kk = 0; kk < k; ++kk) b += q.min_deg + kk + q.coef_offset;
  return b;
}

__global__ void __launch_bounds__(kTpb) loss_grad_kernel(ProposalShape q,
                                                         const float* __restrict__ out,
                                                         const int32_t* __restrict__ n_t,
                                                         const float* __restrict__ c_t, int32_t B,
                                                         float* __restrict__ dout,
                                                         __nv_bfloat16* __restrict__ dout_b,
                                                         double* loss_sum) {
  const int b = blockIdx.x * kTpb + threadIdx.x;
  float loss = 0.0f;
  if (b < B) {
    const float* o = out + (int64_t)b * kOut;
    float g[kOut];
#pragma unroll
    for (int i = 0; i < kOut; ++i) g[i] = 0.0f;
    const int k = n_t[b] - q.min_deg;
    float mx = -INFINITY;
    for (int i = 0; i < q.n_deg; ++i) mx = fmaxf(mx, o[i]);
    float se = 0.0f;
    for (int i = 0; i < q.n_deg; ++i) se += expf(o[i] - mx);
    loss = -(o[k] - mx - logf(se));
    for (int i = 0; i < q.n_deg; ++i) g[i] = expf(o[i] - mx) / se - (i == k ? 1.0f : 0.0f);
    const int ncoef = n_t[b] + q.coef_offset, base = slot_base(q, k);
    for (int j = 0; j < ncoef; ++j) {
      const float om = o[4 + 2 * (base + j)], os = o[5 + 2 * (base + j)];
      const float t = fminf(fmaxf(os, -9.0f), 1.0f);
      const float mu = q.prior_sigma * om, sd = q.prior_sigma * expf(t);
      const float z = (c_t[(int64_t)b * kMaxCoef + j] - mu) / sd;
      loss += 0.91893853320467274f + q.log_prior_sigma + t + 0.5f * z * z;
      g[4 + 2 * (base + j)] = -z / sd * q.prior_sigma;
      g[5 + 2 * (base + j)] = (os > -9.0f && os < 1.0f) ? (1.0f - z * z) : 0.0f;
    }
    const float inv = 1.0f / (float)B;
#pragma unroll
    for (int i = 0; i < kOut; ++i) {
      dout[(int64_t)b * kOut + i] = g[i] * inv;
      dout_b[(int64_t)b * kOut + i] = __float2bfloat16_rn(g[i] * inv);
    }
  }
  loss = warp_sum(loss);
  __shared__ float red[kTpb / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < kTpb / 32; ++w) s += red[w];
    atomicAdd(loss_sum, (double)s);
  }
}

// db[n] = sum over rows of d[m, n] (FP32 or BF16 rows), one thread per column.
template <typename T>
__global__ void colsum_kernel(const T* __restrict__ d, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; ++m) {
    if constexpr (sizeof(T) == 2) s += __bfloat162float(d[(int64_t)m * N + n]);
    else s += d[(int64_t)m * N + n];
  }
  db[n] = s;
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters; refreshes the BF16
// copy of the weights.  step = 1, 2, ... for the bias corrections.
__global__ void __launch_bounds__(kTpb) adam_kernel(float* __restrict__ p,
                                                    const float* __restrict__ g,
                                                    float* __restrict__ m, float* __restrict__ v,
                                                    __nv_bfloat16* __restrict__ pb, int64_t n,
                                                    float lr, float b1, float b2, float eps,
                                                    const int32_t* step) {
  const int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x;
  if (i >= n) return;
  const float t = (float)(*step);
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(b1, t)), vh = vi / (1.0f - powf(b2, t));
  const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb,
                               int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// The step counter advances; the step's summed loss goes to loss_out[step - 1].
__global__ void bump_kernel(int32_t* step, const double* loss, double* loss_out) {
  const int32_t s = *step + 1;
  *step = s;
  if (loss_out) loss_out[s - 1] = *loss;
}

// ---------------------------------------------------------------------------
// Workspace of the network for a batch of B rows.
// ---------------------------------------------------------------------------
struct MlpWs {
  int32_t* status;  // first word: a tensor-core wait that ran out (ppl_workspace_status)
  __nv_bfloat16 *pb, *feat, *h1, *h2, *dout_b, *dh2, *dh1;
  float *out, *dout, *grad;
  int32_t* n_t;
  float* c_t;
  double* loss;
  int32_t* step;
  float* split;  // split-K slices of the products
  size_t total;
};

static size_t a256(size_t v) { return (v + 255) / 256 * 256; }

static MlpWs mlp_ws(char* base, int64_t B) {
  MlpWs w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += a256(bytes);
    return p;
  };
  w.status = (int32_t*)take(sizeof(int32_t));
  w.step = (int32_t*)take(sizeof(int32_t));
  w.loss = (double*)take(sizeof(double) * 2);
  w.pb = (__nv_bfloat16*)take(kNumParams * 2);
  w.grad = (float*)take(kNumParams * 4);
  w.feat = (__nv_bfloat16*)take(B * kIn * 2);
  w.h1 = (__nv_bfloat16*)take(B * kHid * 2);
  w.h2 = (__nv_bfloat16*)take(B * kHid * 2);
  w.out = (float*)take(B * kOut * 4);
  w.dout = (float*)take(B * kOut * 4);
  w.dout_b = (__nv_bfloat16*)take(B * kOut * 2);
  w.dh2 = (__nv_bfloat16*)take(B * kHid * 2);
  w.dh1 = (__nv_bfloat16*)take(B * kHid * 2);
  w.n_t = (int32_t*)take(B * 4);
  w.c_t = (float*)take(B * kMaxCoef * 4);
  w.split = (float*)take(kSplitFloats * 4);
  w.total = off;
  return w;
}

static cudaError_t mlp_forward(const float* params, const MlpWs& w, int B, cudaStream_t s) {
  GemmArgs g{};
  g.A = w.feat; g.sam = kIn; g.sak = 1;
  g.B = w.pb + kOffW1; g.sbn = kIn; g.sbk = 1;
  g.M = B; g.N = kHid; g.K = kIn; g.bias = params + kOffB1; g.relu = 1; g.Cb = w.h1;
  cudaError_t e = gemm(g, w.status, s, w.split);
  if (e != cudaSuccess) return e;
  g = GemmArgs{};
  g.A = w.h1; g.sam = kHid; g.sak = 1;
  g.B = w.pb + kOffW2; g.sbn = kHid; g.sbk = 1;
  g.M = B; g.N = kHid; g.K = kHid; g.bias = params + kOffB2; g.relu = 1; g.Cb = w.h2;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  g = GemmArgs{};
  g.A = w.h2; g.sam = kHid; g.sak = 1;
  g.B = w.pb + kOffW3; g.sbn = kHid; g.sbk = 1;
  g.M = B; g.N = kOut; g.K = kHid; g.bias = params + kOffB3; g.Cf = w.out;
  return gemm(g, w.status, s, w.split);
}

// Gradient of the mean loss over the batch into w.grad (FP32), loss sum into w.loss[0].
static cudaError_t mlp_backward(const ProposalShape& q, const MlpWs& w, int B, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  loss_grad_kernel<<<(B + kTpb - 1) / kTpb, kTpb, 0, s>>>(q, w.out, w.n_t, w.c_t, B, w.dout,
                                                         w.dout_b, w.loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  GemmArgs g{};
  // dW3[o, i] = sum_b dout[b, o] h2[b, i]
  g.A = w.dout_b; g.sam = 1; g.sak = kOut;
  g.B = w.h2; g.sbn = 1; g.sbk = kHid;
  g.M = kOut; g.N = kHid; g.K = B; g.Cf = w.grad + kOffW3;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  colsum_kernel<float><<<1, 64, 0, s>>>(w.dout, B, kOut, w.grad + kOffB3);
  // dh2[b, i] = sum_o dout[b, o] W3[o, i], masked by h2 > 0
  g = GemmArgs{};
  g.A = w.dout_b; g.sam = kOut; g.sak = 1;
  g.B = w.pb + kOffW3; g.sbn = 1; g.sbk = kHid;
  g.M = B; g.N = kHid; g.K = kOut; g.mask = w.h2; g.Cb = w.dh2;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  // dW2[o, i] = sum_b dh2[b, o] h1[b, i]
  g = GemmArgs{};
  g.A = w.dh2; g.sam = 1; g.sak = kHid;
  g.B = w.h1; g.sbn = 1; g.sbk = kHid;
  g.M = kHid; g.N = kHid; g.K = B; g.Cf = w.grad + kOffW2;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  colsum_kernel<__nv_bfloat16><<<1, kHid, 0, s>>>(w.dh2, B, kHid, w.grad + kOffB2);
  // dh1 = (dh2 W2) masked by h1 > 0
  g = GemmArgs{};
  g.A = w.dh2; g.sam = kHid; g.sak = 1;
  g.B = w.pb + kOffW2; g.sbn = 1; g.sbk = kHid;
  g.M = B; g.N = kHid; g.K = kHid; g.mask = w.h1; g.Cb = w.dh1;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  // dW1[o, i] = sum_b dh1[b, o] feat[b, i]
  g = GemmArgs{};
  g.A = w.dh1; g.sam = 1; g.sak = kHid;
  g.B = w.feat; g.sbn = 1; g.sbk = kIn;
  g.M = kHid; g.N = kIn; g.K = B; g.Cf = w.grad + kOffW1;
  if ((e = gemm(g, w.status, s, w.split)) != cudaSuccess) return e;
  colsum_kernel<__nv_bfloat16><<<1, kHid, 0, s>>>(w.dh1, B, kHid, w.grad + kOffB1);
  return cudaGetLastError();
}

static ProposalShape shape_of(const PolyParams& p, float prior_sigma) {
  ProposalShape q;
  q.min_deg = p.min_deg;
  q.n_deg = p.n_deg;
  q.coef_offset = p.coef_offset;
  q.prior_sigma = prior_sigma;
  q.log_prior_sigma = logf(prior_sigma);
  return q;
}

}  // namespace ppl

using namespace ppl;

namespace {

ppl_status mlp_model(const ppl_model* m, PolyParams* p) {
  if (!m || m->id != PPL_MODEL_POLY) return PPL_EINVAL;
  const int n_deg = m->max_deg - m->min_deg + 1;
  if (m->min_deg < 0 || n_deg < 1 || n_deg > kMaxDegrees || m->coef_offset < 0 ||
      m->max_deg + m->coef_offset > kMaxCoef || !(m->obs_sigma > 0.0f) ||
      !(m->prior_sigma > 0.0f))
    return PPL_EINVAL;
  // the 48 outputs hold 4 logits and (mu, log s) for at most 22 coefficient slots
  int slots = 0;
  for (int k = 0; k < n_deg; ++k) slots += m->min_deg + k + m->coef_offset;
  if (4 + 2 * slots > kOut) return PPL_EINVAL;
  p->min_deg = m->min_deg;
  p->n_deg = n_deg;
  p->coef_offset = m->coef_offset;
  p->prior_sigma = m->prior_sigma;
  p->neg_half_inv_var = (float)(-1.0 / (2.0 * (double)m->obs_sigma * (double)m->obs_sigma));
  return PPL_OK;
}

inline ppl_status st(cudaError_t e) { return e == cudaSuccess ? PPL_OK : PPL_ECUDA; }

}  // namespace

extern "C" {

int64_t ppl_proposal_num_params(void) { return (int64_t)kNumParams; }

size_t ppl_proposal_workspace_size(int32_t batch) {
  if (batch < 1) return 0;
  return mlp_ws(nullptr, batch).total;
}

ppl_status ppl_proposal_forward(const ppl_model* model, const float* params, const float* x,
                                const float* y, int32_t n_sets, float* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream) {
  PolyParams p;
  if (mlp_model(model, &p) != PPL_OK || !params || !x || !y || !out_dev || n_sets < 1 || !ws)
    return PPL_EINVAL;
  MlpWs w = mlp_ws(static_cast<char*>(ws), n_sets);
  if (ws_bytes < w.total) return PPL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(w.status, 0, sizeof(int32_t), s) != cudaSuccess) return PPL_ECUDA;
  to_bf16_kernel<<<(unsigned)((kNumParams + kTpb - 1) / kTpb), kTpb, 0, s>>>(params, w.pb,
                                                                            kNumParams);
  features_kernel<<<(unsigned)(((int64_t)n_sets * 32 + kTpb - 1) / kTpb), kTpb, 0, s>>>(
      x, y, n_sets, w.feat);
  w.out = out_dev;
  return st(mlp_forward(params, w, n_sets, s));
}

ppl_status ppl_proposal_features(const float* x, const float* y, int32_t n_sets, void* feat_dev,
                                 ppl_stream stream) {
  if (!x || !y || !feat_dev || n_sets < 1) return PPL_EINVAL;
  features_kernel<<<(unsigned)(((int64_t)n_sets * 32 + kTpb - 1) / kTpb), kTpb, 0,
                    (cudaStream_t)stream>>>(x, y, n_sets,
                                            static_cast<__nv_bfloat16*>(feat_dev));
  return st(cudaGetLastError());
}

ppl_status ppl_proposal_grad(const ppl_model* model, const float* params, int64_t pair0,
                             int32_t batch, uint64_t seed, float* grad_out, double* loss_out,
                             void* ws, size_t ws_bytes, ppl_stream stream) {
  PolyParams p;
  if (mlp_model(model, &p) != PPL_OK || !params || !grad_out || !loss_out || batch < 1 || !ws ||
      pair0 < 0 || pair0 + batch > 0xffffffffll)
    return PPL_EINVAL;
  MlpWs w = mlp_ws(static_cast<char*>(ws), batch);
  if (ws_bytes < w.total) return PPL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(w.status, 0, sizeof(int32_t), s) != cudaSuccess) return PPL_ECUDA;
  to_bf16_kernel<<<(unsigned)((kNumParams + kTpb - 1) / kTpb), kTpb, 0, s>>>(params, w.pb,
                                                                            kNumParams);
  forward_sim_kernel<<<(unsigned)(((int64_t)batch * 32 + kTpb - 1) / kTpb), kTpb, 0, s>>>(
      p, model->obs_sigma, seed, pair0, batch, w.feat, w.n_t, w.c_t);
  ppl_status r = st(mlp_forward(params, w, batch, s));
  if (r != PPL_OK) return r;
  r = st(mlp_backward(shape_of(p, model->prior_sigma), w, batch, s));
  if (r != PPL_OK) return r;
  if (cudaMemcpyAsync(grad_out, w.grad, kNumParams * sizeof(float), cudaMemcpyDeviceToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(loss_out, w.loss, sizeof(double), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return PPL_ECUDA;
  return PPL_OK;
}

ppl_status ppl_proposal_train_init(const float* params, int32_t batch, void* ws,
                                   size_t ws_bytes, ppl_stream stream) {
  if (!params || batch < 1 || !ws) return PPL_EINVAL;
  MlpWs w = mlp_ws(static_cast<char*>(ws), batch);
  if (ws_bytes < w.total) return PPL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(w.status, 0, sizeof(int32_t), s) != cudaSuccess ||
      cudaMemsetAsync(w.step, 0, sizeof(int32_t), s) != cudaSuccess)
    return PPL_ECUDA;
  to_bf16_kernel<<<(unsigned)((kNumParams + kTpb - 1) / kTpb), kTpb, 0, s>>>(params, w.pb,
                                                                            kNumParams);
  return st(cudaGetLastError());
}

ppl_status ppl_proposal_train_steps(const ppl_model* model, float* params, float* adam_m,
                                    float* adam_v, int64_t n_pairs, int32_t batch,
                                    int32_t n_steps, uint64_t seed, float lr,
                                    double* loss_per_step, void* ws, size_t ws_bytes,
                                    ppl_stream stream) {
  PolyParams p;
  if (mlp_model(model, &p) != PPL_OK || !params || !adam_m || !adam_v || batch < 1 ||
      n_pairs < batch || n_steps < 0 || !ws || !(lr > 0.0f) || n_pairs > 0xffffffffll)
    return PPL_EINVAL;
  MlpWs w = mlp_ws(static_cast<char*>(ws), batch);
  if (ws_bytes < w.total) return PPL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const ProposalShape q = shape_of(p, model->prior_sigma);
  const int64_t steps_per_epoch = n_pairs / batch;
  for (int32_t it = 0; it < n_steps; ++it) {
    forward_sim_kernel<<<(unsigned)(((int64_t)batch * 32 + kTpb - 1) / kTpb), kTpb, 0, s>>>(
        p, model->obs_sigma, seed, 0, batch, w.feat, w.n_t, w.c_t, w.step, steps_per_epoch);
    ppl_status r = st(mlp_forward(params, w, batch, s));
    if (r != PPL_OK) return r;
    r = st(mlp_backward(q, w, batch, s));
    if (r != PPL_OK) return r;
    bump_kernel<<<1, 1, 0, s>>>(w.step, w.loss, loss_per_step);
    adam_kernel<<<(unsigned)((kNumParams + kTpb - 1) / kTpb), kTpb, 0, s>>>(
        params, w.grad, adam_m, adam_v, w.pb, kNumParams, lr, 0.9f, 0.999f, 1e-8f, w.step);
  }
  return st(cudaGetLastError());
}

ppl_status ppl_proposal_train(const ppl_model* model, float* params, float* adam_m,
                              float* adam_v, int64_t n_pairs, int32_t batch, int32_t epochs,
                              uint64_t seed, float lr, double* loss_per_step, void* ws,
                              size_t ws_bytes, ppl_stream stream) {
  if (epochs < 1 || batch < 1 || n_pairs < batch) return PPL_EINVAL;
  const int64_t steps = (int64_t)epochs * (n_pairs / batch);
  if (steps > 0x7fffffffll) return PPL_EINVAL;
  ppl_status r = ppl_proposal_train_init(params, batch, ws, ws_bytes, stream);
  if (r != PPL_OK) return r;
  return ppl_proposal_train_steps(model, params, adam_m, adam_v, n_pairs, batch, (int32_t)steps,
                                  seed, lr, loss_per_step, ws, ws_bytes, stream);
}

}  // extern "C"
