// Likelihood weighting (§3.6.2) on the paper's tiny discrete benchmarks
// (Table 1 of §5.1): biasedcoin, binomial and a truncated geometric.  Every
// `sample` draws one Philox word, in program order, from blocks 0, 1, ... of
// the counter (particle, instance 0, step 0, POLY_TRACE); `factor` terms are
// the log-probabilities of the observations.
//
//   biasedcoin: theta = a / 10, a ~ uniform-discrete(1, 9); observe every flip
//               of `data` as bernoulli(theta); return theta.
//   binomial:   k = number of successes among `limit` bernoulli(0.3) samples.
//   geometric:  c = failures of bernoulli(0.5) samples before the first
//               success, at most `limit` samples; a path that reaches the
//               limit lies outside the truncated support (weight 0).
//
// A particle's log-weight is a function of its return value alone, so the
// kernel counts particles per value (integer, exact, order-free) and the
// normalised distribution, evidence and ESS follow from the counts in FP64.
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

struct DiscreteArgs {
  int32_t model;
  const int32_t* data;
  int64_t n_data, N;
  int32_t limit;
  uint64_t seed;
  uint32_t bern_threshold;  // u01(w) < p  <=>  (w >> 9) < threshold
  int32_t n_values;
  int32_t* codes_out;
  float* lw_out;
  unsigned long long* counts;  // [n_values]
  WsHeader* hdr;
  ppl_discrete_result* res;
};

__device__ __forceinline__ uint32_t draw_word(uint64_t seed, uint32_t i, int idx, uint4& blk,
                                              int& blk_id) {
  if ((idx >> 2) != blk_id) {
    blk_id = idx >> 2;
    blk = philox_block(seed, i, 0, 0, kPolyTrace, (uint32_t)blk_id);
  }
  switch (idx & 3) {
    case 0: return blk.x;
    case 1: return blk.y;
    case 2: return blk.z;
    default: return blk.w;
  }
}

// log-weight of a return code: the factor terms of its path
__device__ __forceinline__ float code_lw(int model, int code, int heads, int tails, int limit) {
  if (model == PPL_DISCRETE_BIASEDCOIN) {
    const float theta = (float)(code + 1) / 10.0f;
    return (float)heads * logf(theta) + (float)tails * logf(1.0f - theta);
  }
  if (model == PPL_DISCRETE_GEOMETRIC) return code >= limit ? -INFINITY : 0.0f;
  return 0.0f;
}

__global__ void __launch_bounds__(kTpb) discrete_is_kernel(DiscreteArgs a) {
  __shared__ unsigned int bins[PPL_DISCRETE_MAX_VALUES];
  __shared__ int ht[2];
  const int tid = threadIdx.x;
  for (int v = tid; v < PPL_DISCRETE_MAX_VALUES; v += kTpb) bins[v] = 0;
  if (tid < 2) ht[tid] = 0;
  __syncthreads();
  const int limit = a.limit;
  int heads = 0, tails = 0;
  if (a.model == PPL_DISCRETE_BIASEDCOIN) {  // the same branch for the whole block
    int h = 0, n = 0;
    for (int64_t f = tid; f < a.n_data; f += kTpb) {
      h += a.data[f] != 0;
      ++n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      h += __shfl_xor_sync(0xffffffffu, h, o);
      n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(&ht[0], h);
      atomicAdd(&ht[1], n - h);
    }
    __syncthreads();
    heads = ht[0];
    tails = ht[1];
  }
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + tid; i < a.N; i += stride) {
    uint4 blk = make_uint4(0, 0, 0, 0);
    int blk_id = -1;
    int code = 0;
    if (a.model == PPL_DISCRETE_BIASEDCOIN) {
      code = uniform_discrete(draw_word(a.seed, (uint32_t)i, 0, blk, blk_id), 1, 9) - 1;
    } else if (a.model == PPL_DISCRETE_BINOMIAL) {
      for (int t = 0; t < limit; ++t)
        code += (draw_word(a.seed, (uint32_t)i, t, blk, blk_id) >> 9) < a.bern_threshold;
    } else {
      while (code < limit && !((draw_word(a.seed, (uint32_t)i, code, blk, blk_id) >> 9) <
                               a.bern_threshold))
        ++code;
    }
    if (a.codes_out) a.codes_out[i] = code;
    if (a.lw_out) a.lw_out[i] = code_lw(a.model, code, heads, tails, limit);
    // one shared atomic per distinct code in the warp
    const unsigned peers = __match_any_sync(__activemask(), code);
    if ((tid & 31) == __ffs(peers) - 1) atomicAdd(&bins[code], (unsigned)__popc(peers));
  }
  __syncthreads();
  for (int v = tid; v < a.n_values; v += kTpb)
    if (bins[v]) atomicAdd(a.counts + v, (unsigned long long)bins[v]);
  if (!elect_last_block(&a.hdr->ticket[0])) return;
  if (tid != 0) return;
  // the normalised distribution of the return value, from the counts
  ppl_discrete_result r;
  memset(&r, 0, sizeof(r));
  double lwv[PPL_DISCRETE_MAX_VALUES];
  double M = -INFINITY;
  for (int v = 0; v < a.n_values; ++v) {
    const unsigned long long c = __ldcg(a.counts + v);
    r.count[v] = (int64_t)c;
    if (a.model == PPL_DISCRETE_BIASEDCOIN) {
      const double theta = (v + 1) / 10.0;
      lwv[v] = heads * log(theta) + tails * log(1.0 - theta);
      r.value[v] = theta;
    } else {
      lwv[v] = (a.model == PPL_DISCRETE_GEOMETRIC && v >= limit) ? -INFINITY : 0.0;
      r.value[v] = v;
    }
    if (c && lwv[v] > M) M = lwv[v];
  }
  double s = 0.0, s2 = 0.0;
  for (int v = 0; v < a.n_values; ++v)
    if (r.count[v] && lwv[v] > -INFINITY) {
      const double e = exp(lwv[v] - M);
      s += (double)r.count[v] * e;
      s2 += (double)r.count[v] * e * e;
    }
  r.n_particles = a.N;
  r.n_values = a.n_values;
  if (!(s > 0.0)) {
    record_status(&a.hdr->status, PPL_EEMPTY);
    r.status = PPL_EEMPTY;
    r.log_z = -INFINITY;
  } else {
    r.log_z = M + log(s) - log((double)a.N);
    r.ess = s * s / s2;
    r.max_lw = M;
    for (int v = 0; v < a.n_values; ++v) {
      r.prob[v] = (r.count[v] && lwv[v] > -INFINITY) ? (double)r.count[v] * exp(lwv[v] - M) / s : 0.0;
      r.mean += r.prob[v] * r.value[v];
    }
  }
  *a.res = r;
}

cudaError_t launch_discrete_is(int32_t model, const int32_t* data, int64_t n_data, int32_t limit,
                               int64_t N, uint64_t seed, uint32_t bern_threshold, int32_t n_values,
                               int32_t* codes_out, float* lw_out, void* counts, WsHeader* hdr,
                               ppl_discrete_result* res, cudaStream_t s) {
  DiscreteArgs a;
  a.model = model;
  a.data = data;
  a.n_data = n_data;
  a.limit = limit;
  a.N = N;
  a.seed = seed;
  a.bern_threshold = bern_threshold;
  a.n_values = n_values;
  a.codes_out = codes_out;
  a.lw_out = lw_out;
  a.counts = reinterpret_cast<unsigned long long*>(counts);
  a.hdr = hdr;
  a.res = res;
  cudaError_t e = cudaMemsetAsync(counts, 0, PPL_DISCRETE_MAX_VALUES * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  discrete_is_kernel<<<stream_grid(N), kTpb, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ppl
