// Likelihood weighting on the line-fitting model: the trace kernel (§3.6.2 run
// the model N times; Fig. 1 the model), the statistics pass (log-sum-exp
// normalisation and ESS), and the posterior pass (degree masses, weighted
// coefficient means and variances, the mode).
#include "kernels.h"
#include "poly.cuh"
#include "stats.cuh"

namespace ppl {

// ---------------------------------------------------------------------------
// Trace kernel: every thread runs PPT traces per group; the data set streams
// through shared memory in chunks; the log-weight is the factor
// -sum_l (y_l - f(x_l))^2 / (2 sigma^2) with f evaluated by Horner's rule in
// FP32 FMAs.  The statistics pass is fused: each block leaves a partial and
// the last block merges them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
  const float y = __fsub_rn(v, comp);
  const float t = __fadd_rn(sum, y);
  comp = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

template <int PPT>
__global__ void __launch_bounds__(kTpb) poly_trace_kernel(
    PolyParams p, const float* __restrict__ xs, const float* __restrict__ ys, int64_t L,
    int64_t N, uint64_t seed, uint32_t instance, int chunk, float* __restrict__ lw_out,
    ppl_poly_particle* __restrict__ rec_out, WsHeader* hdr, StatPartial* parts,
    ppl_is_result* res) {
  extern __shared__ float2 sdata[];
  const int64_t group = (int64_t)kTpb * PPT;
  const int64_t n_groups = (N + group - 1) / group;
  const int n_chunks = (int)((L + chunk - 1) / chunk);
  const int tid = threadIdx.x;

  if (n_chunks == 1) {
    for (int l = tid; l < L; l += kTpb) sdata[l] = make_float2(xs[l], ys[l]);
    __syncthreads();
  }

  StatAcc acc;
  acc.init();
  for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
    float c[PPT][kMaxCoef];
    float ss[PPT], comp[PPT];  // compensated (Kahan) sum of the 16-point partial sums
    int n[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int64_t i = g * group + (int64_t)q * kTpb + tid;
      n[q] = poly_draw(p, seed, instance, (uint32_t)(i < N ? i : 0), c[q]);
      ss[q] = 0.0f;
      comp[q] = 0.0f;
    }
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int64_t l0 = (int64_t)ch * chunk;
      const int len = (int)(L - l0 < (int64_t)chunk ? L - l0 : (int64_t)chunk);
      if (n_chunks > 1) {
        __syncthreads();
        for (int l = tid; l < len; l += kTpb) sdata[l] = make_float2(xs[l0 + l], ys[l0 + l]);
        __syncthreads();
      }
      // Inner sums over 16 points keep the FP32 accumulation error small.
      int l = 0;
      for (; l + 16 <= len; l += 16) {
        float part[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) part[q] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
          const float2 d = sdata[l + j];
#pragma unroll
          for (int q = 0; q < PPT; ++q) {
            float f = c[q][5];
            f = fmaf(f, d.x, c[q][4]);
            f = fmaf(f, d.x, c[q][3]);
            f = fmaf(f, d.x, c[q][2]);
            f = fmaf(f, d.x, c[q][1]);
            f = fmaf(f, d.x, c[q][0]);
            const float r = d.y - f;
            part[q] = fmaf(r, r, part[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q) kahan_add(ss[q], comp[q], part[q]);
      }
      if (l < len) {
        float part[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) part[q] = 0.0f;
        for (; l < len; ++l) {
          const float2 d = sdata[l];
#pragma unroll
          for (int q = 0; q < PPT; ++q) {
            float f = c[q][5];
            f = fmaf(f, d.x, c[q][4]);
            f = fmaf(f, d.x, c[q][3]);
            f = fmaf(f, d.x, c[q][2]);
            f = fmaf(f, d.x, c[q][1]);
            f = fmaf(f, d.x, c[q][0]);
            const float r = d.y - f;
            part[q] = fmaf(r, r, part[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < PPT; ++q) kahan_add(ss[q], comp[q], part[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int64_t i = g * group + (int64_t)q * kTpb + tid;
      if (i < N) {
        const float lw = ss[q] * p.neg_half_inv_var;
        if (lw_out) lw_out[i] = lw;
        if (rec_out) {
          float4* dst = reinterpret_cast<float4*>(rec_out + i);
          dst[0] = make_float4(c[q][0], c[q][1], c[q][2], c[q][3]);
          dst[1] = make_float4(c[q][4], c[q][5], __int_as_float(n[q]),
                               __uint_as_float((uint32_t)i));
        }
        acc.add(lw, (int)i, n[q] - p.min_deg);
      }
    }
  }

  StatAcc r = block_reduce_stat(acc);
  if (tid == 0) to_partial(r, parts + blockIdx.x);
  if (elect_last_block(&hdr->ticket[0])) finalize_stats(parts, gridDim.x, N, &p, hdr, res, nullptr);
}

// ---------------------------------------------------------------------------
// Statistics pass over an existing population: lw (NULL = all 0) and, for the
// per-degree bests, the particles' degrees (NULL = no degrees).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTpb) stats_kernel(const float* __restrict__ lw,
                                                     const ppl_poly_particle* __restrict__ rec,
                                                     int64_t N, PolyParams p, int has_model,
                                                     WsHeader* hdr, StatPartial* parts,
                                                     ppl_is_result* res, double* lse_out) {
  StatAcc acc;
  acc.init();
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x; i < N; i += stride) {
    const float v = lw ? lw[i] : 0.0f;
    const int d = rec ? rec[i].n - p.min_deg : -1;
    acc.add(v, (int)i, d);
  }
  StatAcc r = block_reduce_stat(acc);
  if (threadIdx.x == 0) to_partial(r, parts + blockIdx.x);
  if (elect_last_block(&hdr->ticket[0]))
    finalize_stats(parts, gridDim.x, N, has_model ? &p : nullptr, hdr, res, lse_out);
}

// ---------------------------------------------------------------------------
// Posterior pass: per-degree weighted sums around each degree's best trace,
// then the summary.  FROM_RNG regenerates a particle's draws from its counter
// instead of reading a stored record.
// ---------------------------------------------------------------------------
template <bool FROM_RNG>
__global__ void __launch_bounds__(kTpb) posterior_kernel(
    PolyParams p, const ppl_poly_particle* __restrict__ rec, const float* __restrict__ lw,
    int64_t N, uint64_t seed, uint32_t instance, WsHeader* hdr, PostPartial* parts,
    ppl_is_result* res) {
  __shared__ float ref[kMaxDegrees][kMaxCoef];
  __shared__ float dmax[kMaxDegrees];
  const int tid = threadIdx.x;
  if (tid < kMaxDegrees * kMaxCoef) {
    const int d = tid / kMaxCoef, k = tid % kMaxCoef;
    const int j = hdr->deg_arg[d];
    float v = 0.0f;
    if (j >= 0) {
      if (FROM_RNG) {
        float c[kMaxCoef];
        poly_draw(p, seed, instance, (uint32_t)j, c);
        v = c[k];
      } else {
        v = rec[j].c[k];
      }
    }
    ref[d][k] = v;
  }
  if (tid < kMaxDegrees) dmax[tid] = hdr->deg_max[tid];
  __syncthreads();

  float acc[kMaxDegrees][kPostVals];
#pragma unroll
  for (int d = 0; d < kMaxDegrees; ++d)
#pragma unroll
    for (int v = 0; v < kPostVals; ++v) acc[d][v] = 0.0f;

  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + tid; i < N; i += stride) {
    float c[kMaxCoef];
    int n;
    if (FROM_RNG) {
      n = poly_draw(p, seed, instance, (uint32_t)i, c);
    } else {
      const float4* src = reinterpret_cast<const float4*>(rec + i);
      const float4 a = src[0], b = src[1];
      c[0] = a.x;
      c[1] = a.y;
      c[2] = a.z;
      c[3] = a.w;
      c[4] = b.x;
      c[5] = b.y;
      n = __float_as_int(b.z);
    }
    const int d = n - p.min_deg;
    if ((unsigned)d >= (unsigned)p.n_deg) {
      record_status(&hdr->status, PPL_EINVAL);
      continue;
    }
    const float l = lw ? lw[i] : 0.0f;
    const float w = (l > -INFINITY) ? expf(l - dmax[d]) : 0.0f;
    float dc[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) dc[k] = c[k] - ref[d][k];
#pragma unroll
    for (int dd = 0; dd < kMaxDegrees; ++dd) {
      const float wd = (dd == d) ? w : 0.0f;
      acc[dd][0] += wd;
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) {
        const float t = wd * dc[k];
        acc[dd][1 + k] += t;
        acc[dd][1 + kMaxCoef + k] = fmaf(t, dc[k], acc[dd][1 + kMaxCoef + k]);
      }
    }
  }

  // block reduction of the 52 sums
  __shared__ float red[kTpb / 32][kMaxDegrees * kPostVals];
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int d = 0; d < kMaxDegrees; ++d)
#pragma unroll
    for (int v = 0; v < kPostVals; ++v) {
      float x = warp_sum(acc[d][v]);
      if (lane == 0) red[warp][d * kPostVals + v] = x;
    }
  __syncthreads();
  if (tid < kMaxDegrees * kPostVals) {
    float x = 0.0f;
    for (int w = 0; w < kTpb / 32; ++w) x += red[w][tid];
    parts[blockIdx.x].v[tid / kPostVals][tid % kPostVals] = x;
  }
  if (!elect_last_block(&hdr->ticket[1])) return;

  // last block: sum the partials (FP32 over blocks, one warp per value), then
  // form the summary in FP64
  __shared__ double tot[kMaxDegrees * kPostVals];
  for (int v = warp; v < kMaxDegrees * kPostVals; v += kTpb / 32) {
    float x = 0.0f;
    for (int b = lane; b < (int)gridDim.x; b += 32) x += parts[b].v[v / kPostVals][v % kPostVals];
    x = warp_sum(x);
    if (lane == 0) tot[v] = (double)x;
  }
  __syncthreads();
  if (tid == 0 && res) {
    const double M = (double)hdr->max_lw;
    double mass[kMaxDegrees], total = 0.0;
    bool has[kMaxDegrees];
    for (int d = 0; d < kMaxDegrees; ++d) {
      const double S = tot[d * kPostVals];
      has[d] = d < p.n_deg && hdr->deg_arg[d] >= 0 && S > 0.0;
      mass[d] = has[d] ? exp((double)dmax[d] - M) * S : 0.0;
      total += mass[d];
    }
    int best = 0;
    double mean_c[kMaxCoef] = {0, 0, 0, 0, 0, 0};
    for (int d = 0; d < kMaxDegrees; ++d) {
      const double S = tot[d * kPostVals];
      const double pn = total > 0.0 ? mass[d] / total : 0.0;
      res->p_n[d] = pn;
      if (d < p.n_deg && pn > res->p_n[best]) best = d;
      for (int k = 0; k < kMaxCoef; ++k) {
        double mean = 0.0, var = 0.0;
        if (has[d]) {  // defined even when the degree's global mass underflows
          const double A = tot[d * kPostVals + 1 + k] / S;
          const double B = tot[d * kPostVals + 1 + kMaxCoef + k] / S;
          mean = (double)ref[d][k] + A;
          var = fmax(B - A * A, 0.0);
        }
        res->deg_mean[d][k] = mean;
        res->deg_var[d][k] = var;
        mean_c[k] += pn * mean;
      }
    }
    for (int k = 0; k < kMaxCoef; ++k) res->mean_c[k] = mean_c[k];
    res->map_deg = p.min_deg + best;
    res->status = ld_volatile_i32(&hdr->status);
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static int g_num_sms = 0;

int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

constexpr int kTracePpt = 4;
constexpr int kMaxChunk = 4096;

int trace_grid(int64_t N) {
  const int64_t groups = (N + (int64_t)kTpb * kTracePpt - 1) / ((int64_t)kTpb * kTracePpt);
  const int64_t cap = (int64_t)num_sms() * 4;
  return (int)std::max<int64_t>(1, std::min<int64_t>(groups, std::min<int64_t>(cap, kMaxBlocks)));
}

int stream_grid(int64_t N) {
  const int64_t blocks = (N + kTpb - 1) / kTpb;
  const int64_t cap = (int64_t)num_sms() * 4;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, std::min<int64_t>(cap, kMaxBlocks)));
}

cudaError_t launch_poly_trace(const PolyParams& p, const float* x, const float* y, int64_t L,
                              int64_t N, uint64_t seed, uint32_t instance, float* lw_out,
                              ppl_poly_particle* rec_out, WsHeader* hdr, void* parts,
                              ppl_is_result* res, cudaStream_t s) {
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(L, kMaxChunk));
  const size_t smem = (size_t)chunk * sizeof(float2);
  const int grid = trace_grid(N);
  poly_trace_kernel<kTracePpt><<<grid, kTpb, smem, s>>>(p, x, y, L, N, seed, instance, chunk,
                                                         lw_out, rec_out, hdr,
                                                         (StatPartial*)parts, res);
  return cudaGetLastError();
}

cudaError_t launch_stats(const float* lw, const ppl_poly_particle* rec, int64_t N,
                         const PolyParams* p, WsHeader* hdr, void* parts, ppl_is_result* res,
                         double* lse_out, cudaStream_t s) {
  PolyParams pp = p ? *p : PolyParams{0, 0, 0, 0.f, 0.f};
  stats_kernel<<<stream_grid(N), kTpb, 0, s>>>(lw, rec, N, pp, p != nullptr, hdr,
                                               (StatPartial*)parts, res, lse_out);
  return cudaGetLastError();
}

cudaError_t launch_posterior(const PolyParams& p, const ppl_poly_particle* rec, const float* lw,
                             int64_t N, uint64_t seed, uint32_t instance, WsHeader* hdr,
                             void* parts, ppl_is_result* res, cudaStream_t s) {
  const int grid = stream_grid(N);
  if (rec)
    posterior_kernel<false><<<grid, kTpb, 0, s>>>(p, rec, lw, N, seed, instance, hdr,
                                                  (PostPartial*)parts, res);
  else
    posterior_kernel<true><<<grid, kTpb, 0, s>>>(p, rec, lw, N, seed, instance, hdr,
                                                 (PostPartial*)parts, res);
  return cudaGetLastError();
}

size_t partials_bytes() {
  return (size_t)kMaxBlocks * std::max(sizeof(StatPartial), sizeof(PostPartial));
}

}  // namespace ppl
