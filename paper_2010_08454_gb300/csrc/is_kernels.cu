// Likelihood weighting on the line-fitting model: the trace kernel (§3.6.2 run
// the model N times and normalise the log-weights; Fig. 1 the model) with the
// posterior reduction fused in (degree masses, weighted coefficient means and
// variances, the mode), the statistics pass over given log-weights, and the
// one-pass posterior summary of a given population.
#include "kernels.h"
#include "poly.cuh"
#include "posterior.cuh"
#include "stats.cuh"
#include "trace.cuh"

namespace ppl {

// ---------------------------------------------------------------------------
// Final merge of the per-block partials, by the last block: warp k merges
// degree k's partials (FP32, a lane-strided chain then a shuffle tree); the
// sums S, S2 are recombined in FP64 around the merged maximum; thread 0
// writes the summary.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_partials(const DegPartial* parts, int G, int n_deg,
                                                  int min_deg, int64_t N, WsHeader* hdr,
                                                  ppl_is_result* res) {
  __shared__ DegPartial fin[kMaxDegrees];
  __shared__ double fS[kMaxDegrees], fS2[kMaxDegrees];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < kMaxDegrees) {
    DegPartial a;
    deg_empty(a);
    for (int b = lane; b < G; b += 32) deg_merge(a, parts[b * kMaxDegrees + warp]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DegPartial other = deg_shfl_xor(a, o);
      deg_merge(a, other);
    }
    const float M = a.m;
    double s = 0.0, s2 = 0.0;
    if (M != -INFINITY) {
      for (int b = lane; b < G; b += 32) {
        const DegPartial& q = parts[b * kMaxDegrees + warp];
        if (q.m == -INFINITY) continue;
        const double e = (double)expf(q.m - M);
        s += (double)q.S * e;
        s2 += (double)q.S2 * e * e;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      fin[warp] = a;
      fS[warp] = s;
      fS2[warp] = s2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool any = false;
    for (int k = 0; k < n_deg; ++k) any |= fin[k].m != -INFINITY;
    if (!any) record_status(&hdr->status, PPL_EEMPTY);
    if (res) write_summary(fin, fS, fS2, n_deg, min_deg, N, ld_volatile_i32(&hdr->status), res);
  }
}

// ---------------------------------------------------------------------------
// Trace kernel: a persistent grid; each block runs groups of kTpb * PPT traces
// (trace_group: draw, sort by degree, degree-specialised Horner, per-degree
// partials) and merges the groups' partials into its running partial; the
// last block merges the blocks' partials into the summary.
// ---------------------------------------------------------------------------
template <int PPT>
__global__ void __launch_bounds__(kTpb, 4) poly_trace_kernel(
    PolyParams p, const float* __restrict__ xs, const float* __restrict__ ys, int64_t L,
    int64_t N, uint64_t seed, uint32_t instance, int chunk, float* __restrict__ lw_out,
    ppl_poly_particle* __restrict__ rec_out, WsHeader* hdr, DegPartial* parts,
    ppl_is_result* res, const SuffStat* suff_g) {
  extern __shared__ __align__(16) unsigned char smem[];
  TraceSmem<PPT>& ts = *reinterpret_cast<TraceSmem<PPT>*>(smem);
  float2* sdata = reinterpret_cast<float2*>(smem + trace_smem_bytes<PPT>());
  __shared__ DegPartial run[kMaxDegrees];
  __shared__ SuffStat suff_sh;
  const int tid = threadIdx.x;
  // the sufficient-statistics variant: its coefficients, read once per block
  const SuffStat* suff = nullptr;
  if (suff_g) {
    static_assert(sizeof(SuffStat) % 4 == 0, "copied as words");
    for (int i = tid; i < (int)(sizeof(SuffStat) / 4); i += kTpb)
      reinterpret_cast<int*>(&suff_sh)[i] = reinterpret_cast<const int*>(suff_g)[i];
    suff = &suff_sh;
  }
  const int64_t group = (int64_t)kTpb * PPT;
  const int64_t n_groups = (N + group - 1) / group;
  const bool resident = L <= chunk;
  reset_warp_partials(ts);
  if (resident)
    for (int l = tid; l < L; l += kTpb) sdata[l] = make_float2(xs[l], ys[l]);
  __syncthreads();
  int nan = 0;
  for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
    trace_group<PPT>(PriorDraw{p, seed, instance}, p, xs, ys, L, chunk, resident, sdata, N,
                     g * group, lw_out, rec_out, ts, suff);
    if (tid == 0) nan |= ts.nan;
    // the block's running per-degree maxima bound the final maxima from
    // below, so later groups skip traces far beneath them (taken at the group
    // boundary, after trace_group's closing barrier: deterministic)
    if (tid < kMaxDegrees) {
      float m = ts.ext_max[tid];
#pragma unroll
      for (int w = 0; w < kTpb / 32; ++w) m = fmaxf(m, ts.wrun[w * kMaxDegrees + tid].m);
      ts.ext_max[tid] = m;
    }
  }
  merge_warp_partials(ts, run);
  if (tid < kMaxDegrees) parts[blockIdx.x * kMaxDegrees + tid] = run[tid];
  if (tid == 0 && nan) record_status(&hdr->status, PPL_ENAN);
  if (elect_last_block(&hdr->ticket[0]))
    finalize_partials(parts, gridDim.x, p.n_deg, p.min_deg, N, hdr, res);
}

// ---------------------------------------------------------------------------
// Statistics pass over an existing set of log-weights (lw NULL = all 0).
// ---------------------------------------------------------------------------
constexpr int kStatVec = 4;  // float4 loads per thread per round: 16 log-weights in flight

// A thread's batch of log-weights (lowest index first) folded into its running
// statistics: the batch maximum (lowest index on ties) rescales the sums once,
// then every finite weight adds exp(lw - m) and its square; NaNs only raise the
// flag.  Indices increase from batch to batch, so ties keep the earlier index.
template <int B>
__device__ __forceinline__ void add_batch(StatAcc& acc, const float (&v)[B], int64_t i0,
                                          int64_t step) {
  float mb = -INFINITY;
  int64_t ib = 0x7fffffff;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    acc.nan |= v[j] != v[j];
    if (v[j] > mb) {
      mb = v[j];
      ib = i0 + (j / 4) * step + (j % 4);
    }
  }
  if (mb > acc.m) {
    const float e = (acc.m == -INFINITY) ? 0.0f : expf(acc.m - mb);
    acc.s *= e;
    acc.s2 *= e * e;
    acc.m = mb;
    acc.arg = (int)ib;
  }
  if (acc.m > -INFINITY) {
#pragma unroll
    for (int j = 0; j < B; ++j) {
      if (v[j] > -INFINITY) {  // NaN and -inf add nothing
        const float e = expf(v[j] - acc.m);
        acc.s += e;
        acc.s2 = fmaf(e, e, acc.s2);
      }
    }
  }
}

__global__ void __launch_bounds__(kTpb) stats_kernel(const float* __restrict__ lw, int64_t N,
                                                     WsHeader* hdr, StatPartial* parts,
                                                     double* lse_out) {
  StatAcc acc;
  acc.init();
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  int64_t done = 0;  // the prefix handled by the vector loop
  if (lw && (reinterpret_cast<uintptr_t>(lw) & 15) == 0) {
    // coalesced 16-byte loads, kStatVec of them in flight per thread; thread t
    // of the grid takes vectors t, t + stride, ..., kStatVec per round
    const float4* v4 = reinterpret_cast<const float4*>(lw);
    const int64_t n4 = N / 4;
    const int64_t round = stride * kStatVec;
    const int64_t full = n4 / round * round;  // vectors in whole rounds
    for (int64_t q = (int64_t)blockIdx.x * kTpb + threadIdx.x; q < full; q += round) {
      float v[4 * kStatVec];
#pragma unroll
      for (int r = 0; r < kStatVec; ++r) {
        const float4 x = __ldcs(v4 + q + r * stride);
        v[4 * r] = x.x;
        v[4 * r + 1] = x.y;
        v[4 * r + 2] = x.z;
        v[4 * r + 3] = x.w;
      }
      add_batch<4 * kStatVec>(acc, v, 4 * q, 4 * stride);
    }
    done = 4 * full;
  }
  for (int64_t i = done + (int64_t)blockIdx.x * kTpb + threadIdx.x; i < N; i += stride)
    acc.add(lw ? lw[i] : 0.0f, (int)i, -1);
  StatAcc r = block_reduce_stat(acc);
  if (threadIdx.x == 0) to_partial(r, parts + blockIdx.x);
  if (elect_last_block(&hdr->ticket[0]))
    finalize_stats(parts, gridDim.x, N, nullptr, hdr, nullptr, lse_out);
}

// ---------------------------------------------------------------------------
// Posterior summary of an existing weighted population of records, one pass.
// ---------------------------------------------------------------------------
constexpr int kPostPpt = 4;

__global__ void __launch_bounds__(kTpb) posterior_kernel(PolyParams p,
                                                         const ppl_poly_particle* __restrict__ rec,
                                                         const float* __restrict__ lwin,
                                                         int64_t N, WsHeader* hdr,
                                                         DegPartial* parts, ppl_is_result* res) {
  __shared__ GroupScratch gs;
  __shared__ DegPartial run[kMaxDegrees];
  const int tid = threadIdx.x;
  if (tid < kMaxDegrees) deg_empty(run[tid]);
  __syncthreads();
  const int64_t group = (int64_t)kTpb * kPostPpt;
  const int64_t n_groups = (N + group - 1) / group;
  int nan = 0, bad = 0;
  for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
    float lw[kPostPpt], c[kPostPpt][kMaxCoef];
    int d[kPostPpt], idx[kPostPpt];
#pragma unroll
    for (int q = 0; q < kPostPpt; ++q) {
      const int64_t i = g * group + (int64_t)q * kTpb + tid;
      idx[q] = (int)i;
      d[q] = -1;
      lw[q] = -INFINITY;
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) c[q][k] = 0.0f;
      if (i < N) {
        const float4* src = reinterpret_cast<const float4*>(rec + i);
        const float4 a = src[0], b = src[1];
        c[q][0] = a.x;
        c[q][1] = a.y;
        c[q][2] = a.z;
        c[q][3] = a.w;
        c[q][4] = b.x;
        c[q][5] = b.y;
        const int dd = __float_as_int(b.z) - p.min_deg;
        if ((unsigned)dd < (unsigned)p.n_deg) {
          d[q] = dd;
          lw[q] = lwin ? lwin[i] : 0.0f;
        } else {
          bad = 1;
        }
      }
    }
    group_partial<kPostPpt>(lw, d, idx, c, gs);
    if (tid < kMaxDegrees) deg_merge(run[tid], gs.out[tid]);
    if (tid == 0) nan |= gs.nan;
  }
  __syncthreads();
  if (tid < kMaxDegrees) parts[blockIdx.x * kMaxDegrees + tid] = run[tid];
  if (tid == 0 && nan) record_status(&hdr->status, PPL_ENAN);
  if (bad) record_status(&hdr->status, PPL_EINVAL);
  if (elect_last_block(&hdr->ticket[1]))
    finalize_partials(parts, gridDim.x, p.n_deg, p.min_deg, N, hdr, res);
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

constexpr int kTraceKernelPpt = 4;
constexpr int kMaxChunk = 4096;

int trace_grid(int64_t N) {
  const int64_t groups =
      (N + (int64_t)kTpb * kTraceKernelPpt - 1) / ((int64_t)kTpb * kTraceKernelPpt);
  return (int)std::max<int64_t>(1, std::min<int64_t>(groups, kMaxBlocks));
}

int stream_grid(int64_t N) {
  const int64_t blocks = (N + kTpb - 1) / kTpb;
  const int64_t cap = (int64_t)num_sms() * 4;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, std::min<int64_t>(cap, kMaxBlocks)));
}

cudaError_t launch_poly_trace(const PolyParams& p, const float* x, const float* y, int64_t L,
                              int64_t N, uint64_t seed, uint32_t instance, float* lw_out,
                              ppl_poly_particle* rec_out, WsHeader* hdr, void* parts,
                              ppl_is_result* res, cudaStream_t s, const void* suff) {
  constexpr int PPT = kTraceKernelPpt;
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(L, kMaxChunk));
  const size_t smem = trace_smem_bytes<PPT>() + (size_t)chunk * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(poly_trace_kernel<PPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(trace_smem_bytes<PPT>() + kMaxChunk * sizeof(float2)));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, poly_trace_kernel<PPT>,
                                                                kTpb, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(trace_grid(N), num_sms() * std::max(1, per_sm)));
  poly_trace_kernel<PPT><<<grid, kTpb, smem, s>>>(p, x, y, L, N, seed, instance, chunk, lw_out,
                                                  rec_out, hdr, (DegPartial*)parts, res,
                                                  (const SuffStat*)suff);
  return cudaGetLastError();
}

cudaError_t launch_stats(const float* lw, int64_t N, WsHeader* hdr, void* parts,
                         double* lse_out, cudaStream_t s) {
  stats_kernel<<<stream_grid(N), kTpb, 0, s>>>(lw, N, hdr, (StatPartial*)parts, lse_out);
  return cudaGetLastError();
}

cudaError_t launch_posterior(const PolyParams& p, const ppl_poly_particle* rec, const float* lw,
                             int64_t N, WsHeader* hdr, void* parts, ppl_is_result* res,
                             cudaStream_t s) {
  const int64_t groups = (N + (int64_t)kTpb * kPostPpt - 1) / ((int64_t)kTpb * kPostPpt);
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(groups, std::min<int64_t>((int64_t)num_sms() * 4, kMaxBlocks)));
  posterior_kernel<<<grid, kTpb, 0, s>>>(p, rec, lw, N, hdr, (DegPartial*)parts, res);
  return cudaGetLastError();
}

size_t partials_bytes() {
  return (size_t)kMaxBlocks * std::max(sizeof(StatPartial), kMaxDegrees * sizeof(DegPartial));
}

}  // namespace ppl
