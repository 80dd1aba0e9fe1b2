// Likelihood weighting on the line-fitting model: the trace kernel (§3.6.2 run
// the model N times and normalise the log-weights; Fig. 1 the model) with the
// posterior reduction fused in (degree masses, weighted coefficient means and
// variances, the mode), the statistics pass over given log-weights, and the
// one-pass posterior summary of a given population.
#include <map>
#include <mutex>

#include "dfloat.cuh"
#include "kernels.h"
#include "poly.cuh"
#include "posterior.cuh"
#include "stats.cuh"
#include "trace.cuh"

namespace ppl {

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
// Statistics pass over an existing set of log-weights (§3.6.2: the maximum,
// log-sum-exp and ESS that normalise them), one read of lw at HBM speed.
//
// The 16-byte-aligned body of lw is cut into one contiguous range of float4
// vectors per block (balanced to a 128-byte line); a block walks its range in
// tiles of kTpb * kStatU vectors, each thread loading kStatU vectors of the
// next tile while it folds the current one into its running statistics.  The
// (at most three) elements before the first 16-byte boundary go to block 0
// before its range, the (at most three) after the last whole vector to the
// last block after its range, so every thread sees increasing indices.  The
// last block to finish merges the blocks' partials.
// ---------------------------------------------------------------------------
constexpr int kStatThreads = 256;                 // threads per block
constexpr int kStatU = 4;                         // vectors per thread per tile
constexpr int kStatTile = kStatThreads * kStatU;  // vectors per tile
constexpr int kStatBlocksPerSm = 4;
constexpr float kLog2e = 0x1.715476p+0f;

// 2^t by the SFU's base-2 exponential (PTX ex2.approx.ftz: relative error
// about 2^-22, results below 2^-126 flushed to zero, ex2(-inf) = 0).
__device__ __forceinline__ float ex2_sfu(float t) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}

// Running statistics of one thread: maximum m and its (lowest) index, the
// sums of exp(lw - m) and exp(2 (lw - m)), and a NaN flag.
struct LseAcc {
  float m, s, s2;
  int arg, nan;
  __device__ __forceinline__ void init() {
    m = -INFINITY;
    s = 0.0f;
    s2 = 0.0f;
    arg = 0x7fffffff;
    nan = 0;
  }
  // one weight, at an index above every index added before
  __device__ __forceinline__ void add(float v, int i) {
    if (v != v) {
      nan = 1;
      return;
    }
    if (v > m) {
      const float e = (m == -INFINITY) ? 0.0f : ex2_sfu((m - v) * kLog2e);
      s *= e;
      s2 *= e * e;
      m = v;
      arg = i;
    }
    if (m > -INFINITY) {
      const float e = ex2_sfu((v - m) * kLog2e);
      s += e;
      s2 = fmaf(e, e, s2);
    }
  }
};

// A thread's tile folded into its running statistics.  The tile maximum
// (maxNum: NaNs are passed over) is found first; only when it raises the
// running maximum are the tile's values searched for its lowest index and the
// sums rescaled, which after the first tiles is rare.  Every weight then adds
// 2^((lw - m) log2 e) and its square: -inf adds exactly 0, and a NaN (or
// +inf) poisons the tile's sum, whose tile is then summed again with those
// values left out and the flag raised.  Slot j of the tile holds element
// indices i0 + 4 kStatThreads j + 0..3.
__device__ __forceinline__ void add_tile(LseAcc& acc, const float4 (&t)[kStatU], int64_t i0) {
  float mb = -INFINITY;
#pragma unroll
  for (int j = 0; j < kStatU; ++j)
    mb = fmaxf(mb, fmaxf(fmaxf(t[j].x, t[j].y), fmaxf(t[j].z, t[j].w)));
  if (mb > acc.m) {
    int c = 0;
#pragma unroll
    for (int j = kStatU - 1; j >= 0; --j) {  // the last match written is the lowest index
      if (t[j].w == mb) c = 4 * j + 3;
      if (t[j].z == mb) c = 4 * j + 2;
      if (t[j].y == mb) c = 4 * j + 1;
      if (t[j].x == mb) c = 4 * j;
    }
    const float e = (acc.m == -INFINITY) ? 0.0f : ex2_sfu((acc.m - mb) * kLog2e);
    acc.s *= e;
    acc.s2 *= e * e;
    acc.m = mb;
    acc.arg = (int)(i0 + (int64_t)(c >> 2) * 4 * kStatThreads + (c & 3));
  }
  if (acc.m > -INFINITY) {
    const float m = acc.m;
    float s = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int j = 0; j < kStatU; ++j) {
      const float v[4] = {t[j].x, t[j].y, t[j].z, t[j].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float e = ex2_sfu((v[c] - m) * kLog2e);
        s += e;
        s2 = fmaf(e, e, s2);
      }
    }
    if (s != s) {  // a NaN or +inf in the tile
      acc.nan = 1;
      s = 0.0f;
      s2 = 0.0f;
#pragma unroll
      for (int j = 0; j < kStatU; ++j) {
        const float v[4] = {t[j].x, t[j].y, t[j].z, t[j].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float d = v[c] - m;
          if (d == d) {
            const float e = ex2_sfu(d * kLog2e);
            s += e;
            s2 = fmaf(e, e, s2);
          }
        }
      }
    }
    acc.s += s;
    acc.s2 += s2;
  } else {  // nothing finite so far: the tile holds only -inf and NaN
#pragma unroll
    for (int j = 0; j < kStatU; ++j)
      acc.nan |= (t[j].x != t[j].x) | (t[j].y != t[j].y) | (t[j].z != t[j].z) | (t[j].w != t[j].w);
  }
}

// a <- merge(a, b); ties of the maximum keep the lower index
__device__ __forceinline__ void lse_merge(LseAcc& a, const LseAcc& b) {
  const float M = fmaxf(a.m, b.m);
  if (M > -INFINITY) {
    const float ea = (a.m == -INFINITY) ? 0.0f : ex2_sfu((a.m - M) * kLog2e);
    const float eb = (b.m == -INFINITY) ? 0.0f : ex2_sfu((b.m - M) * kLog2e);
    a.s = fmaf(a.s, ea, b.s * eb);
    a.s2 = fmaf(a.s2, ea * ea, b.s2 * eb * eb);
  }
  if (b.m > a.m || (b.m == a.m && b.arg < a.arg)) a.arg = b.arg;
  a.m = M;
  a.nan |= b.nan;
}

__device__ __forceinline__ LseAcc lse_shfl_xor(const LseAcc& a, int o) {
  LseAcc r;
  r.m = __shfl_xor_sync(0xffffffffu, a.m, o);
  r.s = __shfl_xor_sync(0xffffffffu, a.s, o);
  r.s2 = __shfl_xor_sync(0xffffffffu, a.s2, o);
  r.arg = __shfl_xor_sync(0xffffffffu, a.arg, o);
  r.nan = __shfl_xor_sync(0xffffffffu, a.nan, o);
  return r;
}

// Block merge of the threads' statistics; the result is valid in thread 0.
__device__ __forceinline__ LseAcc lse_block_reduce(LseAcc a) {
  __shared__ LseAcc slots[kStatThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lse_merge(a, lse_shfl_xor(a, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) slots[warp] = a;
  __syncthreads();
  if (warp == 0) {
    LseAcc r;
    r.init();
    if (lane < kStatThreads / 32) r = slots[lane];
#pragma unroll
    for (int o = kStatThreads / 64; o > 0; o >>= 1) lse_merge(r, lse_shfl_xor(r, o));
    a = r;
  }
  return a;
}

// Double-float accumulation (Knuth's TwoSum: hi + lo carries the exact sum
// of the FP32 terms added so far, to about 48 bits).
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += err;
}

// Final merge by the last block: the maximum and its lowest index in FP32
// (exact), then every partial's sums rescaled to the merged maximum (FP32
// exp of a difference of two floats) and added in double-float per lane,
// across lanes and across warps; thread 0 takes log s by df_log and the ESS
// as a corrected quotient (no FP64 arithmetic but the final addition).
__device__ __forceinline__ void lse_finalize(const StatPartial* parts, int G, int64_t N,
                                             WsHeader* hdr, double* lse_out) {
  __shared__ float M_sh;
  __shared__ float2 wsum[kStatThreads / 32][2];
  LseAcc a;
  a.init();
  for (int b = threadIdx.x; b < G; b += kStatThreads) {
    const StatPartial p = parts[b];
    LseAcc o;
    o.m = p.m;
    o.s = p.s;
    o.s2 = p.s2;
    o.arg = p.arg;
    o.nan = p.nan;
    lse_merge(a, o);
  }
  const LseAcc r = lse_block_reduce(a);
  if (threadIdx.x == 0) M_sh = r.m;
  __syncthreads();
  const float M = M_sh;
  float sh = 0.0f, sl = 0.0f, qh = 0.0f, ql = 0.0f;
  if (M > -INFINITY) {
    for (int b = threadIdx.x; b < G; b += kStatThreads) {
      const float pm = parts[b].m;
      if (pm == -INFINITY) continue;
      const float e = ex2_sfu((pm - M) * kLog2e);
      df_add(sh, sl, parts[b].s * e);
      df_add(qh, ql, parts[b].s2 * e * e);
    }
  }
  float2 s = df_warp_sum(df_add(make_float2(sh, 0.0f), make_float2(sl, 0.0f)));
  float2 s2 = df_warp_sum(df_add(make_float2(qh, 0.0f), make_float2(ql, 0.0f)));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    wsum[warp][0] = s;
    wsum[warp][1] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s = wsum[0][0];
    s2 = wsum[0][1];
#pragma unroll
    for (int w = 1; w < kStatThreads / 32; ++w) {
      s = df_add(s, wsum[w][0]);
      s2 = df_add(s2, wsum[w][1]);
    }
    int32_t code = 0;
    if (r.nan) code = PPL_ENAN;
    else if (!(M > -INFINITY)) code = PPL_EEMPTY;
    if (code) record_status(&hdr->status, code);
    double lse = -INFINITY, ess = nan("");
    if (s.x > 0.0f) {
      lse = (double)M + df_to_double(df_log(s));
      ess = (double)df_div(df_mul(s, s), s2);
    }
    hdr->max_lw = M;
    hdr->lse = lse;
    hdr->ess = ess;
    hdr->argmax = r.arg;
    if (lse_out) {
      lse_out[0] = lse;
      lse_out[1] = ess;
      lse_out[2] = (double)M;
      lse_out[3] = (double)r.arg;
    }
  }
}

// Vectors [q0 + j kStatThreads + tid] of a whole tile (streamed: read once).
__device__ __forceinline__ void load_tile(float4 (&t)[kStatU], const float4* __restrict__ v4) {
#pragma unroll
  for (int j = 0; j < kStatU; ++j) t[j] = __ldcs(v4 + j * kStatThreads + threadIdx.x);
}

__global__ void __launch_bounds__(kStatThreads, kStatBlocksPerSm) stats_kernel(
    const float* __restrict__ lw, int64_t N, WsHeader* hdr, StatPartial* parts,
    double* lse_out) {
  LseAcc acc;
  acc.init();
  const int tid = threadIdx.x;
  const int G = gridDim.x, b = blockIdx.x;
  const int64_t mis = (int64_t)(((16 - (reinterpret_cast<uintptr_t>(lw) & 15)) & 15) / 4);
  const int head = (int)(mis < N ? mis : N);
  const int64_t n4 = (N - head) / 4;
  const int tail = (int)(N - head - 4 * n4);
  if (b == 0 && tid < head) acc.add(lw[tid], tid);
  // this block's vectors [begin, end), cut at multiples of 8 (128 bytes)
  const int64_t lines = (n4 + 7) / 8;
  const int64_t begin = ::min(n4, lines * b / G * 8);
  const int64_t end = ::min(n4, lines * (b + 1) / G * 8);
  const float4* v4 = reinterpret_cast<const float4*>(lw + head) + begin;
  const int n_vec = (int)(end - begin);
  const int full = n_vec / kStatTile * kStatTile;  // vectors in whole tiles
  const int64_t i_base = head + 4 * (begin + tid);  // element index of slot 0, tile 0
  if (full > 0) {
    float4 cur[kStatU];
    load_tile(cur, v4);
    for (int q0 = 0; q0 < full; q0 += kStatTile) {
      float4 nxt[kStatU];
      const bool more = q0 + kStatTile < full;  // the same for the whole block
      if (more) load_tile(nxt, v4 + q0 + kStatTile);
      add_tile(acc, cur, i_base + 4 * (int64_t)q0);
      if (more) {
#pragma unroll
        for (int j = 0; j < kStatU; ++j) cur[j] = nxt[j];
      }
    }
  }
  if (full < n_vec) {  // the range's last, partial tile
    float4 t[kStatU];
#pragma unroll
    for (int j = 0; j < kStatU; ++j) {
      const int q = full + j * kStatThreads + tid;
      t[j] = q < n_vec ? __ldcs(v4 + q)
                       : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    }
    add_tile(acc, t, i_base + 4 * (int64_t)full);
  }
  if (b == G - 1 && tid < tail) {
    const int64_t i = head + 4 * n4 + tid;
    acc.add(lw[i], (int)i);
  }
  const LseAcc r = lse_block_reduce(acc);
  if (tid == 0) {
    StatPartial p;
    p.m = r.m;
    p.s = r.s;
    p.s2 = r.s2;
    p.arg = r.arg;
    p.nan = r.nan;
    parts[b] = p;
  }
  if (elect_last_block(&hdr->ticket[0])) lse_finalize(parts, G, N, hdr, lse_out);
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
namespace {
std::mutex g_once_mutex;
std::map<std::pair<const void*, int>, int> g_once_value;
}  // namespace

cudaError_t device_once(const void* key, int* value, const std::function<cudaError_t(int*)>& setup) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_once_mutex);
  auto it = g_once_value.find({key, dev});
  if (it == g_once_value.end()) {
    int v = 0;
    e = setup(&v);
    if (e != cudaSuccess) return e;
    it = g_once_value.emplace(std::make_pair(key, dev), v).first;
  }
  *value = it->second;
  return cudaSuccess;
}

int num_sms() {
  int n = 0;
  const cudaError_t e = device_once((const void*)&num_sms, &n, [](int* v) {
    int dev = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
    return r;
  });
  return (e == cudaSuccess && n > 0) ? n : 1;
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
  int unused = 0;
  cudaError_t e = device_once((const void*)poly_trace_kernel<PPT>, &unused, [](int*) {
    return cudaFuncSetAttribute(poly_trace_kernel<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(trace_smem_bytes<PPT>() + kMaxChunk * sizeof(float2)));
  });
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, poly_trace_kernel<PPT>, kTpb, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(trace_grid(N), num_sms() * std::max(1, per_sm)));
  poly_trace_kernel<PPT><<<grid, kTpb, smem, s>>>(p, x, y, L, N, seed, instance, chunk, lw_out,
                                                  rec_out, hdr, (DegPartial*)parts, res,
                                                  (const SuffStat*)suff);
  return cudaGetLastError();
}

cudaError_t launch_stats(const float* lw, int64_t N, WsHeader* hdr, void* parts,
                         double* lse_out, cudaStream_t s) {
  // a few tiles per block at least; up to kStatBlocksPerSm blocks per SM
  const int64_t tiles = (N / 4 + kStatTile - 1) / kStatTile;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((tiles + 1) / 2, (int64_t)num_sms() * kStatBlocksPerSm));
  stats_kernel<<<grid, kStatThreads, 0, s>>>(lw, N, hdr, (StatPartial*)parts, lse_out);
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
