// One-pass posterior reduction of weighted line-fitting traces (§3.6.2 the
// normalisation of the log-weights; Fig. 1 the returned coefficients).
//
// A group of traces (one block's particles of one instance) is reduced to a
// per-degree partial: the best log-weight m and its index, S = sum exp(lw - m),
// S2 = sum exp(2 (lw - m)), and the weighted mean and second central moment
// M2 = sum w (c - mean)^2 of every coefficient.  Within a group the moments are
// formed around the group's best trace of that degree (a shift that keeps the
// FP32 sums well conditioned), and partials merge exactly in real arithmetic:
// rescale by exp(m_a - m), then combine means and M2 by the parallel-variance
// rule (Chan, Golub and LeVeque 1979).  The LSE, ESS, degree masses and pooled
// moments all follow from the per-degree partials.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"
#include "poly.cuh"

namespace ppl {

struct __align__(16) DegPartial {
  float m;
  int arg;
  float S, S2;
  float mean[kMaxCoef];
  float M2[kMaxCoef];
};

__device__ __forceinline__ void deg_empty(DegPartial& p) {
  p.m = -INFINITY;
  p.arg = 0x7fffffff;
  p.S = 0.0f;
  p.S2 = 0.0f;
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) {
    p.mean[k] = 0.0f;
    p.M2[k] = 0.0f;
  }
}

// a <- merge(a, b)
__device__ __forceinline__ void deg_merge(DegPartial& a, const DegPartial& b) {
  if (b.m == -INFINITY) return;
  if (a.m == -INFINITY) {
    a = b;
    return;
  }
  const float M = fmaxf(a.m, b.m);
  const float ea = expf(a.m - M), eb = expf(b.m - M);
  const float wa = a.S * ea, wb = b.S * eb, w = wa + wb;
  const float fb = wb / w, cross = wa * fb;
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) {
    const float d = b.mean[k] - a.mean[k];
    a.mean[k] = fmaf(d, fb, a.mean[k]);
    a.M2[k] = fmaf(d * d, cross, fmaf(a.M2[k], ea, b.M2[k] * eb));
  }
  a.S2 = fmaf(a.S2, ea * ea, b.S2 * eb * eb);
  a.S = w;
  if (b.m > a.m || (b.m == a.m && b.arg < a.arg)) a.arg = b.arg;
  a.m = M;
}

__device__ __forceinline__ DegPartial deg_shfl_xor(const DegPartial& p, int mask) {
  DegPartial o;
  o.m = __shfl_xor_sync(0xffffffffu, p.m, mask);
  o.arg = __shfl_xor_sync(0xffffffffu, p.arg, mask);
  o.S = __shfl_xor_sync(0xffffffffu, p.S, mask);
  o.S2 = __shfl_xor_sync(0xffffffffu, p.S2, mask);
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) {
    o.mean[k] = __shfl_xor_sync(0xffffffffu, p.mean[k], mask);
    o.M2[k] = __shfl_xor_sync(0xffffffffu, p.M2[k], mask);
  }
  return o;
}

// Load a partial written by another block of the running kernel, from L2.
__device__ __forceinline__ DegPartial ld_partial_cg(const DegPartial* src) {
  static_assert(sizeof(DegPartial) == 64, "DegPartial is four 16-byte words");
  DegPartial o;
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(&o);
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = __ldcg(s + i);
  return o;
}

// Shared-memory scratch of group_partial.
struct GroupScratch {
  float wmax[kTpb / 32][kMaxDegrees];
  int warg[kTpb / 32][kMaxDegrees];
  float bmax[kMaxDegrees];
  int barg[kMaxDegrees];
  float ref[kMaxDegrees][kMaxCoef];
  float sums[kTpb / 32][kMaxDegrees * (2 + 2 * kMaxCoef)];
  DegPartial out[kMaxDegrees];
  int nan;
};

// Reduce PPT traces per thread (lw, degree index d in [0, 4) or -1 when the
// slot is empty, coefficients c) over the block into gs.out[0..3].  Every
// thread of the block must call it.  Indices passed as `idx` are global trace
// indices (lowest wins ties).
template <int PPT>
__device__ __forceinline__ void group_partial(const float (&lw)[PPT], const int (&d)[PPT],
                                              const int (&idx)[PPT],
                                              const float (&c)[PPT][kMaxCoef],
                                              GroupScratch& gs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // 1. best trace of every degree
  float m[kMaxDegrees];
  int a[kMaxDegrees];
  int nan = 0;
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) {
    m[k] = -INFINITY;
    a[k] = 0x7fffffff;
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    nan |= (d[q] >= 0) & (lw[q] != lw[q]);
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k)
      if (d[q] == k && (lw[q] > m[k] || (lw[q] == m[k] && idx[q] < a[k]))) {
        m[k] = lw[q];
        a[k] = idx[q];
      }
  }
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, m[k], o);
      const int oa = __shfl_xor_sync(0xffffffffu, a[k], o);
      if (om > m[k] || (om == m[k] && oa < a[k])) {
        m[k] = om;
        a[k] = oa;
      }
    }
    if (lane == 0) {
      gs.wmax[warp][k] = m[k];
      gs.warg[warp][k] = a[k];
    }
  }
  nan = __any_sync(0xffffffffu, nan);
  if (tid == 0) gs.nan = 0;
  __syncthreads();
  if (lane == 0 && nan) gs.nan = 1;
  if (tid < kMaxDegrees) {
    float bm = -INFINITY;
    int ba = 0x7fffffff;
    for (int w = 0; w < kTpb / 32; ++w)
      if (gs.wmax[w][tid] > bm || (gs.wmax[w][tid] == bm && gs.warg[w][tid] < ba)) {
        bm = gs.wmax[w][tid];
        ba = gs.warg[w][tid];
      }
    gs.bmax[tid] = bm;
    gs.barg[tid] = ba;
  }
  __syncthreads();
  // 2. the best trace's coefficients become the shift of its degree
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    if (d[q] >= 0 && idx[q] == gs.barg[d[q]])
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) gs.ref[d[q]][k] = c[q][k];
  __syncthreads();
  // 3. weighted sums around the shift
  constexpr int V = 2 + 2 * kMaxCoef;
  float acc[kMaxDegrees][V];
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[k][v] = 0.0f;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (d[q] < 0) continue;
    const int dd = d[q];
    const float w = (lw[q] > -INFINITY) ? expf(lw[q] - gs.bmax[dd]) : 0.0f;
    float dc[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) dc[k] = c[q][k] - gs.ref[dd][k];
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      const float wk = (k == dd) ? w : 0.0f;
      acc[k][0] += wk;
      acc[k][1] = fmaf(wk, wk, acc[k][1]);
#pragma unroll
      for (int j = 0; j < kMaxCoef; ++j) {
        const float t = wk * dc[j];
        acc[k][2 + j] += t;
        acc[k][2 + kMaxCoef + j] = fmaf(t, dc[j], acc[k][2 + kMaxCoef + j]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float x = warp_sum(acc[k][v]);
      if (lane == 0) gs.sums[warp][k * V + v] = x;
    }
  __syncthreads();
  // 4. one thread per degree forms the partial
  if (tid < kMaxDegrees) {
    const int k = tid;
    float tot[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float x = 0.0f;
      for (int w = 0; w < kTpb / 32; ++w) x += gs.sums[w][k * V + v];
      tot[v] = x;
    }
    DegPartial& p = gs.out[k];
    p.m = gs.bmax[k];
    p.arg = gs.barg[k];
    p.S = tot[0];
    p.S2 = tot[1];
    if (p.m == -INFINITY || !(tot[0] > 0.0f)) {
      deg_empty(p);
      p.m = gs.bmax[k];
      p.arg = gs.barg[k];
    } else {
#pragma unroll
      for (int j = 0; j < kMaxCoef; ++j) {
        const float A = tot[2 + j] / tot[0];
        p.mean[j] = gs.ref[k][j] + A;
        p.M2[j] = fmaxf(tot[2 + kMaxCoef + j] - A * tot[2 + j], 0.0f);
      }
    }
  }
  __syncthreads();
}

// Summary of a population from its four per-degree partials, by the 32 lanes
// of one warp (every lane calls it).  S and S2 are the per-degree sums around
// each degree's maximum as double-floats.  The degree masses, log Z, p(n) and
// the ESS are FP64 (a degree's mass may lie far below FP32's range), but
// GB300's FP64 pipe is narrow and slow, so the work is spread over the lanes
// and every lane's chain of FP64 operations is short: lanes 0-3 take one
// degree's mass (an exp), lane 0 log(s), lane 1 log(N), lane 2 the ESS, lanes
// 0-23 one (degree, coefficient) variance each, lanes 0-5 one pooled mean.
__device__ __forceinline__ void write_summary_warp(const DegPartial (&p)[kMaxDegrees],
                                                   const float2 (&S)[kMaxDegrees],
                                                   const float2 (&S2)[kMaxDegrees], int n_deg,
                                                   int min_deg, int64_t N, int32_t status,
                                                   ppl_is_result* res) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // the best trace (FP32 compares: the conversion to FP64 is exact and monotone)
  float Mf = -INFINITY;
  int32_t arg = -1;
  for (int k = 0; k < n_deg; ++k)
    if (p[k].m != -INFINITY && (p[k].m > Mf || (p[k].m == Mf && p[k].arg < arg))) {
      Mf = p[k].m;
      arg = p[k].arg;
    }
  const double M = (double)Mf;
  // lanes 0-3: degree `lane`'s mass e S and e^2 S2 around the best trace
  const int kd = lane & 3;
  const bool has_k = lane < kMaxDegrees && kd < n_deg && p[kd].m != -INFINITY;
  double mass = 0.0, q2 = 0.0;
  if (has_k && S[kd].x > 0.0f) {
    const double e = exp((double)p[kd].m - M);
    mass = e * df_to_double(S[kd]);
    q2 = e * e * df_to_double(S2[kd]);
  }
  double s = 0.0, s2 = 0.0;
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) {
    s += __shfl_sync(full, mass, k);
    s2 += __shfl_sync(full, q2, k);
  }
  // lane 0: log(s); lane 1: log(N); lane 2: the ESS
  double t = 0.0;
  if (lane == 0) t = log(s);
  else if (lane == 1) t = log((double)N);
  else if (lane == 2) t = s * s / s2;
  const double log_s = __shfl_sync(full, t, 0), log_n = __shfl_sync(full, t, 1);
  const double ess = __shfl_sync(full, t, 2);
  // lanes 0-3: the degree masses p(n)
  const double pn = (lane < kMaxDegrees && s > 0.0) ? mass / s : 0.0;
  double pns[kMaxDegrees];
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) pns[k] = __shfl_sync(full, pn, k);
  // lanes 0-23: (degree k, coefficient j) mean and variance
  if (lane < kMaxDegrees * kMaxCoef) {
    const int k = lane / kMaxCoef, j = lane % kMaxCoef;
    const bool ok = k < n_deg && p[k].m != -INFINITY && S[k].x > 0.0f && p[k].S > 0.0f;
    res->deg_mean[k][j] = ok ? (double)p[k].mean[j] : 0.0;
    res->deg_var[k][j] = ok ? (double)p[k].M2[j] / (double)p[k].S : 0.0;
  }
  // lanes 0-5: pooled coefficient means, summed over degrees in order
  if (lane < kMaxCoef) {
    double mc = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      const bool ok = k < n_deg && p[k].m != -INFINITY && S[k].x > 0.0f && p[k].S > 0.0f;
      mc += pns[k] * (ok ? (double)p[k].mean[lane] : 0.0);
    }
    res->mean_c[lane] = mc;
  }
  if (lane < kMaxDegrees) {
    res->p_n[lane] = pn;
    res->deg_max_lw[lane] = has_k ? (double)p[lane].m : -INFINITY;
    res->deg_argmax[lane] = has_k ? p[lane].arg : -1;
  }
  if (lane == 0) {
    int best = 0;
    for (int k = 1; k < n_deg; ++k)
      if (pns[k] > pns[best]) best = k;
    res->lse = M + log_s;
    res->log_z = res->lse - log_n;
    res->ess = ess;
    res->max_lw = M;
    res->argmax = arg;
    res->n_particles = N;
    res->n_deg = n_deg;
    res->map_deg = min_deg + best;
    res->status = status;
  }
}

// A degree's sums S, S2 over partials q rescaled to the merged maximum M
// (FP32 exp of the difference, double-float products and sums), added by the
// lanes of a warp; every lane gets the totals.
struct DegSums {
  float2 S, S2;
  __device__ __forceinline__ void zero() {
    S = make_float2(0.0f, 0.0f);
    S2 = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void add(float qm, float2 qS, float2 qS2, float M) {
    if (qm == -INFINITY) return;
    const float e = expf(qm - M);
    S = df_add(S, df_mul(qS, e));
    S2 = df_add(S2, df_mul(df_mul(qS2, e), e));
  }
  __device__ __forceinline__ void warp_total() {
    S = df_warp_sum(S);
    S2 = df_warp_sum(S2);
  }
};

// ---------------------------------------------------------------------------
// Final merge of the per-block partials, by the last block: warp k merges
// degree k's partials (FP32, a lane-strided chain then a shuffle tree); the
// sums S, S2 are recombined in FP64 around the merged maximum; thread 0
// writes the summary.
// ---------------------------------------------------------------------------
// Warp `warp` (< kMaxDegrees) merges degree `warp` of G block partials: the
// maximum, its index and the moments in FP32 (a lane-strided chain, then a
// shuffle tree), then the sums S, S2 rescaled to the merged maximum.
__device__ __forceinline__ void merge_degree(const DegPartial* parts, int G, int warp, int lane,
                                             DegPartial& a, DegSums& ds) {
  // the partials come from L2 (written by other blocks of the running
  // kernel); several loads are in flight per lane, since one round trip to L2
  // costs about a microsecond here
  constexpr int U = 4, V = 8;
  deg_empty(a);
  for (int b0 = lane; b0 < G; b0 += 32 * U) {
    DegPartial q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (b0 + 32 * u < G) q[u] = ld_partial_cg(parts + (b0 + 32 * u) * kMaxDegrees + warp);
      else deg_empty(q[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) deg_merge(a, q[u]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DegPartial other = deg_shfl_xor(a, o);
    deg_merge(a, other);
  }
  ds.zero();
  if (a.m != -INFINITY)
    for (int b0 = lane; b0 < G; b0 += 32 * V) {
      float4 h[V];  // (m, arg, S, S2) of each partial
#pragma unroll
      for (int v = 0; v < V; ++v)
        h[v] = b0 + 32 * v < G
                   ? __ldcg(reinterpret_cast<const float4*>(parts + (b0 + 32 * v) * kMaxDegrees + warp))
                   : make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int v = 0; v < V; ++v)
        ds.add(h[v].x, make_float2(h[v].z, 0.0f), make_float2(h[v].w, 0.0f), a.m);
    }
  ds.warp_total();
}

__device__ __forceinline__ void finalize_partials(const DegPartial* parts, int G, int n_deg,
                                                  int min_deg, int64_t N, WsHeader* hdr,
                                                  ppl_is_result* res) {
  __shared__ DegPartial fin[kMaxDegrees];
  __shared__ float2 fS[kMaxDegrees], fS2[kMaxDegrees];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < kMaxDegrees) {
    DegPartial a;
    DegSums ds;
    merge_degree(parts, G, warp, lane, a, ds);
    if (lane == 0) {
      fin[warp] = a;
      fS[warp] = ds.S;
      fS2[warp] = ds.S2;
    }
  }
  __syncthreads();
  if (warp == 0) {
    int32_t st = 0;
    if (lane == 0) {
      bool any = false;
      for (int k = 0; k < n_deg; ++k) any |= fin[k].m != -INFINITY;
      if (!any) record_status(&hdr->status, PPL_EEMPTY);
      st = ld_volatile_i32(&hdr->status);
    }
    if (res) write_summary_warp(fin, fS, fS2, n_deg, min_deg, N, st, res);
  }
}



// ---------------------------------------------------------------------------
// One shard's share of a likelihood-weighting pass whose particles are split
// over several devices: its per-degree partials merged (FP32 means and
// second moments, FP64 sums around each degree's maximum), its particle
// count and device status.  Shards merge exactly like blocks (§3.6.2: the
// normalisation runs over all samples, wherever they were drawn).
// ---------------------------------------------------------------------------
struct __align__(16) IsPartial {
  DegPartial deg[kMaxDegrees];
  float2 S[kMaxDegrees], S2[kMaxDegrees];  // double-float sums around each degree's maximum
  int64_t n;
  int32_t status, n_deg, min_deg, pad0;
  unsigned char pad[32];
};
static_assert(sizeof(IsPartial) == 384, "the public ppl_is_partial is 384 bytes");

// The last block's merge of the block partials into a shard partial (the
// first part of finalize_partials, without the summary).
__device__ __forceinline__ void finalize_to_partial(const DegPartial* parts, int G, int n_deg,
                                                    int min_deg, int64_t N, WsHeader* hdr,
                                                    IsPartial* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < kMaxDegrees) {
    DegPartial a;
    DegSums ds;
    merge_degree(parts, G, warp, lane, a, ds);
    if (lane == 0) {
      out->deg[warp] = a;
      out->S[warp] = ds.S;
      out->S2[warp] = ds.S2;
    }
  }
  if (threadIdx.x == 0) {
    out->n = N;
    out->n_deg = n_deg;
    out->min_deg = min_deg;
    out->status = ld_volatile_i32(&hdr->status);
  }
}

// Merge of P shard partials into the summary of the whole population, by one
// block: warp k merges degree k (the maxima exactly, means and second
// moments by the parallel rule in FP32, the sums rescaled to the merged
// maximum in double-float).  N is the total particle count.
__device__ __forceinline__ void merge_shard_partials(const IsPartial* parts, int P, int64_t N,
                                                     int32_t status, ppl_is_result* res) {
  __shared__ DegPartial fin[kMaxDegrees];
  __shared__ float2 fS[kMaxDegrees], fS2[kMaxDegrees];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_deg = parts[0].n_deg, min_deg = parts[0].min_deg;
  if (warp < kMaxDegrees) {
    DegPartial a;
    deg_empty(a);
    for (int g = lane; g < P; g += 32) deg_merge(a, parts[g].deg[warp]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DegPartial other = deg_shfl_xor(a, o);
      deg_merge(a, other);
    }
    DegSums ds;
    ds.zero();
    if (a.m != -INFINITY)
      for (int g = lane; g < P; g += 32)
        ds.add(parts[g].deg[warp].m, parts[g].S[warp], parts[g].S2[warp], a.m);
    ds.warp_total();
    if (lane == 0) {
      fin[warp] = a;
      fS[warp] = ds.S;
      fS2[warp] = ds.S2;
    }
  }
  __syncthreads();
  if (warp == 0) {
    int32_t st = status;
    for (int g = 0; g < P && st == 0; ++g) st = parts[g].status;
    bool any = false;
    for (int k = 0; k < n_deg; ++k) any |= fin[k].m != -INFINITY;
    if (st == 0 && !any) st = PPL_EEMPTY;
    write_summary_warp(fin, fS, fS2, n_deg, min_deg, N, st, res);
  }
}

}  // namespace ppl
