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
// each degree's maximum as double-floats.  No FP64 arithmetic but single
// conversions and power-of-two scalings (GB300's FP64 pipe is narrow: a chain
// of FP64 exp, log and divisions took about 7 us): the degree weights
// e^(m_k - M) = 2^n_k w_k (exp_split, so a degree's mass keeps its relative
// precision far below FP32's range), the masses w_k S_k and their total s in
// double-float, log s by df_log, p(n) and the ESS as corrected FP32 quotients
// scaled back by 2^n_k in FP64.  Lanes 0-23 take one (degree, coefficient)
// variance each, lanes 0-5 one pooled mean each.
__device__ __forceinline__ void write_summary_warp(const DegPartial (&p)[kMaxDegrees],
                                                   const float2 (&S)[kMaxDegrees],
                                                   const float2 (&S2)[kMaxDegrees], int n_deg,
                                                   int min_deg, int64_t N, int32_t status,
                                                   ppl_is_result* res) {
  const int lane = threadIdx.x & 31;
  float M = -INFINITY;
  int32_t arg = -1;
  for (int k = 0; k < n_deg; ++k)
    if (p[k].m != -INFINITY && (p[k].m > M || (p[k].m == M && p[k].arg < arg))) {
      M = p[k].m;
      arg = p[k].arg;
    }
  // degree k's mass 2^n[k] mw[k] and e^(2 (m_k - M)) S2_k; s, s2 their totals
  // (terms below 2^-120 of the best degree's, which is at least 1, vanish
  // at double-float precision)
  int n[kMaxDegrees];
  float2 mw[kMaxDegrees];
  float2 s = make_float2(0.0f, 0.0f), s2 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) {
    n[k] = 0;
    mw[k] = make_float2(0.0f, 0.0f);
    if (k < n_deg && p[k].m != -INFINITY && S[k].x > 0.0f) {
      // m_k - M = dh + dl exactly (TwoSum of two floats); e^dl = 1 + dl
      const float dh = __fsub_rn(p[k].m, M);
      const float bb = __fsub_rn(dh, p[k].m);
      const float dl = __fsub_rn(__fsub_rn(p[k].m, __fsub_rn(dh, bb)), __fadd_rn(M, bb));
      const ExpSplit e = exp_split(dh);
      const float2 w = df_add(make_float2(e.m, 0.0f), make_float2(__fmul_rn(e.m, dl), 0.0f));
      n[k] = e.n;
      mw[k] = df_mul(S[k], w);
      if (e.n >= -120) {
        s = df_add(s, df_mul(mw[k], exp2i(e.n)));
        if (e.n >= -60) s2 = df_add(s2, df_mul(df_mul(df_mul(S2[k], w), w), exp2i(2 * e.n)));
      }
    }
  }
  // p(n): the FP32 quotient mw / s scaled by 2^n (FP32 value for the pooled
  // means, FP64 for the output)
  float pf[kMaxDegrees], pq[kMaxDegrees];
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k) {
    pq[k] = (s.x > 0.0f && mw[k].x > 0.0f) ? df_div(mw[k], s) : 0.0f;
    pf[k] = n[k] >= -120 ? __fmul_rn(pq[k], exp2i(n[k])) : 0.0f;
  }
  // lanes 0-23: (degree k, coefficient j) mean and variance
  if (lane < kMaxDegrees * kMaxCoef) {
    const int k = lane / kMaxCoef, j = lane % kMaxCoef;
    const bool ok = k < n_deg && p[k].m != -INFINITY && S[k].x > 0.0f && p[k].S > 0.0f;
    res->deg_mean[k][j] = ok ? (double)p[k].mean[j] : 0.0;
    res->deg_var[k][j] = ok ? (double)__fdiv_rn(p[k].M2[j], p[k].S) : 0.0;
  }
  // lanes 0-5: pooled coefficient means
  if (lane < kMaxCoef) {
    float2 mc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      const bool ok = k < n_deg && p[k].m != -INFINITY && S[k].x > 0.0f && p[k].S > 0.0f;
      if (ok) mc = df_add(mc, df_prod(pf[k], p[k].mean[lane]));
    }
    res->mean_c[lane] = df_to_double(mc);
  }
  if (lane < kMaxDegrees) {
    const int k = lane;
    const bool has = k < n_deg && p[k].m != -INFINITY;
    // 2^n as an FP64 value (n >= -1022; smaller masses underflow to 0)
    const double scale = n[k] >= -1022 ? __hiloint2double((n[k] + 1023) << 20, 0) : 0.0;
    res->p_n[k] = (double)pq[k] * scale;
    res->deg_max_lw[k] = has ? (double)p[k].m : -INFINITY;
    res->deg_argmax[k] = has ? p[k].arg : -1;
  }
  if (lane == 0) {
    int best = 0;
    for (int k = 1; k < n_deg; ++k)
      if (pf[k] > pf[best]) best = k;
    if (s.x > 0.0f) {
      const float2 log_s = df_log(s), log_n = df_log(df_from_i64(N));
      res->lse = (double)M + df_to_double(log_s);
      res->log_z = (double)M + df_to_double(df_add(log_s, df_neg(log_n)));
      res->ess = (double)df_div(df_mul(s, s), s2);
    } else {  // no finite weight
      res->lse = -INFINITY;
      res->log_z = -INFINITY;
      res->ess = nan("");
    }
    res->max_lw = (double)M;
    res->argmax = arg;
    res->n_particles = N;
    res->n_deg = n_deg;
    res->map_deg = min_deg + best;
    res->status = status;
    res->pad = 0;  // every field is written: callers need not clear the result
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
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
      S = df_add(S, df_shfl_xor(S, o));
      S2 = df_add(S2, df_shfl_xor(S2, o));
    }
  }
};

// ---------------------------------------------------------------------------
// Final merge of the per-block partials, by the last block: warp k merges
// degree k's partials (FP32, a lane-strided chain then a shuffle tree); the
// sums S, S2 are recombined in double-float around the merged maximum; warp
// 0 writes the summary.
// ---------------------------------------------------------------------------
// Warp `warp` (< kMaxDegrees) merges degree `warp` of G block partials: the
// maximum, its index and the moments in FP32 (a lane-strided chain, then a
// shuffle tree), then the sums S, S2 rescaled to the merged maximum.
__device__ __forceinline__ void merge_degree(const DegPartial* parts, int G, int warp, int lane,
                                             DegPartial& a, DegSums& ds) {
  // This code runs once per launch, by one block, after the kernel's data
  // have streamed through L2: its instructions are fetched cold, so the loops
  // stay rolled (fewer instruction fetches), and the next partial is loaded
  // while the current one is merged.
  deg_empty(a);
  DegPartial nxt;
  if (lane < G) nxt = ld_partial_cg(parts + lane * kMaxDegrees + warp);
#pragma unroll 1
  for (int b = lane; b < G; b += 32) {
    const DegPartial cur = nxt;
    if (b + 32 < G) nxt = ld_partial_cg(parts + (b + 32) * kMaxDegrees + warp);
    deg_merge(a, cur);
  }
#pragma unroll 1
  for (int o = 16; o > 0; o >>= 1) {
    const DegPartial other = deg_shfl_xor(a, o);
    deg_merge(a, other);
  }
  ds.zero();
  if (a.m != -INFINITY) {
    float4 h = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);  // (m, arg, S, S2)
    if (lane < G) h = __ldcg(reinterpret_cast<const float4*>(parts + lane * kMaxDegrees + warp));
#pragma unroll 1
    for (int b = lane; b < G; b += 32) {
      const float4 cur = h;
      if (b + 32 < G)
        h = __ldcg(reinterpret_cast<const float4*>(parts + (b + 32) * kMaxDegrees + warp));
      ds.add(cur.x, make_float2(cur.z, 0.0f), make_float2(cur.w, 0.0f), a.m);
    }
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
// second moments, double-float sums around each degree's maximum), its particle
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
