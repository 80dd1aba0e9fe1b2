// One group of line-fitting traces (Fig. 1) run by one block, with the
// normalisation and posterior reduction of the group fused in (§3.6.2).
//
// The paper notes that branching on the sampled degree costs its GPU code
// performance (§5.1).  Here the block first draws every trace's degree and
// coefficients (counter-addressed, so independent of order), sorts the group
// by degree with a deterministic counting sort in shared memory, and lets each
// warp evaluate 128 consecutive sorted traces with a Horner chain specialised
// to the warp's largest coefficient count.  Warps are then uniform except the
// few that straddle two degrees, which pad the shorter traces with zero
// coefficients (the same value exactly).  Each degree is a contiguous bucket of
// the sorted group, reduced by one warp into a per-degree partial.
#pragma once

#include "posterior.cuh"

namespace ppl {

constexpr int kCStride = 7;  // shared-memory stride of a trace's coefficients (odd: no bank conflicts)

// Shared memory of one group of kTpb * PPT traces.
template <int PPT>
struct TraceSmem {
  float c[kTpb * PPT * kCStride];
  float lw[kTpb * PPT];
  float corr[kTpb * PPT];  // log p - log q of a trace drawn from a proposal (0 under the prior)
  int idx[kTpb * PPT];
  int wcount[PPT][kTpb / 32][kMaxDegrees];
  int wbase[PPT][kTpb / 32][kMaxDegrees];
  int off[kMaxDegrees + 1];
  int nan;
};

template <int PPT>
__host__ __device__ constexpr size_t trace_smem_bytes() {
  return (sizeof(TraceSmem<PPT>) + 15) / 16 * 16;
}

// ss += sum over the staged points of (y - f(x))^2, f by Horner's rule over NC
// coefficients, for PPT traces at once.  Inner sums of 16 points are combined
// by a compensated (Kahan) sum.
template <int PPT, int NC>
__device__ __forceinline__ void accumulate_nc(const float2* sdata, int len,
                                              const float (&c)[PPT][kMaxCoef], float (&ss)[PPT],
                                              float (&comp)[PPT]) {
  int l = 0;
  while (l < len) {
    const int n = (len - l) < 16 ? (len - l) : 16;
    float part[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) part[q] = 0.0f;
    if (n == 16) {
#pragma unroll 4
      for (int j = 0; j < 16; ++j) {
        const float2 d = sdata[l + j];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          float f = c[q][NC - 1];
#pragma unroll
          for (int k = NC - 2; k >= 0; --k) f = fmaf(f, d.x, c[q][k]);
          const float r = d.y - f;
          part[q] = fmaf(r, r, part[q]);
        }
      }
    } else {
      for (int j = 0; j < n; ++j) {
        const float2 d = sdata[l + j];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          float f = c[q][NC - 1];
#pragma unroll
          for (int k = NC - 2; k >= 0; --k) f = fmaf(f, d.x, c[q][k]);
          const float r = d.y - f;
          part[q] = fmaf(r, r, part[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) kahan_add(ss[q], comp[q], part[q]);
    l += n;
  }
}

template <int PPT>
__device__ __forceinline__ void accumulate_dispatch(int nc, const float2* sdata, int len,
                                                    const float (&c)[PPT][kMaxCoef],
                                                    float (&ss)[PPT], float (&comp)[PPT]) {
  switch (nc) {
    case 0:
    case 1: accumulate_nc<PPT, 1>(sdata, len, c, ss, comp); break;
    case 2: accumulate_nc<PPT, 2>(sdata, len, c, ss, comp); break;
    case 3: accumulate_nc<PPT, 3>(sdata, len, c, ss, comp); break;
    case 4: accumulate_nc<PPT, 4>(sdata, len, c, ss, comp); break;
    case 5: accumulate_nc<PPT, 5>(sdata, len, c, ss, comp); break;
    default: accumulate_nc<PPT, 6>(sdata, len, c, ss, comp); break;
  }
}

// Draw policy of the prior (§3.4 `sample` from the model's own distributions):
// log-weight correction 0.
struct PriorDraw {
  PolyParams p;
  uint64_t seed;
  uint32_t instance;
  __device__ __forceinline__ int operator()(uint32_t i, float (&c)[kMaxCoef], float& corr) const {
    corr = 0.0f;
    return poly_draw(p, seed, instance, i, c);
  }
};

// Runs traces [base, base + kTpb * PPT) of an instance with N traces and reduces
// them into out[0..3] (per-degree partials).  Data: L points at xs, ys; when
// `resident` the caller has staged all of them in sdata, otherwise they
// stream through sdata in chunks of `chunk`.  lw_out / rec_out (optional) are
// indexed by trace index.  Every thread of the block must call it.
template <int PPT, class Draw>
__device__ __forceinline__ void trace_group(const Draw& draw, const PolyParams& p, const float* __restrict__ xs,
                                            const float* __restrict__ ys, int64_t L, int chunk,
                                            bool resident, float2* sdata, int64_t N,
                                            int64_t base, float* __restrict__ lw_out,
                                            ppl_poly_particle* __restrict__ rec_out,
                                            TraceSmem<PPT>& ts, DegPartial (&out)[kMaxDegrees]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  // A. draw, write the records, rank every trace within its degree
  float c[PPT][kMaxCoef], corr[PPT];
  int d[PPT], rank[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int64_t i = base + (int64_t)q * kTpb + tid;
    const int n = draw((uint32_t)(i < N ? i : 0), c[q], corr[q]);
    d[q] = (i < N) ? n - p.min_deg : -1;
    if (i < N && rec_out) {
      float4* dst = reinterpret_cast<float4*>(rec_out + i);
      dst[0] = make_float4(c[q][0], c[q][1], c[q][2], c[q][3]);
      dst[1] = make_float4(c[q][4], c[q][5], __int_as_float(n), __uint_as_float((uint32_t)i));
    }
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, d[q] == k);
      if (d[q] == k) rank[q] = __popc(m & lt);
      if (lane == 0) ts.wcount[q][warp][k] = __popc(m);
    }
  }
  __syncthreads();
  // exclusive offsets in (degree, q, warp) order: deterministic sorted order
  if (tid < kMaxDegrees) {
    int tot = 0;
    for (int q = 0; q < PPT; ++q)
      for (int w = 0; w < kTpb / 32; ++w) tot += ts.wcount[q][w][tid];
    ts.off[tid + 1] = tot;
  }
  if (tid == 0) ts.nan = 0;
  __syncthreads();
  if (tid == 0) {
    ts.off[0] = 0;
    for (int k = 0; k < kMaxDegrees; ++k) ts.off[k + 1] += ts.off[k];
  }
  __syncthreads();
  for (int e = tid; e < kMaxDegrees * PPT * (kTpb / 32); e += kTpb) {
    // running offset of (q, warp) within degree k, in (q, warp) order
    const int k = e % kMaxDegrees, qw = e / kMaxDegrees;
    const int q = qw / (kTpb / 32), w = qw % (kTpb / 32);
    int before = ts.off[k];
    for (int qq = 0; qq < PPT; ++qq)
      for (int ww = 0; ww < kTpb / 32; ++ww)
        if (qq * (kTpb / 32) + ww < qw) before += ts.wcount[qq][ww][k];
    ts.wbase[q][w][k] = before;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (d[q] < 0) continue;
    const int slot = ts.wbase[q][warp][d[q]] + rank[q];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) ts.c[slot * kCStride + k] = c[q][k];
    ts.corr[slot] = corr[q];
    ts.idx[slot] = (int)(base + (int64_t)q * kTpb + tid);
  }
  __syncthreads();
  const int n_valid = ts.off[kMaxDegrees];

  // B. evaluate: warp w owns sorted slots [128 w, 128 w + 128), lane l the
  // slots 128 w + 32 j + l; the Horner length is the warp's largest
  int slot[PPT];
  const bool active = warp * 32 * PPT < n_valid;
  const int wlast = min(warp * 32 * PPT + 32 * PPT, n_valid) - 1;
  int dlast = 0;
#pragma unroll
  for (int k = 1; k < kMaxDegrees; ++k)
    if (wlast >= ts.off[k]) dlast = k;
  const int nc = p.min_deg + dlast + p.coef_offset;
  float ss[PPT], comp[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    slot[j] = warp * 32 * PPT + 32 * j + lane;
    ss[j] = 0.0f;
    comp[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k)
      c[j][k] = (slot[j] < n_valid) ? ts.c[slot[j] * kCStride + k] : 0.0f;
  }
  if (resident) {
    if (active) accumulate_dispatch<PPT>(nc, sdata, (int)L, c, ss, comp);
  } else {
    for (int64_t l0 = 0; l0 < L; l0 += chunk) {
      const int len = (int)(L - l0 < (int64_t)chunk ? L - l0 : (int64_t)chunk);
      __syncthreads();
      for (int l = tid; l < len; l += kTpb) sdata[l] = make_float2(xs[l0 + l], ys[l0 + l]);
      __syncthreads();
      if (active) accumulate_dispatch<PPT>(nc, sdata, len, c, ss, comp);
    }
  }
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    if (slot[j] < n_valid) {
      const float lw = ss[j] * p.neg_half_inv_var + ts.corr[slot[j]];
      ts.lw[slot[j]] = lw;
      if (lw_out) lw_out[ts.idx[slot[j]]] = lw;
    }
  __syncthreads();

  // C. one warp per degree bucket: best trace, then sums around it
  if (warp < kMaxDegrees) {
    const int k = warp, s0 = ts.off[k], s1 = ts.off[k + 1];
    float m = -INFINITY;
    int a = 0x7fffffff, as = -1, nan = 0;
    for (int s = s0 + lane; s < s1; s += 32) {
      const float v = ts.lw[s];
      nan |= v != v;
      if (v > m || (v == m && ts.idx[s] < a)) {
        m = v;
        a = ts.idx[s];
        as = s;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, m, o);
      const int oa = __shfl_xor_sync(0xffffffffu, a, o);
      const int os = __shfl_xor_sync(0xffffffffu, as, o);
      if (om > m || (om == m && oa < a)) {
        m = om;
        a = oa;
        as = os;
      }
    }
    nan = __any_sync(0xffffffffu, nan);
    DegPartial r;
    deg_empty(r);
    r.m = m;
    r.arg = a;
    if (m > -INFINITY) {
      float ref[kMaxCoef];
#pragma unroll
      for (int j = 0; j < kMaxCoef; ++j) ref[j] = ts.c[as * kCStride + j];
      float S = 0.0f, S2 = 0.0f, A[kMaxCoef], B[kMaxCoef];
#pragma unroll
      for (int j = 0; j < kMaxCoef; ++j) {
        A[j] = 0.0f;
        B[j] = 0.0f;
      }
      for (int s = s0 + lane; s < s1; s += 32) {
        const float v = ts.lw[s];
        const float w = (v > -INFINITY) ? expf(v - m) : 0.0f;
        S += w;
        S2 = fmaf(w, w, S2);
#pragma unroll
        for (int j = 0; j < kMaxCoef; ++j) {
          const float dc = ts.c[s * kCStride + j] - ref[j];
          const float t = w * dc;
          A[j] += t;
          B[j] = fmaf(t, dc, B[j]);
        }
      }
      S = warp_sum(S);
      S2 = warp_sum(S2);
#pragma unroll
      for (int j = 0; j < kMaxCoef; ++j) {
        A[j] = warp_sum(A[j]);
        B[j] = warp_sum(B[j]);
      }
      r.S = S;
      r.S2 = S2;
      if (S > 0.0f) {
#pragma unroll
        for (int j = 0; j < kMaxCoef; ++j) {
          const float mean_shift = A[j] / S;
          r.mean[j] = ref[j] + mean_shift;
          r.M2[j] = fmaxf(B[j] - mean_shift * A[j], 0.0f);
        }
      }
    }
    if (lane == 0) {
      out[k] = r;
      if (nan) ts.nan = 1;
    }
  }
  __syncthreads();
}

}  // namespace ppl
