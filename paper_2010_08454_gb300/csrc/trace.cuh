// One group of line-fitting traces (Fig. 1) run by one block, with the
// normalisation and posterior reduction of the group fused in (§3.6.2).
//
// The paper notes that branching on the sampled degree costs its GPU code
// performance (§5.1).  Here the block first draws every trace's degree and
// coefficients (counter-addressed, so independent of order), sorts the group
// by degree with a deterministic counting sort in shared memory, and lets each
// warp evaluate rows of consecutive sorted traces with Horner chains
// specialised to each row's largest coefficient count.  Rows are uniform
// except the few that straddle two degrees, which pad the shorter traces with
// zero coefficients (the same value exactly).  Each warp pairs a row from the
// low-degree end of the sort with one from the high-degree end, so the warps
// of a block do nearly equal work and seldom wait at the group's barriers.
#pragma once

#include "posterior.cuh"
#include "suffstat.cuh"

namespace ppl {

constexpr int kCStride = 7;         // shared-memory stride of a trace's coefficients (odd: no bank conflicts)
constexpr float kSkipNats = 50.0f;  // traces this far below their degree's running maximum are skipped
constexpr int kSerialMerges = 4;    // up to this many traces a warp merges one at a time

// Shared memory of one group of kTpb * PPT traces.
template <int PPT>
struct TraceSmem {
  // coefficients of a trace at [slot * 7, slot * 7 + 6); [slot * 7 + 6] holds its
  // log p - log q when it was drawn from a proposal (0 under the prior)
  float c[kTpb * PPT * kCStride];
  int idx[kTpb * PPT];
  int wcount[PPT][kTpb / 32][kMaxDegrees];
  int wbase[PPT][kTpb / 32][kMaxDegrees];
  int off[kMaxDegrees + 1];
  int nan;
  DegPartial wrun[(kTpb / 32) * kMaxDegrees];  // each warp's running per-degree partials
  float ext_max[kMaxDegrees];  // known lower bounds of the final per-degree maxima (or -inf)
};

// Float <-> unsigned keys that order like the floats, with key 0 below every
// float (so a zeroed word means "no maximum yet" and atomicMax on it works).
__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Clear the warps' running partials (before the first group).
template <int PPT>
__device__ __forceinline__ void reset_warp_partials(TraceSmem<PPT>& ts) {
  for (int e = threadIdx.x; e < (kTpb / 32) * kMaxDegrees; e += blockDim.x) deg_empty(ts.wrun[e]);
  if (threadIdx.x < kMaxDegrees) ts.ext_max[threadIdx.x] = -INFINITY;
}

// Merge the warps' running partials into out[0..3] and clear them; every
// thread of the block must call it.  Warp 0 holds partial (warp w, degree d)
// in lane 8 d + w and merges by a three-round shuffle tree.
template <int PPT>
__device__ __forceinline__ void merge_warp_partials(TraceSmem<PPT>& ts,
                                                    DegPartial (&out)[kMaxDegrees]) {
  static_assert(kTpb / 32 == 8 && kMaxDegrees == 4, "one lane per (warp, degree)");
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, w = lane & 7, d = lane >> 3;
    DegPartial r = ts.wrun[w * kMaxDegrees + d];
    deg_empty(ts.wrun[w * kMaxDegrees + d]);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const DegPartial other = deg_shfl_xor(r, o);
      deg_merge(r, other);
    }
    if (w == 0) out[d] = r;
  }
  __syncthreads();
}

template <int PPT>
__host__ __device__ constexpr size_t trace_smem_bytes() {
  return (sizeof(TraceSmem<PPT>) + 15) / 16 * 16;
}

// Paired FP32 arithmetic (PTX f32x2, sm_100 and later): two lanes of IEEE
// single precision in one 64-bit register, each half rounded exactly as the
// scalar instruction would round it.  One instruction does the work of two,
// which halves the issue slots of the Horner chain below.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
  return v;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// One 32-byte record in a single 256-bit store (sm_100 and later; p 32-byte
// aligned): a warp's 32 consecutive records are then 32 whole sectors per
// instruction instead of two half-filled ones each.
__device__ __forceinline__ void st_global_v8(void* p, float a, float b, float c, float d, float e,
                                             float f, float g, float h) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d), "f"(e), "f"(f), "f"(g), "f"(h)
               : "memory");
}

// ss += sum over the staged points of (y - f(x))^2, f by Horner's rule over NC
// coefficients, for PPT traces at once (in pairs when PPT is even: the
// results are those of the scalar chain, bit for bit).  Inner sums of 16
// points are combined by a compensated (Kahan) sum.
template <int PPT, int NC>
__device__ __forceinline__ void accumulate_nc(const float2* sdata, int len,
                                              const float (&c)[PPT][kMaxCoef], float (&ss)[PPT],
                                              float (&comp)[PPT]) {
  if constexpr (PPT % 2 == 0) {
    constexpr int NP = PPT / 2;
    unsigned long long cc[NP][NC];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int k = 0; k < NC; ++k) cc[p][k] = f2_pack(c[2 * p][k], c[2 * p + 1][k]);
    int l = 0;
    while (l < len) {
      const int n = (len - l) < 16 ? (len - l) : 16;
      unsigned long long part[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) part[p] = 0ull;  // +0.0f in both halves
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        const float2 d = sdata[l + j];
        const unsigned long long xx = f2_pack(d.x, d.x), yy = f2_pack(d.y, d.y);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          unsigned long long f = cc[p][NC - 1];
#pragma unroll
          for (int k = NC - 2; k >= 0; --k) f = f2_fma(f, xx, cc[p][k]);
          const unsigned long long r = f2_sub(yy, f);
          part[p] = f2_fma(r, r, part[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float2 v = f2_unpack(part[p]);
        kahan_add(ss[2 * p], comp[2 * p], v.x);
        kahan_add(ss[2 * p + 1], comp[2 * p + 1], v.y);
      }
      l += n;
    }
  } else {
    int l = 0;
    while (l < len) {
      const int n = (len - l) < 16 ? (len - l) : 16;
      float part[PPT];
#pragma unroll
      for (int q = 0; q < PPT; ++q) part[q] = 0.0f;
#pragma unroll 4
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
#pragma unroll
      for (int q = 0; q < PPT; ++q) kahan_add(ss[q], comp[q], part[q]);
      l += n;
    }
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

// One pass over the staged points for traces J0 .. J0 + 3 as two f32x2 pairs
// with their own Horner lengths: (J0, J0 + 1) over NCA coefficients and
// (J0 + 2, J0 + 3) over NCB (NCB = 0: the second pair has no traces).  The
// per-trace arithmetic is that of accumulate_nc, bit for bit.
template <int PPT, int J0, int NCA, int NCB>
__device__ __forceinline__ void accumulate_two(const float2* sdata, int len,
                                               const float (&c)[PPT][kMaxCoef], float (&ss)[PPT],
                                               float (&comp)[PPT]) {
  static_assert(NCA >= 1 && (NCB == 0 || NCB >= NCA) && J0 + 3 < PPT, "sorted pair rows");
  constexpr int NB = NCB > 0 ? NCB : 1;
  unsigned long long ca[NCA], cb[NB];
#pragma unroll
  for (int k = 0; k < NCA; ++k) ca[k] = f2_pack(c[J0][k], c[J0 + 1][k]);
#pragma unroll
  for (int k = 0; k < NB; ++k) cb[k] = f2_pack(c[J0 + 2][k], c[J0 + 3][k]);
  int l = 0;
  while (l < len) {
    const int n = (len - l) < 16 ? (len - l) : 16;
    unsigned long long pa = 0ull, pb = 0ull;  // +0.0f in both halves
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const float2 d = sdata[l + j];
      const unsigned long long xx = f2_pack(d.x, d.x), yy = f2_pack(d.y, d.y);
      unsigned long long f = ca[NCA - 1];
#pragma unroll
      for (int k = NCA - 2; k >= 0; --k) f = f2_fma(f, xx, ca[k]);
      const unsigned long long r = f2_sub(yy, f);
      pa = f2_fma(r, r, pa);
      if constexpr (NCB > 0) {
        unsigned long long g = cb[NCB - 1];
#pragma unroll
        for (int k = NCB - 2; k >= 0; --k) g = f2_fma(g, xx, cb[k]);
        const unsigned long long t = f2_sub(yy, g);
        pb = f2_fma(t, t, pb);
      }
    }
    const float2 va = f2_unpack(pa);
    kahan_add(ss[J0], comp[J0], va.x);
    kahan_add(ss[J0 + 1], comp[J0 + 1], va.y);
    if constexpr (NCB > 0) {
      const float2 vb = f2_unpack(pb);
      kahan_add(ss[J0 + 2], comp[J0 + 2], vb.x);
      kahan_add(ss[J0 + 3], comp[J0 + 3], vb.y);
    }
    l += n;
  }
}

template <int PPT, int J0, int NCA>
__device__ __forceinline__ void accumulate_two_b(int ncb, const float2* sdata, int len,
                                                 const float (&c)[PPT][kMaxCoef],
                                                 float (&ss)[PPT], float (&comp)[PPT]) {
  // ncb >= NCA by the sorted order, or 0 when the second pair row is empty
  switch (ncb) {
    case 0: accumulate_two<PPT, J0, NCA, 0>(sdata, len, c, ss, comp); break;
    case 1:
      if constexpr (NCA <= 1) accumulate_two<PPT, J0, NCA, 1>(sdata, len, c, ss, comp);
      break;
    case 2:
      if constexpr (NCA <= 2) accumulate_two<PPT, J0, NCA, 2>(sdata, len, c, ss, comp);
      break;
    case 3:
      if constexpr (NCA <= 3) accumulate_two<PPT, J0, NCA, 3>(sdata, len, c, ss, comp);
      break;
    case 4:
      if constexpr (NCA <= 4) accumulate_two<PPT, J0, NCA, 4>(sdata, len, c, ss, comp);
      break;
    case 5:
      if constexpr (NCA <= 5) accumulate_two<PPT, J0, NCA, 5>(sdata, len, c, ss, comp);
      break;
    default: accumulate_two<PPT, J0, NCA, 6>(sdata, len, c, ss, comp); break;
  }
}

// Horner lengths nca <= ncb of the two pair rows (0: the row has no traces).
template <int PPT, int J0>
__device__ __forceinline__ void accumulate_two_dispatch(int nca, int ncb, const float2* sdata,
                                                        int len, const float (&c)[PPT][kMaxCoef],
                                                        float (&ss)[PPT], float (&comp)[PPT]) {
  switch (nca) {
    case 0: break;
    case 1: accumulate_two_b<PPT, J0, 1>(ncb, sdata, len, c, ss, comp); break;
    case 2: accumulate_two_b<PPT, J0, 2>(ncb, sdata, len, c, ss, comp); break;
    case 3: accumulate_two_b<PPT, J0, 3>(ncb, sdata, len, c, ss, comp); break;
    case 4: accumulate_two_b<PPT, J0, 4>(ncb, sdata, len, c, ss, comp); break;
    case 5: accumulate_two_b<PPT, J0, 5>(ncb, sdata, len, c, ss, comp); break;
    default: accumulate_two_b<PPT, J0, 6>(ncb, sdata, len, c, ss, comp); break;
  }
}

// Sorted slot of trace j of a lane.  With four or more traces per thread the
// sorted group is cut into pair rows of 64 slots (32 lanes x an f32x2 pair),
// and warp w takes pair rows w and 2W - 1 - w (then 2W + w and 4W - 1 - w): a
// row from the low-degree end of the sort with one from the high-degree end,
// so that the warps of a block do about equal work between its barriers.
// With fewer, warp w takes the 32 PPT consecutive slots from 32 PPT w.
template <int PPT>
__device__ __forceinline__ int sorted_slot(int warp, int lane, int j) {
  constexpr int W = kTpb / 32;
  if constexpr (PPT % 4 == 0) {
    const int p = j >> 1, r = p * W + ((p & 1) ? W - 1 - warp : warp);
    return 64 * r + 32 * (j & 1) + lane;
  } else {
    return warp * 32 * PPT + 32 * j + lane;
  }
}

// Degree index of a sorted slot, from the bucket offsets.
__device__ __forceinline__ int slot_degree(const int* off, int s) {
  int dk = 0;
#pragma unroll
  for (int k = 1; k < kMaxDegrees; ++k)
    if (s >= off[k]) dk = k;
  return dk;
}

// The factor sums of a lane's PPT traces over `len` staged points; nc[u] is
// the Horner length of the lane's u-th row group (pair row, or the warp's
// slots when PPT < 4), 0 when it holds no trace.
template <int PPT>
__device__ __forceinline__ void accumulate_rows(const int (&nc)[PPT], const float2* sdata,
                                                int len, const float (&c)[PPT][kMaxCoef],
                                                float (&ss)[PPT], float (&comp)[PPT]) {
  if constexpr (PPT % 4 == 0) {
    accumulate_two_dispatch<PPT, 0>(nc[0], nc[1], sdata, len, c, ss, comp);
    if constexpr (PPT == 8) accumulate_two_dispatch<PPT, 4>(nc[2], nc[3], sdata, len, c, ss, comp);
    static_assert(PPT <= 8, "at most two passes");
  } else {
    if (nc[0] > 0) accumulate_dispatch<PPT>(nc[0], sdata, len, c, ss, comp);
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

// A warp's candidates for its per-degree partials (phase C of trace_group).
template <int PPT>
struct Cands {
  float lw[PPT];
  int deg[PPT];
  int slot[PPT];
  unsigned cmask[PPT];
};

// More than kSerialMerges candidates folded into the warp's per-degree
// partials by warp reductions, one degree at a time.
template <int PPT>
__device__ __forceinline__ void merge_full(TraceSmem<PPT>* ts, const Cands<PPT> cd, int warp,
                                        int lane) {
  // the degrees that have candidates in this warp
  unsigned dmask = 0;
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    if ((cd.cmask[j] >> lane) & 1u) dmask |= 1u << cd.deg[j];
  dmask = __reduce_or_sync(0xffffffffu, dmask);
  for (int dd = 0; dd < kMaxDegrees; ++dd) {
    if (!((dmask >> dd) & 1u)) continue;
    float m = -INFINITY;
    int a = 0x7fffffff, as = -1;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const bool cj = (cd.cmask[j] >> lane) & 1u;
      if (cj && cd.deg[j] == dd) {
        const int ij = ts->idx[cd.slot[j]];
        if (cd.lw[j] > m || (cd.lw[j] == m && ij < a)) {
          m = cd.lw[j];
          a = ij;
          as = cd.slot[j];
        }
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
    if (!(m > -INFINITY)) continue;  // no finite candidate of this degree
    float ref[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) ref[k] = ts->c[as * kCStride + k];
    float S = 0.0f, S2 = 0.0f, A[kMaxCoef], B[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) {
      A[k] = 0.0f;
      B[k] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const bool cj = (cd.cmask[j] >> lane) & 1u;
      if (!cj || cd.deg[j] != dd) continue;
      const float w = (cd.lw[j] > -INFINITY) ? expf(cd.lw[j] - m) : 0.0f;
      S += w;
      S2 = fmaf(w, w, S2);
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) {
        const float dc = ts->c[cd.slot[j] * kCStride + k] - ref[k];
        const float t = w * dc;
        A[k] += t;
        B[k] = fmaf(t, dc, B[k]);
      }
    }
    S = warp_sum(S);
    S2 = warp_sum(S2);
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) {
      A[k] = warp_sum(A[k]);
      B[k] = warp_sum(B[k]);
    }
    if (lane == 0) {
      DegPartial r;
      deg_empty(r);
      r.m = m;
      r.arg = a;
      r.S = S;
      r.S2 = S2;
      if (S > 0.0f) {
#pragma unroll
        for (int k = 0; k < kMaxCoef; ++k) {
          const float sh = A[k] / S;
          r.mean[k] = ref[k] + sh;
          r.M2[k] = fmaxf(B[k] - sh * A[k], 0.0f);
        }
      }
      deg_merge(ts->wrun[warp * kMaxDegrees + dd], r);
    }
  }
}

// Runs traces [base, base + kTpb * PPT) of an instance with N traces and merges
// them into the warps' running per-degree partials (ts.wrun).  Data: L points at xs, ys; when
// `resident` the caller has staged all of them in sdata, otherwise they
// stream through sdata in chunks of `chunk`.  lw_out / rec_out (optional) are
// indexed by trace index.  Every thread of the block must call it.
template <int PPT, class Draw>
__device__ __forceinline__ void trace_group(const Draw& draw, const PolyParams& p, const float* __restrict__ xs,
                                            const float* __restrict__ ys, int64_t L, int chunk,
                                            bool resident, float2* sdata, int64_t N,
                                            int64_t base, float* __restrict__ lw_out,
                                            ppl_poly_particle* __restrict__ rec_out,
                                            TraceSmem<PPT>& ts, const SuffStat* suff = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const bool rec_v8 = (reinterpret_cast<uintptr_t>(rec_out) & 31) == 0;
  // A. draw, write the records, rank every trace within its degree
  float c[PPT][kMaxCoef], corr[PPT];
  int d[PPT], rank[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int64_t i = base + (int64_t)q * kTpb + tid;
    const int n = draw((uint32_t)(i < N ? i : 0), c[q], corr[q]);
    d[q] = (i < N) ? n - p.min_deg : -1;
    if (i < N && rec_out) {
      if (rec_v8) {
        st_global_v8(rec_out + i, c[q][0], c[q][1], c[q][2], c[q][3], c[q][4], c[q][5],
                     __int_as_float(n), __uint_as_float((uint32_t)i));
      } else {
        float4* dst = reinterpret_cast<float4*>(rec_out + i);
        dst[0] = make_float4(c[q][0], c[q][1], c[q][2], c[q][3]);
        dst[1] = make_float4(c[q][4], c[q][5], __int_as_float(n), __uint_as_float((uint32_t)i));
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, d[q] == k);
      if (d[q] == k) rank[q] = __popc(m & lt);
      if (lane == 0) ts.wcount[q][warp][k] = __popc(m);
    }
  }
  __syncthreads();
  // exclusive offsets in (degree, q, warp) order: deterministic sorted order.
  // One warp scans the 4 PPT 8 counts in that order; the scan at the first
  // entry of degree k is off[k], and every entry's scan is its wbase.
  if (warp == 0) {
    constexpr int W = kTpb / 32, E = kMaxDegrees * PPT * W, R = E / 32;
    static_assert(E % 32 == 0 && (PPT * W) % R == 0, "whole entries per lane");
    int v[R];
    int run = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int f = lane * R + r, k = f / (PPT * W), qw = f % (PPT * W);
      v[r] = run;
      run += ts.wcount[qw / W][qw % W][k];
    }
    int inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const int ex = inc - run;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int f = lane * R + r, k = f / (PPT * W), qw = f % (PPT * W);
      ts.wbase[qw / W][qw % W][k] = ex + v[r];
      if (qw == 0) ts.off[k] = ex + v[r];
    }
    if (lane == 31) ts.off[kMaxDegrees] = inc;
    if (lane == 0) ts.nan = 0;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (d[q] < 0) continue;
    const int slot = ts.wbase[q][warp][d[q]] + rank[q];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) ts.c[slot * kCStride + k] = c[q][k];
    ts.c[slot * kCStride + kMaxCoef] = corr[q];
    ts.idx[slot] = (int)(base + (int64_t)q * kTpb + tid);
  }
  __syncthreads();
  const int n_valid = ts.off[kMaxDegrees];

  // B. evaluate the lane's sorted slots (sorted_slot); each row group runs a
  // Horner chain as long as its largest coefficient count
  int slot[PPT], nc[PPT];
  float ss[PPT], comp[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    slot[j] = sorted_slot<PPT>(warp, lane, j);
    ss[j] = 0.0f;
    comp[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k)
      c[j][k] = (slot[j] < n_valid) ? ts.c[slot[j] * kCStride + k] : 0.0f;
  }
  {
    constexpr int G = PPT % 4 == 0 ? PPT / 2 : 1;  // row groups of a lane
    constexpr int span = PPT % 4 == 0 ? 64 : 32 * PPT;
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      nc[u] = 0;
      if (u < G) {
        const int first = sorted_slot<PPT>(warp, 0, PPT % 4 == 0 ? 2 * u : 0);
        if (first < n_valid) {
          const int last = min(first + span, n_valid) - 1;
          nc[u] = max(1, p.min_deg + slot_degree(ts.off, last) + p.coef_offset);
        }
      }
    }
  }
  if (suff != nullptr && suff->ok) {  // the same branch for the whole block
    // sufficient statistics: O(d^2) per trace, d its own coefficient count
#pragma unroll
    for (int j = 0; j < PPT; ++j)
      if (slot[j] < n_valid)
        ss[j] = suff_residual(*suff, c[j], p.min_deg + slot_degree(ts.off, slot[j]) + p.coef_offset);
  } else if (resident) {
    accumulate_rows<PPT>(nc, sdata, (int)L, c, ss, comp);
  } else {
    for (int64_t l0 = 0; l0 < L; l0 += chunk) {
      const int len = (int)(L - l0 < (int64_t)chunk ? L - l0 : (int64_t)chunk);
      __syncthreads();
      for (int l = tid; l < len; l += kTpb) sdata[l] = make_float2(xs[l0 + l], ys[l0 + l]);
      __syncthreads();
      accumulate_rows<PPT>(nc, sdata, len, c, ss, comp);
    }
  }
  // C. each warp folds its traces into its running per-degree partials.  A
  // trace more than kSkipNats below the running maximum of its degree carries
  // a weight below e^-50 of that maximum: even 2^31 such traces change no sum
  // by more than 4e-13 relative (below FP32 resolution), and the maximum only
  // grows, so such traces are skipped.  The rest are merged: one at a time by
  // lane 0 when there are few, otherwise by a warp reduction per degree.
  float lw[PPT];
  int deg[PPT];
  float thr[kMaxDegrees];
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k)
    thr[k] = fmaxf(ts.wrun[warp * kMaxDegrees + k].m, ts.ext_max[k]) - kSkipNats;
  int ncand = 0, nan = 0;
  unsigned cmask[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    deg[j] = -1;
    lw[j] = -INFINITY;
    bool cand = false;
    if (slot[j] < n_valid) {
      lw[j] = ss[j] * p.neg_half_inv_var + ts.c[slot[j] * kCStride + kMaxCoef];
      if (lw_out) lw_out[ts.idx[slot[j]]] = lw[j];
      const int dj = slot_degree(ts.off, slot[j]);
      deg[j] = dj;
      float t = thr[0];
#pragma unroll
      for (int k = 1; k < kMaxDegrees; ++k)
        if (dj == k) t = thr[k];
      cand = !(lw[j] <= t);  // NaN log-weights are candidates, so they are seen
      nan |= lw[j] != lw[j];
    }
    cmask[j] = __ballot_sync(0xffffffffu, cand);
    ncand += __popc(cmask[j]);
  }
  if (ncand > 0 && ncand <= kSerialMerges) {
    // few candidates: lane 0 merges each as a one-trace partial
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      unsigned msk = cmask[j];
      while (msk) {
        const int src = __ffs(msk) - 1;
        msk &= msk - 1;
        const float v = __shfl_sync(0xffffffffu, lw[j], src);
        const int dv = __shfl_sync(0xffffffffu, deg[j], src);
        const int sv = __shfl_sync(0xffffffffu, slot[j], src);
        if (lane == 0) {
          DegPartial r;
          deg_empty(r);
          r.m = v;
          r.arg = ts.idx[sv];
          if (v > -INFINITY) {
            r.S = 1.0f;
            r.S2 = 1.0f;
#pragma unroll
            for (int k = 0; k < kMaxCoef; ++k) r.mean[k] = ts.c[sv * kCStride + k];
          }
          deg_merge(ts.wrun[warp * kMaxDegrees + dv], r);
        }
      }
    }
  } else if (ncand > kSerialMerges) {
    Cands<PPT> cd;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      cd.lw[j] = lw[j];
      cd.deg[j] = deg[j];
      cd.slot[j] = slot[j];
      cd.cmask[j] = cmask[j];
    }
    merge_full<PPT>(&ts, cd, warp, lane);
  }
  nan = __any_sync(0xffffffffu, nan);
  if (lane == 0 && nan) ts.nan = 1;
  __syncthreads();
}

}  // namespace ppl
