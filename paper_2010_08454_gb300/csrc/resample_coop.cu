// Systematic resampling (the definition in resample.cu: 64-bit fixed-point
// weights q_i, T = sum q, stride = floor(T / M), u = floor(w stride / 2^32),
// a_k = min{j : C_j > u + k stride}) in one persistent, cooperative kernel
// with one grid barrier, and no prefix-sum array in global memory:
//
//   1. the particles are cut into chunks of 4096; blocks sum the weights of
//      their chunks (one read of lw), with one block barrier per 32 chunks;
//   2. barrier: the last arriving block scans the chunk totals, draws u, and
//      gives every chunk its first output K_c = #{k : u + k stride < C_start}
//      -- chunk c holds the ancestors of outputs [K_c, K_c+1) -- and cuts each
//      chunk's outputs into work items of at most 256;
//   3. each block takes a contiguous run of items (weighted so that a chunk's
//      prefix sums count as a number of items; a run never ends inside a
//      chunk with at most two outputs per particle); for each chunk the run
//      touches, the block forms the chunk's inclusive prefix sums in shared
//      memory (lw is L2-resident by now) with a two-level index of every 8th
//      and every 256th sum, and then its warps take the chunk's items
//      independently: a warp finds the item's range of candidate ancestors by
//      three 32-way probes of the index, and its lanes merge those prefix sums
//      with the item's sorted positions (merge path: Green, McColl, Bader, "GPU
//      merge path", ICS 2012), one equal slice of the merge per lane; an item
//      whose outputs all have one ancestor is filled directly.  With a record
//      buffer the warp then copies its outputs' records (the fused gather).
//      A chunk that lies wholly inside one block's run and has at most two
//      outputs per particle (near-uniform weights) is written instead in the
//      scatter form of the same definition: particle j's offspring are the
//      outputs [K(C_{j-1}), K(C_j)), K(c) = #{k : u + k stride < c}; the
//      block writes the chunk's ancestors into a table in shared memory,
//      then the ancestors and the records output by output.
//
// Every item costs at most 4096 weights and 256 outputs whatever the weights
// are: a chunk holding most of the mass (degenerate importance weights)
// becomes many items on many blocks and warps, with no block barrier between
// them.  The ancestors are those of the scan-and-search path bit for bit (both
// are exact integer computations of the same definition).  Traffic: lw twice
// (the second time from L2), the ancestors once, and with the gather every
// output's record once plus each distinct ancestor's record.
#include <algorithm>

#include "gridsync.cuh"
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

constexpr int kRcTpb = 512;                           // two blocks per SM
constexpr int kRcWarps = kRcTpb / 32;
constexpr int kRcItems = 8;                           // weights per thread per chunk
constexpr int64_t kRcChunk = (int64_t)kRcTpb * kRcItems;
constexpr int kRcItemOut = 256;                       // outputs of one work item (one warp)
constexpr int kRcBatch = 32;                          // chunks summed between block barriers
// A chunk's prefix sums cost a block about as much time as this many work
// items; every chunk with outputs is charged it in the partition of the
// items over the blocks, so that a block whose run crosses many sparsely
// used chunks takes correspondingly fewer items.
constexpr int kRcPrefixCost = 128;
constexpr int kRcShort = 4;      // offspring a lane writes alone in the scatter form
constexpr int kRcScatterOut = 2 * (int)kRcChunk;  // outputs of a chunk written in the scatter form
constexpr int kRcJobBlk = 8;     // chunk totals the layout job's first pass loads at once per thread
constexpr int kRcJobPer = 4;     // chunks per thread in a tile of the layout job
constexpr int kRcJobTile = kRcTpb * kRcJobPer;

// 16 bytes of log-weights, marked for eviction last from L2: lw is read
// again after the grid barrier (the prefix sums), while the records gathered
// in between stream through L2.
__device__ __forceinline__ float4 ld_f4_evict_last(const float4* ptr) {
  float4 v;
  asm volatile(
      "{\n .reg .b64 pol;\n createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n"
      " ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], pol;\n}"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(ptr));
  return v;
}

struct RcArgs {
  const float* lw;         // FP32 log-weights, or
  const uint64_t* qf;      // given fixed-point weights
  const double* known_max;
  WsHeader* hdr;
  int64_t n, m;
  uint64_t seed;
  uint32_t instance, t;
  int32_t* anc;
  const int32_t* gate;
  GridCtl* g;
  int64_t n_chunks;
  uint64_t* ctot;   // [n_chunks] chunk totals, then their exclusive prefix
  int64_t* kfirst;  // [n_chunks + 1] first output of each chunk (K_c), K_last = m
  int64_t* ioff;    // [n_chunks + 1] first work item of each chunk
  // fused gather (rec_words > 0): rec_out[k] = rec_in[a_k], records of
  // rec_words words of 16 bytes (or of 4 bytes when rec_word4), rec_in
  // holding the n particles' records
  const void* rec_in;
  void* rec_out;
  int32_t rec_words;
  int32_t rec_word4;
  // one shard of a population split over devices (planned != 0): the
  // weights are quantised for a population of n_scale particles, the layout
  // (stride, u) and this shard's exclusive prefix c_base are given, its
  // outputs are [k_off, k_end) of m, ancestors[k - k_off] = j_off + local
  // ancestor, rec_out[k - k_off]
  int64_t n_scale;
  int32_t planned;
  uint64_t p_stride, p_u, c_base;
  int64_t k_off, k_end, j_off;
};

// The records of outputs k0 .. k0 + nB - 1 of an item, by one warp: output j
// copies the record of ancestor anc_of(j); consecutive lanes take consecutive
// words, so both the loads (ancestors are non-decreasing) and the stores are
// coalesced.
template <typename V, class AncOf>
__device__ __forceinline__ void gather_words(const V* in, V* out_all, int W, int64_t k0, int nB,
                                             AncOf anc_of, int lane) {
  const int total = nB * W;
  V* out = out_all + k0 * W;
  if (W == 1) {
    for (int e = lane; e < total; e += 32) out[e] = in[anc_of(e)];
  } else if (W == 2) {
    for (int e = lane; e < total; e += 32) out[e] = in[(int64_t)anc_of(e >> 1) * 2 + (e & 1)];
  } else {
    for (int e = lane; e < total; e += 32) {
      const int j = e / W;
      out[e] = in[(int64_t)anc_of(j) * W + (e - j * W)];
    }
  }
}

template <class AncOf>
__device__ __forceinline__ void gather_item(const RcArgs& a, int64_t k0, int nB, AncOf anc_of,
                                            int lane) {
  if (a.rec_word4)
    gather_words(reinterpret_cast<const uint32_t*>(a.rec_in), reinterpret_cast<uint32_t*>(a.rec_out),
                 a.rec_words, k0, nB, anc_of, lane);
  else
    gather_words(reinterpret_cast<const uint4*>(a.rec_in), reinterpret_cast<uint4*>(a.rec_out),
                 a.rec_words, k0, nB, anc_of, lane);
}

// The records of outputs k0 .. k0 + n - 1 by the whole block, from the
// ancestors in shared memory: thread t copies words t, t + kRcTpb, .., four
// loads in flight before their stores (coalesced on both sides, the
// ancestors being non-decreasing).
template <typename V>
__device__ __forceinline__ void gather_block_words(const V* __restrict__ in, V* __restrict__ out,
                                                   int W, int64_t k0, int n, const int32_t* sOut,
                                                   int tid) {
  const int total = n * W;
  out += k0 * W;
  for (int e0 = tid; e0 < total; e0 += 4 * kRcTpb) {
    V v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + q * kRcTpb;
      if (e < total) {
        const int j = e / W;
        v[q] = in[(int64_t)sOut[j] * W + (e - j * W)];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + q * kRcTpb;
      if (e < total) out[e] = v[q];
    }
  }
}

__device__ __forceinline__ void gather_block(const RcArgs& a, int64_t k0, int n,
                                             const int32_t* sOut, int tid) {
  if (a.rec_word4)
    gather_block_words(reinterpret_cast<const uint32_t*>(a.rec_in),
                       reinterpret_cast<uint32_t*>(a.rec_out), a.rec_words, k0, n, sOut, tid);
  else
    gather_block_words(reinterpret_cast<const uint4*>(a.rec_in), reinterpret_cast<uint4*>(a.rec_out),
                       a.rec_words, k0, n, sOut, tid);
}

// The weights of one thread's kRcItems particles from `base`: FP32
// log-weights (raw, -inf past n) or given fixed-point words (0 past n).
template <bool FROM_LW>
struct RawWeights {
  float v[kRcItems];
};
template <>
struct RawWeights<false> {
  uint64_t v[kRcItems];
};

template <bool FROM_LW>
__device__ __forceinline__ void load_raw(const RcArgs& a, int64_t base, RawWeights<FROM_LW>& w) {
  if constexpr (FROM_LW) {
    if (base + kRcItems <= a.n && (reinterpret_cast<uintptr_t>(a.lw + base) & 15) == 0) {
      const float4 x = ld_f4_evict_last(reinterpret_cast<const float4*>(a.lw + base));
      const float4 y = ld_f4_evict_last(reinterpret_cast<const float4*>(a.lw + base) + 1);
      w.v[0] = x.x; w.v[1] = x.y; w.v[2] = x.z; w.v[3] = x.w;
      w.v[4] = y.x; w.v[5] = y.y; w.v[6] = y.z; w.v[7] = y.w;
    } else {
#pragma unroll
      for (int r = 0; r < kRcItems; ++r)
        w.v[r] = base + r < a.n ? __ldcg(a.lw + base + r) : -INFINITY;
    }
  } else {
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) w.v[r] = base + r < a.n ? __ldcg(a.qf + base + r) : 0ull;
  }
}

// Fixed-point weights from raw ones (log-weights quantised against m_lw).
// A log-weight more than 44.5 below the maximum quantises to 0; when that
// holds for all of a warp's weights (most of them, for degenerate importance
// weights) the exponentials are skipped.
template <bool FROM_LW>
__device__ __forceinline__ void to_fixed(const RawWeights<FROM_LW>& w, float m_lw, float scale,
                                         uint64_t (&q)[kRcItems], int& bad) {
  if constexpr (FROM_LW) {
    bool near = false;
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) {
      // a log-weight above the maximum is an error (a wrong known maximum);
      // otherwise q <= 2^S and no sum of the n weights exceeds 2^61
      bad |= w.v[r] > m_lw;
      near |= __fsub_rn(w.v[r], m_lw) >= -44.5f;
      q[r] = 0ull;
    }
    if (__any_sync(0xffffffffu, near)) {
#pragma unroll
      for (int r = 0; r < kRcItems; ++r)
        q[r] = w.v[r] > m_lw ? 0ull : quantize(w.v[r], m_lw, scale);
    }
  } else {
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) {
      bad |= w.v[r] > (1ull << 61);
      q[r] = w.v[r] > kLimit ? kLimit : w.v[r];
    }
  }
}

template <bool FROM_LW>
__device__ __forceinline__ void load_weights(const RcArgs& a, int64_t base, float m_lw, float scale,
                                             uint64_t (&q)[kRcItems], int& bad) {
  RawWeights<FROM_LW> w;
  load_raw<FROM_LW>(a, base, w);
  to_fixed<FROM_LW>(w, m_lw, scale, q, bad);
}

// Sums of fixed-point weights: plain for quantised log-weights (they cannot
// pass 2^61, see to_fixed), saturating for given fixed-point words.
template <bool FROM_LW>
__device__ __forceinline__ uint64_t acc_add(uint64_t a, uint64_t b) {
  if constexpr (FROM_LW) return a + b;
  else return sat_add(a, b);
}

template <bool FROM_LW>
__device__ __forceinline__ uint64_t warp_sum_acc(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = acc_add<FROM_LW>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <bool FROM_LW>
__device__ __forceinline__ uint64_t warp_scan_acc(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = acc_add<FROM_LW>(v, u);
  }
  return v;
}

// First j in [lo, hi) with v[j] > x, by one warp over a sorted global array
// (hi if none): each round the 32 lanes probe 32 evenly spaced entries.
__device__ __forceinline__ int64_t warp_first_above(const int64_t* v, int64_t lo, int64_t hi,
                                                    int64_t x, int lane) {
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t q = lo + (int64_t)(lane + 1) * step - 1;
    const unsigned m = __ballot_sync(0xffffffffu, q >= hi || __ldcg(v + q) > x);
    if (m == 0) return hi;  // every probe below hi holds <= x, lane 31 probes hi - 1
    const int f = __ffs(m) - 1;
    const int64_t qf = lo + (int64_t)(f + 1) * step - 1;
    lo = lo + (int64_t)f * step;  // probe f - 1 holds <= x
    hi = qf < hi ? qf : hi;       // the answer is at most probe f
  }
  const int64_t q = lo + lane;
  const unsigned m = __ballot_sync(0xffffffffu, q < hi && __ldcg(v + q) > x);
  return m ? lo + __ffs(m) - 1 : hi;
}

// First index of the chunk's prefix sums sA[0..kRcChunk) above x, by one
// warp, for x below the chunk's last sum: the first 256-block whose last sum
// is above x (L1: every 256th sum), then the first 8-block within it (L2:
// every 8th), then the entry.  Each probe reads at most 32 consecutive words.
__device__ __forceinline__ int chunk_first_above(const uint64_t* sA, const uint64_t* sL2,
                                                 const uint64_t* sL1, uint64_t x, int lane) {
  constexpr int nL1 = (int)(kRcChunk / 256);
  static_assert(kRcChunk % 256 == 0 && nL1 <= 32, "three levels of at most 32");
  unsigned m = __ballot_sync(0xffffffffu, lane < nL1 && sL1[lane < nL1 ? lane : 0] > x);
  const int f1 = m ? __ffs(m) - 1 : nL1 - 1;
  m = __ballot_sync(0xffffffffu, sL2[32 * f1 + lane] > x);
  const int t = 8 * (32 * f1 + (m ? __ffs(m) - 1 : 31));
  m = __ballot_sync(0xffffffffu, lane < 8 && sA[t + (lane & 7)] > x);
  return t + (m ? __ffs(m) - 1 : 7);
}

// Descriptor of the chunk that holds cost unit `it` (the last chunk with
// ioff <= it), by one warp: chunk, ioff of it and of the next, first output
// of it and of the next, and its prefix start.  With a hint (a chunk whose
// ioff is it) the warp first probes the 32 chunks from the hint at once, so
// the next chunk of a run costs one round trip; otherwise, or when all 32 lie
// at or below it, a 32-way search.  ioff[0] = 0 <= it < ioff[n_chunks].
__device__ __forceinline__ void seg_lookup(const RcArgs& a, int64_t it, int64_t hint, int64_t* out,
                                           int lane) {
  int64_t ch = -1;
  if (hint >= 0) {
    const int64_t q = hint + lane;
    const unsigned m = __ballot_sync(0xffffffffu, q <= a.n_chunks && __ldcg(a.ioff + q) <= it);
    if (m != 0xffffffffu) ch = hint + __popc(m) - 1;  // ioff is non-decreasing: m is a prefix
  }
  if (ch < 0) ch = warp_first_above(a.ioff, hint > 0 ? hint : 0, a.n_chunks + 1, it, lane) - 1;
  ch = ch < 0 ? 0 : (ch < a.n_chunks ? ch : a.n_chunks - 1);
  int64_t v = ch;
  if (lane == 1) v = __ldcg(a.ioff + ch);
  if (lane == 2) v = __ldcg(a.ioff + ch + 1);
  if (lane == 3) v = __ldcg(a.kfirst + ch);
  if (lane == 4) v = __ldcg(a.kfirst + ch + 1);
  if (lane == 5) v = (int64_t)__ldcg(a.ctot + ch);
  if (lane < 6) out[lane] = v;
}

template <bool FROM_LW>
__global__ void __launch_bounds__(kRcTpb, 2) resample_coop_kernel(RcArgs a) {
  if (a.gate && *a.gate == 0) return;  // every block reads the same flag
  extern __shared__ __align__(16) unsigned char rc_dyn[];
  uint64_t* sA = reinterpret_cast<uint64_t*>(rc_dyn);  // [kRcChunk] prefix sums of a chunk
  uint64_t* sL2 = sA + kRcChunk;                        // [kRcTpb] every 8th of them
  int32_t* sW = reinterpret_cast<int32_t*>(sL2 + kRcTpb);  // [warp][kRcItemOut] ancestors
  int32_t* sOut = sW + kRcWarps * kRcItemOut;  // [kRcScatterOut] a scattered chunk's ancestors
  __shared__ uint64_t sL1[kRcChunk / 256];  // every 256th prefix sum
  static_assert(3 * kRcJobTile * 8 <= kRcChunk * 8 + kRcTpb * 8 + kRcWarps * kRcItemOut * 4,
                "the layout job's tile tables fit in the dynamic shared memory");
  __shared__ uint64_t wtot[kRcWarps], jtot[kRcWarps];
  __shared__ int64_t jitem[kRcWarps];
  __shared__ unsigned long long rel;
  __shared__ uint64_t view[3];  // T, stride, u
  __shared__ int64_t seg_sh[2][6];  // chunk, its first and end unit, first and end output, C at its start
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  float m_lw = 0.0f, scale = 0.0f;
  if (FROM_LW) {
    m_lw = a.known_max ? (float)*a.known_max : a.hdr->max_lw;
    int S = 0;
    while (((int64_t)1 << S) < a.n_scale) ++S;
    scale = __int_as_float((127 + 61 - S) << 23);  // 2^(61 - ceil(log2 n))
  }

  // 1. chunk totals: block b sums chunks b, b + G, ...; warps leave their
  // partial sums of up to kRcBatch chunks in shared memory (aliasing sW), two
  // chunks' loads in flight per thread, and warp r then adds chunk r's
  int bad = 0;
  {
    uint64_t* wt = reinterpret_cast<uint64_t*>(sW);  // [kRcBatch][kRcWarps]
    static_assert(kRcBatch * kRcWarps * 8 <= kRcWarps * kRcItemOut * 4, "fits in sW");
    const int64_t nk = a.n_chunks > (int64_t)blockIdx.x
                           ? (a.n_chunks - (int64_t)blockIdx.x + G - 1) / G : 0;
    for (int64_t k0 = 0; k0 < nk; k0 += kRcBatch) {
      const int nb = (int)(nk - k0 < kRcBatch ? nk - k0 : kRcBatch);
      // kP1 chunks' loads in flight per thread (two for 64-bit input words)
      constexpr int kP1 = FROM_LW ? 4 : 2;
      static_assert(kRcBatch % kP1 == 0, "whole rounds per batch");
      for (int r = 0; r < nb; r += kP1) {
        RawWeights<FROM_LW> w[kP1];
#pragma unroll
        for (int i = 0; i < kP1; ++i)
          if (r + i < nb)
            load_raw<FROM_LW>(a, ((int64_t)blockIdx.x + (k0 + r + i) * G) * kRcChunk +
                                     (int64_t)tid * kRcItems, w[i]);
#pragma unroll
        for (int i = 0; i < kP1; ++i) {
          if (r + i >= nb) break;  // the same for the whole block
          uint64_t q[kRcItems], t = 0;
          to_fixed<FROM_LW>(w[i], m_lw, scale, q, bad);
#pragma unroll
          for (int e = 0; e < kRcItems; ++e) t = acc_add<FROM_LW>(t, q[e]);
          t = warp_sum_acc<FROM_LW>(t);
          if (lane == 0) wt[(r + i) * kRcWarps + warp] = t;
        }
      }
      __syncthreads();
      for (int r = warp; r < nb; r += kRcWarps) {
        const uint64_t t = warp_sum_acc<FROM_LW>(lane < kRcWarps ? wt[r * kRcWarps + lane] : 0ull);
        if (lane == 0) a.ctot[(int64_t)blockIdx.x + (k0 + r) * G] = t;
      }
      __syncthreads();  // wt is rewritten by the next batch
    }
  }
  if (bad) record_status(&a.hdr->status, PPL_EINVAL);
  // 2. barrier: the last block scans the chunk totals, checks T, draws u, and
  // lays out the work items; the item count is the release word's payload
  const bool ok = grid_sync<true>(a.g, &a.hdr->status, G, 1, &rel, [&]() -> unsigned long long {
    // T, the saturating sum of the chunk totals: coalesced loads, kRcJobBlk
    // in flight per thread
    uint64_t run = 0;
    for (int64_t c0 = tid; c0 < a.n_chunks; c0 += (int64_t)kRcTpb * kRcJobBlk) {
      uint64_t t[kRcJobBlk];
#pragma unroll
      for (int r = 0; r < kRcJobBlk; ++r) {
        const int64_t c = c0 + (int64_t)r * kRcTpb;
        t[r] = c < a.n_chunks ? __ldcg(a.ctot + c) : 0ull;
      }
#pragma unroll
      for (int r = 0; r < kRcJobBlk; ++r) run = sat_add(run, t[r]);
    }
    run = warp_sum_acc<false>(run);
    if (lane == 0) jtot[warp] = run;
    __syncthreads();
    const uint64_t T = warp_sum_acc<false>(lane < kRcWarps ? jtot[lane] : 0ull);
    bool valid;
    uint64_t stride = 0, u = 0;
    if (a.planned) {  // a shard: the population's layout is given
      valid = T <= (1ull << 61) && a.p_stride > 0;
      stride = a.p_stride;
      u = a.p_u;
    } else {
      valid = T > 0 && T <= (1ull << 61) && T >= (uint64_t)a.m;
      if (valid) {
        stride = T / (uint64_t)a.m;
        const uint64_t w = philox_block(a.seed, 0, a.instance, a.t, kResample, 0).x;
        u = (__umul64hi(w, stride) << 32) | ((w * stride) >> 32);
      }
    }
    const DivInv sv = div_inv(stride);
    // a chunk with outputs costs its items plus kRcPrefixCost
    auto cost = [](int64_t k0, int64_t k1) -> int64_t {
      return k1 > k0 ? (k1 - k0 + kRcItemOut - 1) / kRcItemOut + kRcPrefixCost : 0;
    };
    // Tiles of kRcJobTile chunks: the totals come into shared memory with
    // coalesced loads; thread t takes the tile's chunks kRcJobPer t ..
    // kRcJobPer t + kRcJobPer - 1 in order, the block scans the exclusive
    // prefixes C, the first outputs K = positions_below(C) and the cost units
    // (ioff); the three tables leave with coalesced stores.
    uint64_t* jC = reinterpret_cast<uint64_t*>(rc_dyn);
    int64_t* jK = reinterpret_cast<int64_t*>(rc_dyn + kRcJobTile * 8);
    int64_t* jI = reinterpret_cast<int64_t*>(rc_dyn + 2 * kRcJobTile * 8);
    uint64_t carry_c = a.planned ? a.c_base : 0ull;  // prefixes in the population's terms
    int64_t carry_i = 0;
    for (int64_t t0 = 0; t0 < a.n_chunks; t0 += kRcJobTile) {
      const int nt = (int)(a.n_chunks - t0 < kRcJobTile ? a.n_chunks - t0 : kRcJobTile);
      __syncthreads();  // jtot, jitem and the previous tile's tables have been read
      for (int i = tid; i < kRcJobTile; i += kRcTpb) jC[i] = i < nt ? __ldcg(a.ctot + t0 + i) : 0ull;
      __syncthreads();
      uint64_t cs[kRcJobPer + 1];  // the prefix at each of this thread's chunks, then past the last
      uint64_t own = 0;
#pragma unroll
      for (int r = 0; r < kRcJobPer; ++r) own = sat_add(own, jC[tid * kRcJobPer + r]);
      const uint64_t inc = warp_scan_u64(own, lane);
      if (lane == 31) jtot[warp] = inc;
      __syncthreads();
      const uint64_t jv = lane < kRcWarps ? jtot[lane] : 0ull, ji = warp_scan_u64(jv, lane);
      cs[0] = sat_add(carry_c, sat_add(__shfl_sync(0xffffffffu, ji - jv, warp), inc - own));
#pragma unroll
      for (int r = 0; r < kRcJobPer; ++r) cs[r + 1] = sat_add(cs[r], jC[tid * kRcJobPer + r]);
      int64_t k[kRcJobPer + 1];  // independent divisions
#pragma unroll
      for (int r = 0; r <= kRcJobPer; ++r) k[r] = valid ? positions_below_inv(cs[r], u, sv, a.m) : 0;
      int64_t own_i = 0;
#pragma unroll
      for (int r = 0; r < kRcJobPer; ++r) own_i += cost(k[r], k[r + 1]);
      int64_t ii = own_i;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, ii, o);
        if (lane >= o) ii += y;
      }
      if (lane == 31) jitem[warp] = ii;
      __syncthreads();
      const int64_t iv = lane < kRcWarps ? jitem[lane] : 0;
      int64_t iw = iv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, iw, o);
        if (lane >= o) iw += y;
      }
      int64_t ix = carry_i + __shfl_sync(0xffffffffu, iw - iv, warp) + (ii - own_i);
#pragma unroll
      for (int r = 0; r < kRcJobPer; ++r) {
        const int e = tid * kRcJobPer + r;
        jC[e] = cs[r];
        jK[e] = k[r];
        jI[e] = ix;
        ix += cost(k[r], k[r + 1]);
      }
      carry_c = sat_add(carry_c, __shfl_sync(0xffffffffu, ji, 31));
      carry_i += __shfl_sync(0xffffffffu, iw, 31);
      __syncthreads();
      for (int i = tid; i < nt; i += kRcTpb) {
        a.ctot[t0 + i] = jC[i];
        a.kfirst[t0 + i] = jK[i];
        a.ioff[t0 + i] = jI[i];
      }
    }
    const int64_t n_items = carry_i;
    if (tid == 0) {
      if (!a.planned && T == 0) record_status(&a.hdr->status, PPL_EEMPTY);
      else if (!valid) record_status(&a.hdr->status, PPL_EINVAL);
      a.g->total = T;
      a.g->stride = stride;
      a.g->offset = u;
      a.kfirst[a.n_chunks] = a.planned ? a.k_end : a.m;
      a.ioff[a.n_chunks] = n_items;
    }
    return valid ? (unsigned long long)n_items : 0ull;
  }, [&] {
    view[0] = __ldcg(&a.g->total);
    view[1] = __ldcg(&a.g->stride);
    view[2] = __ldcg(&a.g->offset);
  });
  if (!ok) return;
  const int64_t n_items = (int64_t)(rel & ((1ull << 34) - 1));
  const uint64_t stride = view[1], u = view[2];
  const DivInv sv = div_inv(stride);

  // 3. work items: block b takes the contiguous run [I b / G, I (b + 1) / G)
  // of cost units and walks it chunk by chunk.  Chunk c's units are
  // [ioff_c, ioff_c+1): kRcPrefixCost that stand for its prefix sums, then one
  // per item; a run that holds none of the chunk's items skips the chunk.
  // An end of the run that falls inside a chunk with at most kRcScatterOut
  // outputs moves to the nearer end of that chunk (block b's last end is
  // block b + 1's first, moved the same way), so such a chunk is never split
  // between two blocks: one block builds its prefix sums and writes it in the
  // scatter form.  Moving the ends is monotone, so the runs still tile the
  // units in order.
  int64_t it1 = n_items * (blockIdx.x + 1) / G;
  int32_t* sWw = sW + warp * kRcItemOut;
  int64_t it = n_items * blockIdx.x / G;
  {
    __shared__ int64_t ends[2];
    if (warp < 2) {  // warp 0 the first end, warp 1 the last
      int64_t x = warp == 0 ? it : it1;
      if (x > 0 && x < n_items) {
        seg_lookup(a, x, -1, seg_sh[warp], lane);
        __syncwarp();
        const int64_t io0 = seg_sh[warp][1], io1 = seg_sh[warp][2];
        if (seg_sh[warp][4] - seg_sh[warp][3] <= kRcScatterOut)
          x = 2 * (x - io0) <= io1 - io0 ? io0 : io1;
      }
      if (lane == 0) ends[warp] = x;
    }
    __syncthreads();
    // warp 0's descriptor is the first chunk's unless the first end moved
    // (or was not looked up)
    const bool again = ends[0] != it || it == 0;
    it = ends[0];
    it1 = ends[1];
    __syncthreads();  // seg_sh[1] is the next chunk's slot from here on
    if (warp == 0 && it < it1 && again) seg_lookup(a, it, -1, seg_sh[0], lane);
  }
  __syncthreads();
  for (int cur = 0; it < it1; cur ^= 1) {
    const int64_t ch = seg_sh[cur][0], io0 = seg_sh[cur][1];
    const int64_t io1 = seg_sh[cur][2] < it1 ? seg_sh[cur][2] : it1;
    const int64_t kc = seg_sh[cur][3], kn = seg_sh[cur][4];
    const uint64_t cstart = (uint64_t)seg_sh[cur][5];
    const bool more = io1 < it1;  // another chunk follows in this block's run
    const int64_t cb = ch * kRcChunk;
    const int64_t xs = it > io0 + kRcPrefixCost ? it : io0 + kRcPrefixCost;  // first item unit
    // a chunk wholly inside this block's run, with at most two outputs per
    // particle on average, is written in the scatter form (below)
    const int nCw = (int)(a.n - cb < kRcChunk ? a.n - cb : kRcChunk);
    const bool scatter = it <= io0 && seg_sh[cur][2] <= it1 && kn - kc <= kRcScatterOut;
    if (xs < io1) {  // the same for every thread of the block: the chunk's inclusive
      // prefix sums, every 8th and every 256th
      uint64_t p[kRcItems];
      load_weights<FROM_LW>(a, cb + (int64_t)tid * kRcItems, m_lw, scale, p, bad);
#pragma unroll
      for (int r = 1; r < kRcItems; ++r) p[r] = acc_add<FROM_LW>(p[r], p[r - 1]);
      const uint64_t own = p[kRcItems - 1];
      const uint64_t inc = warp_scan_acc<FROM_LW>(own, lane);
      if (lane == 31) wtot[warp] = inc;
      __syncthreads();
      const uint64_t v = lane < kRcWarps ? wtot[lane] : 0ull;
      const uint64_t wi = warp_scan_acc<FROM_LW>(v, lane);
      const uint64_t base = acc_add<FROM_LW>(
          cstart, acc_add<FROM_LW>(__shfl_sync(0xffffffffu, wi - v, warp), inc - own));
#pragma unroll
      for (int r = 0; r < kRcItems; ++r) sA[tid * kRcItems + r] = acc_add<FROM_LW>(base, p[r]);
      const uint64_t last = acc_add<FROM_LW>(base, own);
      sL2[tid] = last;
      if ((tid & 31) == 31) sL1[tid >> 5] = last;  // thread 32 i + 31 ends 256-block i
      __syncthreads();
    }
    // warp 0 fetches the next chunk's descriptor while the others take this
    // chunk's items
    if (more && warp == 0) seg_lookup(a, io1, ch + 1, seg_sh[cur ^ 1], lane);
    if (xs < io1 && scatter) {
      // the scatter form of the same definition: particle j's offspring are
      // the outputs k with C_{j-1} <= u + k stride < C_j, i.e. [K(C_{j-1}),
      // K(C_j)) with K(c) = positions below c.  Lane l of a warp takes
      // particle 32 w + l of each 512-particle slice and writes its
      // ancestor index into the chunk's output table in shared memory (a
      // particle with more than kRcShort offspring by its whole warp); the
      // block then writes the ancestors and gathers the records output by
      // output, several loads in flight per thread.
      const int n_out = (int)(kn - kc);
      for (int j0 = 0; j0 < nCw; j0 += kRcTpb) {
        const int j = j0 + tid;  // the same slice for the whole warp
        const bool has = j < nCw;
        const int64_t ke = has ? positions_below_inv(sA[j], u, sv, a.m) : a.m;
        int64_t ks = __shfl_up_sync(0xffffffffu, ke, 1);
        if (lane == 0)
          ks = has ? positions_below_inv(j == 0 ? cstart : sA[j - 1], u, sv, a.m) : a.m;
        const int32_t an = (int32_t)(cb + j);
        const bool longr = has && ke - ks > kRcShort;
        if (has && !longr)
          for (int64_t k = ks; k < ke; ++k) sOut[k - kc] = an;
        unsigned lm = __ballot_sync(0xffffffffu, longr);
        while (lm) {
          const int src = __ffs(lm) - 1;
          lm &= lm - 1;
          const int s0 = (int)(__shfl_sync(0xffffffffu, ks, src) - kc);
          const int s1 = (int)(__shfl_sync(0xffffffffu, ke, src) - kc);
          const int32_t as = __shfl_sync(0xffffffffu, an, src);
          for (int k = s0 + lane; k < s1; k += 32) sOut[k] = as;
        }
      }
      __syncthreads();
      for (int e = tid; e < n_out; e += kRcTpb) a.anc[kc - a.k_off + e] = sOut[e] + (int32_t)a.j_off;
      if (a.rec_words > 0) gather_block(a, kc - a.k_off, n_out, sOut, tid);
    } else if (xs < io1 && !(more && warp == 0)) {
      const int nC = (int)(a.n - cb < kRcChunk ? a.n - cb : kRcChunk);
      const int w0 = more ? 1 : 0, nw = kRcWarps - w0;
      for (int64_t x = xs + (warp - w0); x < io1; x += nw) {
        const int64_t k0 = kc + (x - io0 - kRcPrefixCost) * kRcItemOut;
        const int nB = (int)(kn - k0 < kRcItemOut ? kn - k0 : kRcItemOut);
        const uint64_t pos0 = u + (uint64_t)k0 * stride;  // position of output k0
        const uint64_t posl = pos0 + (uint64_t)(nB - 1) * stride;
        // only A's from the first above pos0 to the first above the last
        // position can be ancestors (with degenerate weights, a handful)
        const int ia = chunk_first_above(sA, sL2, sL1, pos0, lane);
        if (posl < sA[ia]) {  // one ancestor for the whole item (degenerate weights)
          const int32_t an = (int32_t)(cb + ia);
          for (int jj = lane; jj < nB; jj += 32) a.anc[k0 - a.k_off + jj] = an + (int32_t)a.j_off;
          if (a.rec_words > 0)
            gather_item(a, k0 - a.k_off, nB, [an](int) { return an; }, lane);
          continue;
        }
        const int ib = min(chunk_first_above(sA, sL2, sL1, posl, lane) + 1, nC);
        const uint64_t* A = sA + ia;
        const int nA = ib - ia;
        const int L = nA + nB;
        const int d0 = L * lane / 32, d1 = L * (lane + 1) / 32;
        int lo = d0 > nB ? d0 - nB : 0, hi = d0 < nA ? d0 : nA;
        while (lo < hi) {  // the prefix sums among the first d0 merged items (ties: A first)
          const int mid = (lo + hi) >> 1;
          if (A[mid] <= pos0 + (uint64_t)(d0 - 1 - mid) * stride) lo = mid + 1;
          else hi = mid;
        }
        int i = lo, j = d0 - lo;
        uint64_t bj = pos0 + (uint64_t)j * stride;
        uint64_t ai = i < nA ? A[i] : ~0ull;
        for (int s = d0; s < d1; ++s) {
          if (j >= nB || ai <= bj) {
            ++i;
            ai = i < nA ? A[i] : ~0ull;
          } else {  // output k0 + j: ancestor cb + ia + i (A_i > its position, so i < nA)
            sWw[j] = (int32_t)(cb + ia + (i < nA ? i : nA - 1));
            ++j;
            bj += stride;
          }
        }
        __syncwarp();
        for (int jj = lane; jj < nB; jj += 32) a.anc[k0 - a.k_off + jj] = sWw[jj] + (int32_t)a.j_off;
        if (a.rec_words > 0)
          gather_item(a, k0 - a.k_off, nB, [sWw](int j) { return sWw[j]; }, lane);
        __syncwarp();  // sWw is rewritten by the warp's next item
      }
    }
    __syncthreads();  // sA, its index and seg_sh are rewritten for the next chunk
    it = io1;
  }
}

// The sum of one shard's fixed-point weights, quantised exactly as the whole
// population's (its maximum, the scale of n_total particles): block sums of
// u64 integers added atomically (integer addition, so the order does not
// matter).  A weight above the given maximum is an error.
__global__ void __launch_bounds__(kTpb) shard_total_kernel(const float* __restrict__ lw, int64_t n,
                                                           int64_t n_total,
                                                           const double* known_max,
                                                           uint64_t* total, WsHeader* hdr) {
  __shared__ uint64_t wsum[kTpb / 32];
  const float m = (float)*known_max;
  int S = 0;
  while (((int64_t)1 << S) < n_total) ++S;
  const float scale = __int_as_float((127 + 61 - S) << 23);
  uint64_t t = 0;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x; i < n; i += (int64_t)gridDim.x * kTpb) {
    const float v = lw[i];
    bad |= v > m;
    t += v > m ? 0ull : quantize(v, m, scale);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t b = 0;
    for (int w = 0; w < kTpb / 32; ++w) b += wsum[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(total), (unsigned long long)b);
  }
  if (bad) record_status(&hdr->status, PPL_EINVAL);
}

cudaError_t launch_shard_total(const float* lw, int64_t n, int64_t n_total,
                               const double* known_max, uint64_t* total, WsHeader* hdr,
                               cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((n + kTpb - 1) / kTpb, (int64_t)num_sms() * 8));
  shard_total_kernel<<<grid, kTpb, 0, s>>>(lw, n, n_total, known_max, total, hdr);
  return cudaGetLastError();
}

size_t resample_coop_scratch(int64_t n) {
  const int64_t chunks = (n + kRcChunk - 1) / kRcChunk;
  return (size_t)chunks * 8 + 2 * (size_t)(chunks + 1) * 8 + 2 * 16;
}

size_t resample_coop_barrier_bytes() { return sizeof(GridCtl); }

cudaError_t launch_resample_coop(const float* lw, const uint64_t* q_fixed, const double* known_max,
                                 int64_t n, int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                 WsHeader* hdr, void* barrier, char* scratch, size_t scratch_bytes,
                                 int32_t* anc, const int32_t* gate, cudaStream_t s,
                                 const void* rec_in, int64_t rec_bytes, void* rec_out,
                                 const ResampleShard* shard) {
  if (scratch_bytes < resample_coop_scratch(n) || (reinterpret_cast<uintptr_t>(scratch) & 15) ||
      (reinterpret_cast<uintptr_t>(barrier) & 127))
    return cudaErrorInvalidValue;
  RcArgs a;
  a.lw = lw;
  a.qf = q_fixed;
  a.known_max = known_max;
  a.hdr = hdr;
  a.n = n;
  a.m = m;
  a.seed = seed;
  a.instance = instance;
  a.t = t;
  a.anc = anc;
  a.gate = gate;
  a.n_chunks = (n + kRcChunk - 1) / kRcChunk;
  a.n_scale = shard ? shard->n_total : n;
  a.planned = shard ? 1 : 0;
  a.p_stride = shard ? shard->stride : 0;
  a.p_u = shard ? shard->offset : 0;
  a.c_base = shard ? shard->c_base : 0;
  a.k_off = shard ? shard->k_first : 0;
  a.k_end = shard ? shard->k_end : m;
  a.j_off = shard ? shard->first_particle : 0;
  a.rec_in = rec_in;
  a.rec_out = rec_out;
  a.rec_words = 0;
  a.rec_word4 = 0;
  if (rec_in) {
    const uintptr_t al = reinterpret_cast<uintptr_t>(rec_in) | reinterpret_cast<uintptr_t>(rec_out);
    if (!rec_out || rec_bytes <= 0 || rec_bytes > 1024 || rec_bytes % 4 || (al & 3))
      return cudaErrorInvalidValue;
    const bool w16 = rec_bytes % 16 == 0 && (al & 15) == 0;
    a.rec_word4 = w16 ? 0 : 1;
    a.rec_words = (int32_t)(w16 ? rec_bytes / 16 : rec_bytes / 4);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = scratch + off;
    off += (bytes + 15) / 16 * 16;
    return q;
  };
  a.g = reinterpret_cast<GridCtl*>(barrier);
  a.ctot = reinterpret_cast<uint64_t*>(take((size_t)a.n_chunks * 8));
  a.kfirst = reinterpret_cast<int64_t*>(take((size_t)(a.n_chunks + 1) * 8));
  a.ioff = reinterpret_cast<int64_t*>(take((size_t)(a.n_chunks + 1) * 8));
  constexpr size_t dyn = (size_t)kRcChunk * sizeof(uint64_t) + (size_t)kRcTpb * sizeof(uint64_t) +
                         (size_t)kRcWarps * kRcItemOut * sizeof(int32_t) +
                         (size_t)kRcScatterOut * sizeof(int32_t);
  const void* fn = lw ? (const void*)resample_coop_kernel<true> : (const void*)resample_coop_kernel<false>;
  // once per kernel and device: the shared-memory attribute and the residency
  int per_sm = 0;
  const cudaError_t e = device_once(fn, &per_sm, [fn](int* v) {
    cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (r != cudaSuccess) return r;
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, fn, kRcTpb, dyn);
    if (r == cudaSuccess && *v < 1) *v = 1;
    return r;
  });
  if (e != cudaSuccess) return e;
  const int64_t grid = (int64_t)num_sms() * per_sm;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kRcTpb), args, dyn, s);
}

}  // namespace ppl
