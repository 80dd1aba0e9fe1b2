// Systematic resampling (the definition in resample.cu: 64-bit fixed-point
// weights q_i, T = sum q, stride = floor(T / M), u = floor(w stride / 2^32),
// a_k = min{j : C_j > u + k stride}) in one persistent, cooperative kernel
// with one grid barrier, and no prefix-sum array in global memory:
//
//   1. the particles are cut into chunks of 8192; blocks sum the weights of
//      their chunks (one read of lw);
//   2. barrier: the last arriving block scans the chunk totals, draws u, and
//      gives every chunk its first output K_c = #{k : u + k stride < C_start}
//      -- chunk c holds the ancestors of outputs [K_c, K_c+1) -- and cuts each
//      chunk's outputs into work items of at most 8192;
//   3. blocks take the items in turn: an item forms its chunk's inclusive
//      prefix sums in shared memory (lw is L2-resident by now) and finds its
//      outputs' ancestors by merging the sorted prefix sums with the sorted
//      positions (merge path: Green, McColl, Bader, "GPU merge path", ICS
//      2012), one equal slice of the merge per thread.
//
// Every item costs at most 8192 weights and 8192 outputs whatever the
// weights are: a chunk holding most of the mass (degenerate importance
// weights) becomes many items on many blocks.  The ancestors are those of the
// scan-and-search path bit for bit (both are exact integer computations of the
// same definition).  Traffic: lw twice (the second time from L2), the
// ancestors once.
#include <algorithm>

#include "gridsync.cuh"
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

constexpr int kRcTpb = 1024;                          // one block per SM
constexpr int kRcItems = 8;                           // weights per thread per chunk
constexpr int64_t kRcChunk = (int64_t)kRcTpb * kRcItems;
constexpr int64_t kRcItemOut = 8192;                  // outputs of one work item

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
};

template <bool FROM_LW>
__device__ __forceinline__ void load_weights(const RcArgs& a, int64_t base, float m_lw, float scale,
                                             uint64_t (&q)[kRcItems], int& bad) {
  if (FROM_LW) {
    float v[kRcItems];
    if (base + kRcItems <= a.n && (reinterpret_cast<uintptr_t>(a.lw + base) & 15) == 0) {
      const float4 x = __ldcg(reinterpret_cast<const float4*>(a.lw + base));
      const float4 y = __ldcg(reinterpret_cast<const float4*>(a.lw + base) + 1);
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
      v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
#pragma unroll
      for (int r = 0; r < kRcItems; ++r) v[r] = base + r < a.n ? __ldcg(a.lw + base + r) : -INFINITY;
    }
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) q[r] = quantize(v[r], m_lw, scale);
  } else {
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) {
      const uint64_t x = base + r < a.n ? __ldcg(a.qf + base + r) : 0ull;
      bad |= x > (1ull << 61);
      q[r] = x > kLimit ? kLimit : x;
    }
  }
}

template <bool FROM_LW>
__global__ void __launch_bounds__(kRcTpb, 1) resample_coop_kernel(RcArgs a) {
  if (a.gate && *a.gate == 0) return;  // every block reads the same flag
  extern __shared__ __align__(16) unsigned char rc_dyn[];
  uint64_t* sA = reinterpret_cast<uint64_t*>(rc_dyn);         // [kRcChunk] prefix sums of a chunk
  int32_t* sO = reinterpret_cast<int32_t*>(sA + kRcChunk);    // [kRcItemOut] an item's ancestors
  __shared__ uint64_t wtot[kRcTpb / 32], jtot[kRcTpb / 32];
  __shared__ int64_t jitem[kRcTpb / 32];
  __shared__ unsigned long long rel;
  __shared__ uint64_t view[3];  // T, stride, u
  __shared__ int64_t item_sh[5];  // chunk, C at its start, first and end output, new chunk
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  float m_lw = 0.0f, scale = 0.0f;
  if (FROM_LW) {
    m_lw = a.known_max ? (float)*a.known_max : a.hdr->max_lw;
    int S = 0;
    while (((int64_t)1 << S) < a.n) ++S;
    scale = __int_as_float((127 + 61 - S) << 23);  // 2^(61 - ceil(log2 n))
  }

  // 1. chunk totals
  int bad = 0;
  for (int64_t ch = blockIdx.x; ch < a.n_chunks; ch += G) {
    uint64_t q[kRcItems];
    load_weights<FROM_LW>(a, ch * kRcChunk + (int64_t)tid * kRcItems, m_lw, scale, q, bad);
    uint64_t tot = 0;
#pragma unroll
    for (int r = 0; r < kRcItems; ++r) tot = sat_add(tot, q[r]);
    const uint64_t wi = warp_scan_u64(tot, lane);
    __syncthreads();  // wtot of the previous chunk is read
    if (lane == 31) wtot[warp] = wi;
    __syncthreads();
    if (warp == 0) {
      const uint64_t bt = warp_scan_u64(wtot[lane], lane);
      if (lane == 31) a.ctot[ch] = bt;
    }
  }
  if (bad) record_status(&a.hdr->status, PPL_EINVAL);
  // 2. barrier: the last block scans the chunk totals, checks T, draws u, and
  // lays out the work items; the item count is the release word's payload
  const bool ok = grid_sync<true>(a.g, &a.hdr->status, G, 1, &rel, [&]() -> unsigned long long {
    // thread tid takes chunks [c0, c1) in order
    const int64_t per = (a.n_chunks + kRcTpb - 1) / kRcTpb;
    const int64_t c0 = (int64_t)tid * per, c1 = c0 + per < a.n_chunks ? c0 + per : a.n_chunks;
    uint64_t run = 0;
    for (int64_t ch = c0; ch < c1; ++ch) run = sat_add(run, __ldcg(a.ctot + ch));
    const uint64_t wi = warp_scan_u64(run, lane);
    if (lane == 31) jtot[warp] = wi;
    __syncthreads();
    const uint64_t jv = jtot[lane], ji = warp_scan_u64(jv, lane);
    const uint64_t T = __shfl_sync(0xffffffffu, ji, 31);
    uint64_t cx = sat_add(__shfl_sync(0xffffffffu, ji - jv, warp), wi - run);
    const bool valid = T > 0 && T <= (1ull << 61) && T >= (uint64_t)a.m;
    uint64_t stride = 0, u = 0;
    if (valid) {
      stride = T / (uint64_t)a.m;
      const uint64_t w = philox_block(a.seed, 0, a.instance, a.t, kResample, 0).x;
      u = (__umul64hi(w, stride) << 32) | ((w * stride) >> 32);
    }
    // exclusive chunk prefixes, first outputs and item counts of this thread's chunks
    int64_t items = 0;
    for (int64_t ch = c0; ch < c1; ++ch) {
      const uint64_t t_ch = __ldcg(a.ctot + ch);
      const int64_t k0 = valid ? positions_below(cx, u, stride, a.m) : 0;
      const int64_t k1 = valid ? positions_below(sat_add(cx, t_ch), u, stride, a.m) : 0;
      a.ctot[ch] = cx;
      a.kfirst[ch] = k0;
      items += (k1 - k0 + kRcItemOut - 1) / kRcItemOut;
      cx = sat_add(cx, t_ch);
    }
    // exclusive scan of the item counts
    int64_t ii = items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, ii, o);
      if (lane >= o) ii += y;
    }
    if (lane == 31) jitem[warp] = ii;
    __syncthreads();
    int64_t iv = jitem[lane], iw = iv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, iw, o);
      if (lane >= o) iw += y;
    }
    int64_t ix = __shfl_sync(0xffffffffu, iw - iv, warp) + (ii - items);
    const int64_t n_items = __shfl_sync(0xffffffffu, iw, 31);
    for (int64_t ch = c0; ch < c1; ++ch) {  // K of the next chunk: written before the barrier above
      a.ioff[ch] = ix;
      const int64_t k0 = __ldcg(a.kfirst + ch);
      const int64_t k1 = ch + 1 < a.n_chunks ? __ldcg(a.kfirst + ch + 1) : a.m;
      ix += (k1 - k0 + kRcItemOut - 1) / kRcItemOut;
    }
    if (tid == 0) {
      if (T == 0) record_status(&a.hdr->status, PPL_EEMPTY);
      else if (T > (1ull << 61) || T < (uint64_t)a.m) record_status(&a.hdr->status, PPL_EINVAL);
      a.g->total = T;
      a.g->stride = stride;
      a.g->offset = u;
      a.kfirst[a.n_chunks] = a.m;
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

  // 3. work items: block b takes the contiguous run [I b / G, I (b + 1) / G),
  // so consecutive items usually share a chunk, whose prefix sums then stay
  // in shared memory
  const int64_t it0 = n_items * blockIdx.x / G, it1 = n_items * (blockIdx.x + 1) / G;
  int64_t ch_t0 = -1;  // thread 0: chunk of the previous item
  for (int64_t it = it0; it < it1; ++it) {
    __syncthreads();  // the previous item has read sO and item_sh
    if (tid == 0) {
      int64_t lo = ch_t0 < 0 ? 0 : ch_t0;
      if (ch_t0 < 0 || __ldcg(a.ioff + ch_t0 + 1) <= it) {
        int64_t hi = a.n_chunks;  // the last chunk with ioff <= it (ioff[n_chunks] > it)
        while (hi - lo > 1) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldcg(a.ioff + mid) <= it) lo = mid;
          else hi = mid;
        }
      }
      const int64_t kc = __ldcg(a.kfirst + lo), kn = __ldcg(a.kfirst + lo + 1);
      const int64_t first = kc + (it - __ldcg(a.ioff + lo)) * kRcItemOut;
      item_sh[0] = lo;
      item_sh[1] = (int64_t)__ldcg(a.ctot + lo);
      item_sh[2] = first;
      item_sh[3] = first + kRcItemOut < kn ? first + kRcItemOut : kn;
      item_sh[4] = lo != ch_t0;  // new chunk: its prefix sums are formed below
      ch_t0 = lo;
    }
    __syncthreads();
    const int64_t ch = item_sh[0], k0 = item_sh[2], k1 = item_sh[3];
    const uint64_t cstart = (uint64_t)item_sh[1];
    const int64_t cb = ch * kRcChunk;
    if (item_sh[4]) {  // the same for every thread of the block
      uint64_t p[kRcItems];
      load_weights<FROM_LW>(a, cb + (int64_t)tid * kRcItems, m_lw, scale, p, bad);
#pragma unroll
      for (int r = 1; r < kRcItems; ++r) p[r] = sat_add(p[r], p[r - 1]);
      const uint64_t own = p[kRcItems - 1];
      const uint64_t inc = warp_scan_u64(own, lane);
      if (lane == 31) wtot[warp] = inc;
      __syncthreads();
      const uint64_t v = wtot[lane], wi = warp_scan_u64(v, lane);
      const uint64_t base = sat_add(cstart, sat_add(__shfl_sync(0xffffffffu, wi - v, warp), inc - own));
#pragma unroll
      for (int r = 0; r < kRcItems; ++r) sA[tid * kRcItems + r] = sat_add(base, p[r]);
      __syncthreads();
    }
    {
      const int nC = (int)(a.n - cb < kRcChunk ? a.n - cb : kRcChunk);
      const int nB = (int)(k1 - k0);
      const uint64_t pos0 = u + (uint64_t)k0 * stride;  // position of output k0
      const uint64_t posl = pos0 + (uint64_t)(nB - 1) * stride;
      // only A's between the first above pos0 and the first above the last
      // position can be ancestors (with degenerate weights, a handful)
      auto upper = [&](uint64_t v) {
        int lo = 0, hi = nC;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sA[mid] <= v) lo = mid + 1;
          else hi = mid;
        }
        return lo;
      };
      const int ia = upper(pos0), ib = min(upper(posl) + 1, nC);
      const uint64_t* A = sA + ia;
      const int nA = ib - ia;
      const int L = nA + nB;
      const int d0 = (int)((int64_t)L * tid / kRcTpb), d1 = (int)((int64_t)L * (tid + 1) / kRcTpb);
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
          sO[j] = (int32_t)(cb + ia + (i < nA ? i : nA - 1));
          ++j;
          bj += stride;
        }
      }
      __syncthreads();
      for (int jj = tid; jj < nB; jj += kRcTpb) a.anc[k0 + jj] = sO[jj];
    }
  }
}

size_t resample_coop_scratch(int64_t n) {
  const int64_t chunks = (n + kRcChunk - 1) / kRcChunk;
  return sizeof(GridCtl) + (size_t)chunks * 8 + 2 * (size_t)(chunks + 1) * 8 + 3 * 16;
}

cudaError_t launch_resample_coop(const float* lw, const uint64_t* q_fixed, const double* known_max,
                                 int64_t n, int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                 WsHeader* hdr, char* scratch, size_t scratch_bytes,
                                 int32_t* anc, const int32_t* gate, cudaStream_t s) {
  if (scratch_bytes < resample_coop_scratch(n) || (reinterpret_cast<uintptr_t>(scratch) & 127))
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
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = scratch + off;
    off += (bytes + 15) / 16 * 16;
    return q;
  };
  a.g = reinterpret_cast<GridCtl*>(take(sizeof(GridCtl)));
  a.ctot = reinterpret_cast<uint64_t*>(take((size_t)a.n_chunks * 8));
  a.kfirst = reinterpret_cast<int64_t*>(take((size_t)(a.n_chunks + 1) * 8));
  a.ioff = reinterpret_cast<int64_t*>(take((size_t)(a.n_chunks + 1) * 8));
  constexpr size_t dyn = (size_t)kRcChunk * sizeof(uint64_t) + (size_t)kRcItemOut * sizeof(int32_t);
  const void* fn = lw ? (const void*)resample_coop_kernel<true> : (const void*)resample_coop_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRcTpb, dyn);
  if (e != cudaSuccess) return e;
  const int64_t grid = (int64_t)num_sms() * std::max(per_sm, 1);
  e = cudaMemsetAsync(a.g, 0, sizeof(GridCtl), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kRcTpb), args, dyn, s);
}

}  // namespace ppl
