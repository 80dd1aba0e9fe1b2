// Systematic resampling with 64-bit fixed-point weights, exact prefix sums by a
// single-pass decoupled-lookback scan (Merrill and Garland, "Single-pass
// Parallel Prefix Scan with Decoupled Look-back", 2016), output-parallel
// ancestor search, and the gather of resampled particle state.
//
// Definition (particle methods are the paper's stated future work, §6; the
// scheme is systematic resampling, Kitagawa 1996):
//   m = max lw,  S = 61 - ceil(log2 N),  q_i = floor(E32(lw_i - m) * 2^S)
//   (0 when lw_i - m < -44.5),  T = sum q,  stride = floor(T / M),
//   u = floor(w * stride / 2^32),  a_k = min{ j : C_j > u + k * stride }.
// E32 is a fixed FP32 exponential (Cody-Waite reduction by ln 2, degree-7
// Taylor polynomial in Horner form, each step one rounded FP32 operation), so
// the integers q_i, and hence the ancestors, are reproducible bit for bit.
#include "fixedpoint.cuh"
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

__device__ __forceinline__ uint64_t warp_sum_sat(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = sat_add(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One tile of kScanTile weights per block; tiles are taken in launch order
// from an atomic counter so every predecessor of a tile is already running.
template <bool FROM_LW, bool VEC>
__global__ void __launch_bounds__(kTpb) resample_scan_kernel(
    const float* __restrict__ lw, const uint64_t* __restrict__ qf, int64_t N, int64_t M,
    uint64_t seed, uint32_t instance, uint32_t t, WsHeader* hdr, uint64_t* tile_status,
    uint64_t* __restrict__ prefix, const int32_t* gate, int64_t n_tiles,
    const double* known_max, int64_t silent_tile, int max_spin) {
  if (gate && *gate == 0) return;
  __shared__ int64_t tile_sh;
  __shared__ uint64_t warp_tot[kTpb / 32];
  __shared__ uint64_t excl_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) tile_sh = (int64_t)atomicAdd(&hdr->tile_counter[0], 1u);
  __syncthreads();
  const int64_t tile = tile_sh;
  const int64_t base = tile * kScanTile + (int64_t)tid * kScanItems;

  uint64_t q[kScanItems];
  int bad = 0;
  if (FROM_LW) {
    const float m = known_max ? (float)*known_max : hdr->max_lw;
    int S = 0;
    while (((int64_t)1 << S) < N) ++S;
    const float scale = __int_as_float((127 + 61 - S) << 23);
    float v[kScanItems];
    if (VEC && base + kScanItems <= N) {
      const float4 a = *reinterpret_cast<const float4*>(lw + base);
      const float4 b = *reinterpret_cast<const float4*>(lw + base + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < N) ? lw[base + j] : -INFINITY;
    }
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) q[j] = quantize(v[j], m, scale);
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const uint64_t x = (base + j < N) ? qf[base + j] : 0ull;
      bad |= x > (1ull << 61);
      q[j] = x > kLimit ? kLimit : x;
    }
  }

  // thread-local inclusive scan
#pragma unroll
  for (int j = 1; j < kScanItems; ++j) q[j] = sat_add(q[j], q[j - 1]);
  const uint64_t own = q[kScanItems - 1];
  // warp inclusive scan of the thread totals
  uint64_t inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = sat_add(inc, y);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  uint64_t warp_excl = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kTpb / 32; ++w) {
    if (w < warp) warp_excl = sat_add(warp_excl, warp_tot[w]);
    agg = sat_add(agg, warp_tot[w]);
  }
  const uint64_t thread_excl = sat_add(warp_excl, inc - own);

  // A silent tile publishes nothing (self-test of the bounded wait only).
  if (tile == silent_tile) return;
  // publish the aggregate, then look back for the exclusive prefix
  if (warp == 0) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (lane == 0) st_release_u64(tile_status, kFlagIncl | agg);
    } else {
      if (lane == 0) st_release_u64(tile_status + tile, kFlagAgg | agg);
      int64_t j = tile - 1;
      bool timed_out = false;
      while (true) {
        const int64_t idx = j - lane;
        uint64_t v = (idx < 0) ? kFlagIncl : ld_acquire_u64(tile_status + idx);
        int spins = 0;
        while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
          if (++spins > max_spin) {
            timed_out = true;
            break;
          }
          if (spins > 64) __nanosleep(32);
          if ((v >> 62) == 0) v = ld_acquire_u64(tile_status + idx);
        }
        if (timed_out) {
          if (lane == 0) record_status(&hdr->status, PPL_ETIMEOUT);
          break;
        }
        const unsigned incl = __ballot_sync(0xffffffffu, (v >> 62) == 2);
        if (incl) {
          const int first = __ffs(incl) - 1;
          excl = sat_add(excl, warp_sum_sat(lane <= first ? (v & kValMask) : 0ull));
          break;
        }
        excl = sat_add(excl, warp_sum_sat(v & kValMask));
        j -= 32;
      }
      if (lane == 0) st_release_u64(tile_status + tile, kFlagIncl | sat_add(excl, agg));
    }
    if (lane == 0) excl_sh = excl;
  }
  __syncthreads();
  const uint64_t tile_excl = excl_sh;
  const uint64_t off = sat_add(tile_excl, thread_excl);
  if (base + kScanItems <= N) {
    uint4* dst = reinterpret_cast<uint4*>(prefix + base);
#pragma unroll
    for (int j = 0; j < kScanItems; j += 2) {
      const uint64_t a = sat_add(off, q[j]), b = sat_add(off, q[j + 1]);
      dst[j / 2] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
      if (base + j < N) prefix[base + j] = sat_add(off, q[j]);
  }

  if (bad) record_status(&hdr->status, PPL_EINVAL);
  if (tile == n_tiles - 1 && tid == 0) {
    const uint64_t T = sat_add(tile_excl, agg);
    if (T > (1ull << 61)) {
      record_status(&hdr->status, PPL_EINVAL);
    } else if (T == 0) {
      record_status(&hdr->status, PPL_EEMPTY);
    } else if (T < (uint64_t)M) {
      record_status(&hdr->status, PPL_EINVAL);
    } else {
      const uint64_t stride = T / (uint64_t)M;
      const uint32_t w = philox_block(seed, 0, instance, t, kResample, 0).x;
      const uint64_t lo = (uint64_t)w * stride, hi = __umul64hi((uint64_t)w, stride);
      hdr->total = T;
      hdr->stride = stride;
      hdr->offset = (hi << 32) | (lo >> 32);
    }
  }
}

constexpr int kAncItems = 8;
constexpr int64_t kAncChunk = (int64_t)kTpb * kAncItems;
constexpr int kAncSmem = 4096;

// bounds[2c], bounds[2c + 1]: the first ancestor of the first and of the last
// output of chunk c (one warp per bound).
__global__ void __launch_bounds__(kTpb) chunk_bounds_kernel(const uint64_t* __restrict__ C,
                                                            int64_t N, int64_t M,
                                                            const WsHeader* hdr,
                                                            int64_t* __restrict__ bounds,
                                                            const int32_t* gate) {
  if (gate && *gate == 0) return;
  if (ld_volatile_i32(&hdr->status) != 0) return;
  const int64_t w = ((int64_t)blockIdx.x * kTpb + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t n_chunks = (M + kAncChunk - 1) / kAncChunk;
  if (w >= 2 * n_chunks) return;
  const int64_t c = w >> 1;
  const int64_t k = (w & 1) ? ((M < (c + 1) * kAncChunk ? M : (c + 1) * kAncChunk) - 1)
                            : c * kAncChunk;
  const int64_t j = warp_upper_bound(C, 0, N, hdr->offset + (uint64_t)k * hdr->stride, lane);
  if (lane == 0) bounds[w] = j < N - 1 ? j : N - 1;
}

// First index j in [lo, hi) with C[j] > p (hi if none).
__device__ __forceinline__ int64_t upper_bound_global(const uint64_t* C, int64_t lo, int64_t hi,
                                                      uint64_t p) {
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (C[mid] > p) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Output-parallel search: a block owns kAncChunk consecutive outputs, so the
// work is balanced whatever the weights; the prefix sums it needs (between the
// chunk's precomputed bounds) are staged in shared memory when they fit.
__global__ void __launch_bounds__(kTpb) ancestors_kernel(const uint64_t* __restrict__ C,
                                                         int64_t N, int64_t M,
                                                         const WsHeader* hdr,
                                                         const int64_t* __restrict__ bounds,
                                                         int32_t* __restrict__ anc,
                                                         const int32_t* gate) {
  if (gate && *gate == 0) return;
  if (ld_volatile_i32(&hdr->status) != 0) return;
  __shared__ uint64_t sC[kAncSmem];
  const uint64_t stride = hdr->stride, off = hdr->offset;
  const int tid = threadIdx.x;
  const int64_t n_chunks = (M + kAncChunk - 1) / kAncChunk;
  for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int64_t k0 = ch * kAncChunk;
    const int64_t k1 = (M < k0 + kAncChunk ? M : k0 + kAncChunk) - 1;
    const int64_t jlo = bounds[2 * ch], jhi = bounds[2 * ch + 1];
    const int64_t span = jhi - jlo + 1;
    const bool staged = span <= kAncSmem;
    __syncthreads();
    if (staged)
      for (int64_t j = tid; j < span; j += kTpb) sC[j] = C[jlo + j];
    __syncthreads();
    const int64_t kb = k0 + (int64_t)tid * kAncItems;
    int32_t out[kAncItems];
    int64_t j = -1;
#pragma unroll
    for (int it = 0; it < kAncItems; ++it) {
      const int64_t k = kb + it;
      if (k > k1) {
        out[it] = 0;
        continue;
      }
      const uint64_t p = off + (uint64_t)k * stride;
      if (staged) {
        int64_t r;
        if (j >= 0) {  // walk on from the previous answer
          r = j;
          int steps = 0;
          while (r < span && sC[r] <= p && steps < 8) {
            ++r;
            ++steps;
          }
          if (r < span && sC[r] <= p) {
            int64_t lo = r, hi = span;
            while (lo < hi) {
              const int64_t mid = lo + ((hi - lo) >> 1);
              if (sC[mid] > p) hi = mid;
              else lo = mid + 1;
            }
            r = lo;
          }
        } else {
          int64_t lo = 0, hi = span;
          while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (sC[mid] > p) hi = mid;
            else lo = mid + 1;
          }
          r = lo;
        }
        j = r;
        out[it] = (int32_t)(jlo + r);
      } else {
        const int64_t r = upper_bound_global(C, j >= 0 ? jlo + j : jlo, jhi + 1, p);
        j = r - jlo;
        out[it] = (int32_t)r;
      }
    }
    if (kb + kAncItems - 1 <= k1 && ((reinterpret_cast<uintptr_t>(anc + kb) & 15) == 0)) {
      reinterpret_cast<int4*>(anc + kb)[0] = make_int4(out[0], out[1], out[2], out[3]);
      reinterpret_cast<int4*>(anc + kb)[1] = make_int4(out[4], out[5], out[6], out[7]);
    } else {
#pragma unroll
      for (int it = 0; it < kAncItems; ++it)
        if (kb + it <= k1) anc[kb + it] = out[it];
    }
    __syncthreads();
  }
}

// state_out[k] = state_in[anc[k]]: one thread per vector word of the output,
// so stores are fully coalesced; ancestors are non-decreasing, so loads are
// nearly so.  Out-of-range ancestors give zero records.  W > 0 fixes the words
// per record at compile time (the index split is then a shift or a constant
// division); W = 0 reads it from `words`.  Each thread takes kGatherUnroll
// words per round, so that many ancestor loads are in flight at once.
constexpr int kGatherUnroll = 4;

template <typename V, int W>
__global__ void __launch_bounds__(kTpb) gather_kernel(const V* __restrict__ in, int64_t n_in,
                                                      int64_t words_rt,
                                                      const int32_t* __restrict__ anc,
                                                      int64_t M, V* __restrict__ out,
                                                      const int32_t* gate) {
  if (gate && *gate == 0) return;
  const int64_t words = W > 0 ? (int64_t)W : words_rt;
  const int64_t total = M * words;
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t u0 = (int64_t)blockIdx.x * kTpb + threadIdx.x; u0 < total;
       u0 += stride * kGatherUnroll) {
    int64_t a[kGatherUnroll];
#pragma unroll
    for (int r = 0; r < kGatherUnroll; ++r) {
      const int64_t u = u0 + r * stride;
      a[r] = u < total ? (int64_t)anc[u / words] : -1;
    }
#pragma unroll
    for (int r = 0; r < kGatherUnroll; ++r) {
      const int64_t u = u0 + r * stride;
      if (u >= total) break;
      const int64_t v = u % words;
      V val;
      if (a[r] >= 0 && a[r] < n_in) val = in[a[r] * words + v];
      else memset(&val, 0, sizeof(V));
      out[u] = val;
    }
  }
}

cudaError_t launch_resample_scan(const float* lw, const uint64_t* q_fixed, int64_t N, int64_t M,
                                 uint64_t seed, uint32_t instance, uint32_t t, WsHeader* hdr,
                                 uint64_t* tile_status, uint64_t* prefix, const int32_t* gate,
                                 cudaStream_t s, const double* known_max) {
  const int64_t tiles = scan_tiles(N);
  if (lw) {
    const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15) == 0;
    if (vec)
      resample_scan_kernel<true, true><<<(unsigned)tiles, kTpb, 0, s>>>(
          lw, nullptr, N, M, seed, instance, t, hdr, tile_status, prefix, gate, tiles, known_max, -1,
          kMaxSpin);
    else
      resample_scan_kernel<true, false><<<(unsigned)tiles, kTpb, 0, s>>>(
          lw, nullptr, N, M, seed, instance, t, hdr, tile_status, prefix, gate, tiles, known_max, -1,
          kMaxSpin);
  } else {
    resample_scan_kernel<false, false><<<(unsigned)tiles, kTpb, 0, s>>>(
        nullptr, q_fixed, N, M, seed, instance, t, hdr, tile_status, prefix, gate, tiles, nullptr, -1,
        kMaxSpin);
  }
  return cudaGetLastError();
}

// Self-test of the bounded look-back wait: tile 0 of a fixed-point scan
// publishes nothing, so every other tile's wait runs out after max_spin polls
// and records PPL_ETIMEOUT; each still publishes, so no tile waits forever.
cudaError_t launch_scan_timeout_selftest(const uint64_t* q, int64_t N, WsHeader* hdr,
                                         uint64_t* tile_status, uint64_t* prefix, int max_spin,
                                         cudaStream_t s) {
  const int64_t tiles = scan_tiles(N);
  resample_scan_kernel<false, false><<<(unsigned)tiles, kTpb, 0, s>>>(
      nullptr, q, N, N, 0, 0, 0, hdr, tile_status, prefix, nullptr, tiles, nullptr, 0, max_spin);
  return cudaGetLastError();
}

int64_t ancestor_bounds_count(int64_t M) { return 2 * ((M + kAncChunk - 1) / kAncChunk); }

cudaError_t launch_ancestors(const uint64_t* prefix, int64_t N, int64_t M, const WsHeader* hdr,
                             int64_t* bounds, int32_t* ancestors, const int32_t* gate,
                             cudaStream_t s) {
  const int64_t chunks = (M + kAncChunk - 1) / kAncChunk;
  const int64_t warps = 2 * chunks;
  chunk_bounds_kernel<<<(unsigned)((warps * 32 + kTpb - 1) / kTpb), kTpb, 0, s>>>(
      prefix, N, M, hdr, bounds, gate);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)num_sms() * 8));
  ancestors_kernel<<<grid, kTpb, 0, s>>>(prefix, N, M, hdr, bounds, ancestors, gate);
  return cudaGetLastError();
}

template <typename V>
static void launch_gather_t(const V* in, int64_t n_in, int64_t words, const int32_t* anc,
                            int64_t M, V* out, const int32_t* gate, cudaStream_t s) {
  const int64_t cap = (int64_t)num_sms() * 8;
  const int64_t want = (M * words + (int64_t)kTpb * kGatherUnroll - 1) / ((int64_t)kTpb * kGatherUnroll);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
  switch (words) {
    case 1: gather_kernel<V, 1><<<grid, kTpb, 0, s>>>(in, n_in, words, anc, M, out, gate); break;
    case 2: gather_kernel<V, 2><<<grid, kTpb, 0, s>>>(in, n_in, words, anc, M, out, gate); break;
    case 4: gather_kernel<V, 4><<<grid, kTpb, 0, s>>>(in, n_in, words, anc, M, out, gate); break;
    default: gather_kernel<V, 0><<<grid, kTpb, 0, s>>>(in, n_in, words, anc, M, out, gate); break;
  }
}

cudaError_t launch_gather(const void* in, int64_t n_in, int64_t stride_bytes, const int32_t* anc,
                          int64_t M, void* out, const int32_t* gate, cudaStream_t s) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out);
  if (stride_bytes % 16 == 0 && (a & 15) == 0)
    launch_gather_t<uint4>((const uint4*)in, n_in, stride_bytes / 16, anc, M, (uint4*)out, gate, s);
  else if (stride_bytes % 4 == 0 && (a & 3) == 0)
    launch_gather_t<uint32_t>((const uint32_t*)in, n_in, stride_bytes / 4, anc, M, (uint32_t*)out,
                              gate, s);
  else
    launch_gather_t<uint8_t>((const uint8_t*)in, n_in, stride_bytes, anc, M, (uint8_t*)out, gate, s);
  return cudaGetLastError();
}

}  // namespace ppl
