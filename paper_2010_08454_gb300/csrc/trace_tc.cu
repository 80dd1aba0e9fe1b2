// Likelihood weighting on the line-fitting model (Fig. 1; §3.6.2 runs the
// model N times and normalises the log-weights) with the factor's polynomial
// evaluations on the fifth-generation tensor cores.
//
// For a tile of 128 traces and a chunk of up to 128 data points, the
// residuals of every (trace, point) pair form one matrix product:
//   D[t, l] = sum_k A[t, k] B[l, k],  A[t] = (c_0, .., c_5, 1, 1),
//   B[l] = (1, x_l, .., x_l^5, -yh_l, -yr_l),  yh = tf32(y), yr = y - yh,
// so D[t, l] = f_t(x_l) - y_l, and the trace's factor is
// -sum_l D[t, l]^2 / (2 sigma^2).  Coefficients past a trace's count are 0,
// so every degree shares one product and nothing branches on the sampled
// degree (the cost the paper reports for its GPU code, §5.1).
//
// Accuracy: each FP32 operand v is split into two TF32 parts, v = hi + lo
// (hi rounded to nearest; the data's lo rounded to nearest, a coefficient's
// lo = v - hi passed exactly as FP32, of which the tensor cores use the TF32
// part: within 2^-21 of v), and D accumulates A_hi B_hi + A_hi B_lo +
// A_lo B_hi in FP32 in tensor memory (three kind::tf32 MMAs of K = 8); the
// dropped A_lo B_lo is below 2^-22 of each product.  The powers x^k are
// formed in FP64 before their split, and y is carried exactly by the two
// columns (yh, yr).  The sum of squares is taken in FP32 by each trace's
// thread (eight running sums in f32x2 pairs per 64-point block; the block
// sums add plainly up to 512 points, with Kahan's compensation beyond).
//
// Layout: one CTA per SM; its four warpgroups hold all 512 tensor-memory
// columns, 128 FP32 columns of D each.  Warpgroup g takes tiles g, g + 4, ..
// of its CTA's share; thread r of a warpgroup owns trace r of the tile and
// TMEM lane r.  While the tensor cores run a tile's first chunk, the
// warpgroup draws its next tile (two Philox blocks and three Box-Muller
// pairs per trace) and writes those records; the four warpgroups
// interleave, so one's products overlap the others' draws and sums.
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8 x 4 core matrices of 128 contiguous bytes, the two K-halves of
// a row group 128 B apart (leading byte offset), row groups 256 B apart
// (stride byte offset).  The data's B operand (hi and lo, 32 bytes per point
// each) is staged once per CTA.
//
// The per-degree posterior partials are folded per warp with the trace
// kernel's rules (traces more than 50 nats below the warp's running maximum
// of their degree, or below the best of their degree in the tile, are
// skipped), and the last CTA merges the CTAs' partials.
// Every mbarrier wait is bounded; a wait that runs out records PPL_ETIMEOUT,
// and the CTA still frees its tensor memory.
#include "kernels.h"
#include "poly.cuh"
#include "posterior.cuh"
#include "trace.cuh"

namespace ppl {
namespace {

constexpr int kTcM = 128;           // traces per tile (tensor-memory lanes)
constexpr int kTcWGs = 4;           // warpgroups per CTA, each with its own accumulator
constexpr int kTcChunk = 128;       // data points per product (MMA N): 512 columns / kTcWGs
constexpr int kTcThreads = 128 * kTcWGs;
constexpr int kTcSpin = 1 << 18;    // bound of one mbarrier wait (polls)
constexpr uint32_t kTcSuspendNs = 4096;  // a poll may suspend the warp this long (hint)
constexpr float kTcSkipNats = 50.0f;
constexpr int kTcSerialMerges = 4;  // up to this many traces a warp merges one at a time
constexpr uint32_t kTcTmemCols = 512;
constexpr int kTcMaxPoints = 2048;  // the data's B operand (64 B per point) stays in shared memory

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), TF32 A
// and B (bits 7-9, 10-12 = 2), both K-major, M >> 4 at bit 24; N >> 3 at bit
// 17 is added per product.
constexpr uint32_t kTcIdescBase = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Byte offset of element (row r, k) of a K = 8 operand in the core layout.
__device__ __forceinline__ uint32_t kcore(int r, int k) {
  return (uint32_t)((((r >> 3) * 2 + (k >> 2)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// TF32 rounding to nearest (PTX cvt.rna.tf32.f32: ties away from zero); the
// result is an FP32 value whose low 13 significand bits are zero.
__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Wait for the mbarrier phase of the given parity.  Each poll may suspend the
// warp (up to the hint) instead of spinning, so a waiting warpgroup leaves the
// issue slots to the others; at most kTcSpin polls (well under a minute).
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
  for (int i = 0; i < kTcSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(phase), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Barrier of one warpgroup (named barrier 1 + g, 128 threads) that also
// returns, to every thread, whether any thread of the warpgroup passed `bad`.
__device__ __forceinline__ bool wg_sync_any(int g, bool bad) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n"
      " bar.red.or.pred pout, %2, 128, pin;\n selp.u32 %0, 1, 0, pout;\n}"
      : "=r"(out)
      : "r"((uint32_t)bad), "r"(1 + g)
      : "memory");
  return out != 0;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Paired FP32 multiply and add (PTX f32x2), each half rounded as the scalar
// instruction would round it.
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// One 32-byte record in a single 256-bit store (p 32-byte aligned).
__device__ __forceinline__ void st_record_v8(void* p, const float (&c)[kMaxCoef], int n,
                                             uint32_t i) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(c[0]),
               "f"(c[1]), "f"(c[2]), "f"(c[3]), "f"(c[4]), "f"(c[5]), "f"(__int_as_float(n)),
               "f"(__uint_as_float(i))
               : "memory");
}

struct TcShared {
  DegPartial wrun[(kTcThreads / 32) * kMaxDegrees];  // each warp's running per-degree partials
  uint64_t mbar[kTcWGs];
  uint32_t tmem_base;
  int nan;
};

// A warpgroup's trace row of the A operand, hi and lo parts.
__device__ __forceinline__ void write_a_row(unsigned char* a_hi, unsigned char* a_lo, int r,
                                            const float (&c)[kMaxCoef], bool valid) {
  float h[8], l[8];
#pragma unroll
  for (int k = 0; k < kMaxCoef; ++k) {
    const float v = valid ? c[k] : 0.0f;
    h[k] = tf32_rna(v);
    l[k] = v - h[k];  // exact; the tensor cores read its TF32 part
  }
  h[6] = h[7] = valid ? 1.0f : 0.0f;  // the y columns
  l[6] = l[7] = 0.0f;
  *reinterpret_cast<float4*>(a_hi + kcore(r, 0)) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(a_hi + kcore(r, 4)) = make_float4(h[4], h[5], h[6], h[7]);
  *reinterpret_cast<float4*>(a_lo + kcore(r, 0)) = make_float4(l[0], l[1], l[2], l[3]);
  *reinterpret_cast<float4*>(a_lo + kcore(r, 4)) = make_float4(l[4], l[5], l[6], l[7]);
}

// The three products of one chunk into the warpgroup's accumulator columns,
// committed to its mbarrier.  Every thread of the warpgroup calls it after
// writing its A row (or after reading the previous chunk's columns), with
// `bad` set when its last wait ran out; then nothing is issued and every
// thread of the warpgroup gets true.
__device__ __forceinline__ bool issue_chunk(int g, int r, uint32_t tmem_d, uint32_t a_hi,
                                            uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                            int n_cols, uint32_t mbar, bool bad) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A rows visible to the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if (wg_sync_any(g, bad)) return true;
  if (r == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = kTcIdescBase | ((uint32_t)(n_cols >> 3) << 17);
    const uint64_t ah = tc_desc(a_hi, 128, 256), al = tc_desc(a_lo, 128, 256);
    const uint64_t bh = tc_desc(b_hi, 128, 256), bl = tc_desc(b_lo, 128, 256);
    asm volatile(
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %3, 1;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %5, %2, %3, 1;\n"
        ::"r"(tmem_d), "l"(ah), "l"(bh), "r"(idesc), "l"(bl), "l"(al)
        : "memory");
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar)
                 : "memory");
  }
  return false;
}

// Fold the warp's traces (one per lane: log-weight, degree index d in [0, 4)
// or -1, global index, coefficients) into the warp's running per-degree
// partials.  A trace more than kTcSkipNats below its degree's running
// maximum carries a weight below e^-50 of it and is skipped; NaN log-weights
// only raise the flag.
__device__ __forceinline__ void fold_warp(DegPartial* wr, float lw, int d, int idx,
                                          const float (&c)[kMaxCoef], int lane, int& nan) {
  float thr = -INFINITY;
#pragma unroll
  for (int k = 0; k < kMaxDegrees; ++k)
    if (d == k) thr = wr[k].m - kTcSkipNats;
  const bool is_nan = d >= 0 && lw != lw;
  nan |= is_nan;
  bool cand = d >= 0 && !is_nan && lw > thr;
  unsigned cm = __ballot_sync(0xffffffffu, cand);
  if (!cm) return;
  if (__popc(cm) > kTcSerialMerges) {
    // many traces above the running thresholds (a warp's first tiles): a
    // trace more than kTcSkipNats below the best of its degree in this tile
    // is negligible as well
    float tmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < kMaxDegrees; ++k) {
      float m = (cand && d == k) ? lw : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (d == k) tmax = m;
    }
    cand = cand && lw > tmax - kTcSkipNats;
    cm = __ballot_sync(0xffffffffu, cand);
  }
  if (__popc(cm) <= kTcSerialMerges) {
    while (cm) {
      const int src = __ffs(cm) - 1;
      cm &= cm - 1;
      const float v = __shfl_sync(0xffffffffu, lw, src);
      const int dv = __shfl_sync(0xffffffffu, d, src);
      const int iv = __shfl_sync(0xffffffffu, idx, src);
      float cc[kMaxCoef];
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) cc[k] = __shfl_sync(0xffffffffu, c[k], src);
      if (lane == 0) {
        DegPartial p;
        deg_empty(p);
        p.m = v;
        p.arg = iv;
        if (v > -INFINITY) {
          p.S = 1.0f;
          p.S2 = 1.0f;
#pragma unroll
          for (int k = 0; k < kMaxCoef; ++k) p.mean[k] = cc[k];
        }
        deg_merge(wr[dv], p);
      }
      __syncwarp();
    }
    return;
  }
  for (int dd = 0; dd < kMaxDegrees; ++dd) {
    const bool mine = cand && d == dd;
    if (!__any_sync(0xffffffffu, mine)) continue;
    float m = mine ? lw : -INFINITY;
    int a = mine ? idx : 0x7fffffff, src = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float om = __shfl_xor_sync(0xffffffffu, m, o);
      const int oa = __shfl_xor_sync(0xffffffffu, a, o);
      const int os = __shfl_xor_sync(0xffffffffu, src, o);
      if (om > m || (om == m && oa < a)) {
        m = om;
        a = oa;
        src = os;
      }
    }
    if (!(m > -INFINITY)) continue;  // only -inf traces of this degree
    float ref[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) ref[k] = __shfl_sync(0xffffffffu, c[k], src);
    const float w = (mine && lw > -INFINITY) ? expf(lw - m) : 0.0f;
    const float S = warp_sum(w), S2 = warp_sum(w * w);
    float A[kMaxCoef], B[kMaxCoef];
#pragma unroll
    for (int k = 0; k < kMaxCoef; ++k) {
      const float dc = mine ? c[k] - ref[k] : 0.0f;
      const float t = w * dc;
      A[k] = warp_sum(t);
      B[k] = warp_sum(t * dc);
    }
    if (lane == 0) {
      DegPartial p;
      deg_empty(p);
      p.m = m;
      p.arg = a;
      p.S = S;
      p.S2 = S2;
      if (S > 0.0f) {
#pragma unroll
        for (int k = 0; k < kMaxCoef; ++k) {
          const float sh = A[k] / S;
          p.mean[k] = ref[k] + sh;
          p.M2[k] = fmaxf(B[k] - sh * A[k], 0.0f);
        }
      }
      deg_merge(wr[dd], p);
    }
    __syncwarp();
  }
}

}  // namespace

// kComp: the 64-point block sums of a trace add with Kahan's compensation
// (data sets above 512 points) or plainly (at most 7 additions: below 2^-21
// relative).
template <bool kComp>
__global__ void __launch_bounds__(kTcThreads, 1) poly_trace_tc_kernel(
    PolyParams p, const float* __restrict__ xs, const float* __restrict__ ys, int L, int Lp,
    int64_t N, int64_t first, uint64_t seed, uint32_t instance, float* __restrict__ lw_out,
    ppl_poly_particle* __restrict__ rec_out, WsHeader* hdr, DegPartial* parts,
    ppl_is_result* res, IsPartial* part_out) {
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  // A operands: [warpgroup][hi, lo] x 4 KB; then B hi and lo, Lp x 32 B each
  unsigned char* a_base = tc_dyn;
  unsigned char* b_hi = tc_dyn + kTcWGs * 8192;
  unsigned char* b_lo = b_hi + (size_t)Lp * 32;
  __shared__ TcShared sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid >> 7, r = tid & 127;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&sh.tmem_base)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    sh.nan = 0;
    for (int q = 0; q < kTcWGs; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sh.mbar[q]))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < (kTcThreads / 32) * kMaxDegrees; e += kTcThreads) deg_empty(sh.wrun[e]);
  // the data's B operand: powers of x in FP64, split into TF32 hi and lo; y
  // exactly as (yh, yr); padded points are zero rows (they add nothing)
  for (int l = tid; l < Lp; l += kTcThreads) {
    float h[8], lo[8];
    if (l < L) {
      const double x = (double)xs[l];
      double pw = 1.0;
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) {
        const float f = (float)pw;
        h[k] = tf32_rna(f);
        lo[k] = tf32_rna((float)(pw - (double)h[k]));
        pw *= x;
      }
      const float y = ys[l];
      const float yh = tf32_rna(y);
      const float yr = y - yh;  // exact
      h[6] = -yh;
      lo[6] = 0.0f;
      h[7] = -tf32_rna(yr);
      lo[7] = -(yr - tf32_rna(yr));  // exact, and TF32-representable
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] = lo[k] = 0.0f;
    }
    *reinterpret_cast<float4*>(b_hi + kcore(l, 0)) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(b_hi + kcore(l, 4)) = make_float4(h[4], h[5], h[6], h[7]);
    *reinterpret_cast<float4*>(b_lo + kcore(l, 0)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<float4*>(b_lo + kcore(l, 4)) = make_float4(lo[4], lo[5], lo[6], lo[7]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const uint32_t tmem_d = sh.tmem_base + (uint32_t)(g * kTcChunk);
  const uint32_t t_lane = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lanes
  unsigned char* a_hi = a_base + g * 8192;
  unsigned char* a_lo = a_hi + 4096;
  const uint32_t sa_hi = smem_addr(a_hi), sa_lo = smem_addr(a_lo);
  const uint32_t sb_hi = smem_addr(b_hi), sb_lo = smem_addr(b_lo);
  const uint32_t mbar = smem_addr(&sh.mbar[g]);
  const int n_chunks = (Lp + kTcChunk - 1) / kTcChunk;
  const int64_t n_tiles = (N + kTcM - 1) / kTcM;
  const int64_t step = kTcWGs * (int64_t)gridDim.x;
  const bool rec_v8 = (reinterpret_cast<uintptr_t>(rec_out) & 31) == 0;
  DegPartial* wr = &sh.wrun[warp * kMaxDegrees];
  const PriorDraw draw{p, seed, instance};
  uint32_t phase = 0;
  int nan = 0;

  int64_t tile = kTcWGs * (int64_t)blockIdx.x + g;
  float c[kMaxCoef];
  int n = 0;
  // trace i of this call is particle first + i of the population: its draws
  // and its recorded origin use the particle index
  auto draw_tile = [&](int64_t t, float (&cc)[kMaxCoef], int& nn) {
    const int64_t i = t * kTcM + r;
    const uint32_t gi = (uint32_t)(first + (i < N ? i : 0));
    float corr;
    nn = draw(gi, cc, corr);
    if (i < N && rec_out) {
      if (rec_v8) {
        st_record_v8(rec_out + i, cc, nn, gi);
      } else {
        float4* dst = reinterpret_cast<float4*>(rec_out + i);
        dst[0] = make_float4(cc[0], cc[1], cc[2], cc[3]);
        dst[1] = make_float4(cc[4], cc[5], __int_as_float(nn), __uint_as_float(gi));
      }
    }
  };
  bool bad = false;  // a wait of this thread ran out
  if (tile < n_tiles) {
    draw_tile(tile, c, n);
    if (n_chunks > 0) {
      write_a_row(a_hi, a_lo, r, c, tile * kTcM + r < N);
      issue_chunk(g, r, tmem_d, sa_hi, sa_lo, sb_hi, sb_lo, min(Lp, kTcChunk), mbar, false);
    }
  }
  bool stop = false;  // the same in every thread of the warpgroup
  for (; tile < n_tiles && !stop; tile += step) {
    const int64_t i = tile * kTcM + r;
    const bool valid = i < N;
    // the next tile's draws run while this tile's products are computed
    const int64_t next = tile + step;
    float cn[kMaxCoef];
    int nn = 0;
    if (next < n_tiles) draw_tile(next, cn, nn);
    float ss = 0.0f, comp = 0.0f;
    for (int j = 0; j < n_chunks; ++j) {
      const int cols = min(kTcChunk, Lp - j * kTcChunk);
      if (!tc_wait(mbar, phase)) {
        bad = true;
        record_status(&hdr->status, PPL_ETIMEOUT);
      }
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int c0 = 0; c0 < cols; c0 += 64) {
        float v0[32], v1[32];
        tmem_ld32(tmem_d + t_lane + (uint32_t)c0, v0);
        const bool two = c0 + 32 < cols;  // the same for the whole warp
        if (two) tmem_ld32(tmem_d + t_lane + (uint32_t)(c0 + 32), v1);
        tmem_wait_ld();
        // squares summed in f32x2 pairs, four pair accumulators
        unsigned long long acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned long long d = f2_pack(v0[2 * q], v0[2 * q + 1]);
          acc[q] = f2_mul(d, d);
        }
#pragma unroll
        for (int q = 4; q < 16; ++q) {
          const unsigned long long d = f2_pack(v0[2 * q], v0[2 * q + 1]);
          acc[q & 3] = f2_fma(d, d, acc[q & 3]);
        }
        if (two) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const unsigned long long d = f2_pack(v1[2 * q], v1[2 * q + 1]);
            acc[q & 3] = f2_fma(d, d, acc[q & 3]);
          }
        }
        const float2 a01 = f2_unpack(f2_add(acc[0], acc[1]));
        const float2 a23 = f2_unpack(f2_add(acc[2], acc[3]));
        const float block = (a01.x + a01.y) + (a23.x + a23.y);
        if (kComp) kahan_add(ss, comp, block);
        else ss += block;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (j + 1 < n_chunks &&
          issue_chunk(g, r, tmem_d, sa_hi, sa_lo, sb_hi + (uint32_t)((j + 1) * kTcChunk * 32),
                      sb_lo + (uint32_t)((j + 1) * kTcChunk * 32),
                      min(kTcChunk, Lp - (j + 1) * kTcChunk), mbar, bad)) {
        stop = true;
        break;
      }
    }
    if (stop) break;
    const float lw = ss * p.neg_half_inv_var;
    if (valid && lw_out) lw_out[i] = lw;
    fold_warp(wr, lw, valid ? n - p.min_deg : -1, (int)(first + i), c, lane, nan);
    if (next < n_tiles) {
#pragma unroll
      for (int k = 0; k < kMaxCoef; ++k) c[k] = cn[k];
      n = nn;
      if (n_chunks > 0) {
        write_a_row(a_hi, a_lo, r, c, next * kTcM + r < N);
        stop = issue_chunk(g, r, tmem_d, sa_hi, sa_lo, sb_hi, sb_lo, min(Lp, kTcChunk), mbar,
                           bad);
      }
    }
  }

  nan = __any_sync(0xffffffffu, nan);
  if (lane == 0 && nan) sh.nan = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem_base),
                 "r"(kTcTmemCols)
                 : "memory");
  // merge the warps' partials: warp d merges degree d over the 16 warps
  // (lane w < 16 holds warp w's partial; lanes 16-31 an empty one)
  if (warp < kMaxDegrees) {
    DegPartial q;
    deg_empty(q);
    if (lane < kTcThreads / 32) q = sh.wrun[lane * kMaxDegrees + warp];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const DegPartial other = deg_shfl_xor(q, o);
      deg_merge(q, other);
    }
    if (lane == 0) parts[blockIdx.x * kMaxDegrees + warp] = q;
  }
  if (tid == 0 && sh.nan) record_status(&hdr->status, PPL_ENAN);
  if (elect_last_block(&hdr->ticket[0])) {
    if (part_out) finalize_to_partial(parts, gridDim.x, p.n_deg, p.min_deg, N, hdr, part_out);
    else finalize_partials(parts, gridDim.x, p.n_deg, p.min_deg, N, hdr, res);
  }
}

// The summary of a population from its shards' partials (one block); the
// population's size is the sum of the shards'.
__global__ void __launch_bounds__(256) merge_shards_kernel(const IsPartial* parts, int P,
                                                           ppl_is_result* res) {
  __shared__ int64_t n_sh;
  if (threadIdx.x == 0) {
    int64_t n = 0;
    for (int g = 0; g < P; ++g) n += parts[g].n;
    n_sh = n;
  }
  __syncthreads();
  merge_shard_partials(parts, P, n_sh, 0, res);
}

// Largest data set the tensor-core trace kernel stages in shared memory.
int trace_tc_max_points() { return kTcMaxPoints; }

size_t trace_tc_smem(int64_t L) {
  const int64_t Lp = (L + 31) / 32 * 32;
  return (size_t)kTcWGs * 8192 + (size_t)Lp * 64;
}

cudaError_t launch_merge_shards(const void* parts, int P, ppl_is_result* res, cudaStream_t s) {
  merge_shards_kernel<<<1, 256, 0, s>>>((const IsPartial*)parts, P, res);
  return cudaGetLastError();
}

cudaError_t launch_poly_trace_tc(const PolyParams& p, const float* x, const float* y, int64_t L,
                                 int64_t N, uint64_t seed, uint32_t instance, float* lw_out,
                                 ppl_poly_particle* rec_out, WsHeader* hdr, void* parts,
                                 ppl_is_result* res, cudaStream_t s, int64_t first,
                                 void* part_out) {
  if (L < 0 || L > kTcMaxPoints) return cudaErrorInvalidValue;
  const int Lp = (int)((L + 31) / 32 * 32);
  const size_t smem = trace_tc_smem(L);
  // the largest shared-memory size, once per device (the attribute is per
  // device; setting it is a slow host call)
  const bool comp = Lp > 4 * kTcChunk;
  const void* fn = comp ? (const void*)poly_trace_tc_kernel<true>
                        : (const void*)poly_trace_tc_kernel<false>;
  int unused = 0;
  cudaError_t e = device_once(fn, &unused, [fn](int*) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)trace_tc_smem(kTcMaxPoints));
  });
  if (e != cudaSuccess) return e;
  const int64_t tiles = (N + kTcM - 1) / kTcM;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((tiles + kTcWGs - 1) / kTcWGs, num_sms()));
  if (comp)
    poly_trace_tc_kernel<true><<<grid, kTcThreads, smem, s>>>(
        p, x, y, (int)L, Lp, N, first, seed, instance, lw_out, rec_out, hdr, (DegPartial*)parts,
        res, (IsPartial*)part_out);
  else
    poly_trace_tc_kernel<false><<<grid, kTcThreads, smem, s>>>(
        p, x, y, (int)L, Lp, N, first, seed, instance, lw_out, rec_out, hdr, (DegPartial*)parts,
        res, (IsPartial*)part_out);
  return cudaGetLastError();
}

}  // namespace ppl
