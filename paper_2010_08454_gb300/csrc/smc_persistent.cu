// The whole bootstrap particle filter on the linear-Gaussian state-space model
// in one persistent, cooperative kernel (particle methods: the paper's stated
// future work, §6; observe as in §3.4, Fig. 2).  Each thread keeps its
// particles' state and log-weights in registers for all T steps; the steps are
// separated by grid barriers instead of kernel launches.  The arithmetic of a
// step is exactly that of ppl_smc_step (same draws, same FP32 operations, same
// fixed-point systematic resampling), so both give the same particles.
//
// Barriers spin on a generation counter with a bound; a block whose wait runs
// out records PPL_ETIMEOUT and every block leaves at its next barrier, so the
// kernel always ends.  The launch is cooperative, which guarantees that all
// blocks are resident at once (or fails to launch).
#include <algorithm>

#include "fixedpoint.cuh"
#include "kernels.h"
#include "rng.cuh"
#include "stats.cuh"

namespace ppl {

constexpr int kSmcSpin = 1 << 22;      // bound of one barrier wait (polls)
constexpr int kSmcSmem = 4096;         // prefix sums staged per block for the ancestor search

// Control words at offset 0 of the workspace: the status first, where
// ppl_workspace_status reads it.
struct SmcCtl {
  int32_t status;
  unsigned count, gen;  // barrier
  int32_t pad;
};

// Grid barrier with a bounded wait.  Returns false when the kernel must stop.
__device__ __forceinline__ bool grid_barrier(SmcCtl* ctl, unsigned nblocks) {
  __shared__ bool ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = true;
    if (ld_volatile_i32(&ctl->status) != 0) {
      ok = false;
    } else {
      const unsigned g = *reinterpret_cast<volatile unsigned*>(&ctl->gen);
      __threadfence();
      if (atomicAdd(&ctl->count, 1u) == nblocks - 1) {
        atomicExch(&ctl->count, 0u);
        __threadfence();
        atomicAdd(&ctl->gen, 1u);
      } else {
        int spins = 0;
        while (*reinterpret_cast<volatile unsigned*>(&ctl->gen) == g) {
          if (ld_volatile_i32(&ctl->status) != 0) {  // another block gave up
            ok = false;
            break;
          }
          if (++spins > kSmcSpin) {
            record_status(&ctl->status, PPL_ETIMEOUT);
            ok = false;
            break;
          }
          if (spins > 32) __nanosleep(64);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return ok;
}

struct SmcArgs {
  LgssmParams p;
  const float* y;  // [T]
  int32_t T;
  uint64_t seed;
  int64_t N;
  float* x_out;
  float* lw_out;
  double* logz;        // [1]
  int32_t* resampled;  // [T]
  double* ess;         // [T]
  SmcCtl* ctl;
  StatPartial* parts;  // [2 x grid]
  uint64_t* bsum;      // [grid]
  uint64_t* C;         // [N]
  float* xbuf;         // [N]
};

// Thread `tid` of block b holds particles i0 .. i0 + R - 1, i0 = (b kTpb + tid) R,
// so a thread's fixed-point weights are consecutive terms of the prefix sum.
template <int R>
__global__ void __launch_bounds__(kTpb, 4) smc_persistent_kernel(SmcArgs a) {
  __shared__ uint64_t sC[kSmcSmem];
  __shared__ uint64_t warp_tot[kTpb / 32];
  __shared__ uint64_t red[2][kTpb / 32];
  __shared__ int64_t bound_sh[2];
  __shared__ double stat_sh[3];
  __shared__ float M_sh;
  __shared__ int nan_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  const int64_t base = (int64_t)blockIdx.x * kTpb * R;
  const int64_t i0 = base + (int64_t)tid * R;
  const int64_t N = a.N;
  float x[R], lw[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    x[r] = 0.0f;
    lw[r] = 0.0f;
  }
  double logz_acc = 0.0, last_lse = 0.0;
  bool last_resampled = false;
  const double log_n = log((double)N);
  int S = 0;
  while (((int64_t)1 << S) < N) ++S;
  const float scale = __int_as_float((127 + 61 - S) << 23);  // 2^(61 - ceil(log2 N))

  for (int t = 1; t <= a.T; ++t) {
    const float yt = a.y[t - 1];
    StatAcc acc;
    acc.init();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = i0 + r;
      if (i < N) {
        // the FP32 operations of ppl_smc_step, in its order, one rounding each
        const uint4 w = philox_block(a.seed, (uint32_t)i, 0, (uint32_t)t, kLgssmPropagate, 0);
        const float z0 = normal32(w.x, w.y);
        const float xi = __fadd_rn(__fmul_rn(a.p.phi, x[r]), __fmul_rn(a.p.q_sigma, z0));
        const float d = __fsub_rn(yt, xi);
        const float li = __fadd_rn(
            lw[r], __fadd_rn(a.p.obs_const, __fmul_rn(__fmul_rn(a.p.neg_half_inv_r2, d), d)));
        x[r] = xi;
        lw[r] = li;
        acc.add(li, (int)i, -1);
      }
    }
    // partials are double-buffered by step parity: a block can be at most one
    // barrier ahead, so it never overwrites partials another block still reads
    StatPartial* parts = a.parts + (size_t)(t & 1) * G;
    {
      StatAcc br = block_reduce_stat(acc);
      if (tid == 0) to_partial(br, parts + blockIdx.x);
    }
    if (!grid_barrier(a.ctl, G)) return;
    // every block merges all partials in the same fixed order, so every block
    // holds the same LSE and ESS and takes the same resampling decision
    {
      StatAcc m;
      m.init();
      for (unsigned b = tid; b < G; b += kTpb) {
        const StatPartial* q = parts + b;
        StatAcc o;
        o.init();
        o.m = __ldcg(&q->m);
        o.s = __ldcg(&q->s);
        o.s2 = __ldcg(&q->s2);
        o.arg = __ldcg(&q->arg);
        o.nan = __ldcg(&q->nan);
        m.merge(o);
      }
      StatAcc rr = block_reduce_stat(m);
      if (tid == 0) {
        M_sh = rr.m;
        nan_sh = rr.nan;
      }
      __syncthreads();
      const float M = M_sh;
      double s = 0.0, s2 = 0.0;
      if (M > -INFINITY)
        for (unsigned b = tid; b < G; b += kTpb) {
          const StatPartial* q = parts + b;
          const float qm = __ldcg(&q->m);
          if (qm == -INFINITY) continue;
          const double e = (double)expf(qm - M);
          s += (double)__ldcg(&q->s) * e;
          s2 += (double)__ldcg(&q->s2) * e * e;
        }
      s = block_sum_f64(s);
      s2 = block_sum_f64(s2);
      if (tid == 0) {
        stat_sh[0] = (double)M + log(s);
        stat_sh[1] = s * s / s2;
        stat_sh[2] = (double)M;
        if (nan_sh) record_status(&a.ctl->status, PPL_ENAN);
        else if (!(M > -INFINITY)) record_status(&a.ctl->status, PPL_EEMPTY);
      }
      __syncthreads();
    }
    const double lse = stat_sh[0], ess = stat_sh[1];
    const float M = (float)stat_sh[2];
    const bool resample = ess < 0.5 * (double)N;
    if (blockIdx.x == 0 && tid == 0) {
      a.ess[t - 1] = ess;
      a.resampled[t - 1] = resample ? 1 : 0;
    }
    last_lse = lse;
    last_resampled = resample;
    if (!resample) continue;
    logz_acc += lse - log_n;

    // 1. this thread's sum of fixed-point weights, then the block's exclusive scan
    uint64_t own = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i0 + r < N) own = sat_add(own, quantize(lw[r], M, scale));
    uint64_t inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = sat_add(inc, v);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint64_t texcl = inc - own, btot = 0;
#pragma unroll
    for (int w = 0; w < kTpb / 32; ++w) {
      if (w < warp) texcl = sat_add(texcl, warp_tot[w]);
      btot = sat_add(btot, warp_tot[w]);
    }
    if (tid == 0) a.bsum[blockIdx.x] = btot;
    // the state goes to global memory for the gather
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i0 + r < N) a.xbuf[i0 + r] = x[r];
    if (!grid_barrier(a.ctl, G)) return;
    // 2. the grid's exclusive prefix of this block and the total T
    uint64_t bexcl = 0, T = 0;
    {
      uint64_t be = 0, tt = 0;
      for (unsigned b = tid; b < G; b += kTpb) {
        const uint64_t v = __ldcg(a.bsum + b);
        tt = sat_add(tt, v);
        if (b < blockIdx.x) be = sat_add(be, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        be = sat_add(be, __shfl_xor_sync(0xffffffffu, be, o));
        tt = sat_add(tt, __shfl_xor_sync(0xffffffffu, tt, o));
      }
      if (lane == 0) {
        red[0][warp] = be;
        red[1][warp] = tt;
      }
      __syncthreads();
#pragma unroll
      for (int w = 0; w < kTpb / 32; ++w) {
        bexcl = sat_add(bexcl, red[0][w]);
        T = sat_add(T, red[1][w]);
      }
      __syncthreads();
    }
    if (T == 0 || T > (1ull << 61)) {  // every block sees the same T and leaves here
      if (blockIdx.x == 0 && tid == 0)
        record_status(&a.ctl->status, T == 0 ? PPL_EEMPTY : PPL_EINVAL);
      return;
    }
    // 3. inclusive prefix sums C_i (the weights are recomputed: same values)
    {
      uint64_t run = sat_add(bexcl, texcl);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r < N) {
          run = sat_add(run, quantize(lw[r], M, scale));
          a.C[i0 + r] = run;
        }
    }
    if (!grid_barrier(a.ctl, G)) return;
    // 4. systematic positions u + k stride and their ancestors a_k = min{j : C_j > u + k stride}
    const uint64_t stride = T / (uint64_t)N;
    const uint32_t w0 = philox_block(a.seed, 0, 0, (uint32_t)t, kResample, 0).x;
    const uint64_t offset =
        (__umul64hi((uint64_t)w0, stride) << 32) | (((uint64_t)w0 * stride) >> 32);
    const int64_t k_last = (base + kTpb * R < N ? base + kTpb * R : N) - 1;
    if (warp < 2) {
      const int64_t k = warp == 0 ? base : k_last;
      const int64_t j = warp_upper_bound<true>(a.C, 0, N, offset + (uint64_t)k * stride, lane);
      if (lane == 0) bound_sh[warp] = j < N - 1 ? j : N - 1;
    }
    __syncthreads();
    const int64_t jlo = bound_sh[0], jhi = bound_sh[1];
    const int64_t span = jhi - jlo + 1;
    const bool staged = span <= kSmcSmem;
    if (staged)
      for (int64_t j = tid; j < span; j += kTpb) sC[j] = __ldcg(a.C + jlo + j);
    __syncthreads();
    int64_t lo = 0;  // ancestors are non-decreasing in k: each search starts at the last
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t k = i0 + r;
      if (k < N) {
        const uint64_t pk = offset + (uint64_t)k * stride;
        int64_t hi = span;
        if (staged) {
          while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (sC[mid] > pk) hi = mid;
            else lo = mid + 1;
          }
        } else {
          while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (__ldcg(a.C + jlo + mid) > pk) hi = mid;
            else lo = mid + 1;
          }
        }
        x[r] = __ldcg(a.xbuf + jlo + (lo < span ? lo : span - 1));
        lw[r] = 0.0f;
      }
    }
    __syncthreads();  // sC and bound_sh are reused by the next resampling step
  }
  // evidence: accumulated normalisers plus the unnormalised last step
  if (blockIdx.x == 0 && tid == 0)
    a.logz[0] = logz_acc + (last_resampled ? 0.0 : last_lse - log_n);
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (i0 + r < N) {
      a.x_out[i0 + r] = x[r];
      a.lw_out[i0 + r] = lw[r];
    }
}

size_t smc_run_workspace(int64_t N) {
  const size_t grid = (size_t)kMaxBlocks;
  return 5 * 256 + grid * (2 * sizeof(StatPartial) + 8) + (size_t)N * (8 + 4);
}

template <int R>
static cudaError_t launch_r(SmcArgs& a, int64_t max_blocks, cudaStream_t s, bool* fits) {
  const int64_t grid = (a.N + (int64_t)kTpb * R - 1) / ((int64_t)kTpb * R);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smc_persistent_kernel<R>,
                                                                kTpb, 0);
  if (e != cudaSuccess) return e;
  *fits = grid <= std::min<int64_t>((int64_t)num_sms() * per_sm, max_blocks);
  if (!*fits) return cudaSuccess;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)smc_persistent_kernel<R>, dim3((unsigned)grid),
                                     dim3(kTpb), args, 0, s);
}

cudaError_t launch_smc_persistent(const LgssmParams& p, const float* y, int32_t T, uint64_t seed,
                                  int64_t N, float* x_out, float* lw_out, double* logz,
                                  int32_t* resampled, double* ess, char* ws, size_t ws_bytes,
                                  int32_t** status_out, cudaStream_t s) {
  SmcArgs a;
  a.p = p;
  a.y = y;
  a.T = T;
  a.seed = seed;
  a.N = N;
  a.x_out = x_out;
  a.lw_out = lw_out;
  a.logz = logz;
  a.resampled = resampled;
  a.ess = ess;
  const int64_t max_blocks = kMaxBlocks;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = ws + off;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  a.ctl = reinterpret_cast<SmcCtl*>(take(sizeof(SmcCtl)));
  a.parts = reinterpret_cast<StatPartial*>(take(2 * (size_t)max_blocks * sizeof(StatPartial)));
  a.bsum = reinterpret_cast<uint64_t*>(take((size_t)max_blocks * 8));
  a.C = reinterpret_cast<uint64_t*>(take((size_t)N * 8));
  a.xbuf = reinterpret_cast<float*>(take((size_t)N * 4));
  if (off > ws_bytes) return cudaErrorInvalidValue;
  *status_out = &a.ctl->status;
  cudaError_t e = cudaMemsetAsync(a.ctl, 0, sizeof(SmcCtl), s);
  if (e != cudaSuccess) return e;
  // fewest particles per thread whose grid is resident at once
  bool fits = false;
  if ((e = launch_r<1>(a, max_blocks, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<2>(a, max_blocks, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<4>(a, max_blocks, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<8>(a, max_blocks, s, &fits)) != cudaSuccess || fits) return e;
  return cudaErrorInvalidValue;  // more particles than resident threads can hold
}

}  // namespace ppl
