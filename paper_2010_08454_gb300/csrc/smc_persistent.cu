// The whole bootstrap particle filter on the linear-Gaussian state-space model
// in one persistent, cooperative kernel (particle methods: the paper's stated
// future work, §6; observe as in §3.4, Fig. 2).  One block of 1024 threads per
// SM; each thread keeps its R particles' state and log-weights in registers
// for all T steps; the steps are separated by grid barriers instead of kernel
// launches.  The arithmetic of a step is exactly that of ppl_smc_step (same
// draws, same FP32 operations, same fixed-point systematic resampling), so
// both give the same particles.
//
// A step is: propagate and weight (registers) -> block partial -> barrier 1,
// after which every block merges all the partials itself, in one fixed order,
// so that all take the same resampling decision; when resampling: fixed-point
// weights and block totals -> barrier 2, after which every block scans all
// the totals itself and finds which output slots its particles are the
// ancestors of -> each block finds those ancestors by a merge of its prefix
// sums with the slots' positions, in shared memory, and writes the slots ->
// barrier 3 -> every thread reads its slots.  The three barriers are plain
// arrival counts: a merge or scan done once by the last arriving block and
// published to the others would add its own latency and that of the release
// to every step, for a few kilobytes that every block reads from L2 in one
// round trip.
//
// Every barrier wait is bounded; a block whose wait runs out records
// PPL_ETIMEOUT and every block leaves at its next wait, so the kernel always
// ends.  The launch is cooperative, which guarantees that all blocks are
// resident at once (or fails to launch).
#include <algorithm>

#include "dfloat.cuh"
#include "gridsync.cuh"
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

constexpr int kSmcTpb = 1024;          // threads of a block: one block per SM
constexpr int kSmcWarps = kSmcTpb / 32;
constexpr int kSmcMaxGrid = kSmcTpb;   // the merging block holds one partial per thread
constexpr int kSmcOut = 24576;         // outputs a block stages in shared memory

// A block's normalisation partial: m = max lw, s = sum exp(lw - m),
// s2 = sum exp(2 (lw - m)), nan = some lw is NaN.  One 16-byte load.
struct __align__(16) SmcPart {
  float m, s, s2;
  int nan;
};

// What one step leaves for the evidence and ESS outputs, which are formed in
// FP64 once after the last step: M the maximum log-weight, S and S2 the sums of
// exp(lw - M) and exp(2 (lw - M)) as unevaluated FP32 pairs.
struct __align__(16) SmcStep {
  float M, s_hi, s_lo, s2_hi, s2_lo;
  int32_t flag, pad[2];
};

// Control block at offset 0 of the workspace: the status word (first, where
// ppl_workspace_status reads it) on its own line, then the barrier words.
struct __align__(128) SmcCtl {
  int32_t status;
  int32_t pad[31];
  GridCtl g;
};

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
  SmcPart* parts;      // [2][grid] block partials of even and odd steps
  uint64_t* bsum;      // [grid] block totals of the fixed-point weights
  SmcStep* stash;      // [T]
  float* xbuf;         // [N] the resampled states, by output slot
};

// Thread `tid` of block b holds particles i0 .. i0 + R - 1, i0 = (b kSmcTpb + tid) R,
// so a thread's fixed-point weights are consecutive terms of the prefix sum.
template <int R>
__global__ void __launch_bounds__(kSmcTpb, 1) smc_persistent_kernel(SmcArgs a) {
  constexpr int64_t P = (int64_t)kSmcTpb * R;  // particles of one block
  extern __shared__ __align__(16) unsigned char smc_dyn[];
  uint64_t* sA = reinterpret_cast<uint64_t*>(smc_dyn);  // [P] weights, then local prefix sums
  float* sX = reinterpret_cast<float*>(sA + P);           // [P] states
  float* sx = sX + P;                                     // [kSmcOut] this block's outputs
  __shared__ float sh_max[kSmcWarps];
  __shared__ int sh_nan[kSmcWarps];
  __shared__ float2 sh_s[kSmcWarps];
  __shared__ float j_max[kSmcWarps];
  __shared__ int j_nan[kSmcWarps];
  __shared__ float2 j_s[kSmcWarps], j_s2[kSmcWarps];
  __shared__ uint64_t sh_tot[kSmcWarps], j_tot[kSmcWarps];
  __shared__ double sh_z[kSmcWarps];
  __shared__ unsigned long long rel;
  __shared__ uint64_t view[6];  // T, stride, u, C at the block start, K_b, K_b+1
  __shared__ unsigned long long decision;  // bad << 33 | resample << 32 | bits of M
  __shared__ uint32_t resample_word;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * P + (int64_t)tid * R;
  const int64_t N = a.N;
  SmcCtl* ctl = a.ctl;
  float x[R], lw[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    x[r] = 0.0f;
    lw[r] = 0.0f;
  }
  int S = 0;
  while (((int64_t)1 << S) < N) ++S;
  const float scale = __int_as_float((127 + 61 - S) << 23);  // 2^(61 - ceil(log2 N))
  const float half_n = 0.5f * (float)N;                      // exact: N < 2^24
  unsigned long long e = 0;                                  // barriers passed
  float y_next = a.y[0];

  for (int t = 1; t <= a.T; ++t) {
    if (tid == 0) resample_word = philox_block(a.seed, 0, 0, (uint32_t)t, kResample, 0).x;
    const float yt = y_next;
    if (t < a.T) y_next = __ldg(a.y + t);  // in flight during this step
    // this step's half of the partials: a block may write step t + 1's
    // partial while slower blocks still read step t's, but not step t + 2's
    // (it has to pass barrier 1 of step t + 1 first, which they reach only
    // after reading)
    SmcPart* const parts_t = a.parts + (size_t)(t & 1) * G;
    int nan = 0;
    float tm = -INFINITY;
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
        nan |= (li != li);
        tm = fmaxf(tm, li);
      }
    }
    // block partial: the maximum (every warp reduces the 32 warp maxima), then
    // the sums around it (warp 0 adds the 32 warp sums)
    tm = warp_max(tm);
    nan = __any_sync(0xffffffffu, nan);
    if (lane == 0) {
      sh_max[warp] = tm;
      sh_nan[warp] = nan;
    }
    __syncthreads();
    const float bm = warp_max(sh_max[lane]);
    float ts = 0.0f, ts2 = 0.0f;
    if (bm > -INFINITY) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r < N && lw[r] > -INFINITY) {
          const float ex = expf(lw[r] - bm);
          ts += ex;
          ts2 = fmaf(ex, ex, ts2);
        }
    }
    ts = warp_sum(ts);
    ts2 = warp_sum(ts2);
    if (lane == 0) sh_s[warp] = make_float2(ts, ts2);
    __syncthreads();
    if (warp == 0) {
      const float bs = warp_sum(sh_s[lane].x), bs2 = warp_sum(sh_s[lane].y);
      const int bn = __any_sync(0xffffffffu, sh_nan[lane]);
      if (lane == 0) {
        SmcPart q;
        q.m = bm;
        q.s = bs;
        q.s2 = bs2;
        q.nan = bn;
        *reinterpret_cast<float4*>(parts_t + blockIdx.x) = *reinterpret_cast<const float4*>(&q);
      }
    }
    // barrier 1, then every block merges all partials in the same fixed order
    // (thread b reads block b's): the maximum M, the sums around it as
    // double-float pairs, the NaN and empty checks and the decision
    if (!grid_sync<false>(&ctl->g, &ctl->status, G, ++e, &rel, [] { return 0ull; }, [] {})) return;
    {
      SmcPart q;
      if ((unsigned)tid < G) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(parts_t + tid));
        q = *reinterpret_cast<const SmcPart*>(&v);
      } else {
        q.m = -INFINITY;
        q.s = q.s2 = 0.0f;
        q.nan = 0;
      }
      const float gm = warp_max(q.m);
      const int gn = __any_sync(0xffffffffu, q.nan);
      if (lane == 0) {
        j_max[warp] = gm;
        j_nan[warp] = gn;
      }
      __syncthreads();
      const float M = warp_max(j_max[lane]);
      const int any_nan = __any_sync(0xffffffffu, j_nan[lane]);
      float2 Ss = make_float2(0.0f, 0.0f), Ss2 = make_float2(0.0f, 0.0f);
      if (M > -INFINITY && q.m > -INFINITY) {
        const float ex = expf(q.m - M);
        Ss = df_prod(q.s, ex);
        Ss2 = df_prod(q.s2, ex * ex);
      }
      Ss = df_warp_sum(Ss);
      Ss2 = df_warp_sum(Ss2);
      if (lane == 0) {
        j_s[warp] = Ss;
        j_s2[warp] = Ss2;
      }
      __syncthreads();
      if (warp == 0) {
        Ss = df_warp_sum(j_s[lane]);
        Ss2 = df_warp_sum(j_s2[lane]);
        if (lane == 0) {
          // ESS = S^2 / S2 < N / 2  <=>  S^2 - (N / 2) S2 < 0, in double-float
          const float2 lhs = df_mul(Ss, Ss), rhs = df_mul(make_float2(half_n, 0.0f), Ss2);
          const bool bad = any_nan || !(M > -INFINITY);
          const bool res =
              !bad && __fadd_rn(__fsub_rn(lhs.x, rhs.x), __fsub_rn(lhs.y, rhs.y)) < 0.0f;
          if (blockIdx.x == 0) {  // one block records the step
            if (any_nan) record_status(&ctl->status, PPL_ENAN);
            else if (bad) record_status(&ctl->status, PPL_EEMPTY);
            SmcStep st;
            st.M = M;
            st.s_hi = Ss.x;
            st.s_lo = Ss.y;
            st.s2_hi = Ss2.x;
            st.s2_lo = Ss2.y;
            st.flag = res ? 1 : 0;
            st.pad[0] = st.pad[1] = 0;
            a.stash[t - 1] = st;
          }
          decision = ((unsigned long long)bad << 33) | ((unsigned long long)res << 32) |
                     (unsigned long long)__float_as_uint(M);
        }
      }
      __syncthreads();
    }
    const unsigned long long r1 = decision;
    if ((r1 >> 33) & 1) return;  // a NaN or no finite weight: every block leaves
    if (!((r1 >> 32) & 1)) continue;
    const float M = __uint_as_float((uint32_t)r1);

    // 1. this thread's fixed-point weights and states (kept in shared memory in
    // particle order) and their sum, then the block's exclusive scan
    uint64_t own = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t q = i0 + r < N ? quantize(lw[r], M, scale) : 0ull;
      sA[tid * R + r] = q;
      sX[tid * R + r] = x[r];
      own = sat_add(own, q);
    }
    const uint64_t inc = warp_scan_u64(own, lane);
    if (lane == 31) sh_tot[warp] = inc;
    __syncthreads();
    uint64_t texcl, btot;
    {
      const uint64_t v = sh_tot[lane], wi = warp_scan_u64(v, lane);
      texcl = sat_add(__shfl_sync(0xffffffffu, wi - v, warp), inc - own);
      btot = __shfl_sync(0xffffffffu, wi, 31);
    }
    if (tid == 0) a.bsum[blockIdx.x] = btot;
    // barrier 2, then every block scans the G block totals itself (the same
    // integer sums in every block): T, the stride floor(T / N), the systematic
    // offset u, and the first outputs whose ancestors this block and the next
    // hold, K_b = cnt(C at the block's start), where cnt(c) = #{k >= 0 : u + k
    // stride < c} (K_G = N)
    if (!grid_sync<false>(&ctl->g, &ctl->status, G, ++e, &rel, [] { return 0ull; }, [] {})) return;
    {
      const uint64_t v = (unsigned)tid < G ? __ldcg(a.bsum + tid) : 0ull;
      const uint64_t wi = warp_scan_u64(v, lane);
      if (lane == 31) j_tot[warp] = wi;
      __syncthreads();
      const uint64_t jv = j_tot[lane], ji = warp_scan_u64(jv, lane);
      const uint64_t ex = sat_add(__shfl_sync(0xffffffffu, ji - jv, warp), wi - v);  // C at block tid's start
      const uint64_t T = __shfl_sync(0xffffffffu, ji, 31);
      const bool valid = T >= (uint64_t)N && T <= (1ull << 61);
      const unsigned b = blockIdx.x;
      if ((unsigned)tid == b || (unsigned)tid == b + 1) {  // b + 1 < G <= kSmcTpb when taken
        uint64_t stride = 0, u = 0;
        if (valid) {
          const uint64_t w0 = resample_word;
          stride = T / (uint64_t)N;
          u = (__umul64hi(w0, stride) << 32) | ((w0 * stride) >> 32);
        }
        const uint64_t k = valid ? (uint64_t)positions_below(ex, u, stride, N) : 0ull;
        if ((unsigned)tid == b) {
          view[0] = T;
          view[1] = stride;
          view[2] = u;
          view[3] = ex;
          view[4] = k;
          if (b + 1 == G) view[5] = (uint64_t)N;
        } else if (b + 1 < G) {
          view[5] = k;
        }
        if (b == 0 && tid == 0 && !valid) record_status(&ctl->status, T == 0 ? PPL_EEMPTY : PPL_EINVAL);
      }
      __syncthreads();
    }
    const uint64_t T = view[0];
    if (T < (uint64_t)N || T > (1ull << 61)) return;  // every block sees the same T and leaves
    // 2. systematic resampling of this block's outputs k in [K_b, K_b+1), whose
    // ancestors a_k = min{j : C_j > u + k stride} are all in this block: with
    // A_i the block-local inclusive prefix sums and B_j = u + (K_b + j) stride
    // - C_start, a_k is the number of A's not above B_j, i.e. B_j's place in
    // the merge of the two sorted lists (ties: A first).  The merge is cut
    // into equal slices, one per thread (merge path: Green, McColl, Bader,
    // "GPU merge path", ICS 2012); the outputs are assembled in shared memory
    // and stored to global memory whole.
    const uint64_t stride = view[1], offset = view[2], cstart = view[3];
    const int64_t Kb = (int64_t)view[4], nB = (int64_t)view[5] - Kb;
    {
      uint64_t run = texcl;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        run += sA[tid * R + r];
        sA[tid * R + r] = run;
      }
    }
    __syncthreads();
    {
      const int nA = (int)P, nBi = (int)nB;
      const int64_t L = (int64_t)nA + nB;
      const int d0 = (int)(L * tid / kSmcTpb), d1 = (int)(L * (tid + 1) / kSmcTpb);
      // B_j relative to the block start (>= 0: the outputs from K_b on lie at or past it)
      const uint64_t b0 = offset + (uint64_t)Kb * stride - cstart;
      int lo = d0 > nBi ? d0 - nBi : 0, hi = d0 < nA ? d0 : nA;
      while (lo < hi) {  // the A's among the first d0 merged items
        const int mid = (lo + hi) >> 1;
        if (sA[mid] <= b0 + (uint64_t)(d0 - 1 - mid) * stride) lo = mid + 1;
        else hi = mid;
      }
      int i = lo, j = d0 - lo;
      uint64_t bj = b0 + (uint64_t)j * stride;
      uint64_t ai = i < nA ? sA[i] : ~0ull;
      for (int s = d0; s < d1; ++s) {
        if (j >= nBi || ai <= bj) {
          ++i;
          ai = i < nA ? sA[i] : ~0ull;
        } else {  // output K_b + j: ancestor i (A_i > B_j, so i < nA)
          const float v = sX[i < nA ? i : nA - 1];
          if (j < kSmcOut) sx[j] = v;
          else a.xbuf[Kb + j] = v;  // beyond the staging area: straight to global memory
          ++j;
          bj += stride;
        }
      }
    }
    __syncthreads();
    {
      const int64_t n_staged = nB < kSmcOut ? nB : kSmcOut;
      for (int64_t j = tid; j < n_staged; j += kSmcTpb) a.xbuf[Kb + j] = sx[j];
    }
    if (!grid_sync<false>(&ctl->g, &ctl->status, G, ++e, &rel, [] { return 0ull; }, [] {})) return;
    // 3. the new population: this thread's outputs are i0 .. i0 + R - 1
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (i0 + r < N) x[r] = __ldcg(a.xbuf + i0 + r);
      lw[r] = 0.0f;
    }
  }
  // evidence and ESS of every step, in FP64, by block 0 after the last step:
  // log Z = sum over resampling steps of (lse_t - log N), plus lse_T - log N
  // when the last step did not resample (its weights are carried unnormalised)
  if (blockIdx.x == 0) {
    const double log_n = log((double)N);
    double z = 0.0;
    for (int t = tid; t < a.T; t += kSmcTpb) {
      const float4 h0 = __ldcg(reinterpret_cast<const float4*>(a.stash + t));
      const float4 h1 = __ldcg(reinterpret_cast<const float4*>(a.stash + t) + 1);
      const double S1 = (double)h0.y + (double)h0.z;
      const double S2 = (double)h0.w + (double)h1.x;
      const int flag = __float_as_int(h1.y);
      const double lse = (double)h0.x + log(S1);
      a.ess[t] = S1 * S1 / S2;
      a.resampled[t] = flag;
      if (flag || t == a.T - 1) z += lse - log_n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) sh_z[warp] = z;
    __syncthreads();
    if (warp == 0) {
      z = sh_z[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
      if (lane == 0) a.logz[0] = z;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (i0 + r < N) {
      a.x_out[i0 + r] = x[r];
      a.lw_out[i0 + r] = lw[r];
    }
}

// The filter's grid barriers with nothing between them: what the step
// separators alone cost at the filter's launch shape.
__global__ void __launch_bounds__(kSmcTpb) grid_barrier_probe_kernel(SmcCtl* ctl, int n) {
  __shared__ unsigned long long rel;
  for (int e = 1; e <= n; ++e)
    if (!grid_sync<false>(&ctl->g, &ctl->status, gridDim.x, (unsigned long long)e, &rel,
                          [] { return 0ull; }, [] {}))
      return;
}

cudaError_t launch_grid_barrier_probe(int blocks, int n_barriers, void* ws, cudaStream_t s) {
  SmcCtl* ctl = static_cast<SmcCtl*>(ws);
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(SmcCtl), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&ctl, &n_barriers};
  return cudaLaunchCooperativeKernel((const void*)grid_barrier_probe_kernel, dim3((unsigned)blocks),
                                     dim3(kSmcTpb), args, 0, s);
}

size_t smc_run_workspace(int64_t N, int64_t T) {
  return 8 * 256 + (size_t)kSmcMaxGrid * (2 * sizeof(SmcPart) + 8) +
         (size_t)std::max<int64_t>(T, 0) * sizeof(SmcStep) + (size_t)N * 4;
}

template <int R>
static cudaError_t launch_r(SmcArgs& a, cudaStream_t s, bool* fits) {
  const int64_t grid = (a.N + (int64_t)kSmcTpb * R - 1) / ((int64_t)kSmcTpb * R);
  constexpr size_t dyn = (size_t)R * kSmcTpb * (8 + 4) + (size_t)kSmcOut * 4;
  cudaError_t e = cudaFuncSetAttribute(smc_persistent_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smc_persistent_kernel<R>, kSmcTpb,
                                                    dyn);
  if (e != cudaSuccess) return e;
  *fits = grid <= std::min<int64_t>((int64_t)num_sms() * per_sm, kSmcMaxGrid);
  if (!*fits) return cudaSuccess;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)smc_persistent_kernel<R>, dim3((unsigned)grid),
                                     dim3(kSmcTpb), args, dyn, s);
}

cudaError_t launch_smc_persistent(const LgssmParams& p, const float* y, int32_t T, uint64_t seed,
                                  int64_t N, float* x_out, float* lw_out, double* logz,
                                  int32_t* resampled, double* ess, char* ws, size_t ws_bytes,
                                  int32_t** status_out, cudaStream_t s) {
  if (T < 1 || T > (1 << 27)) return cudaErrorInvalidValue;  // barrier numbers fit 30 bits
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
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = ws + off;
    off += (bytes + 255) / 256 * 256;
    return q;
  };
  a.ctl = reinterpret_cast<SmcCtl*>(take(sizeof(SmcCtl)));
  a.parts = reinterpret_cast<SmcPart*>(take(2 * (size_t)kSmcMaxGrid * sizeof(SmcPart)));
  a.bsum = reinterpret_cast<uint64_t*>(take((size_t)kSmcMaxGrid * 8));
  a.stash = reinterpret_cast<SmcStep*>(take((size_t)T * sizeof(SmcStep)));
  a.xbuf = reinterpret_cast<float*>(take((size_t)N * 4));
  if (off > ws_bytes) return cudaErrorInvalidValue;
  *status_out = &a.ctl->status;
  cudaError_t e = cudaMemsetAsync(a.ctl, 0, sizeof(SmcCtl), s);
  if (e != cudaSuccess) return e;
  // fewest particles per thread whose grid is resident at once
  bool fits = false;
  if ((e = launch_r<1>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<2>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<3>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<4>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<5>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<6>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<7>(a, s, &fits)) != cudaSuccess || fits) return e;
  if ((e = launch_r<8>(a, s, &fits)) != cudaSuccess || fits) return e;
  return cudaErrorInvalidValue;  // more particles than resident threads can hold
}

}  // namespace ppl
