// One step of the bootstrap particle filter on the linear-Gaussian state-space
// model (particle methods: the paper's stated future work, §6), with the
// observation entering through observe(dist, y) = factor(dist-score(dist, y))
// (§3.4, Fig. 2).  The step's propagate, weight and normalisation statistics
// are one kernel; its last block decides whether the step resamples and
// publishes that decision to the gated resampling kernels that follow.
#include "kernels.h"
#include "rng.cuh"
#include "stats.cuh"

namespace ppl {

__global__ void __launch_bounds__(kTpb) smc_propagate_kernel(
    LgssmParams p, float y_t, uint32_t t, uint64_t seed, float* __restrict__ x,
    float* __restrict__ lw, int64_t N, double* logz_acc, int32_t* resampled, double* logz_est,
    WsHeader* hdr, StatPartial* parts) {
  StatAcc acc;
  acc.init();
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x; i < N; i += stride) {
    // x_t = phi x_{t-1} + q e_t, e_t the reproducible FP32 normal of words 0, 1;
    // lw += -log(2 pi r^2)/2 - (y_t - x_t)^2 / (2 r^2).  FP32, one rounding per
    // operation in the order written (no contraction), so the state is the
    // value any FP32 filter of this definition holds, bit for bit, and the
    // resampling decisions taken from it agree exactly.
    const uint4 w = philox_block(seed, (uint32_t)i, 0, t, kLgssmPropagate, 0);
    const float z0 = normal32(w.x, w.y);
    const float xi = __fadd_rn(__fmul_rn(p.phi, x[i]), __fmul_rn(p.q_sigma, z0));
    const float d = __fsub_rn(y_t, xi);
    const float li =
        __fadd_rn(lw[i], __fadd_rn(p.obs_const, __fmul_rn(__fmul_rn(p.neg_half_inv_r2, d), d)));
    x[i] = xi;
    lw[i] = li;
    acc.add(li, (int)i, -1);
  }
  StatAcc r = block_reduce_stat(acc);
  if (threadIdx.x == 0) to_partial(r, parts + blockIdx.x);
  if (!elect_last_block(&hdr->ticket[0])) return;
  finalize_stats(parts, gridDim.x, N, nullptr, hdr, nullptr, nullptr);
  if (threadIdx.x == 0) {
    const double lse = hdr->lse, ess = hdr->ess;
    const double log_n = log((double)N);
    const int flag = (ess < 0.5 * (double)N) ? 1 : 0;
    double acc_z = *logz_acc;
    double est;
    if (flag) {
      acc_z += lse - log_n;
      *logz_acc = acc_z;
      est = acc_z;  // the weights are reset to equal: LSE(0) - log N = 0
    } else {
      est = acc_z + lse - log_n;
    }
    hdr->resample_flag = flag;
    *resampled = flag;
    logz_est[0] = est;
    logz_est[1] = ess;
  }
}

// After a resampling step: x = gathered x, lw = 0.
__global__ void __launch_bounds__(kTpb) smc_commit_kernel(float* __restrict__ x,
                                                          const float* __restrict__ x_tmp,
                                                          float* __restrict__ lw, int64_t N,
                                                          const int32_t* gate) {
  if (*gate == 0) return;
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t i = (int64_t)blockIdx.x * kTpb + threadIdx.x; i < N; i += stride) {
    x[i] = x_tmp[i];
    lw[i] = 0.0f;
  }
}

cudaError_t launch_smc_propagate(const LgssmParams& p, float y_t, int32_t t, uint64_t seed,
                                 float* x, float* lw, int64_t N, double* logz_acc,
                                 int32_t* resampled, double* logz_est, WsHeader* hdr,
                                 void* parts, cudaStream_t s) {
  smc_propagate_kernel<<<stream_grid(N), kTpb, 0, s>>>(p, y_t, (uint32_t)t, seed, x, lw, N,
                                                       logz_acc, resampled, logz_est, hdr,
                                                       (StatPartial*)parts);
  return cudaGetLastError();
}

cudaError_t launch_smc_commit(float* x, const float* x_tmp, float* lw, int64_t N,
                              const int32_t* gate, cudaStream_t s) {
  smc_commit_kernel<<<stream_grid(N), kTpb, 0, s>>>(x, x_tmp, lw, N, gate);
  return cudaGetLastError();
}

}  // namespace ppl
