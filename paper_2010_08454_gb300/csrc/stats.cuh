// Block-level reductions of the normalisation statistics and the last-block
// finalisation shared by the likelihood-weighting and SMC kernels.
#pragma once

#include "common.cuh"
#include "poly.cuh"

namespace ppl {

// ---------------------------------------------------------------------------
// Block-level reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ StatAcc block_reduce_stat(StatAcc a) {
  __shared__ StatPartial slots[kTpb / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a.merge(a.shfl_xor(o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    StatPartial& p = slots[warp];
    p.m = a.m;
    p.s = a.s;
    p.s2 = a.s2;
    p.arg = a.arg;
    p.nan = a.nan;
    for (int k = 0; k < kMaxDegrees; ++k) {
      p.dm[k] = a.dm[k];
      p.darg[k] = a.darg[k];
    }
  }
  __syncthreads();
  StatAcc r;
  r.init();
  if (warp == 0) {
    if (lane < kTpb / 32) {
      const StatPartial& p = slots[lane];
      r.m = p.m;
      r.s = p.s;
      r.s2 = p.s2;
      r.arg = p.arg;
      r.nan = p.nan;
      for (int k = 0; k < kMaxDegrees; ++k) {
        r.dm[k] = p.dm[k];
        r.darg[k] = p.darg[k];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r.merge(r.shfl_xor(o));
  }
  __syncthreads();
  return r;  // valid in warp 0
}

__device__ __forceinline__ void to_partial(const StatAcc& a, StatPartial* p) {
  p->m = a.m;
  p->s = a.s;
  p->s2 = a.s2;
  p->arg = a.arg;
  p->nan = a.nan;
  for (int k = 0; k < kMaxDegrees; ++k) {
    p->dm[k] = a.dm[k];
    p->darg[k] = a.darg[k];
  }
}

__device__ __forceinline__ double block_sum_f64(double v) {
  __shared__ double slots[kTpb / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) slots[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (lane < kTpb / 32) ? slots[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in warp 0
}

// Final merge of the statistics partials, by the last block.  The maximum,
// argmax and per-degree bests are exact; the sums are rescaled with FP32 exp
// and accumulated in FP64.
__device__ __forceinline__ void finalize_stats(const StatPartial* parts, int G, int64_t N, const PolyParams* pp,
                               WsHeader* hdr, ppl_is_result* res, double* lse_out) {
  StatAcc a;
  a.init();
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    StatAcc o;
    const StatPartial& p = parts[b];
    o.m = p.m;
    o.s = p.s;
    o.s2 = p.s2;
    o.arg = p.arg;
    o.nan = p.nan;
    for (int k = 0; k < kMaxDegrees; ++k) {
      o.dm[k] = p.dm[k];
      o.darg[k] = p.darg[k];
    }
    a.merge(o);
  }
  StatAcc r = block_reduce_stat(a);
  __shared__ float M_sh;
  if (threadIdx.x == 0) M_sh = r.m;
  __syncthreads();
  const float M = M_sh;
  double s = 0.0, s2 = 0.0;
  if (M > -INFINITY) {
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
      const StatPartial& p = parts[b];
      if (p.m == -INFINITY) continue;
      const double e = (double)expf(p.m - M);
      s += (double)p.s * e;
      s2 += (double)p.s2 * e * e;
    }
  }
  s = block_sum_f64(s);
  s2 = block_sum_f64(s2);
  if (threadIdx.x == 0) {
    int32_t code = 0;
    if (r.nan) code = PPL_ENAN;
    else if (!(M > -INFINITY)) code = PPL_EEMPTY;
    if (code) record_status(&hdr->status, code);
    const double lse = (double)M + log(s);
    const double ess = s * s / s2;
    hdr->max_lw = M;
    hdr->lse = lse;
    hdr->ess = ess;
    hdr->argmax = r.arg;
    for (int k = 0; k < kMaxDegrees; ++k) {
      hdr->deg_max[k] = r.dm[k];
      hdr->deg_arg[k] = (r.darg[k] == 0x7fffffff) ? -1 : r.darg[k];
    }
    if (res) {
      res->lse = lse;
      res->log_z = lse - log((double)N);
      res->ess = ess;
      res->max_lw = M;
      res->argmax = r.arg;
      res->n_particles = N;
      res->n_deg = pp ? pp->n_deg : 0;
      for (int k = 0; k < kMaxDegrees; ++k) {
        const bool has = pp && k < pp->n_deg && r.darg[k] != 0x7fffffff;
        res->deg_max_lw[k] = has ? (double)r.dm[k] : -INFINITY;
        res->deg_argmax[k] = has ? r.darg[k] : -1;
      }
      res->status = ld_volatile_i32(&hdr->status);
    }
    if (lse_out) {
      lse_out[0] = lse;
      lse_out[1] = ess;
      lse_out[2] = (double)M;
      lse_out[3] = (double)r.arg;
    }
  }
}

}  // namespace ppl
