// Shared device-side definitions of the particle-inference library: workspace
// layout, status words, warp/block reductions and memory-ordering helpers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ppl.h"

namespace ppl {

constexpr int kMaxDegrees = 4;  // values of the degree prior
constexpr int kMaxCoef = 6;     // coefficients of one trace
constexpr int kTpb = 256;       // threads per block of the streaming kernels
constexpr int kMaxBlocks = 4096;  // cap on persistent grids (partials live in the workspace)

// Device status word semantics: the first error recorded wins.
__device__ __forceinline__ void record_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

// Workspace header, at offset 0 of every workspace.  Cleared by a memset at the
// start of every entry point (so every call starts with status PPL_OK).
struct WsHeader {
  int32_t status;
  uint32_t ticket[7];        // last-block election counters, one per kernel kind
  uint32_t tile_counter[4];  // dynamic tile ids of the decoupled-lookback scan
  float max_lw;              // maximum log-weight found by the statistics pass
  int32_t resample_flag;     // SMC: 1 when the current step resamples
  uint64_t total;            // resampling: T = sum of fixed-point weights
  uint64_t stride;           // resampling: floor(T / M)
  uint64_t offset;           // resampling: u = floor(w * stride / 2^32)
  uint64_t stride_inv;       // floor((2^64 - 1) / stride), for exact division
  double lse, ess;           // statistics pass
  float deg_max[kMaxDegrees];
  int32_t deg_arg[kMaxDegrees];
  int32_t argmax;
  int32_t pad;
  uint64_t reserved[8];
};
static_assert(sizeof(WsHeader) <= 512, "header must fit its slot");

// Workspace regions (byte offsets), computed on the host for one call.
struct WsLayout {
  size_t header;      // WsHeader
  size_t partials;    // per-block partial results
  size_t tiles;       // scan tile status words
  size_t prefix;      // inclusive prefix sums C_j (u64)
  size_t bounds;      // first ancestor of every output chunk's first and last output
  size_t lw;          // FP32 log-weights when the caller keeps none
  size_t scratch;     // SMC: ancestors + gathered state; host API: data copies
  size_t total;
};

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Memory-ordering helpers for the decoupled-lookback scan (PTX ISA 8.x
// ld.acquire / st.release at GPU scope).
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// Last-block election: every block calls this once after writing its partial;
// it returns true in exactly one block, after all partials are visible.
__device__ __forceinline__ bool elect_last_block(uint32_t* ticket) {
  __shared__ bool last;
  __threadfence();  // every thread's partial writes are device-visible before the ticket
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    uint32_t t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace ppl
