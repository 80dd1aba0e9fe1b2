// Raw Philox4x32-10 words as the traces draw them, exposed so the random
// streams can be checked bit for bit.
#include "kernels.h"
#include "rng.cuh"

namespace ppl {

// out[(i * n_blocks + j) * 4 + w] = word w of block j of counter
// (particle i, instance, step, purpose << 16 | j).
__global__ void __launch_bounds__(kTpb) rng_words_kernel(uint64_t seed, uint32_t instance,
                                                         uint32_t step, uint32_t purpose,
                                                         int64_t n, int32_t n_blocks,
                                                         uint4* __restrict__ out) {
  const int64_t total = n * n_blocks;
  const int64_t stride = (int64_t)gridDim.x * kTpb;
  for (int64_t u = (int64_t)blockIdx.x * kTpb + threadIdx.x; u < total; u += stride) {
    const int64_t i = u / n_blocks;
    const uint32_t j = (uint32_t)(u - i * n_blocks);
    out[u] = philox_block(seed, (uint32_t)i, instance, step, purpose, j);
  }
}

cudaError_t launch_rng_words(uint64_t seed, uint32_t instance, uint32_t step, uint32_t purpose,
                             int64_t n, int32_t n_blocks, uint32_t* out, cudaStream_t s) {
  rng_words_kernel<<<stream_grid(n * n_blocks), kTpb, 0, s>>>(seed, instance, step, purpose, n,
                                                             n_blocks, (uint4*)out);
  return cudaGetLastError();
}

}  // namespace ppl
