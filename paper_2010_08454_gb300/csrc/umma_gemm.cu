// BF16 GEMM on the fifth-generation tensor cores (tcgen05, sm_100 family):
//   C[m, n] = sum_k A(m, k) B(n, k)  (+ bias[n]) (relu) (* [mask(m, n) > 0])
// with A(m, k) = A[m sam + k sak], B(n, k) = B[n sbn + k sbk] (any layout, so
// the network's backward products read transposed operands in place), FP32
// accumulation in tensor memory.
//
// Per CTA: a 128 x 64 tile of C in 64 TMEM columns (lane = row).  Each K step
// of 64, the 128 threads stage A (128 x 64) and B (64 x 64) in shared memory
// in the canonical K-major layout without swizzle -- 8 x 8 core matrices of
// 128 contiguous bytes, K-adjacent cores 128 B apart (leading byte offset),
// row-group-adjacent cores 1024 B apart (stride byte offset) -- then one
// thread issues four tcgen05.mma (K = 16 each) and commits them to an
// mbarrier that all threads wait on before the tile is overwritten.  The
// epilogue reads the accumulator with tcgen05.ld (each warp its 32 lanes).
// Every wait is bounded; a wait that runs out records an error in *status,
// and the CTA still frees its tensor memory.
#include <cuda_bf16.h>

#include "kernels.h"

namespace ppl {

constexpr int kUM = 128, kUN = 64, kUK = 64;
constexpr int kUmmaSpin = 1 << 24;   // bound of one mbarrier wait (polls)
constexpr uint32_t kUTmemCols = 64;  // FP32 accumulator columns (power of two, >= 32)

struct UmmaArgs {
  const __nv_bfloat16* A;
  int64_t sam, sak;
  const __nv_bfloat16* B;
  int64_t sbn, sbk;
  int M, N, K;
  const float* bias;
  const __nv_bfloat16* mask;  // [M x N] row-major, multiply by (mask > 0)
  int relu;
  float* Cf;          // FP32 output [M x N], optional
  __nv_bfloat16* Cb;  // BF16 output [M x N], optional
  int32_t* status;    // set to PPL_ETIMEOUT when a wait runs out
  int vec_a, vec_b;   // K contiguous, rows 16-byte aligned: 8 elements per load
  // split-K: CTA z of grid.z takes K range [z k_split, (z + 1) k_split) and
  // writes its raw FP32 tile to partial[z][M][N]; a second kernel sums the
  // slices in order and applies the epilogue
  float* partial;
  int k_split;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kUIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kUN >> 3) << 17) |
                             ((uint32_t)(kUM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (int i = 0; i < kUmmaSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Core-matrix layout of a 64-wide K tile: element (r, k) of a rows x 64 tile.
__device__ __forceinline__ int core_index(int r, int k) {
  return (((r >> 3) * (kUK / 8) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__global__ void __launch_bounds__(128) umma_gemm_kernel(UmmaArgs g) {
  extern __shared__ __align__(1024) unsigned char um_dyn[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(um_dyn);  // 128 x 64, 16 KB
  __nv_bfloat16* Bs = As + kUM * kUK;                              // 64 x 64, 8 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * kUM, n0 = blockIdx.x * kUN;
  const uint32_t mb = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(kUTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  uint32_t phase = 0;
  bool any = false;
  const int k_begin = g.partial ? (int)blockIdx.z * g.k_split : 0;
  const int k_end = g.partial ? min(g.K, k_begin + g.k_split) : g.K;
  for (int k0 = k_begin; k0 < k_end; k0 += kUK) {
    // stage the K tile (the previous tile's MMAs have completed)
    if (g.vec_a) {  // one core-matrix row (8 consecutive k) per 16-byte load
      for (int e = tid; e < kUM * (kUK / 8); e += 128) {
        const int r = e / (kUK / 8), k = (e % (kUK / 8)) * 8;
        const int gm = m0 + r, gk = k0 + k;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gm < g.M && gk < g.K)  // K % 8 == 0: the whole row is in range
          v = *reinterpret_cast<const uint4*>(g.A + (int64_t)gm * g.sam + gk);
        *reinterpret_cast<uint4*>(As + core_index(r, k)) = v;
      }
    } else if (g.sam == 1) {  // rows contiguous: consecutive threads take consecutive rows
      for (int e = tid; e < kUM * kUK; e += 128) {
        const int r = e % kUM, k = e / kUM;
        const int gm = m0 + r, gk = k0 + k;
        As[core_index(r, k)] =
            (gm < g.M && gk < g.K) ? g.A[gm + (int64_t)gk * g.sak] : zero;
      }
    } else {
      for (int e = tid; e < kUM * kUK; e += 128) {
        const int r = e / kUK, k = e % kUK;
        const int gm = m0 + r, gk = k0 + k;
        As[core_index(r, k)] = (gm < g.M && gk < g.K) ? g.A[gm * g.sam + gk * g.sak] : zero;
      }
    }
    if (g.vec_b) {
      for (int e = tid; e < kUN * (kUK / 8); e += 128) {
        const int r = e / (kUK / 8), k = (e % (kUK / 8)) * 8;
        const int gn = n0 + r, gk = k0 + k;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gn < g.N && gk < g.K)
          v = *reinterpret_cast<const uint4*>(g.B + (int64_t)gn * g.sbn + gk);
        *reinterpret_cast<uint4*>(Bs + core_index(r, k)) = v;
      }
    } else if (g.sbn == 1) {  // columns contiguous: consecutive threads take consecutive columns
      for (int e = tid; e < kUN * kUK; e += 128) {
        const int r = e % kUN, k = e / kUN;
        const int gn = n0 + r, gk = k0 + k;
        Bs[core_index(r, k)] =
            (gn < g.N && gk < g.K) ? g.B[gn + (int64_t)gk * g.sbk] : zero;
      }
    } else {
      for (int e = tid; e < kUN * kUK; e += 128) {
        const int r = e / kUK, k = e % kUK;
        const int gn = n0 + r, gk = k0 + k;
        Bs[core_index(r, k)] = (gn < g.N && gk < g.K) ? g.B[gn * g.sbn + gk * g.sbk] : zero;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kUK / 16; ++kk) {
        const uint64_t ad = umma_desc(smem_u32(As) + kk * 2 * 128, 128, 1024);
        const uint64_t bd = umma_desc(smem_u32(Bs) + kk * 2 * 128, 128, 1024);
        const uint32_t acc = (k0 > k_begin || kk > 0) ? 1u : 0u;  // first step of the slice: overwrite
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(kUIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(mb) : "memory");
    }
    if (!mbar_wait(mb, phase)) {
      atomicExch(&failed, 1);
      record_status(g.status, PPL_ETIMEOUT);
    }
    phase ^= 1u;
    any = true;
    __syncthreads();
    if (failed) break;  // the same for every thread
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile in its TMEM lanes
    const int m = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < kUN; c0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < g.M && g.partial) {  // a K slice: the raw tile
        float* dst = g.partial + ((int64_t)blockIdx.z * g.M + m) * g.N;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + c0 + j;
          if (n < g.N) dst[n] = any ? __uint_as_float(v[j]) : 0.0f;
        }
      } else if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + c0 + j;
          if (n >= g.N) continue;
          float x = any ? __uint_as_float(v[j]) : 0.0f;
          if (g.bias) x += g.bias[n];
          if (g.relu) x = fmaxf(x, 0.0f);
          if (g.mask && !(__bfloat162float(g.mask[(int64_t)m * g.N + n]) > 0.0f)) x = 0.0f;
          if (g.Cf) g.Cf[(int64_t)m * g.N + n] = x;
          if (g.Cb) g.Cb[(int64_t)m * g.N + n] = __float2bfloat16_rn(x);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kUTmemCols) : "memory");
}

// The sum of the K slices in order (deterministic), then the epilogue.
__global__ void __launch_bounds__(256) splitk_reduce_kernel(UmmaArgs g, int S) {
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t MN = (int64_t)g.M * g.N;
  if (e >= MN) return;
  const int n = (int)(e % g.N);
  float x = 0.0f;
  for (int z = 0; z < S; ++z) x += g.partial[z * MN + e];
  if (g.bias) x += g.bias[n];
  if (g.relu) x = fmaxf(x, 0.0f);
  if (g.mask && !(__bfloat162float(g.mask[e]) > 0.0f)) x = 0.0f;
  if (g.Cf) g.Cf[e] = x;
  if (g.Cb) g.Cb[e] = __float2bfloat16_rn(x);
}

// Shared memory per CTA (dynamic), sized so that at most four CTAs share an
// SM: 4 x 64 tensor-memory columns stay within the SM's 512.
constexpr size_t kUmmaSmem = 48 * 1024;

cudaError_t launch_umma_gemm(const __nv_bfloat16* A, int64_t sam, int64_t sak,
                             const __nv_bfloat16* B, int64_t sbn, int64_t sbk, int M, int N, int K,
                             const float* bias, const __nv_bfloat16* mask, int relu, float* Cf,
                             __nv_bfloat16* Cb, int32_t* status, cudaStream_t s,
                             float* split_ws, size_t split_floats) {
  int unused = 0;
  const cudaError_t e = device_once((const void*)umma_gemm_kernel, &unused, [](int*) {
    return cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kUmmaSmem);
  });
  if (e != cudaSuccess) return e;
  UmmaArgs g;
  g.A = A; g.sam = sam; g.sak = sak;
  g.B = B; g.sbn = sbn; g.sbk = sbk;
  g.M = M; g.N = N; g.K = K;
  g.bias = bias; g.mask = mask; g.relu = relu; g.Cf = Cf; g.Cb = Cb; g.status = status;
  // 16-byte loads need K contiguous, K and the row stride multiples of 8, and
  // a 16-byte aligned base
  g.vec_a = sak == 1 && K % 8 == 0 && sam % 8 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  g.vec_b = sbk == 1 && K % 8 == 0 && sbn % 8 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  g.partial = nullptr;
  g.k_split = K;
  dim3 grid((N + kUN - 1) / kUN, (M + kUM - 1) / kUM);
  // split K while the output tiles leave most SMs idle and each slice keeps
  // at least one 64-wide step
  int S = 1;
  const int64_t tiles = (int64_t)grid.x * grid.y;
  while (split_ws && tiles * S * 2 <= (int64_t)num_sms() * 2 && K / (S * 2) >= kUK &&
         (size_t)S * 2 * M * N <= split_floats)
    S *= 2;
  if (S > 1) {
    g.partial = split_ws;
    g.k_split = ((K + S - 1) / S + kUK - 1) / kUK * kUK;
    S = (K + g.k_split - 1) / g.k_split;
    grid.z = S;
  }
  umma_gemm_kernel<<<grid, 128, kUmmaSmem, s>>>(g);
  cudaError_t r = cudaGetLastError();
  if (r != cudaSuccess || S == 1) return r;
  splitk_reduce_kernel<<<(unsigned)(((int64_t)M * N + 255) / 256), 256, 0, s>>>(g, S);
  return cudaGetLastError();
}

}  // namespace ppl
