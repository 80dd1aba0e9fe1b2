// Building blocks of the persistent, cooperative kernels: a bounded grid
// barrier whose last arriving block runs a job before it releases the others,
// warp scans of saturating 64-bit sums, and exact 64-bit division by an FP32
// estimate plus integer corrections (no 64-bit integer/float conversion
// instructions).
#pragma once

#include "fixedpoint.cuh"

namespace ppl {

constexpr int kGridSpin = 1 << 22;  // bound of one barrier wait (polls)

// Barrier words.  Line 0: the arrival counter (barrier e is complete at
// e * grid); line 1: the release word, (barrier number << 34) | payload, and
// what the job publishes with it.
struct __align__(128) GridCtl {
  unsigned long long arrive;
  char pad0[120];
  unsigned long long release;
  unsigned long long total, stride, offset;
};

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* p,
                                                               unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
               : "=l"(old)
               : "l"(p), "l"(v)
               : "memory");
  return old;
}

// Grid barrier number e (1-based; every block counts its own).  After a block
// barrier, thread 0 arrives with an acquire-release atomic.  Without a job the
// others poll the arrival count.  With one, the block whose arrival completes
// the count runs `job` with all its threads (thread 0's return value is the
// payload, below 2^34) and releases the others, which poll the release word;
// every block finds the release word in *rel.  Thread 0 then runs `after`
// before the closing block barrier.  A wait that runs out records
// PPL_ETIMEOUT in *status; a block that sees a status set while waiting gives
// up too.  Returns false when the kernel must stop.
template <bool kJob, class Job, class After>
__device__ __forceinline__ bool grid_sync(GridCtl* g, int32_t* status, unsigned G,
                                          unsigned long long e, unsigned long long* rel,
                                          Job&& job, After&& after) {
  __shared__ int role;  // 1: ran the job, 0: released, -1: stop
  __syncthreads();      // the block's writes precede thread 0's release
  if (threadIdx.x == 0) {
    const unsigned long long target = e * G;
    const unsigned long long old = atom_add_acq_rel(&g->arrive, 1ull);
    int r = 0;
    if (old == target - 1) {
      r = kJob ? 1 : 0;
    } else {
      const uint64_t* word = reinterpret_cast<const uint64_t*>(kJob ? &g->release : &g->arrive);
      int spins = 0;
      for (;;) {
        const unsigned long long v = ld_acquire_u64(word);
        if (kJob ? (v >> 34) >= e : v >= target) {
          if (kJob) *rel = v;
          break;
        }
        if ((spins & 15) == 15 && ld_volatile_i32(status) != 0) {  // another block gave up
          r = -1;
          break;
        }
        if (++spins > kGridSpin) {
          record_status(status, PPL_ETIMEOUT);
          r = -1;
          break;
        }
        if (spins > 32) __nanosleep(32);
      }
    }
    role = r;
  }
  __syncthreads();
  const int r = role;
  if (r == 1) {
    const unsigned long long payload = job();
    __syncthreads();  // the job's writes precede the release
    if (threadIdx.x == 0) {
      const unsigned long long v = (e << 34) | payload;
      st_release_u64(reinterpret_cast<uint64_t*>(&g->release), v);
      *rel = v;
    }
  }
  if (r >= 0 && threadIdx.x == 0) after();
  __syncthreads();
  return r >= 0;
}

// Inclusive warp scan of saturating 64-bit sums.
__device__ __forceinline__ uint64_t warp_scan_u64(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = sat_add(v, u);
  }
  return v;
}

// The leading 24 bits of v as an FP32 number (relative error below 2^-23;
// 0 for 0), through 32-bit conversions only.
__device__ __forceinline__ float lead_f32(uint64_t v) {
  const int sh = max(0, 40 - __clzll(v));  // v >> sh < 2^24
  return __fmul_rn(__uint2float_rn((uint32_t)(v >> sh)), __int_as_float((127 + sh) << 23));
}

// floor(num / den) for num < 2^62, 1 <= den and a quotient below 2^33: an FP32
// estimate (relative error below 2^-20), one FP32 correction from the signed
// remainder, then exact integer steps (at most two each way).
__device__ __forceinline__ uint64_t floor_div_u64(uint64_t num, uint64_t den) {
  const float fd = lead_f32(den);
  uint64_t q = floor_u64(__fdividef(lead_f32(num), fd));
  int64_t r = (int64_t)(num - q * den);  // |r| < 2^13 den
  const float fr = r >= 0 ? lead_f32((uint64_t)r) : -lead_f32((uint64_t)(-r));
  const int64_t dq = (int64_t)(int)floorf(__fdividef(fr, fd));  // |dq| < 2^14
  q += (uint64_t)dq;
  r -= dq * (int64_t)den;
  for (int i = 0; i < 4 && r < 0; ++i) {
    --q;
    r += (int64_t)den;
  }
  for (int i = 0; i < 4 && r >= (int64_t)den; ++i) {
    ++q;
    r -= (int64_t)den;
  }
  if (r < 0 || r >= (int64_t)den) q = num / den;  // not reached for the stated ranges
  return q;
}

// #{k >= 0 : u + k stride < c}, capped at m: the number of systematic
// positions below c (stride >= 1, u < stride, c <= 2^61).
__device__ __forceinline__ int64_t positions_below(uint64_t c, uint64_t u, uint64_t stride,
                                                   int64_t m) {
  if (c <= u) return 0;
  const uint64_t k = floor_div_u64(c - u + stride - 1, stride);
  return k < (uint64_t)m ? (int64_t)k : m;
}

// Division by an invariant divisor d (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): with
// inv = floor((2^64 - 1) / d), the high word of num * inv never exceeds
// floor(num / d) and, for num < 2^62, falls short of it by at most one, which
// one remainder test corrects.
struct DivInv {
  uint64_t d, inv;
};
__device__ __forceinline__ DivInv div_inv(uint64_t d) { return DivInv{d, d ? ~0ull / d : 0ull}; }
__device__ __forceinline__ uint64_t div_by(uint64_t num, const DivInv& v) {
  uint64_t q = __umul64hi(num, v.inv);
  const uint64_t r = num - q * v.d;  // < 2 d
  if (r >= v.d) ++q;
  return q;
}

// positions_below with the stride's reciprocal precomputed (num < 2^62 holds:
// c <= 2^61 and stride <= 2^61).
__device__ __forceinline__ int64_t positions_below_inv(uint64_t c, uint64_t u, const DivInv& sv,
                                                       int64_t m) {
  if (c <= u) return 0;
  const uint64_t k = div_by(c - u + sv.d - 1, sv);
  return k < (uint64_t)m ? (int64_t)k : m;
}

}  // namespace ppl
