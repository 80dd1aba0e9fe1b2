// Internal launch interface between the C ABI (abi.cu) and the kernels.
#pragma once

#include <cuda_bf16.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <functional>

#include "common.cuh"

namespace ppl {

struct PolyParams;

// Host set-up that must run once per device (a kernel's shared-memory
// attribute, a residency count): runs `setup` the first time `key` is seen
// with the current device, under a lock, and returns the int it produced
// then and on every later call for that (key, device).  A failed set-up is
// not cached.
cudaError_t device_once(const void* key, int* value, const std::function<cudaError_t(int*)>& setup);

int num_sms();
int trace_grid(int64_t N);
int stream_grid(int64_t N);
size_t partials_bytes();

// is_kernels.cu
cudaError_t launch_poly_trace(const PolyParams& p, const float* x, const float* y, int64_t L,
                              int64_t N, uint64_t seed, uint32_t instance, float* lw_out,
                              ppl_poly_particle* rec_out, WsHeader* hdr, void* parts,
                              ppl_is_result* res, cudaStream_t s, const void* suff = nullptr);
// trace_tc.cu: the same pass with the factor's polynomial evaluations on the
// tensor cores (data sets of up to trace_tc_max_points() points).
// With part_out, the shard partial of particles [first, first + N) of a
// larger population instead of the summary (trace i is particle first + i).
int trace_tc_max_points();
cudaError_t launch_poly_trace_tc(const PolyParams& p, const float* x, const float* y, int64_t L,
                                 int64_t N, uint64_t seed, uint32_t instance, float* lw_out,
                                 ppl_poly_particle* rec_out, WsHeader* hdr, void* parts,
                                 ppl_is_result* res, cudaStream_t s, int64_t first = 0,
                                 void* part_out = nullptr);
// The summary of a population from P shard partials.
cudaError_t launch_merge_shards(const void* parts, int P, ppl_is_result* res, cudaStream_t s);
// Sufficient statistics of a data set for the line-fitting factor (one
// block); `out` holds suffstat_bytes() bytes, 16-byte aligned.
size_t suffstat_bytes();
// With split_ws (split_floats FP32 words of device scratch) the product may
// be split along K over more CTAs, the slices summed in order by a second
// kernel (the same result on every run).
cudaError_t launch_umma_gemm(const __nv_bfloat16* A, int64_t sam, int64_t sak,
                             const __nv_bfloat16* B, int64_t sbn, int64_t sbk, int M, int N, int K,
                             const float* bias, const __nv_bfloat16* mask, int relu, float* Cf,
                             __nv_bfloat16* Cb, int32_t* status, cudaStream_t s,
                             float* split_ws = nullptr, size_t split_floats = 0);
cudaError_t launch_customdist(const ppl_customdist_model& m, uint32_t comp_threshold,
                              const float* y, int64_t n, int64_t N, uint64_t seed, float* x_out,
                              float* lw_out, void* parts, WsHeader* hdr,
                              ppl_customdist_result* res, cudaStream_t s);
cudaError_t launch_discrete_is(int32_t model, const int32_t* data, int64_t n_data, int32_t limit,
                               int64_t N, uint64_t seed, uint32_t bern_threshold, int32_t n_values,
                               int32_t* codes_out, float* lw_out, void* counts, WsHeader* hdr,
                               ppl_discrete_result* res, cudaStream_t s);
cudaError_t launch_suffstat(const float* x, const float* y, int64_t L, int d_max, void* out,
                            cudaStream_t s);
cudaError_t launch_stats(const float* lw, int64_t N, WsHeader* hdr, void* parts,
                         double* lse_out, cudaStream_t s);
cudaError_t launch_posterior(const PolyParams& p, const ppl_poly_particle* rec, const float* lw,
                             int64_t N, WsHeader* hdr, void* parts, ppl_is_result* res,
                             cudaStream_t s);

// resample.cu
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kTpb * kScanItems;
inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
// gate: when non-null, the kernels do nothing unless *gate != 0 (SMC steps).
// known_max (optional, device): the maximum log-weight, when a previous pass
// already found it (the statistics pass is then skipped by the caller).
cudaError_t launch_resample_scan(const float* lw, const uint64_t* q_fixed, int64_t N, int64_t M,
                                 uint64_t seed, uint32_t instance, uint32_t t, WsHeader* hdr,
                                 uint64_t* tile_status, uint64_t* prefix, const int32_t* gate,
                                 cudaStream_t s, const double* known_max = nullptr);
int64_t ancestor_bounds_count(int64_t M);
cudaError_t launch_scan_timeout_selftest(const uint64_t* q, int64_t N, WsHeader* hdr,
                                         uint64_t* tile_status, uint64_t* prefix, int max_spin,
                                         cudaStream_t s);
cudaError_t launch_ancestors(const uint64_t* prefix, int64_t N, int64_t M, const WsHeader* hdr,
                             int64_t* bounds, int32_t* ancestors, const int32_t* gate,
                             cudaStream_t s);
cudaError_t launch_gather(const void* in, int64_t n_in, int64_t stride_bytes, const int32_t* anc,
                          int64_t M, void* out, const int32_t* gate, cudaStream_t s);

// rng_kernels.cu
cudaError_t launch_rng_words(uint64_t seed, uint32_t instance, uint32_t step, uint32_t purpose,
                             int64_t n, int32_t n_blocks, uint32_t* out, cudaStream_t s);

// smc.cu
struct LgssmParams {
  float phi, q_sigma;
  float obs_const;      // -log(2 pi r^2) / 2
  float neg_half_inv_r2;  // -1 / (2 r^2)
};
cudaError_t launch_smc_propagate(const LgssmParams& p, float y_t, int32_t t, uint64_t seed,
                                 float* x, float* lw, int64_t N, double* logz_acc,
                                 int32_t* resampled, double* logz_est, WsHeader* hdr,
                                 void* parts, cudaStream_t s);
size_t smc_run_workspace(int64_t N, int64_t T);
// Systematic resampling in one cooperative kernel: the ancestors, and with
// rec_in the gathered records too (rec_out[k] = rec_in[anc[k]], rec_bytes a
// multiple of 4 up to 1024, both pointers 4-byte aligned; copied in 16-byte
// words when size and pointers allow).  `barrier` holds
// the grid barrier's words (resample_coop_barrier_bytes(), 128-byte aligned,
// zeroed by the caller before the launch); `scratch` the per-chunk tables
// (resample_coop_scratch(n) bytes, 16-byte aligned).
// With `shard`, one shard of a population split over devices: n is the
// shard's particle count, m the population's output count; the weights are
// quantised for n_total particles with the population's maximum (known_max),
// the layout is the shard plan's, and the call writes the shard's outputs
// [k_first, k_end): anc[k - k_first] = first_particle + local ancestor.
struct ResampleShard {
  int64_t n_total, first_particle, k_first, k_end;
  uint64_t stride, offset, c_base;
};
size_t resample_coop_scratch(int64_t n);
size_t resample_coop_barrier_bytes();
cudaError_t launch_resample_coop(const float* lw, const uint64_t* q_fixed, const double* known_max,
                                 int64_t n, int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                 WsHeader* hdr, void* barrier, char* scratch, size_t scratch_bytes,
                                 int32_t* anc, const int32_t* gate, cudaStream_t s,
                                 const void* rec_in = nullptr, int64_t rec_bytes = 0,
                                 void* rec_out = nullptr, const ResampleShard* shard = nullptr);
// The sum of a shard's fixed-point weights (quantised for n_total particles
// against *known_max) added to *total (zeroed by the caller).
cudaError_t launch_shard_total(const float* lw, int64_t n, int64_t n_total,
                               const double* known_max, uint64_t* total, WsHeader* hdr,
                               cudaStream_t s);
cudaError_t launch_smc_persistent(const LgssmParams& p, const float* y, int32_t T, uint64_t seed,
                                  int64_t N, float* x_out, float* lw_out, double* logz,
                                  int32_t* resampled, double* ess, char* ws, size_t ws_bytes,
                                  int32_t** status_out, cudaStream_t s);
cudaError_t launch_grid_barrier_probe(int blocks, int n_barriers, void* ws, cudaStream_t s);
cudaError_t launch_smc_commit(float* x, const float* x_tmp, float* lw, int64_t N,
                              const int32_t* gate, cudaStream_t s);

}  // namespace ppl
