// C ABI of libppl.so (declared in include/ppl.h): argument checks, workspace
// layout and the launch sequence of every entry point.  No entry point
// allocates memory; every launch is stream-ordered on the caller's stream.
#include <math.h>
#include <string.h>

#include "kernels.h"
#include "poly.cuh"

namespace ppl {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t kHeaderBytes = 512;
constexpr int64_t kMaxParticles = 0x7fffffffll;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Header and tile status words are contiguous so one memset clears both.
WsLayout layout(int64_t n, int64_t data_len) {
  WsLayout w;
  size_t off = 0;
  w.header = off;
  off += kHeaderBytes;
  w.tiles = off;  // scan tile status words, or the cooperative resampler's barrier words
  off += align_up(std::max((size_t)scan_tiles(std::max<int64_t>(n, 1)) * sizeof(uint64_t),
                           resample_coop_barrier_bytes()));
  w.partials = off;
  off += align_up(partials_bytes());
  w.prefix = off;  // prefix sums C, or the cooperative resampler's tables
  off += align_up(std::max((size_t)n * sizeof(uint64_t), resample_coop_scratch(n)));
  w.bounds = off;
  off += align_up((size_t)ancestor_bounds_count(n) * sizeof(int64_t));
  w.lw = off;
  off += align_up((size_t)n * sizeof(float));
  w.scratch = off;
  off += std::max(align_up((size_t)n * sizeof(int32_t)) + align_up((size_t)n * sizeof(float)),
                  align_up((size_t)std::max<int64_t>(data_len, 0) * 2 * sizeof(float)));
  w.total = off;
  return w;
}

struct Ws {
  char* base;
  WsLayout l;
  WsHeader* hdr() const { return reinterpret_cast<WsHeader*>(base + l.header); }
  uint64_t* tiles() const { return reinterpret_cast<uint64_t*>(base + l.tiles); }
  void* partials() const { return base + l.partials; }
  uint64_t* prefix() const { return reinterpret_cast<uint64_t*>(base + l.prefix); }
  int64_t* bounds() const { return reinterpret_cast<int64_t*>(base + l.bounds); }
  float* lw() const { return reinterpret_cast<float*>(base + l.lw); }
  char* scratch() const { return base + l.scratch; }
};

ppl_status check_ws(void* ws, size_t ws_bytes, int64_t n, int64_t data_len, Ws* out) {
  if (!ws) return PPL_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return PPL_EINVAL;
  out->base = static_cast<char*>(ws);
  out->l = layout(n, data_len);
  if (ws_bytes < out->l.total) return PPL_EINVAL;
  return PPL_OK;
}

ppl_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PPL_OK : PPL_ECUDA; }

// Clear the header (status, tickets, tile counters) and, when `tiles`, the
// scan tile status words.
ppl_status reset_ws(const Ws& w, bool tiles, cudaStream_t s) {
  const size_t bytes = tiles ? (w.l.partials - w.l.header) : kHeaderBytes;
  return cuda_status(cudaMemsetAsync(w.base + w.l.header, 0, bytes, s));
}

ppl_status poly_params(const ppl_model* m, PolyParams* p) {
  if (!m || m->id != PPL_MODEL_POLY) return PPL_EINVAL;
  const int n_deg = m->max_deg - m->min_deg + 1;
  if (m->min_deg < 0 || n_deg < 1 || n_deg > kMaxDegrees) return PPL_EINVAL;
  if (m->coef_offset < 0 || m->min_deg + m->coef_offset < 0 ||
      m->max_deg + m->coef_offset > kMaxCoef)
    return PPL_EINVAL;
  if (!(m->obs_sigma > 0.0f) || !isfinite(m->obs_sigma) || !isfinite(m->prior_sigma))
    return PPL_EINVAL;
  p->min_deg = m->min_deg;
  p->n_deg = n_deg;
  p->coef_offset = m->coef_offset;
  p->prior_sigma = m->prior_sigma;
  p->neg_half_inv_var = (float)(-1.0 / (2.0 * (double)m->obs_sigma * (double)m->obs_sigma));
  return PPL_OK;
}

// Word 0 of Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) on the
// host, with the counter layout of the device draws: key = (seed lo, seed
// hi), counter = (particle, instance, step, purpose << 16 | block).
uint32_t host_philox_word0(uint64_t seed, uint32_t particle, uint32_t instance, uint32_t step,
                           uint32_t purpose, uint32_t block) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = particle, c1 = instance, c2 = step, c3 = (purpose << 16) | block;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return c0;
}

#define PPL_TRY(expr)                      \
  do {                                     \
    const ppl_status _st = (expr);         \
    if (_st != PPL_OK) return _st;         \
  } while (0)

}  // namespace
}  // namespace ppl

using namespace ppl;

extern "C" {

const char* ppl_status_string(int32_t status) {
  switch (status) {
    case PPL_OK: return "ok";
    case PPL_EINVAL: return "invalid argument";
    case PPL_ENOMEM: return "out of memory";
    case PPL_ECUDA: return "CUDA error";
    case PPL_ENAN: return "NaN log-weight";
    case PPL_EEMPTY: return "all weights are zero";
    case PPL_ETIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
  }
}

size_t ppl_workspace_size(const ppl_model* model, int64_t n_particles, int64_t data_len) {
  if (!model || n_particles < 1 || n_particles > kMaxParticles || data_len < 0) return 0;
  const size_t total = layout(n_particles, data_len).total;
  if (model->id == PPL_MODEL_LGSSM) return std::max(total, smc_run_workspace(n_particles, data_len));
  return total;
}

ppl_status ppl_workspace_status(const void* ws, ppl_stream stream) {
  if (!ws) return PPL_EINVAL;
  int32_t st = 0;
  if (cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
      cudaSuccess)
    return PPL_ECUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PPL_ECUDA;
  return (ppl_status)st;
}

ppl_status ppl_infer_is_instance(const ppl_model* model, const ppl_data* data,
                                 int64_t n_particles, uint64_t seed, uint32_t instance,
                                 ppl_is_result* out_dev, float* lw_out,
                                 ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                 ppl_stream stream) {
  PolyParams p;
  PPL_TRY(poly_params(model, &p));
  if (!data || data->len < 0 || (data->len > 0 && (!data->x || !data->y))) return PPL_EINVAL;
  if (n_particles < 1 || n_particles > kMaxParticles || !out_dev) return PPL_EINVAL;
  if (particles_out && (reinterpret_cast<uintptr_t>(particles_out) & 15)) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_particles, data->len, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  // (the last block writes every field of *out_dev)
  // the polynomial evaluations on the tensor cores while the data set fits in
  // shared memory, in FP32 on the CUDA cores beyond
  if (data->len <= trace_tc_max_points())
    PPL_TRY(cuda_status(launch_poly_trace_tc(p, data->x, data->y, data->len, n_particles, seed,
                                             instance, lw_out, particles_out, w.hdr(),
                                             w.partials(), out_dev, s)));
  else
    PPL_TRY(cuda_status(launch_poly_trace(p, data->x, data->y, data->len, n_particles, seed,
                                          instance, lw_out, particles_out, w.hdr(), w.partials(),
                                          out_dev, s)));
  return PPL_OK;
}

ppl_status ppl_infer_is_suffstat(const ppl_model* model, const ppl_data* data,
                                 int64_t n_particles, uint64_t seed, uint32_t instance,
                                 ppl_is_result* out_dev, float* lw_out,
                                 ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                 ppl_stream stream) {
  PolyParams p;
  PPL_TRY(poly_params(model, &p));
  if (!data || data->len < 0 || (data->len > 0 && (!data->x || !data->y))) return PPL_EINVAL;
  if (n_particles < 1 || n_particles > kMaxParticles || !out_dev) return PPL_EINVAL;
  if (particles_out && (reinterpret_cast<uintptr_t>(particles_out) & 15)) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_particles, data->len, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(cudaMemsetAsync(out_dev, 0, sizeof(ppl_is_result), s)));
  // the statistics live in the scratch region, unused by likelihood weighting
  const int d_max = p.min_deg + p.n_deg - 1 + p.coef_offset;
  PPL_TRY(cuda_status(launch_suffstat(data->x, data->y, data->len, d_max, w.scratch(), s)));
  PPL_TRY(cuda_status(launch_poly_trace(p, data->x, data->y, data->len, n_particles, seed,
                                        instance, lw_out, particles_out, w.hdr(), w.partials(),
                                        out_dev, s, w.scratch())));
  return PPL_OK;
}

ppl_status ppl_infer_discrete(int32_t model, const int32_t* flips, int64_t n_flips, int32_t limit,
                              int64_t n_particles, uint64_t seed, ppl_discrete_result* out_dev,
                              int32_t* codes_out, float* lw_out, void* ws, size_t ws_bytes,
                              ppl_stream stream) {
  if (!out_dev || n_particles < 1 || n_particles > kMaxParticles) return PPL_EINVAL;
  int32_t n_values = 0;
  double p = 0.0;
  if (model == PPL_DISCRETE_BIASEDCOIN) {
    if (n_flips < 0 || n_flips > 0x7fffffff || (n_flips > 0 && !flips)) return PPL_EINVAL;
    n_values = 9;
  } else if (model == PPL_DISCRETE_BINOMIAL) {
    if (limit < 0 || limit >= PPL_DISCRETE_MAX_VALUES) return PPL_EINVAL;
    n_values = limit + 1;
    p = 0.3;
  } else if (model == PPL_DISCRETE_GEOMETRIC) {
    if (limit < 1 || limit >= PPL_DISCRETE_MAX_VALUES) return PPL_EINVAL;
    n_values = limit + 1;
    p = 0.5;
  } else {
    return PPL_EINVAL;
  }
  // u01(w) = ((w >> 9) + 0.5) 2^-23 < p  <=>  (w >> 9) < ceil(p 2^23 - 0.5), exact in FP64
  const uint32_t threshold = (uint32_t)ceil(p * 8388608.0 - 0.5);
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, 1, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(launch_discrete_is(model, flips, model == PPL_DISCRETE_BIASEDCOIN ? n_flips : 0,
                                         limit, n_particles, seed, threshold, n_values, codes_out,
                                         lw_out, w.partials(), w.hdr(), out_dev, s)));
  return PPL_OK;
}

ppl_status ppl_infer_customdist(const ppl_customdist_model* model, const float* y, int64_t n_obs,
                                int64_t n_particles, uint64_t seed,
                                ppl_customdist_result* out_dev, float* x_out, float* lw_out,
                                void* ws, size_t ws_bytes, ppl_stream stream) {
  if (!model || !out_dev || n_particles < 1 || n_particles > kMaxParticles) return PPL_EINVAL;
  if (n_obs < 0 || (n_obs > 0 && !y)) return PPL_EINVAL;
  if (!(model->w1 >= 0.0f && model->w1 <= 1.0f) || !(model->sigma1 > 0.0f) ||
      !(model->sigma2 > 0.0f) || !(model->obs_sigma > 0.0f) || !isfinite(model->mu1) ||
      !isfinite(model->mu2))
    return PPL_EINVAL;
  // u01(w) = ((w >> 9) + 0.5) 2^-23 < w1  <=>  (w >> 9) < ceil(w1 2^23 - 0.5), exact in FP64
  const uint32_t threshold = (uint32_t)std::max(0.0, ceil((double)model->w1 * 8388608.0 - 0.5));
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_particles, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(launch_customdist(*model, threshold, y, n_obs, n_particles, seed, x_out,
                                        lw_out, w.partials(), w.hdr(), out_dev, s)));
  return PPL_OK;
}

ppl_status ppl_gemm_bf16(const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbn,
                         int64_t sbk, int32_t M, int32_t N, int32_t K, float* C, void* ws,
                         size_t ws_bytes, ppl_stream stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || M >= (1 << 24) || N >= (1 << 24) ||
      K >= (1 << 24))
    return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, 1, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  return cuda_status(launch_umma_gemm(reinterpret_cast<const __nv_bfloat16*>(A), sam, sak,
                                      reinterpret_cast<const __nv_bfloat16*>(B), sbn, sbk, M, N,
                                      K, nullptr, nullptr, 0, C, nullptr, &w.hdr()->status, s));
}

ppl_status ppl_infer_is(const ppl_model* model, const ppl_data* data, int64_t n_particles,
                        uint64_t seed, ppl_is_result* out_dev, float* lw_out,
                        ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                        ppl_stream stream) {
  return ppl_infer_is_instance(model, data, n_particles, seed, 0, out_dev, lw_out,
                               particles_out, ws, ws_bytes, stream);
}

ppl_status ppl_infer_is_host(const ppl_model* model, const float* x_host, const float* y_host,
                             int64_t data_len, int64_t n_particles, uint64_t seed,
                             ppl_is_result* out_host, void* ws, size_t ws_bytes,
                             ppl_stream stream) {
  if (!out_host || data_len < 0 || (data_len > 0 && (!x_host || !y_host))) return PPL_EINVAL;
  if (n_particles < 1 || n_particles > kMaxParticles) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_particles, data_len, &w));
  cudaStream_t s = (cudaStream_t)stream;
  float* xd = reinterpret_cast<float*>(w.scratch());
  float* yd = xd + data_len;
  // the summary lands in the scan-prefix region, unused by likelihood weighting
  ppl_is_result* res = reinterpret_cast<ppl_is_result*>(w.prefix());
  if (data_len > 0) {
    PPL_TRY(cuda_status(cudaMemcpyAsync(xd, x_host, data_len * sizeof(float),
                                        cudaMemcpyHostToDevice, s)));
    PPL_TRY(cuda_status(cudaMemcpyAsync(yd, y_host, data_len * sizeof(float),
                                        cudaMemcpyHostToDevice, s)));
  }
  ppl_data d{xd, yd, data_len};
  PPL_TRY(ppl_infer_is(model, &d, n_particles, seed, res, nullptr, nullptr, ws, ws_bytes, stream));
  PPL_TRY(cuda_status(cudaMemcpyAsync(out_host, res, sizeof(ppl_is_result),
                                      cudaMemcpyDeviceToHost, s)));
  PPL_TRY(cuda_status(cudaStreamSynchronize(s)));
  return (ppl_status)out_host->status;
}

ppl_status ppl_logsumexp(const float* lw, int64_t n, double* out_dev, void* ws, size_t ws_bytes,
                         ppl_stream stream) {
  if (!lw || !out_dev || n < 1 || n > kMaxParticles) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(launch_stats(lw, n, w.hdr(), w.partials(), out_dev, s)));
  return PPL_OK;
}

static ppl_status resample_impl(const float* lw, const uint64_t* q_fixed, const double* known_max,
                                int64_t n, int64_t m, uint64_t seed, uint32_t instance,
                                uint32_t t, int32_t* ancestors, void* ws, size_t ws_bytes,
                                ppl_stream stream, const void* rec_in = nullptr,
                                int64_t rec_bytes = 0, void* rec_out = nullptr) {
  if ((lw == nullptr) == (q_fixed == nullptr)) return PPL_EINVAL;
  if (!ancestors || n < 1 || n > kMaxParticles || m < 1 || m > kMaxParticles) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, std::max(n, m), 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, true, s));
  if (lw && !known_max)
    PPL_TRY(cuda_status(launch_stats(lw, n, w.hdr(), w.partials(), nullptr, s)));
  // the scan-tile region (cleared with the header above) holds the
  // resampling kernel's barrier words, the prefix-sum region its per-chunk
  // tables (a few bytes per 4096 particles)
  PPL_TRY(cuda_status(launch_resample_coop(lw, q_fixed, known_max, n, m, seed, instance, t,
                                           w.hdr(), w.tiles(), reinterpret_cast<char*>(w.prefix()),
                                           w.l.bounds - w.l.prefix, ancestors, nullptr, s, rec_in,
                                           rec_bytes, rec_out)));
  return PPL_OK;
}

ppl_status ppl_resample_gather(const float* lw, const double* max_lw_dev, int64_t n, int64_t m,
                               uint64_t seed, uint32_t instance, uint32_t t, const void* state_in,
                               int64_t stride_bytes, void* state_out, int32_t* ancestors,
                               void* ws, size_t ws_bytes, ppl_stream stream) {
  if (!lw || !state_in || !state_out || stride_bytes <= 0) return PPL_EINVAL;
  const bool fused = stride_bytes % 4 == 0 && stride_bytes <= 1024 &&
                     ((reinterpret_cast<uintptr_t>(state_in) |
                       reinterpret_cast<uintptr_t>(state_out)) & 3) == 0;
  if (fused)
    return resample_impl(lw, nullptr, max_lw_dev, n, m, seed, instance, t, ancestors, ws,
                         ws_bytes, stream, state_in, stride_bytes, state_out);
  PPL_TRY(resample_impl(lw, nullptr, max_lw_dev, n, m, seed, instance, t, ancestors, ws, ws_bytes,
                        stream));
  return cuda_status(launch_gather(state_in, n, stride_bytes, ancestors, m, state_out, nullptr,
                                   (cudaStream_t)stream));
}

ppl_status ppl_resample(const float* lw, const uint64_t* q_fixed, int64_t n, int64_t m,
                        uint64_t seed, uint32_t instance, uint32_t t, int32_t* ancestors,
                        void* ws, size_t ws_bytes, ppl_stream stream) {
  return resample_impl(lw, q_fixed, nullptr, n, m, seed, instance, t, ancestors, ws, ws_bytes,
                       stream);
}

ppl_status ppl_selftest_scan_timeout(const uint64_t* q_fixed, int64_t n, int32_t max_spin,
                                     void* ws, size_t ws_bytes, ppl_stream stream) {
  if (!q_fixed || n <= kScanTile || n > kMaxParticles || max_spin < 1 || max_spin > (1 << 22))
    return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, true, s));
  PPL_TRY(cuda_status(launch_scan_timeout_selftest(q_fixed, n, w.hdr(), w.tiles(), w.prefix(),
                                                   max_spin, s)));
  return ppl_workspace_status(ws, stream);
}

ppl_status ppl_resample_known_max(const float* lw, const double* max_lw_dev, int64_t n,
                                  int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                  int32_t* ancestors, void* ws, size_t ws_bytes,
                                  ppl_stream stream) {
  if (!lw || !max_lw_dev) return PPL_EINVAL;
  return resample_impl(lw, nullptr, max_lw_dev, n, m, seed, instance, t, ancestors, ws, ws_bytes,
                       stream);
}

ppl_status ppl_gather(const void* state_in, int64_t n_in, int64_t stride_bytes,
                      const int32_t* ancestors, int64_t m, void* state_out, ppl_stream stream) {
  if (!state_in || !state_out || !ancestors || stride_bytes <= 0 || m < 0 || n_in < 0)
    return PPL_EINVAL;
  if (m == 0) return PPL_OK;
  return cuda_status(launch_gather(state_in, n_in, stride_bytes, ancestors, m, state_out,
                                   nullptr, (cudaStream_t)stream));
}

ppl_status ppl_smc_step(const ppl_model* model, float y_t, int32_t t, uint64_t seed, float* x,
                        float* lw, int64_t n, double* logz_acc, int32_t* resampled,
                        double* logz_est, void* ws, size_t ws_bytes, ppl_stream stream) {
  if (!model || model->id != PPL_MODEL_LGSSM) return PPL_EINVAL;
  if (!(model->obs_sigma > 0.0f) || !isfinite(model->phi) || !isfinite(model->q_sigma))
    return PPL_EINVAL;
  if (!x || !lw || !logz_acc || !resampled || !logz_est || t < 1 || n < 1 || n > kMaxParticles)
    return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  const double r2 = (double)model->obs_sigma * (double)model->obs_sigma;
  LgssmParams p;
  p.phi = model->phi;
  p.q_sigma = model->q_sigma;
  p.obs_const = (float)(-0.5 * log(2.0 * M_PI * r2));
  p.neg_half_inv_r2 = (float)(-1.0 / (2.0 * r2));
  int32_t* anc = reinterpret_cast<int32_t*>(w.scratch());
  float* x_tmp = reinterpret_cast<float*>(w.scratch() + align_up((size_t)n * sizeof(int32_t)));
  const int32_t* gate = &w.hdr()->resample_flag;
  PPL_TRY(reset_ws(w, true, s));
  PPL_TRY(cuda_status(launch_smc_propagate(p, y_t, t, seed, x, lw, n, logz_acc, resampled,
                                           logz_est, w.hdr(), w.partials(), s)));
  // resampling with the states' gather fused (4-byte records)
  PPL_TRY(cuda_status(launch_resample_coop(lw, nullptr, nullptr, n, n, seed, 0, (uint32_t)t,
                                           w.hdr(), w.tiles(), reinterpret_cast<char*>(w.prefix()),
                                           w.l.bounds - w.l.prefix, anc, gate, s, x,
                                           (int64_t)sizeof(float), x_tmp)));
  PPL_TRY(cuda_status(launch_smc_commit(x, x_tmp, lw, n, gate, s)));
  return PPL_OK;
}

ppl_status ppl_rng_words(uint64_t seed, uint32_t instance, uint32_t step, uint32_t purpose,
                         int64_t n_particles, int32_t n_blocks, uint32_t* out_dev,
                         ppl_stream stream) {
  if (!out_dev || n_particles < 1 || n_particles > kMaxParticles || n_blocks < 1 ||
      n_blocks > 65535 || purpose > 0xffff)
    return PPL_EINVAL;
  if (reinterpret_cast<uintptr_t>(out_dev) & 15) return PPL_EINVAL;
  return cuda_status(launch_rng_words(seed, instance, step, purpose, n_particles, n_blocks,
                                      out_dev, (cudaStream_t)stream));
}

ppl_status ppl_smc_run(const ppl_model* model, const float* y, int32_t T, uint64_t seed,
                       int64_t n, float* x_out, float* lw_out, double* logz_out,
                       int32_t* resampled_out, double* ess_out, void* ws, size_t ws_bytes,
                       ppl_stream stream) {
  if (!model || model->id != PPL_MODEL_LGSSM) return PPL_EINVAL;
  if (!(model->obs_sigma > 0.0f) || !isfinite(model->phi) || !isfinite(model->q_sigma))
    return PPL_EINVAL;
  if (!y || T < 1 || n < 1 || n > kMaxParticles || !x_out || !lw_out || !logz_out ||
      !resampled_out || !ess_out || !ws || (reinterpret_cast<uintptr_t>(ws) % kAlign))
    return PPL_EINVAL;
  if (ws_bytes < smc_run_workspace(n, T)) return PPL_EINVAL;
  const double r2 = (double)model->obs_sigma * (double)model->obs_sigma;
  LgssmParams p;
  p.phi = model->phi;
  p.q_sigma = model->q_sigma;
  p.obs_const = (float)(-0.5 * log(2.0 * M_PI * r2));
  p.neg_half_inv_r2 = (float)(-1.0 / (2.0 * r2));
  int32_t* status = nullptr;
  const cudaError_t e =
      launch_smc_persistent(p, y, T, seed, n, x_out, lw_out, logz_out, resampled_out, ess_out,
                            static_cast<char*>(ws), ws_bytes, &status, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return PPL_EINVAL;
  return cuda_status(e);
}

ppl_status ppl_grid_barrier_probe(int32_t blocks, int32_t n_barriers, void* ws, size_t ws_bytes,
                                  ppl_stream stream) {
  if (blocks < 1 || blocks > num_sms() || n_barriers < 1 || n_barriers > (1 << 27) || !ws ||
      ws_bytes < 1024 || (reinterpret_cast<uintptr_t>(ws) % kAlign))
    return PPL_EINVAL;
  return cuda_status(launch_grid_barrier_probe(blocks, n_barriers, ws, (cudaStream_t)stream));
}

ppl_status ppl_posterior_reduce(const ppl_model* model, const ppl_poly_particle* particles,
                                const float* lw, int64_t n, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream) {
  PolyParams p;
  PPL_TRY(poly_params(model, &p));
  if (!particles || !out_dev || n < 1 || n > kMaxParticles) return PPL_EINVAL;
  if (reinterpret_cast<uintptr_t>(particles) & 15) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(cudaMemsetAsync(out_dev, 0, sizeof(ppl_is_result), s)));
  PPL_TRY(cuda_status(launch_posterior(p, particles, lw, n, w.hdr(), w.partials(), out_dev, s)));
  return PPL_OK;
}

ppl_status ppl_infer_is_partial(const ppl_model* model, const ppl_data* data,
                                int64_t first_particle, int64_t n_particles, uint64_t seed,
                                uint32_t instance, ppl_is_partial* partial_dev, float* lw_out,
                                ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                ppl_stream stream) {
  PolyParams p;
  PPL_TRY(poly_params(model, &p));
  if (!data || data->len < 0 || (data->len > 0 && (!data->x || !data->y))) return PPL_EINVAL;
  if (data->len > trace_tc_max_points()) return PPL_EINVAL;
  if (first_particle < 0 || n_particles < 1 || first_particle + n_particles > kMaxParticles ||
      !partial_dev || (reinterpret_cast<uintptr_t>(partial_dev) & 15))
    return PPL_EINVAL;
  if (particles_out && (reinterpret_cast<uintptr_t>(particles_out) & 15)) return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_particles, data->len, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(launch_poly_trace_tc(p, data->x, data->y, data->len, n_particles, seed,
                                           instance, lw_out, particles_out, w.hdr(),
                                           w.partials(), nullptr, s, first_particle,
                                           partial_dev)));
  return PPL_OK;
}

ppl_status ppl_is_merge(const ppl_is_partial* partials_dev, int32_t n_partials,
                        ppl_is_result* out_dev, ppl_stream stream) {
  if (!partials_dev || !out_dev || n_partials < 1 || n_partials > 65536 ||
      (reinterpret_cast<uintptr_t>(partials_dev) & 15))
    return PPL_EINVAL;
  return cuda_status(launch_merge_shards(partials_dev, n_partials, out_dev,
                                         (cudaStream_t)stream));
}

ppl_status ppl_resample_shard_total(const float* lw, int64_t n_local, const double* max_lw_dev,
                                    int64_t n_total, uint64_t* total_dev, void* ws,
                                    size_t ws_bytes, ppl_stream stream) {
  if (!lw || !max_lw_dev || !total_dev || n_local < 1 || n_total < n_local ||
      n_total > kMaxParticles)
    return PPL_EINVAL;
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, 1, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, false, s));
  PPL_TRY(cuda_status(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s)));
  return cuda_status(launch_shard_total(lw, n_local, n_total, max_lw_dev, total_dev, w.hdr(), s));
}

ppl_status ppl_resample_shard_plan(const uint64_t* totals, int32_t n_shards, int64_t n_total,
                                   int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                   ppl_resample_plan* plans) {
  if (!totals || !plans || n_shards < 1 || m < 1 || m > kMaxParticles || n_total < 1 ||
      n_total > kMaxParticles)
    return PPL_EINVAL;
  // T = sum of the shards' totals (each at most 2^61: the quantisation
  // bounds the whole population's sum by 2^61)
  uint64_t T = 0;
  for (int32_t g = 0; g < n_shards; ++g) {
    if (totals[g] > (1ull << 61) || T + totals[g] > (1ull << 61)) return PPL_EINVAL;
    T += totals[g];
  }
  if (T == 0) return PPL_EEMPTY;
  if (T < (uint64_t)m) return PPL_EINVAL;
  const uint64_t stride = T / (uint64_t)m;
  const uint32_t w = host_philox_word0(seed, 0, instance, t, 3 /* resampling offset */, 0);
  const uint64_t u = (uint64_t)(((unsigned __int128)w * stride) >> 32);
  // K(c) = #{k < m : u + k stride < c}
  auto K = [&](uint64_t c) -> int64_t {
    if (c <= u) return 0;
    const uint64_t k = (c - u + stride - 1) / stride;
    return k < (uint64_t)m ? (int64_t)k : m;
  };
  uint64_t c = 0;
  for (int32_t g = 0; g < n_shards; ++g) {
    ppl_resample_plan& p = plans[g];
    p.total = T;
    p.stride = stride;
    p.offset = u;
    p.c_base = c;
    p.k_first = K(c);
    c += totals[g];
    p.k_end = K(c);
    p.m = m;
    p.n_total = n_total;
  }
  return PPL_OK;
}

ppl_status ppl_resample_shard(const float* lw, int64_t n_local, int64_t first_particle,
                              const double* max_lw_dev, const ppl_resample_plan* plan,
                              int32_t* ancestors, const void* state_in, int64_t stride_bytes,
                              void* state_out, void* ws, size_t ws_bytes, ppl_stream stream) {
  if (!lw || !max_lw_dev || !plan || n_local < 1 || first_particle < 0 ||
      first_particle + n_local > plan->n_total || plan->n_total > kMaxParticles ||
      plan->k_first < 0 || plan->k_end < plan->k_first || plan->k_end > plan->m ||
      plan->stride == 0)
    return PPL_EINVAL;
  if (plan->k_end > plan->k_first && !ancestors) return PPL_EINVAL;
  if (state_in || state_out) {
    if (!state_in || !state_out || stride_bytes <= 0 || stride_bytes > 1024 || stride_bytes % 4 ||
        ((reinterpret_cast<uintptr_t>(state_in) | reinterpret_cast<uintptr_t>(state_out)) & 3))
      return PPL_EINVAL;
  }
  Ws w;
  PPL_TRY(check_ws(ws, ws_bytes, n_local, 0, &w));
  cudaStream_t s = (cudaStream_t)stream;
  PPL_TRY(reset_ws(w, true, s));
  ResampleShard sh;
  sh.n_total = plan->n_total;
  sh.first_particle = first_particle;
  sh.k_first = plan->k_first;
  sh.k_end = plan->k_end;
  sh.stride = plan->stride;
  sh.offset = plan->offset;
  sh.c_base = plan->c_base;
  PPL_TRY(cuda_status(launch_resample_coop(
      lw, nullptr, max_lw_dev, n_local, plan->m, 0, 0, 0, w.hdr(), w.tiles(),
      reinterpret_cast<char*>(w.prefix()), w.l.bounds - w.l.prefix, ancestors, nullptr, s,
      state_in, state_in ? stride_bytes : 0, state_out, &sh)));
  return PPL_OK;
}

}  // extern "C"
