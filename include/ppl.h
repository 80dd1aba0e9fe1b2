/*
 * ppl.h -- C ABI of the GB300 particle-inference library (libppl.so).
 *
 * The library runs the data-parallel hot path of likelihood-weighting
 * importance sampling (§3.6.2): many particles each run one execution trace of
 * a model function, where `sample` draws from a built-in distribution and
 * `factor` adds to the trace's log-weight (§3.4, Fig. 2); the log-weights are
 * normalised by log-sum-exp; sequential Monte Carlo (the particle methods named
 * as future work in §6) adds systematic resampling; the weighted empirical
 * posterior is reduced to the summary the line-fitting example asks for
 * (Fig. 1, §1.1).
 *
 * Conventions shared by every entry point:
 *  - Buffers marked [dev] are device memory owned by the caller; [host] are
 *    host memory.  Nothing is allocated on these paths.
 *  - `ws` is a caller-allocated device workspace of `ws_bytes` bytes, at least
 *    ppl_workspace_size(...) for the largest call it serves, 256-byte aligned.
 *    One workspace must not be used by two calls that run concurrently.
 *  - Calls are stream-ordered and asynchronous on `stream` (a cudaStream_t;
 *    NULL is the legacy default stream) unless stated otherwise.
 *  - A return value reports argument errors and launch failures.  Errors found
 *    on the device (NaN log-weights, an expired bounded wait, empty weights)
 *    are recorded in the workspace status word and in the `status` field of a
 *    result struct; read them with ppl_workspace_status after the stream
 *    reaches the call.
 *  - Random draws come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *    `seed`, with counter (particle, instance, step, purpose << 16 | block):
 *    results do not depend on launch configuration or control flow.
 */
#ifndef PPL_H
#define PPL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ppl_stream; /* cudaStream_t */

typedef enum {
  PPL_OK = 0,
  PPL_EINVAL = 1,   /* invalid argument (null pointer, bad size, workspace too small) */
  PPL_ENOMEM = 2,   /* reserved: the library never allocates on these paths */
  PPL_ECUDA = 3,    /* a CUDA launch or call failed */
  PPL_ENAN = 4,     /* a log-weight was NaN */
  PPL_EEMPTY = 5,   /* every weight is zero (all log-weights -inf) */
  PPL_ETIMEOUT = 6  /* a bounded device-side wait expired */
} ppl_status;

typedef enum { PPL_MODEL_POLY = 1, PPL_MODEL_LGSSM = 2 } ppl_model_id;

/* Model registry entry.  Fields a model does not use are ignored.
 *  PPL_MODEL_POLY (Fig. 1): n ~ uniform-discrete(min_deg, max_deg), at most 4
 *    values; n + coef_offset coefficients (at most 6) ~ normal(0, prior_sigma);
 *    factor(-sum_l (y_l - f(x_l))^2 / (2 obs_sigma^2)), f(x) = sum_k c_k x^k.
 *  PPL_MODEL_LGSSM: x_0 = 0, x_t = phi x_{t-1} + q_sigma e_t; observe(normal(x_t,
 *    obs_sigma), y_t) adds the normalised log-density (§3.4, Fig. 2). */
typedef struct {
  int32_t id;
  int32_t min_deg, max_deg, coef_offset;
  float obs_sigma;
  float prior_sigma;
  float phi, q_sigma;
} ppl_model;

/* Observed data set [dev]: x[len], y[len] in FP32. */
typedef struct {
  const float* x;
  const float* y;
  int64_t len;
} ppl_data;

/* One line-fitting particle, 32 bytes: the coefficients (zero beyond the
 * trace's count), the sampled degree, and the index of the trace it came from. */
typedef struct {
  float c[6];
  int32_t n;
  uint32_t origin;
} ppl_poly_particle;

/* Posterior summary of a weighted population (§3.6.2, Fig. 1).  FP64 fields,
 * formed from FP32 partials with double-float sums (about 48 significant
 * bits); the kernels write every field, so the buffer needs no clearing.
 *  log_z   = lse - log N: estimate of the evidence E_prior[exp(sum of factors)]
 *  ess     = (sum w)^2 / sum w^2
 *  argmax  = the mode: index of the highest log-weight (lowest index on ties)
 *  p_n[d]  = posterior mass of degree min_deg + d; map_deg its argmax
 *  mean_c  = weighted mean coefficients, zero beyond each trace's count
 *  deg_mean/deg_var[d][k] = weighted mean/variance of c_k among degree min_deg + d
 *  deg_max_lw/deg_argmax  = best trace of each degree (-inf / -1 if none) */
typedef struct {
  double log_z, lse, ess, max_lw;
  int64_t argmax, n_particles;
  int32_t map_deg, n_deg;
  double p_n[4];
  double mean_c[6];
  double deg_mean[4][6];
  double deg_var[4][6];
  double deg_max_lw[4];
  int64_t deg_argmax[4];
  int32_t status, pad;
} ppl_is_result;

/* The paper's tiny discrete benchmarks (Table 1 of §5.1). */
typedef enum {
  PPL_DISCRETE_BIASEDCOIN = 0, /* theta = a/10, a ~ uniform-discrete(1,9); observe flips */
  PPL_DISCRETE_BINOMIAL = 1,   /* successes among `limit` bernoulli(0.3) samples */
  PPL_DISCRETE_GEOMETRIC = 2   /* bernoulli(0.5) failures before a success, < `limit` */
} ppl_discrete_model;

#define PPL_DISCRETE_MAX_VALUES 64

/* The normalised distribution of a discrete model's return value.  Value code
 * v: biasedcoin theta = (v + 1)/10 (9 codes); binomial k = v (limit + 1
 * codes); geometric c = v (limit + 1 codes, the last one -- the limit reached
 * -- outside the truncated support).  [dev] like ppl_is_result. */
typedef struct {
  double log_z, ess, max_lw;
  double mean;  /* sum over codes of prob * value */
  int64_t n_particles;
  int32_t n_values, status;
  double value[PPL_DISCRETE_MAX_VALUES];
  double prob[PPL_DISCRETE_MAX_VALUES];
  int64_t count[PPL_DISCRETE_MAX_VALUES]; /* particles that returned each code */
} ppl_discrete_result;

/* The customdist benchmark (Table 1 of §5.1): a user-defined distribution
 * whose density is w1 N(mu1, sigma1^2) + (1 - w1) N(mu2, sigma2^2), its draw
 * observed through normal(x, obs_sigma) at every data point. */
typedef struct {
  float w1, mu1, sigma1, mu2, sigma2, obs_sigma;
} ppl_customdist_model;

typedef struct {
  double log_z, lse, ess, max_lw;
  double mean_x, var_x; /* posterior mean and variance of x under the normalised weights */
  int64_t n_particles;
  int32_t status, pad;
} ppl_customdist_result;

/* Readable name of a status code.  Never NULL. */
const char* ppl_status_string(int32_t status);

/* Workspace bytes needed by any call below for this model and sizes
 * (n_particles particles, data_len data points or time steps).  Returns 0 for
 * invalid arguments. */
size_t ppl_workspace_size(const ppl_model* model, int64_t n_particles, int64_t data_len);

/* Synchronise `stream` and return the device-side status recorded in `ws`
 * by the calls issued before (PPL_OK if none failed). */
ppl_status ppl_workspace_status(const void* ws, ppl_stream stream);

/* Likelihood weighting (§3.6.2) on the line-fitting model (Fig. 1): particle i
 * runs one trace, lw_i = sum of its factors; the population is normalised and
 * reduced into *out_dev [dev].  lw_out [dev, n_particles] and particles_out
 * [dev, n_particles] are optional (NULL to skip).  1 <= n_particles < 2^31;
 * data->len >= 0. */
ppl_status ppl_infer_is(const ppl_model* model, const ppl_data* data, int64_t n_particles,
                        uint64_t seed, ppl_is_result* out_dev, float* lw_out,
                        ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                        ppl_stream stream);

/* ppl_infer_is for instance `instance` of a batch: the counter field
 * `instance` of every draw is set to it, so independent instances (or ranks)
 * with one seed draw independent traces.  ppl_infer_is uses instance 0.  The
 * whole summary (normalisation and posterior) comes out of one fused kernel. */
ppl_status ppl_infer_is_instance(const ppl_model* model, const ppl_data* data,
                                 int64_t n_particles, uint64_t seed, uint32_t instance,
                                 ppl_is_result* out_dev, float* lw_out,
                                 ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                 ppl_stream stream);

/* One shard's share of a likelihood-weighting pass whose particles are split
 * over several GPUs (or calls) by contiguous ranges of the global particle
 * index: the particle-based inference the paper names as future work (§6)
 * scales out because its normalisation (§3.6.2) is a reduction over all
 * samples, and per-degree partials merge like the blocks of one kernel.
 * Opaque, 384 bytes; [dev] buffers of it must be 16-byte aligned. */
typedef struct {
  unsigned char opaque[384];
} ppl_is_partial;

/* Likelihood weighting on particles [first_particle, first_particle +
 * n_particles) of a population: trace i of this call draws as particle
 * first_particle + i of ppl_infer_is_instance (same seed and instance), so a
 * population split over shards draws exactly the traces of the unsplit call.
 * Writes this shard's partial to *partial_dev [dev]; lw_out and
 * particles_out [dev, n_particles] (optional) are indexed by i, and a
 * record's origin is its global particle index.  Data sets of at most 2048
 * points (the tensor-core trace kernel); first_particle + n_particles <
 * 2^31.  Workspace: ppl_workspace_size(model, n_particles, data->len). */
ppl_status ppl_infer_is_partial(const ppl_model* model, const ppl_data* data,
                                int64_t first_particle, int64_t n_particles, uint64_t seed,
                                uint32_t instance, ppl_is_partial* partial_dev, float* lw_out,
                                ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                ppl_stream stream);

/* The summary of a population from its shards' partials, partials_dev [dev,
 * n_partials] (e.g. gathered from every rank), into *out_dev [dev].  The
 * result is that of ppl_infer_is_instance on the whole population up to the
 * order of FP32 and double-float roundings in the merge (maxima, argmax and counts are
 * exact).  A shard's device error is reported in out_dev->status; no finite
 * weight anywhere -> PPL_EEMPTY. */
ppl_status ppl_is_merge(const ppl_is_partial* partials_dev, int32_t n_partials,
                        ppl_is_result* out_dev, ppl_stream stream);

/* Sharded systematic resampling (particle methods across devices, §6): a
 * population of n_total particles split by contiguous ranges of the global
 * index, m outputs.  The fixed-point weights are those of ppl_resample on the
 * whole population (its maximum log-weight, the scale 2^(61 - ceil(log2
 * n_total))), so the ancestors are those of the unsplit call bit for bit:
 *  1. each shard: ppl_logsumexp gives its maximum; the maximum over shards
 *     (an all-reduce) is the population's;
 *  2. each shard: ppl_resample_shard_total -> its sum of fixed-point weights;
 *  3. every shard, from all shards' sums in shard order (an all-gather):
 *     ppl_resample_shard_plan -> each shard's plan;
 *  4. each shard: ppl_resample_shard -> the ancestors (global indices) of its
 *     outputs [k_first, k_end), which all descend from its own particles,
 *     and optionally their gathered records. */
typedef struct {
  uint64_t total, stride, offset; /* the population's T, floor(T / m), u */
  uint64_t c_base;                /* sum of the fixed-point weights of the shards before */
  int64_t k_first, k_end;         /* this shard's outputs */
  int64_t m, n_total;
} ppl_resample_plan;

/* The sum of the shard's fixed-point weights into *total_dev [dev, u64]:
 * lw [dev, n_local], *max_lw_dev [dev, FP64] the population's maximum.  A
 * log-weight above it sets PPL_EINVAL in the workspace status.  Workspace:
 * ppl_workspace_size(any model, 1, 0). */
ppl_status ppl_resample_shard_total(const float* lw, int64_t n_local, const double* max_lw_dev,
                                    int64_t n_total, uint64_t* total_dev, void* ws,
                                    size_t ws_bytes, ppl_stream stream);

/* Host only (no device work): the plans of n_shards shards from their sums
 * totals [host, n_shards], in shard order, into plans [host, n_shards].  The
 * offset u is the resampling draw of ppl_resample (step t, instance).
 * Every weight zero -> PPL_EEMPTY; sums above 2^61 or below m -> PPL_EINVAL. */
ppl_status ppl_resample_shard_plan(const uint64_t* totals, int32_t n_shards, int64_t n_total,
                                   int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                   ppl_resample_plan* plans);

/* One shard's resampling: ancestors [dev, k_end - k_first] gets, for output
 * k of the population, the global index of its ancestor at ancestors[k -
 * k_first].  With state_in [dev, n_local records of stride_bytes, a multiple
 * of 4 up to 1024, 4-byte aligned] the records of those outputs' ancestors
 * are copied to state_out [dev, k_end - k_first records].  `plan` [host] is
 * this shard's entry.  Workspace: ppl_workspace_size(any model, n_local, 0). */
ppl_status ppl_resample_shard(const float* lw, int64_t n_local, int64_t first_particle,
                              const double* max_lw_dev, const ppl_resample_plan* plan,
                              int32_t* ancestors, const void* state_in, int64_t stride_bytes,
                              void* state_out, void* ws, size_t ws_bytes, ppl_stream stream);

/* ppl_infer_is_instance with the factor evaluated from the data's
 * sufficient statistics instead of point by point.  The model of Fig. 1 is
 * linear in its coefficients, so with Phi the matrix of powers x_l^j,
 * G = Phi^T Phi = R^T R and w = R^-T Phi^T y, a trace with d coefficients has
 * sum_l (y_l - f(x_l))^2 = (y^T y - sum_{i<d} w_i^2) + |R_d c - w_d|^2 (exact in
 * real arithmetic; both terms are non-negative, so nothing cancels).  One
 * small kernel forms G, R and w in FP64; each trace then costs O(d^2) instead
 * of O(L d).  The draws, and so the traces, are those of ppl_infer_is_instance
 * bit for bit; log-weights differ by rounding only.  When G is singular to
 * working precision (fewer distinct points than coefficients) the point-by-
 * point sum is used.  Same arguments and workspace as ppl_infer_is_instance. */
ppl_status ppl_infer_is_suffstat(const ppl_model* model, const ppl_data* data,
                                 int64_t n_particles, uint64_t seed, uint32_t instance,
                                 ppl_is_result* out_dev, float* lw_out,
                                 ppl_poly_particle* particles_out, void* ws, size_t ws_bytes,
                                 ppl_stream stream);

/* Likelihood weighting (§3.6.2) on a tiny discrete benchmark (Table 1 of
 * §5.1).  Each `sample` takes one Philox word, in program order, from blocks
 * 0, 1, ... of counter (particle, 0, 0, POLY_TRACE); bernoulli(p) is
 * u01(w) < p, decided exactly on the word's top 23 bits.  flips [dev, int32,
 * 0/1, n_flips] are biasedcoin's observations; `limit` is binomial's number
 * of trials (0..63) or geometric's depth (1..63).  Writes *out_dev; codes_out
 * and lw_out [dev, n_particles] are optional per-particle outputs.  `ws` needs
 * ppl_workspace_size(model, 1, 0) bytes for any model.  Invalid model, limit
 * or n_particles -> PPL_EINVAL; no finite weight -> PPL_EEMPTY in the status. */
ppl_status ppl_infer_discrete(int32_t model, const int32_t* flips, int64_t n_flips, int32_t limit,
                              int64_t n_particles, uint64_t seed, ppl_discrete_result* out_dev,
                              int32_t* codes_out, float* lw_out, void* ws, size_t ws_bytes,
                              ppl_stream stream);

/* Likelihood weighting (§3.6.2) on customdist: x from the user-defined
 * density (component 1 when u01(w0) < w1, then mu + sigma z with z the first
 * Box-Muller normal of words 1, 2; block 0 of counter (particle, 0, 0,
 * POLY_TRACE)); lw = sum_j log N(y_j; x, obs_sigma^2).  y [dev, FP32, n_obs];
 * writes *out_dev; x_out and lw_out [dev, n_particles] optional.  `ws` needs
 * ppl_workspace_size(model, n_particles, 0) bytes for any ppl_model.  Invalid
 * weights (w1 outside [0, 1]) or scales (not positive) -> PPL_EINVAL. */
ppl_status ppl_infer_customdist(const ppl_customdist_model* model, const float* y, int64_t n_obs,
                                int64_t n_particles, uint64_t seed,
                                ppl_customdist_result* out_dev, float* x_out, float* lw_out,
                                void* ws, size_t ws_bytes, ppl_stream stream);

/* The proposal network's matrix product on the fifth-generation tensor
 * cores: C[m, n] = sum_k A(m, k) B(n, k), A(m, k) = A[m sam + k sak],
 * B(n, k) = B[n sbn + k sbk] (BF16, any strides: transposed operands are read
 * in place), C [dev, FP32, M x N row-major], FP32 accumulation.  A wait that
 * runs out is reported through ppl_workspace_status(ws); `ws` needs
 * ppl_workspace_size(model, 1, 0) bytes for any model.  M, N, K >= 1 and
 * below 2^24 (else PPL_EINVAL). */
ppl_status ppl_gemm_bf16(const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbn,
                         int64_t sbk, int32_t M, int32_t N, int32_t K, float* C, void* ws,
                         size_t ws_bytes, ppl_stream stream);

/* Same as ppl_infer_is with the data and the result in host memory: copies x,
 * y in, runs, copies the summary out, and synchronises `stream` before it
 * returns.  The workspace must also hold the data (see ppl_workspace_size). */
ppl_status ppl_infer_is_host(const ppl_model* model, const float* x_host, const float* y_host,
                             int64_t data_len, int64_t n_particles, uint64_t seed,
                             ppl_is_result* out_host, void* ws, size_t ws_bytes,
                             ppl_stream stream);

/* Log-sum-exp normalisation (§3.6.2) of lw[n] [dev, FP32]: writes FP64
 * out_dev[0] = LSE, out_dev[1] = ESS, out_dev[2] = max lw, and the argmax (lowest
 * index on ties) as a double in out_dev[3].  NaN -> PPL_ENAN status; all -inf ->
 * PPL_EEMPTY status. */
ppl_status ppl_logsumexp(const float* lw, int64_t n, double* out_dev, void* ws, size_t ws_bytes,
                         ppl_stream stream);

/* Systematic resampling with 64-bit fixed-point weights.  Exactly one of lw
 * [dev, FP32, n] and q_fixed [dev, u64, n] is non-NULL.  From lw:
 * q_i = floor(E32(lw_i - max lw) * 2^(61 - ceil(log2 n))), E32 the library's
 * fixed FP32 exponential; q_fixed must sum to at most 2^61.  With T = sum q,
 * step = floor(T / m) and u = floor(w * step / 2^32) (w: word 0 of counter
 * (0, instance, t, RESAMPLE)), ancestors[k] [dev, m] = min{j : q_0 + .. + q_j >
 * u + k * step}.  The prefix sums are exact, so ancestors are bit-exact.  The
 * workspace must be sized for max(n, m) particles. */
ppl_status ppl_resample(const float* lw, const uint64_t* q_fixed, int64_t n, int64_t m,
                        uint64_t seed, uint32_t instance, uint32_t t, int32_t* ancestors,
                        void* ws, size_t ws_bytes, ppl_stream stream);

/* ppl_resample from lw when the maximum log-weight is already known on the
 * device, e.g. &out_dev->max_lw of the ppl_infer_is that produced lw (whose
 * status was PPL_OK): saves a pass over lw.  NaN log-weights are not detected;
 * a log-weight above *max_lw_dev is reported as PPL_EINVAL. */
ppl_status ppl_resample_known_max(const float* lw, const double* max_lw_dev, int64_t n,
                                  int64_t m, uint64_t seed, uint32_t instance, uint32_t t,
                                  int32_t* ancestors, void* ws, size_t ws_bytes,
                                  ppl_stream stream);

/* Resampling and the gather of the resampled state in one pass: the same
 * ancestors as ppl_resample (max_lw_dev may be NULL, as there) or
 * ppl_resample_known_max written to ancestors [dev, int32, m], and
 * state_out[k] = state_in[ancestors[k]] for k < m, records of stride_bytes
 * bytes [dev]; state_in holds the n particles' records.  Records whose size
 * is a multiple of 4 bytes (up to 1024) with 4-byte aligned buffers are
 * copied by the resampling kernel's own work items as their ancestors are
 * found (in 16-byte words when size and buffers allow); other records go
 * through ppl_gather after it.  Errors as ppl_resample and ppl_gather. */
ppl_status ppl_resample_gather(const float* lw, const double* max_lw_dev, int64_t n, int64_t m,
                               uint64_t seed, uint32_t instance, uint32_t t, const void* state_in,
                               int64_t stride_bytes, void* state_out, int32_t* ancestors,
                               void* ws, size_t ws_bytes, ppl_stream stream);

/* Self-test of failure detection in the resampler's bounded wait: runs the
 * decoupled-lookback scan over q_fixed [dev, u64, n > 2048] with its first tile
 * silenced, so every later tile's wait on it expires after max_spin polls
 * (1..2^22); synchronises and returns the device status, PPL_ETIMEOUT when the
 * waits ran out as designed.  Nothing hangs: a tile that gives up publishes. */
ppl_status ppl_selftest_scan_timeout(const uint64_t* q_fixed, int64_t n, int32_t max_spin,
                                     void* ws, size_t ws_bytes, ppl_stream stream);

/* Gather of the resampled particle state: state_out[k] = state_in[ancestors[k]]
 * for k < m, records of stride_bytes bytes [dev]; state_in holds n_in records.
 * An ancestor outside [0, n_in) yields a zero-filled record instead of a read
 * out of bounds.  stride_bytes > 0; in and out must not overlap. */
ppl_status ppl_gather(const void* state_in, int64_t n_in, int64_t stride_bytes,
                      const int32_t* ancestors, int64_t m, void* state_out, ppl_stream stream);

/* One step t >= 1 of the bootstrap particle filter on PPL_MODEL_LGSSM with
 * adaptive resampling, over x[n], lw[n] [dev, FP32].  Propagates every
 * particle, adds observe(normal(x, obs_sigma), y_t), computes ESS; if
 * ESS < n/2 it adds LSE - log n to *logz_acc [dev, FP64], resamples x with
 * ppl_resample's scheme (instance 0, step t) and zeroes lw.  Writes
 * *resampled [dev] = 1 or 0 and logz_est[0] [dev, FP64] = logz_acc + LSE(lw) -
 * log n, the running evidence estimate; logz_est[1] = ESS before resampling. */
ppl_status ppl_smc_step(const ppl_model* model, float y_t, int32_t t, uint64_t seed, float* x,
                        float* lw, int64_t n, double* logz_acc, int32_t* resampled,
                        double* logz_est, void* ws, size_t ws_bytes, ppl_stream stream);

/* The whole bootstrap filter of ppl_smc_step for t = 1..T in one persistent
 * cooperative kernel: x_0 = 0, lw_0 = 0, observations y [dev, FP32, T]; the
 * particles stay in registers between steps, which are separated by bounded
 * grid barriers.  Each step computes exactly what ppl_smc_step computes.
 * Writes x_out, lw_out [dev, n] (the final population), *logz_out [dev, FP64]
 * (the evidence estimate), resampled_out [dev, int32, T] and ess_out [dev,
 * FP64, T] (ESS before resampling).  n must fit the resident threads, at
 * most 8 particles each (about 1.2 million on a GB300: one block of 1024
 * threads per SM); larger n, or T > 2^27, -> PPL_EINVAL.  A
 * barrier wait that runs out records PPL_ETIMEOUT in `ws` (read with
 * ppl_workspace_status) and ends the kernel.  `ws` holds at least
 * ppl_workspace_size(model, n, T) bytes.  The per-step normalising sums are
 * kept as FP32 pairs (about 48 significant bits); log Z and the ESS are formed
 * from them in FP64 after the last step.  Capturable in a CUDA graph. */
ppl_status ppl_smc_run(const ppl_model* model, const float* y, int32_t T, uint64_t seed,
                       int64_t n, float* x_out, float* lw_out, double* logz_out,
                       int32_t* resampled_out, double* ess_out, void* ws, size_t ws_bytes,
                       ppl_stream stream);

/* The cost floor of ppl_smc_run's step separators (§6: the particle filter's
 * steps meet at population-wide reductions): one cooperative launch of
 * `blocks` blocks of 1024 threads (the filter's launch shape; 1 <= blocks <=
 * the SMs) passing n_barriers (>= 1) bounded grid barriers of the filter's
 * kind and doing nothing else.  The caller times it on `stream` (CUDA events)
 * to see what the barriers alone cost.  `ws` [dev] holds at least 1024 bytes
 * (its first 512 are cleared by the call); a barrier wait that runs out
 * records PPL_ETIMEOUT there (ppl_workspace_status).  Bad sizes ->
 * PPL_EINVAL. */
ppl_status ppl_grid_barrier_probe(int32_t blocks, int32_t n_barriers, void* ws, size_t ws_bytes,
                                  ppl_stream stream);

/* Posterior summary (as ppl_infer_is) of an existing weighted population of
 * line-fitting particles [dev] with log-weights lw [dev]; lw == NULL means
 * equal weights.  Writes *out_dev [dev]. */
ppl_status ppl_posterior_reduce(const ppl_model* model, const ppl_poly_particle* particles,
                                const float* lw, int64_t n, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream);

/* The raw random words behind every `sample` (§3.4): out_dev [dev, u32,
 * 16-byte aligned] receives, for particle i < n_particles and block j <
 * n_blocks, the four Philox4x32-10 words of counter (i, instance, step,
 * purpose << 16 | j) at out_dev[(i * n_blocks + j) * 4 ...].  Purposes: 1 line-
 * fitting trace, 2 state-space propagation, 3 resampling offset. */
ppl_status ppl_rng_words(uint64_t seed, uint32_t instance, uint32_t step, uint32_t purpose,
                         int64_t n_particles, int32_t n_blocks, uint32_t* out_dev,
                         ppl_stream stream);

/* Batched likelihood weighting: many independent line-fitting data sets of
 * uneven size in one persistent launch.  Instance b has data x, y [dev] at
 * [data_off[b], data_off[b+1]) and part_off[b+1] - part_off[b] >= 1 particles;
 * its draws use counter field instance = b.  The work is cut into (instance,
 * tile of 256 * ppt particles) items taken heaviest first (longest data first)
 * from an atomic queue by num_SMs * blocks_per_sm resident blocks; the last
 * item of an instance writes out_dev[b] [dev].
 *  ppl_batched_workspace_size: bytes for any configuration (host offsets).
 *  ppl_batched_prepare: builds the item plan on the host from host copies of
 *    the offsets, copies it into `ws` and synchronises `stream`; fills *plan.
 *  ppl_infer_is_batched: the launch (a memset, a device copy and one kernel);
 *    it can be captured in a CUDA graph and replayed.
 *  ppl_batched_autotune: times every ppt in {1,2,4,8} x blocks_per_sm in
 *    {1..4} on the caller's data, keeps the fastest (cached as one JSON line in
 *    cache_path, reused when the batch's shape matches), and prepares it. */
typedef struct {
  int32_t ppt, blocks_per_sm, n_inst, pad;
  int64_t n_items, max_len, total_particles;
  double work; /* sum over instances of particles x data points */
} ppl_batch_plan;

size_t ppl_batched_workspace_size(const int64_t* data_off_host, const int64_t* part_off_host,
                                  int32_t n_inst, int32_t ppt);
ppl_status ppl_batched_prepare(const ppl_model* model, const int64_t* data_off_host,
                               const int64_t* part_off_host, int32_t n_inst, int32_t ppt,
                               int32_t blocks_per_sm, ppl_batch_plan* plan, void* ws,
                               size_t ws_bytes, ppl_stream stream);
ppl_status ppl_infer_is_batched(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off, const int64_t* part_off,
                                int32_t n_inst, uint64_t seed, const ppl_batch_plan* plan,
                                ppl_is_result* out_dev, void* ws, size_t ws_bytes,
                                ppl_stream stream);
ppl_status ppl_batched_autotune(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off_dev, const int64_t* part_off_dev,
                                const int64_t* data_off_host, const int64_t* part_off_host,
                                int32_t n_inst, uint64_t seed, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, const char* cache_path, ppl_batch_plan* best,
                                ppl_stream stream);
ppl_status ppl_batched_status(const void* ws, ppl_stream stream);

/* Learned proposal (inference compilation: Le, Baydin and Wood, AISTATS 2017).
 * A network maps a 32-point line-fitting data set to a proposal q(n, c | data)
 * over the trace's random choices; importance weights p/q correct it to the
 * posterior (§3.6.2).  Network: in[64] = the points sorted by x, (x, y/10),
 * BF16; h1 = relu(W1 in + b1), h2 = relu(W2 h1 + b2) with 256 units, out =
 * W3 h2 + b3 with 48 outputs; BF16 weights and activations on the tensor
 * cores (tcgen05, accumulator in tensor memory; ppl_gemm_bf16), FP32
 * accumulation, FP32 biases.  A tensor-core wait that runs out sets the first
 * word of the proposal workspace (read it with ppl_workspace_status).  out[0..n_deg) are degree logits;
 * coefficient j of degree slot k (slots in order, ncoef_k = min_deg + k +
 * coef_offset) has mu = prior_sigma out[4 + 2 i], s = prior_sigma exp(clamp(
 * out[5 + 2 i], -9, 1)), i = ncoef_0 + .. + ncoef_{k-1} + j.
 * params [dev, FP32, ppl_proposal_num_params()] = W1 | b1 | W2 | b2 | W3 | b3
 * (row-major [out x in]).  Training pairs are forward simulations of the model
 * (purpose FORWARD_SIM): pair p draws a prior trace and 32 points x ~ U[-1, 1],
 * y = f(x) + obs_sigma e.
 *  ppl_proposal_features: BF16 features [dev, n_sets x 64] of x, y [n_sets x 32].
 *  ppl_proposal_forward: out_dev [dev, FP32, n_sets x 48] for data sets x, y.
 *  ppl_proposal_grad: gradient [dev, FP32] of the mean -log q over pairs
 *    pair0 .. pair0 + batch - 1, and the summed loss in loss_out [dev, FP64].
 *  ppl_proposal_train: Adam (lr, 0.9, 0.999, 1e-8) on params with moments
 *    adam_m, adam_v [dev, FP32, zero-initialised], epochs x (n_pairs / batch)
 *    steps over pairs 0 .. n_pairs - 1; loss_per_step [dev, FP64] optional.
 *    It is ppl_proposal_train_init followed by ppl_proposal_train_steps of
 *    every step.
 *  ppl_proposal_train_init: zeroes the training run's step counter in `ws`
 *    and converts params to the BF16 copy the products read.
 *  ppl_proposal_train_steps: n_steps more steps of the run that `ws` holds.
 *    Step s (the counter, kept on the device) trains on pairs (s mod
 *    (n_pairs / batch)) batch .. + batch - 1 and writes its summed loss to
 *    loss_per_step[s]; nothing a step does depends on host values, so the
 *    enqueued work of one call (about 17 launches per step) can be captured
 *    once in a CUDA graph by the caller and replayed for every later block of
 *    steps.
 *  ppl_infer_is_learned: ppl_infer_is_batched with each instance's draws from
 *    its proposal (proposal [dev, FP32, n_inst x 48], e.g. from
 *    ppl_proposal_forward); a proposal equal to the prior gives the prior run. */
int64_t ppl_proposal_num_params(void);
size_t ppl_proposal_workspace_size(int32_t batch);
ppl_status ppl_proposal_features(const float* x, const float* y, int32_t n_sets, void* feat_dev,
                                 ppl_stream stream);
ppl_status ppl_proposal_forward(const ppl_model* model, const float* params, const float* x,
                                const float* y, int32_t n_sets, float* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream);
ppl_status ppl_proposal_grad(const ppl_model* model, const float* params, int64_t pair0,
                             int32_t batch, uint64_t seed, float* grad_out, double* loss_out,
                             void* ws, size_t ws_bytes, ppl_stream stream);
ppl_status ppl_proposal_train(const ppl_model* model, float* params, float* adam_m,
                              float* adam_v, int64_t n_pairs, int32_t batch, int32_t epochs,
                              uint64_t seed, float lr, double* loss_per_step, void* ws,
                              size_t ws_bytes, ppl_stream stream);
ppl_status ppl_proposal_train_init(const float* params, int32_t batch, void* ws,
                                   size_t ws_bytes, ppl_stream stream);
ppl_status ppl_proposal_train_steps(const ppl_model* model, float* params, float* adam_m,
                                    float* adam_v, int64_t n_pairs, int32_t batch,
                                    int32_t n_steps, uint64_t seed, float lr,
                                    double* loss_per_step, void* ws, size_t ws_bytes,
                                    ppl_stream stream);
ppl_status ppl_infer_is_learned(const ppl_model* model, const float* x, const float* y,
                                const int64_t* data_off, const int64_t* part_off,
                                int32_t n_inst, uint64_t seed, const ppl_batch_plan* plan,
                                const float* proposal, ppl_is_result* out_dev, void* ws,
                                size_t ws_bytes, ppl_stream stream);

/* ppl_resample without a workspace, for callers that cannot allocate device
 * memory: a plugin whose host application owns every device allocation
 * through its own pool, or a real-time loop that must not risk the implicit
 * device synchronisation of cudaMalloc.  The paper has no counterpart; this is
 * a library convenience.  Same arguments and result as ppl_resample, but the
 * scratch is a static device array of about 9.4 MB per device, so n and m must
 * be at most 2^20 (1048576); larger sizes return PPL_EINVAL.  Nothing is
 * allocated.  The first call on a device looks the array's address up and
 * caches it (make that first call before any stream capture).  All calls on a
 * device share the array: calls whose work overlaps on the GPU race, so issue
 * them in one stream.  Device-side errors are read with
 * ppl_resample_noalloc_status, which synchronises `stream`. */
ppl_status ppl_resample_noalloc(const float* lw, const uint64_t* q_fixed, int64_t n, int64_t m,
                                uint64_t seed, uint32_t instance, uint32_t t, int32_t* ancestors,
                                ppl_stream stream);
ppl_status ppl_resample_noalloc_status(ppl_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* PPL_H */
