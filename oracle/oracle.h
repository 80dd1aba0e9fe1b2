/*
 * Oracle for the particle-inference hot path: a plain, slow FP64 restatement
 * in C of what the CUDA library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load, call or link this code.
 * It shares no code, header, constant table or helper with the CUDA library
 * (paper_2010_08454_gb300/csrc), and neither side includes the other.  The two
 * sides agree only on a written specification (counter layout, uniform and
 * normal transforms, fixed-point weights), each implemented independently.
 *
 * Floating point is FP64 throughout, except the conversion of log-weights to
 * fixed-point resampling weights, which the method defines in FP32 (the
 * integer it produces must be decided in the same precision on both sides).
 */
#ifndef PPL_ORACLE_H
#define PPL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- random numbers (philox.c) ---------------------------------------- */
enum {
  ORC_PURPOSE_POLY_TRACE = 1,
  ORC_PURPOSE_LGSSM_PROPAGATE = 2,
  ORC_PURPOSE_RESAMPLE = 3,
  ORC_PURPOSE_LEARNED_TRACE = 4,
  ORC_PURPOSE_FORWARD_SIM = 5
};

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_block(uint64_t seed, uint32_t particle, uint32_t instance, uint32_t step,
                      uint32_t purpose, uint32_t block, uint32_t out[4]);
double orc_u01(uint32_t w);
void orc_box_muller(uint32_t wa, uint32_t wb, double* z0, double* z1);
int orc_uniform_discrete(uint32_t w, int lo, int hi);
float orc_ln32(float u);
float orc_cos2pi32(float u);
float orc_normal32(uint32_t wa, uint32_t wb);

/* ---- polynomial line-fitting model (poly.c) ---------------------------- */
typedef struct {
  int min_deg, max_deg; /* degree prior: uniform-discrete{min_deg..max_deg} */
  int coef_offset;      /* a degree-n trace draws n + coef_offset coefficients */
  double obs_sigma;     /* distance scale: factor = -sum r^2 / (2 obs_sigma^2) */
  double prior_sigma;   /* coefficient prior: normal(0, prior_sigma) */
} orc_poly;

double orc_poly_trace(const orc_poly* m, const double* x, const double* y, int64_t L,
                      uint64_t seed, uint32_t instance, uint32_t particle, int* n_out,
                      double c_out[6]);
void orc_is_poly(const orc_poly* m, const double* x, const double* y, int64_t L, int64_t N,
                 uint64_t seed, uint32_t instance, double* lw, int32_t* n, double* c);
void orc_is_poly_indices(const orc_poly* m, const double* x, const double* y, int64_t L,
                         const int64_t* idx, int64_t K, uint64_t seed, uint32_t instance,
                         double* lw, int32_t* n, double* c);

/* ---- normalisation and posterior summary (normalize.c) ---------------- */
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
} orc_is_result;

void orc_lse_ess(const double* lw, int64_t N, double* lse, double* ess, double* max_lw,
                 int64_t* argmax);
void orc_posterior_poly(const orc_poly* m, const double* lw, const int32_t* n, const double* c,
                        int64_t N, orc_is_result* out);

/* ---- fixed-point systematic resampling (resample.c) ------------------- */
float orc_exp32(float d);
int orc_fixed_shift(int64_t N);
void orc_quantize_weights(const float* lw, int64_t N, uint64_t* q);
int orc_resample_systematic(const uint64_t* q, int64_t N, int64_t M, uint64_t seed,
                            uint32_t instance, uint32_t step, int32_t* ancestors);
int orc_resample_from_lw(const float* lw, int64_t N, int64_t M, uint64_t seed,
                         uint32_t instance, uint32_t step, int32_t* ancestors);
void orc_gather(const void* in, int64_t stride_bytes, const int32_t* anc, int64_t M, void* out);

/* ---- linear-Gaussian state-space model (lgssm.c) ---------------------- */
typedef struct {
  double phi, q_sigma, r_sigma;
} orc_lgssm;

double orc_kalman_logz(const orc_lgssm* m, const double* y, int64_t T);
double orc_smc_lgssm(const orc_lgssm* m, const double* y, int64_t T, int64_t N, uint64_t seed,
                     int state_f32, double* ess_t, int32_t* resampled_t, double* x_out,
                     double* lw_out);

/* ---- conjugate evidence (conjugate.c) --------------------------------- */
double orc_blr_evidence(const double* x, const double* y, int64_t L, int ncoef, double sigma,
                        double prior_sigma, double* mean, double* var);
double orc_poly_exact(const orc_poly* m, const double* x, const double* y, int64_t L,
                      double* p_n, double* deg_mean, double* deg_var);

/* ---- exact enumeration of tiny discrete models (enumerate.c) ---------- */
int orc_enumerate(int model, const int32_t* data, int64_t n_data, int max_depth,
                  double* values, double* probs, int max_out);
/* customdist (customdist.c): prm = {w1, mu1, s1, mu2, s2, obs_sigma}. */
void orc_customdist_is(const double* prm, const float* y, int64_t n, int64_t N, uint64_t seed,
                       double* x_out, double* lw_out);
void orc_customdist_exact(const double* prm, const float* y, int64_t n, double* out);
void orc_is_discrete(int model, const int32_t* data, int64_t n_data, int64_t N, uint64_t seed,
                     double* values, double* lw);

/* ---- threads for the embarrassingly parallel particle loops ----------- */
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
