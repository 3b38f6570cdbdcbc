/*
 * cf_oracle.h -- plain, slow FP64 CPU oracle for the exact circulant-embedding
 * survey-field sampler of Carron, Wolk & Szapudi (2014), "On fast generation of
 * cosmological random fields".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path (the
 * CUDA library and its Python binding) never links, imports or calls it, and
 * shares no code, header, table or constant generator with it.
 *
 * Every function follows one passage of the paper; the citation is given at the
 * definition in cf_oracle.c.  All floating point is IEEE binary64 unless a
 * function is explicitly the single-precision noise specification.
 *
 * Parity status: every function here is pinned by a CPU test (see the
 * test_oracle_*.py files) against closed forms, brute force or an independent
 * library routine.  Nothing here is "parity unpinned".
 */
#ifndef CF_ORACLE_H
#define CF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based generator (Salmon et al., SC'11, Philox4x32-10) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- own elementary functions used by the noise specification ---- */
double or_log_unit(double u);                 /* ln u, u in (0,1] */
float or_logf_unit(float u);                  /* ln u, u in (0,1], binary32 */
void or_cossin_2pi(double u, double* c, double* s);   /* cos(2 pi u), sin(2 pi u) */
void or_cossin_2pif(float u, float* c, float* s);     /* binary32 */

/* ---- noise: complex standard normal per embedded cell ----
 * dtype 0 = binary64 noise, 1 = binary32 noise (promoted to double on output).
 * out: [R][ncells][2] doubles (re, im). m_last = size of the last embedding
 * axis (needed by the binary32 pairing rule); ncells must be a multiple of it. */
void or_draw_noise(uint64_t seed, uint64_t r0, int32_t R, int64_t ncells,
                   int64_t m_last, int32_t dtype, double* out);

/* ---- 1-D transforms (unnormalised; sign = -1 forward, +1 inverse) ---- */
void or_dft_naive(const double* in, double* out, int64_t n, int sign);  /* interleaved complex */
void or_fft_recursive(double* a, int64_t n, int sign);                  /* n power of two */
/* Axis-by-axis N-D transform of an interleaved complex row-major array. */
void or_fft_nd(double* a, int32_t ndim, const int64_t* dims, int sign);

/* ---- circulant embedding, section 2 ---- */
enum { OR_XI_GAUSSIAN = 0, OR_XI_GEN_CAUCHY = 1, OR_XI_EXPONENTIAL = 2, OR_XI_TABLE = 3 };
typedef struct {
    double lambda_min, lambda_max, tau, neg_mass, cov_error;
    int64_t n_negative, n_zeroed;
    int32_t clamped, status; /* status 0 ok, 2 not positive semi-definite */
} or_embed_report;

/* c: first row of the circulant on the embedded grid M (M_i = 2 n_i for the
 * paper's box of twice the survey side, or any larger even size), lag of
 * index m_i: m_i for 2 m_i < M_i, m_i - M_i otherwise. */
void or_embed_row(int32_t ndim, const int64_t* M, const double* cell, int32_t kind,
                  double amp, double scale, double beta, const double* table, double* c);
/* lambda = unnormalised forward DFT of c (real part). */
void or_eigenvalues(int32_t ndim, const int64_t* M, const double* c, double* lambda);
/* Positivity check, threshold tau = 1e-12 * lambda_max, lambda+ and sqrt(lambda+).
 * clamp != 0 sets negative eigenvalues to zero instead of failing.  When
 * clamped, the realised-covariance error on survey lags is computed. */
void or_psd(int32_t ndim, const int64_t* n, const int64_t* M, const double* c, const double* lambda,
            int32_t clamp, double* lambda_plus, double* sqrt_lambda, or_embed_report* rep);

/* ---- per-realization Gaussian fields, section 2 ----
 * s: sqrt(lambda+) on M^d.  fields: [R][2][N^d] doubles (Re, Im). */
void or_sample(int32_t ndim, const int64_t* n, const int64_t* M, const double* s, uint64_t seed,
               uint64_t r0, int32_t R, int32_t dtype, double* fields);
/* Same map with the complex noise given explicitly: eps [M^d][2] -> W [N^d][2]. */
void or_sample_given_noise(int32_t ndim, const int64_t* n, const int64_t* M, const double* s,
                           const double* eps, double* w);

/* ---- lognormal transform and Poisson sampling, section 3.1 ---- */
double or_poisson_uniform(uint64_t seed, uint64_t cell, uint64_t field);
int32_t or_poisson_icdf(double U, double mu, double* margin);
void or_lognormal_poisson(const double* G, int64_t cells, int64_t nfields, double sigma2,
                          double nbar, const double* f_or_null, uint64_t seed,
                          uint64_t field0, double* delta_out, int32_t* counts_out,
                          double* margin_out);

/* ---- binned power spectrum, section 3.2 ---- */
enum { OR_BINS_LINEAR = 0, OR_BINS_LOG = 1, OR_BINS_EDGES = 2 };
void or_bin_edges(int32_t kind, int32_t nbins, double kmin, double kmax,
                  const double* edges_in, double* edges_out);
void or_power_spectrum(const double* fields, int32_t ndim, const int64_t* n, const double* cell,
                       int64_t nfields, int32_t nbins, const double* edges,
                       double* pk, int64_t* nmodes);
void or_counts_to_delta(const int32_t* counts, const double* f_or_null, int64_t cells,
                        int64_t nfields, double* delta_g);
void or_mean_cov(const double* pk, int64_t nfields, int32_t nbins, double* mean, double* cov);

#ifdef __cplusplus
}
#endif
#endif
