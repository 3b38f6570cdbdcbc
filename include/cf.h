/*
 * cf.h -- C ABI of the GB300 (sm_103a) exact survey-field sampler.
 *
 * Method: Carron, Wolk & Szapudi (2014), "On fast generation of cosmological
 * random fields".  A stationary Gaussian field with covariance xi on a survey
 * grid of n_i cells per axis is sampled exactly by embedding the grid in a
 * periodic grid of M_i = 2 n_i cells (section 2, eq. (grid)), taking the DFT
 * of the embedded correlation row (eq. (Specd)), drawing independent Fourier
 * modes with variance lambda (eq. (Papos2)), inverse transforming and keeping
 * the survey box (closing paragraph of section 2).  Section 3.1 exponentiates
 * the field into a lognormal density and Poisson-samples galaxy counts (eqs.
 * (Lncov), (sampling)); section 3.2 validates with the binned power spectrum
 * (eq. (Def spec)).
 *
 * Conventions shared by every entry point
 *  - Status: every function returns a cf_status; CF_OK on success.  Nothing
 *    throws across the ABI.  cf_last_error() returns a thread-local message
 *    describing the most recent failure on the calling thread.
 *  - Memory: unless stated otherwise, array arguments are DEVICE pointers of
 *    the current CUDA device, owned by the caller; structs passed by pointer
 *    are host memory.  The library owns cf_embedding and cf_server objects.
 *  - Asynchrony: work is enqueued on the caller's stream and returns without
 *    waiting, except cf_embed / cf_embed_from_lambda, which synchronise the
 *    stream to fill the report (once, or twice when the clamped covariance
 *    error is computed).
 *    The first call on a device performs a one-time set-up (twiddle tables)
 *    with a device synchronisation; make it before any stream capture.
 *  - Device: calls run on the device of the stream passed (the legacy
 *    default stream, NULL, means the calling thread's current device).
 *  - Layouts: row-major (C order).  Complex values are interleaved (re, im).
 *    Sampled fields are [R][2][n0][n1][n2]: field 2r is Re and 2r+1 is Im of
 *    realization r0 + r (two independent exact fields per complex draw).
 *  - Sizes: M_i = 2 n_i must be a power of two between 2 and 4096 (8192
 *    cells along one axis at most are not supported: CF_ERR_UNSUPPORTED).
 *  - Randomness: counter-based Philox4x32-10 (Salmon et al., SC'11) keyed by
 *    the 64-bit seed; any realization range [r0, r0+R) is reproducible on its
 *    own.  The realization index r0+R-1 must fit in 32 bits.
 */
#ifndef CF_H
#define CF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CF_API __attribute__((visibility("default")))
#else
#define CF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cf_stream_t; /* == cudaStream_t; NULL = legacy default stream */
typedef struct CUevent_st* cf_event_t;   /* == cudaEvent_t */

typedef enum {
    CF_OK = 0,
    CF_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad enum)  */
    CF_ERR_NOT_PSD = 2,      /* an embedding eigenvalue < -tau and no clamping       */
    CF_ERR_NOMEM = 3,        /* device or host allocation failed / workspace small   */
    CF_ERR_UNSUPPORTED = 4,  /* size or mode not supported by the library or call   */
    CF_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the detail)  */
    CF_ERR_TIMEOUT = 6,      /* cf_serve_wait ran out of time                        */
    CF_ERR_BUSY = 7,         /* server queue full / shutting down                    */
    CF_ERR_NOT_FOUND = 8     /* unknown ticket                                       */
} cf_status;

typedef enum {
    CF_F64 = 0,      /* binary64 noise, transforms and fields                         */
    CF_F32 = 1,      /* binary32 noise, transforms and fields (eigenvalues stay FP64) */
    CF_BF16_TC = 2,  /* binary32 noise; bf16 DFT-matrix tensor-core stages with binary32
                        accumulation; binary32 fields (cf_sample only, 2D, embedded
                        sides 256, 512, 1024, 2048 or 4096) */
    CF_F16_TC = 3    /* as CF_BF16_TC with fp16 stage inputs                               */
} cf_dtype;

/* Survey grid (section 2, eq. (grid)): ndim in {1,2,3}; n[i] survey cells on
 * axis i (unused axes ignored); cell[i] the physical cell side (the L/N of
 * the paper), used for the lag r of xi and the volume of the power spectrum.
 * embed_factor p: the periodic embedding grid has M_i points per axis, the
 * smallest power of two >= p n_i (p = 0 or 2: the paper's box of twice the
 * survey side, exactly 2 n_i when n_i is a power of two; 4 or 8: a larger box,
 * in which every survey-sized sub-box still has the target covariance
 * (section 2, Fig. 1) and whose spectrum is non-negative for more two-point
 * functions, at about (p/2)^d times the work and memory).  Any n_i >= 1 is
 * accepted (M_i <= 4096); the lag of embedded index m_i is m_i for
 * 2 m_i < M_i and m_i - M_i otherwise, and the fields are the first n_i points
 * per axis.  Calls that take fields only (lognormal / Poisson, counts in
 * cells) ignore p; the power spectrum needs power-of-two n_i; the tensor-core
 * modes and cf_embed_periodic need M_i = 2 n_i. */
typedef struct {
    int32_t ndim;
    int32_t embed_factor;
    int64_t n[3];
    double cell[3];
} cf_grid;

typedef enum {
    CF_XI_GAUSSIAN = 0,     /* amp * exp(-r^2 / (2 scale^2))                        */
    CF_XI_GEN_CAUCHY = 1,   /* amp / (1 + (r/scale)^2)^beta                         */
    CF_XI_EXPONENTIAL = 2,  /* amp * exp(-r / scale)                                */
    CF_XI_TABLE = 3         /* caller's embedded first row c, M^d doubles           */
} cf_xi_kind;

/* Two-point function to embed.  For CF_XI_TABLE, table holds the embedded first
 * row c(m) = xi(lag(m)) on the M^d periodic grid, row-major, with lag(m_i) =
 * m_i for m_i < n_i and m_i - M_i otherwise; table_on_device says whether
 * table is a device (1) or host (0) pointer.  Other kinds ignore table. */
typedef struct {
    int32_t kind;
    int32_t table_on_device;
    double amp;
    double scale;
    double beta;
    const double* table;
} cf_xi;

/* cf_embed flags */
#define CF_EMBED_CLAMP 1u        /* set eigenvalues < -tau to zero instead of failing */
#define CF_EMBED_SKIP_ERROR 2u   /* with CF_EMBED_CLAMP: skip the covariance-error pass */
#define CF_EMBED_DF 8u           /* parametric xi: the transforms of the eigenvalues and of
                                    the covariance-error pass run in double-float arithmetic
                                    (pairs of binary32, about 48 bits): eigenvalues within
                                    about 1e-14 lambda_max of binary64 ones (inside the 1e-12
                                    tolerance), several times faster on this GPU, whose
                                    binary64 rate is low.  For binary32 and lower-precision
                                    fields; binary64 fields want the default binary64
                                    transforms (their tolerance is 1e-10 on the fields) */
#define CF_EMBED_LOG1P 4u        /* xi is the correlation function of the lognormal
                                    density delta; the Gaussian covariance embedded is
                                    ln(1 + xi) (section 3.1, eq. (Lncov)).  xi must stay
                                    above -1 (a table entry <= -1 gives CF_ERR_NOT_PSD);
                                    the lognormal variance is then sigma^2 = ln(1 + xi(0)).
                                    Not accepted by the serving loop (its cache scales
                                    amplitudes linearly). */

/* Outcome of the positivity check (section 2, eq. (condition)).
 * tau = 1e-12 lambda_max.  Eigenvalues in [-tau, tau] are set to zero (n_zeroed);
 * eigenvalues below -tau are "negative" (n_negative, neg_mass = sum of |lambda|).
 * exact = 1 when no eigenvalue was clamped: the realised covariance then equals
 * xi on every survey lag to within tau.  When clamped, cov_error is the largest
 * |IDFT(lambda+)/M^d - c| over survey lags (the realised covariance error). */
typedef struct {
    double lambda_min;
    double lambda_max;
    double tau;
    double neg_mass;
    double cov_error;
    int64_t n_negative;
    int64_t n_zeroed;
    int32_t clamped;
    int32_t exact;
} cf_embed_report;

typedef struct cf_embedding cf_embedding;

/* Steps a1-a3 (section 2, eqs. (grid), (Specd), (condition)): builds the
 * embedded row c on the device, computes lambda = DFT(c) in binary64 (the cell
 * volume of eq. (Specd) is absorbed: lambda_k = sum_m c_m e^{-2 pi i k.m/M}),
 * checks positivity, and keeps lambda, sqrt(lambda+) on the device.
 * Synchronises stream s once to fill *rep (may be NULL).  On CF_ERR_NOT_PSD
 * *out is NULL and *rep still describes the spectrum. */
CF_API cf_status cf_embed(const cf_grid* g, const cf_xi* xi, uint32_t flags, cf_stream_t s,
                   cf_embedding** out, cf_embed_report* rep);

/* As cf_embed, with the spectrum lambda (M^d doubles, device) given instead of
 * xi (e.g. the periodic-box spectrum of section 3.3, eq. (Periodicboxmodes)).
 * The covariance-error pass compares against IDFT(lambda) itself. */
CF_API cf_status cf_embed_from_lambda(const cf_grid* g, const double* lambda, uint32_t flags,
                               cf_stream_t s, cf_embedding** out, cf_embed_report* rep);

/* k-space (periodic box) sampler of section 3.3, eq. (Periodicboxmodes): the
 * survey grid g (n per axis) is observed inside a periodic box of side
 * B = box_factor * n (1, 2 or 4) whose modes k = 2 pi m / (B cell) have
 * variance P(k) / cell^d, P the continuous Fourier transform of xi (of
 * ln(1 + xi) with CF_EMBED_LOG1P), and the DC mode is zero.  P is the Fourier
 * sum of xi on a grid of spacing cell / resolution over resolution * extent * B
 * points per axis (both 1..16, powers of two; the product must stay <= 4096):
 * aliasing sits at k = 2 pi resolution / cell and xi is truncated at
 * |r| = extent B cell / 2.  The returned embedding samples like cf_embed's:
 * cf_sample gives fields of n per axis for box_factor 1 and 2 and of 2n for
 * box_factor 4 (the survey is then the first n per axis).  No covariance-error
 * pass (the target is the periodised covariance).  Parametric xi only. */
CF_API cf_status cf_embed_periodic(const cf_grid* g, const cf_xi* xi, int32_t box_factor, int32_t extent,
                                   int32_t resolution, uint32_t flags, cf_stream_t s, cf_embedding** out,
                                   cf_embed_report* report);

/* Frees an embedding without waiting on the host: the memory is released on
 * a library-owned stream after the last work that any library call enqueued
 * on it (on any stream) has finished. */
CF_API cf_status cf_embedding_free(cf_embedding* e);

/* Copies of the embedding's arrays into caller device memory (M^d doubles),
 * enqueued on s: the raw eigenvalues lambda and sqrt(lambda+). */
CF_API cf_status cf_embedding_lambda(const cf_embedding* e, double* dst, cf_stream_t s);
CF_API cf_status cf_embedding_sqrt_lambda(const cf_embedding* e, double* dst, cf_stream_t s);
/* Grid and report of an embedding (host structs). */
CF_API cf_status cf_embedding_info(const cf_embedding* e, cf_grid* g, cf_embed_report* rep);

/* Step b1 alone (section 2, eq. (Papos2): independent zero-mean Gaussian
 * modes).  Writes the complex standard-normal noise of cells [0, ncells) of
 * realizations [r0, r0+R) to out: [R][ncells] complex of dtype dt (float2 or
 * double2).  m_last is the size of the last embedding axis (the binary32
 * specification pairs column c with c + m_last/2); ncells must be a multiple
 * of m_last.  Bit-exact reference for the noise fused into cf_sample. */
CF_API cf_status cf_draw_noise(uint64_t seed, uint64_t r0, int32_t R, int64_t ncells, int64_t m_last,
                        cf_dtype dt, void* out, cf_stream_t s);

/* Self-check of the binary32 noise arithmetic (section 2, eq. (Papos2): the
 * draws are the specification's only if every operation rounds as it
 * specifies).  The noise kernels form the logarithm's quotient
 * (m - 1) / (m + 1) and the Box-Muller square root with short sequences; this
 * call compares them with the IEEE correctly rounded quotient and square root
 * over every binary32 input of their domains (m from sqrt(1/2) to sqrt(2):
 * 8.4 M inputs; x = +-0 and x from 2^-24 to 34: 0.24 G inputs) on the current
 * device, synchronously.  mismatches (host, 2 entries): quotient, square root
 * (both 0: the draws are the specification's).  examples (host, 2 entries,
 * may be NULL): the bit pattern of the first mismatching m and x found (0
 * where none).  Allocates 24 bytes of device memory for the call. */
CF_API cf_status cf_noise_selfcheck(uint64_t* mismatches, uint32_t* examples);

/* Workspace (bytes, device) that cf_sample / cf_sample_lp need for R
 * realizations; realizations are processed in chunks whose intermediate
 * fits 1 GiB (or the chunk cf_tune_sample recorded for this grid), so the size
 * saturates for large R. */
CF_API cf_status cf_sample_workspace_size(const cf_embedding* e, int32_t R, cf_dtype dt, size_t* bytes);

/* Steps b1-b4 (section 2, eq. (Papos2) and the closing paragraph): for each
 * realization r in [r0, r0+R), draws eps_k (Philox stream 0), scales it by
 * sqrt(lambda+_k), computes W_m = M^{-d/2} sum_k sqrt(lambda_k) eps_k
 * e^{+2 pi i k.m/M} for survey cells m (pruned axis-by-axis inverse FFT), and
 * writes fields_out [R][2][n...] (float for CF_F32, double for CF_F64):
 * Re W then Im W.  ws: device workspace of at least cf_sample_workspace_size
 * bytes (fewer bytes -> smaller chunks; below one realization -> CF_ERR_NOMEM). */
CF_API cf_status cf_sample(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, cf_dtype dt,
                    void* fields_out, void* ws, size_t ws_bytes, cf_stream_t s);

/* cf_sample (binary32) without a caller workspace.  The paper has no
 * counterpart: this entry exists for callers that cannot allocate device
 * memory where they sample -- code running while another thread captures a
 * CUDA graph in global capture mode, where cudaMalloc is an error, and
 * programs whose device memory is fixed up front by a budget or another
 * allocator.  They pass the embedding and fields_out ([R][2][n...] float) as
 * for cf_sample; the intermediate lives in a 16 MiB array inside the library
 * that every device loading the library holds until the process exits.
 *  - Sizes whose single realization needs more than 16 MiB of intermediate
 *    (e.g. 2D surveys above 1024x1024, 3D above 64^3) are rejected with
 *    CF_ERR_UNSUPPORTED and a message giving the bytes needed.  An embedding
 *    built on another device than s's is rejected with CF_ERR_ARG.
 *  - Nothing is allocated on the device: no cudaMalloc, cudaFree or allocator
 *    call.  The first call on a device does a one-time set-up (the array's
 *    device address, an ordering event, the twiddle tables) that synchronises
 *    the device: make it before any stream capture.  The first use of an
 *    embedding on a stream other than the one it was built on creates one
 *    CUDA event (host-side object) so that cf_embedding_free can wait for the
 *    work.
 *  - While another thread captures in global mode, s must be a stream created
 *    with cudaStreamNonBlocking: work on the legacy default stream (s = NULL,
 *    or a default stream of a framework that maps to it) synchronises with
 *    every other stream and invalidates that capture.
 *  - All calls share the array, which keeps the last call's contents; every
 *    element a call reads it has written first, so nothing needs clearing.
 *    The library orders successive direct calls on a device (host lock +
 *    device event); calls whose work nevertheless overlaps on the GPU race on
 *    the array. */
CF_API cf_status cf_sample_noalloc(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R,
                                   void* fields_out, cf_stream_t s);

/* Autotuner of the sampler's schedule.  Times cf_sample on R realizations of
 * e for each candidate chunk that fits ws_bytes (realizations per launch of
 * the transform passes: 1, 2, 4, ... up to R), then, in binary32 on grids
 * with a side of 256 or more, each of the 3 CTA shapes of the row pass
 * (and of the paired column pass, where it is enabled) at the best
 * chunk, writing into fields_scratch
 * ([R][2][n...] of dt), and records the fastest for this device, grid shape
 * and dtype (on small binary32 grids also the persistent single launch);
 * later cf_sample / cf_sample_lp / cf_sample_workspace_size calls and served
 * batches with that shape use it (cf_tune_info reads it).
 * Synchronises s.  *chunk_out (may be NULL) receives the chosen chunk,
 * *ms_out (may be NULL) its time per realization. */
CF_API cf_status cf_tune_sample(const cf_embedding* e, cf_dtype dt, int32_t R, void* ws, size_t ws_bytes,
                                void* fields_scratch, cf_stream_t s, int32_t* chunk_out, double* ms_out);

/* The sampler schedule recorded for e's grid and dt on the current device:
 * realizations per launch (0: the default, chunks of up to 1 GiB of
 * intermediate), the CTA shapes (0, 1, 2; 0 the default) of the binary32
 * row pass (rows of 256 or 1024 points: 8, 4 or 16 warps per block; other
 * rows: 128, 256 or 512 threads) and of the paired column pass (where it is
 * enabled), and whether each chunk runs as one
 * persistent cooperative launch (1; binary32 grids whose embedded sides are
 * all 64 or 128, else CF_ERR_UNSUPPORTED) instead of one launch per pass (0).
 * cf_tune_sample records the fastest; cf_tune_set records a given one (all
 * zero clears the record).  No schedule changes a result bit.  Output
 * pointers may be NULL. */
CF_API cf_status cf_tune_info(const cf_embedding* e, cf_dtype dt, int32_t* chunk, int32_t* rows_shape,
                              int32_t* cols_shape, int32_t* persistent);
CF_API cf_status cf_tune_set(const cf_embedding* e, cf_dtype dt, int32_t chunk, int32_t rows_shape,
                             int32_t cols_shape, int32_t persistent);

/* Tensor-core modes: number of tensor-core waits that ran out of time (1 s
 * each) on the current device since the last call; synchronises s and
 * resets the count.  A non-zero count means the affected fields are invalid. */
CF_API cf_status cf_tc_faults(cf_stream_t s, uint32_t* count);

/* ---------------------------------------------------------------- counts in cells
 * Section 3.4.  Counts are int32 maps [nfields][cells]; f is the surface
 * fraction [cells] (NULL: f = 1); cells with f = 0 are ignored.  All device
 * pointers, asynchronous on s. */

/* Histogram P(N) = #{i : f_i != 0, N_i = N} for N < nbins (larger counts are
 * not binned) of every map: hist_out [nfields][nbins] (binary64 holding
 * integers); optionally its mean [nbins] and unbiased covariance
 * [nbins][nbins] over the maps.  nbins <= 1024, nfields <= 65535. */
CF_API cf_status cf_cic_histogram(const int32_t* counts, int64_t cells, int64_t nfields, const float* f,
                                  int32_t nbins, double* hist_out, double* mean_or_null, double* cov_or_null,
                                  cf_stream_t s);

/* Mean histogram of the Poisson-lognormal model, section 3.4:
 * <P(N)> = int dA N(A; -sigma2_A/2, sigma2_A) sum_{f_i != 0} Poisson(N; nbar f_i e^A),
 * N < nbins <= 64, by a 512-node trapezoid rule over +-10 standard deviations
 * (pred_out [nbins], binary64). */
CF_API cf_status cf_cic_prediction(double sigma2_A, double nbar, const float* f, int64_t cells, int32_t nbins,
                                   double* pred_out, cf_stream_t s);

/* The non-linear transform of eq. (As): out = A*, the root of
 * exp(A) nbar_i sigma2_A + A = sigma2_A (N - 1/2), nbar_i = nbar f_i, per cell
 * of every map (binary32 out [nfields][cells]; 0 where f = 0). */
CF_API cf_status cf_astar(const int32_t* counts, const float* f, int64_t cells, int64_t nfields, double nbar,
                          double sigma2_A, float* out, cf_stream_t s);

/* Copies the first g_out->n[a] cells of every axis of each of nfields fields
 * laid out on g_in (e.g. the survey corner of a box-sampled field); binary32
 * or binary64, device pointers. */
CF_API cf_status cf_copy_corner(const void* in, cf_dtype dt, const cf_grid* g_in, const cf_grid* g_out,
                                int64_t nfields, void* out, cf_stream_t s);

/* Mean over rows [ncols] and unbiased covariance (1/(nrows - 1)) [ncols][ncols]
 * of x [nrows][ncols] (binary64, device); either output may be NULL.  The
 * estimator used by cf_power_spectrum and cf_cic_histogram, for spectra
 * gathered over several calls. */
CF_API cf_status cf_mean_cov(const double* x, int64_t nrows, int32_t ncols, double* mean_or_null,
                             double* cov_or_null, cf_stream_t s);

/* Cumulative information of section 3.3, eq. (cuminfo), from the mean [nbins]
 * and covariance [nbins][nbins] of binned power spectra (cf_power_spectrum):
 * info_out[b] = sum_{b1, b2 <= b} [C^{-1}]_{b1 b2} over the bins up to b, with
 * C_{12} = cov_{12} / (mean_1 mean_2).  Bins with mean <= 0 are left out (their
 * entry repeats the previous one); from a bin whose pivot is not positive
 * (too few fields for the number of bins) on, the entries are NaN.
 * ws: device scratch of 8 (nbins^2 + nbins) + 4 nbins bytes; nbins <= 4096. */
CF_API cf_status cf_cumulative_information(const double* mean, const double* cov, int32_t nbins, double* info_out,
                                           void* ws, size_t ws_bytes, cf_stream_t s);

/* Lognormal + Poisson parameters (section 3.1, eqs. (Lncov), (sampling)). */
typedef struct {
    double sigma2;          /* variance of G: rho = exp(G - sigma2/2), delta = rho - 1 */
    double nbar;            /* Poisson intensity of a cell with f = 1                 */
    const float* f;         /* device [cells] unmasked fraction f_i, or NULL (f = 1)  */
    uint64_t seed;          /* key of Philox stream 1 (the Poisson uniforms)          */
    float* delta_out;       /* device [nfields][cells] or NULL                        */
    int32_t* counts_out;    /* device [nfields][cells], required                      */
} cf_lp_params;

/* cf_sample with steps c1-c2 fused into the last inverse-FFT pass: writes the
 * fields (if fields_out is not NULL) and the lognormal delta / Poisson counts
 * of every field, with field index 2(r0+r) + {0,1}.  Binary32 only. */
CF_API cf_status cf_sample_lp(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, cf_dtype dt,
                       void* fields_out, const cf_lp_params* lp, void* ws, size_t ws_bytes,
                       cf_stream_t s);

/* Steps c1-c2 standalone (section 3.1): for fields j in [0, nfields) with
 * global index field0 + j and cells i in [0, cells_per_field):
 *   rho = exp(G - sigma2/2); delta = rho - 1; mu = nbar f_i rho;
 *   count = min{ k >= 0 : U < F(k; mu) }, F the Poisson CDF, U in [0,1) from
 *   Philox key seed, counter (i_lo, i_hi, (field0+j) >> 1, 1), words (0,1) for
 *   even and (2,3) for odd fields, U = ((a>>5) 2^26 + (b>>6)) 2^-53.
 * G: [nfields][cells] of dtype dt; f_or_null: [cells] float or NULL;
 * delta_out_or_null: [nfields][cells] float; counts_out: [nfields][cells] int32. */
CF_API cf_status cf_lognormal_poisson(const void* G, cf_dtype dt, int64_t cells_per_field,
                               int64_t nfields, double sigma2, double nbar,
                               const float* f_or_null, uint64_t seed, uint64_t field0,
                               float* delta_out_or_null, int32_t* counts_out, cf_stream_t s);

typedef enum { CF_BINS_LINEAR = 0, CF_BINS_LOG = 1, CF_BINS_EDGES = 2 } cf_bins_kind;

/* Bins of the mode length |k| in units of the fundamental frequency 2 pi/L_ref
 * of the longest side L_ref = max_i n_i cell_i: q = sqrt(sum_i (s_i r_i)^2),
 * s_i in (-n_i/2, n_i/2] the signed mode index and r_i = L_ref/(n_i cell_i),
 * each operation rounded in binary64 in this order (on a cube r_i = 1 and q is
 * the index length sqrt(sum_i s_i^2)).  Bin b is [e_b, e_{b+1}).  LINEAR:
 * e_b = kmin + b (kmax - kmin)/nbins; LOG: e_b = kmin exp(b ln(kmax/kmin)/nbins)
 * (the paper's 20 ln-spaced bins); EDGES: host array edges[nbins+1],
 * increasing.  kmax <= 0 means the smallest axis Nyquist frequency in these
 * units, min_i n_i r_i / 2 (n/2 on a cube).  The DC mode is never binned. */
typedef struct {
    int32_t nbins;
    int32_t kind;
    double kmin;
    double kmax;
    const double* edges;
} cf_bins;

/* Workspace bytes for cf_power_spectrum / cf_power_spectrum_counts. */
CF_API cf_status cf_power_spectrum_workspace_size(const cf_grid* g, int64_t nfields, const cf_bins* b,
                                           cf_dtype dt, size_t* bytes);

/* Step d1 (section 3.2, eq. (Def spec)): for each real field phi of fields
 * [nfields][n...] (float for CF_F32, double for CF_F64):
 *   pk_out[f][b] = cell^d / (prod n_i * N_b) * sum_{|n| in bin b} |DFT(phi)_n|^2
 * over all modes of the full grid (both +n and -n); nmodes_out[b] = N_b
 * (int64).  Any box of 1 to 3 dimensions: sides up to 4096
 * (powers of two) or 2048 (other lengths, through Bluestein transforms),
 * rectangular and with unequal cells (cubes with power-of-two sides take a
 * faster path with the same results).  If mean_or_null / cov_or_null are
 * given, the mean over fields [nbins] and the unbiased (1/(F-1)) covariance
 * [nbins][nbins] are written too (section 3.2, "prediction and covariance from
 * a very large number of simulations").  Outputs are device doubles/int64. */
CF_API cf_status cf_power_spectrum(const void* fields, cf_dtype dt, const cf_grid* g, int64_t nfields,
                            const cf_bins* bins, double* pk_out, int64_t* nmodes_out,
                            double* mean_or_null, double* cov_or_null, void* ws,
                            size_t ws_bytes, cf_stream_t s);

/* Step d1 on count maps (section 3.2, eq. (Estim) and the map before it):
 * each count field N [nfields][n...] (int32) becomes
 * delta_g = (N/f - Nhat)/Nhat where f != 0 (0 elsewhere), Nhat = N_tot / sum f,
 * and its spectrum is computed as in cf_power_spectrum (binary32 transforms). */
CF_API cf_status cf_power_spectrum_counts(const int32_t* counts, const float* f_or_null, const cf_grid* g,
                                   int64_t nfields, const cf_bins* bins, double* pk_out,
                                   int64_t* nmodes_out, double* mean_or_null, double* cov_or_null,
                                   void* ws, size_t ws_bytes, cf_stream_t s);

/* cf_sample (binary32) or cf_sample_lp (lp non-NULL) followed by
 * cf_power_spectrum of the 2R fields, with the sampler's last pass fused with
 * the first axis of the spectra (sections 2 and 3.2): the column pass keeps
 * each cropped column in shared memory and transforms it forward, so the
 * fields are not read back for their spectra.  Square 2D grids only (n0 = n1
 * = n, 128 <= n <= 2048, equal cell sides, embed_factor 2), R <= 32767.  Same outputs as the
 * separate calls: fields and counts identical, spectra equal up to rounding
 * (another order of the transform's axes).  ws / ws_bytes: the sampler
 * workspace (cf_sample_workspace_size); pk_ws: pk_ws_bytes >=
 * cf_sample_spectra_workspace_size(e, R, bins) bytes of device memory for the
 * half spectra and accumulators.  The count maps' spectra, if wanted, come
 * from cf_power_spectrum_counts on lp->counts_out; sampled_or_null, if given,
 * is recorded on s once the fields and counts are complete and before the
 * spectra, so that work on another stream may start from them.  Errors:
 * CF_ERR_UNSUPPORTED for other grids, CF_ERR_NOMEM for a short workspace, else
 * as the separate calls. */
CF_API cf_status cf_sample_spectra_workspace_size(const cf_embedding* e, int32_t R, const cf_bins* bins,
                                                  size_t* pk_ws_bytes);
CF_API cf_status cf_sample_spectra(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, float* fields_out,
                                   const cf_lp_params* lp_or_null, const cf_bins* bins, double* pk_out,
                                   int64_t* nmodes_out, double* mean_or_null, double* cov_or_null, void* ws,
                                   size_t ws_bytes, void* pk_ws, size_t pk_ws_bytes, cf_event_t sampled_or_null,
                                   cf_stream_t s);

/* ---------------------------------------------------------------- plans
 * The binary32 per-realization path of one embedding recorded once as a CUDA
 * graph: R realizations drawn with `seed` (cf_sample's noise), the optional
 * lognormal + Poisson step (lp: sigma2, nbar, seed, counts_out; no mask, no
 * delta output) and, with bins, the power spectra of the 2R fields
 * (pk_out [2R][nbins], nmodes_out, optional mean/cov) and of the count maps
 * (pk_counts_out and its optional mean/cov; needs lp).  Each cf_plan_launch
 * replays the graph on s and draws the next R realizations: launch k after
 * creation (or after cf_plan_seek(r0)) covers [r0 + kR, r0 + (k+1)R), with
 * results identical to cf_sample_lp / cf_power_spectrum on that range.  The
 * realization counter lives on the device and advances inside the graph.
 * The plan owns its workspaces; all output arrays are the caller's and must
 * outlive the plan.  cf_plan_create synchronises s (one eager pass fills the
 * library's caches before the capture). */
typedef struct cf_plan cf_plan;
CF_API cf_status cf_plan_create(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R,
                                const cf_lp_params* lp_or_null, const cf_bins* bins_or_null, float* fields_out,
                                double* pk_out, int64_t* nmodes_out, double* mean_or_null, double* cov_or_null,
                                double* pk_counts_out, double* mean_counts_or_null, double* cov_counts_or_null,
                                cf_stream_t s, cf_plan** out);
CF_API cf_status cf_plan_launch(cf_plan* p, cf_stream_t s);
/* Next launch starts at realization r0; synchronises s. */
CF_API cf_status cf_plan_seek(cf_plan* p, uint64_t r0, cf_stream_t s);
CF_API cf_status cf_plan_destroy(cf_plan* p);


/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching (not in the paper; it
 * serves the paper's sampler, sections 2 and 3.1, to many clients).
 *
 * A server owns one device.  Requests (grid, xi, realization range, optional
 * lognormal + Poisson step) are queued by cf_serve_submit and run by a worker
 * thread: requests are admitted while a slot (stream) is free and their
 * device memory fits the HBM budget; queued requests of the same grid shape
 * are batched into one launch (even with different xi or seeds); the
 * eigenvalues of each spectrum are kept on the device (LRU cache keyed by
 * grid, family, scale, beta and flags -- the amplitude is applied as
 * sqrt(amp) at sampling, since lambda is linear in amp).  Results stay in
 * server-owned device memory until cf_serve_release; optionally they are also
 * copied to host memory (pinned memory keeps the worker from blocking).
 * Binary32 fields only; the Poisson step uses f = 1 (no survey mask).
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t device;                  /* CUDA device index                                  */
    int32_t max_inflight;            /* concurrent batches (streams), >= 1                 */
    int32_t queue_capacity;          /* queued requests before submit returns CF_ERR_BUSY  */
    int32_t cache_entries;           /* embeddings kept on the device                      */
    int32_t max_batch_realizations;  /* realizations per batched launch (and per request)  */
    int32_t small_request_cells;     /* > 0: one more slot, on a stream of the highest
                                        priority, reserved for requests of at most this many
                                        output cells (2 R prod n), so that they need not wait
                                        behind large batches; 0: none                       */
    size_t hbm_budget;               /* bytes: cached embeddings + in-flight + unreleased results */
} cf_serve_cfg;

typedef struct {
    cf_grid grid;
    cf_xi xi;                        /* CF_XI_GAUSSIAN / GEN_CAUCHY / EXPONENTIAL          */
    uint32_t embed_flags;            /* CF_EMBED_CLAMP etc.                                */
    int32_t want_counts;             /* 1: also lognormal + Poisson counts                 */
    uint64_t seed;                   /* noise seed                                         */
    uint64_t r0;                     /* first realization                                  */
    int32_t R;                       /* realizations (two fields each)                     */
    int32_t pad_;
    double sigma2, nbar;             /* lognormal / Poisson parameters (want_counts)       */
    uint64_t lp_seed;                /* Poisson seed                                       */
    float* host_fields;              /* optional host copy [R][2][n...] float              */
    int32_t* host_counts;            /* optional host copy [R][2][n...] int32              */
} cf_request;

typedef struct {
    cf_status status;                /* CF_OK, CF_ERR_NOT_PSD, CF_ERR_NOMEM, ...           */
    int32_t cache_hit;               /* embedding served from the cache                    */
    double queue_ms, run_ms, latency_ms;  /* submit->start, start->done, submit->done    */
    const float* dev_fields;         /* server-owned device results, valid until release   */
    const int32_t* dev_counts;
    cf_embed_report embed;           /* report of the request's spectrum (at its amp)      */
} cf_result;

typedef struct {
    uint64_t submitted, completed, failed, rejected;
    int64_t queued, inflight;
    uint64_t cache_hits, cache_misses, cache_evictions;
    uint64_t batches, batched_requests, realizations;
    size_t bytes_in_use, bytes_peak, budget;
    double p50_ms, p99_ms, mean_ms;  /* submit->done latency over completed requests       */
    double realizations_per_s;       /* completed realizations / (last done - first submit) */
} cf_serve_statistics;

typedef struct cf_server cf_server;

/* Starts a server (worker thread, streams) on cfg->device. */
CF_API cf_status cf_serve_create(const cf_serve_cfg* cfg, cf_server** out);
/* Queues a request; *ticket identifies it.  CF_ERR_ARG for an invalid
 * request, CF_ERR_BUSY when the queue is full. */
CF_API cf_status cf_serve_submit(cf_server* sv, const cf_request* req, uint64_t* ticket);
/* CF_OK and *res when the request has finished (res->status is its
 * outcome); CF_ERR_BUSY while it is queued or running; CF_ERR_NOT_FOUND for
 * an unknown or released ticket. */
CF_API cf_status cf_serve_poll(cf_server* sv, uint64_t ticket, cf_result* res);
/* As cf_serve_poll, waiting up to timeout_us microseconds (< 0: no limit);
 * CF_ERR_TIMEOUT if it has not finished by then. */
CF_API cf_status cf_serve_wait(cf_server* sv, uint64_t ticket, int64_t timeout_us, cf_result* res);
/* Frees a finished request's device results (and forgets the ticket). */
CF_API cf_status cf_serve_release(cf_server* sv, uint64_t ticket);
CF_API cf_status cf_serve_stats(cf_server* sv, cf_serve_statistics* st);
/* Stops the worker after the running batches finish; queued requests end
 * with CF_ERR_BUSY; frees everything. */
CF_API cf_status cf_serve_destroy(cf_server* sv);

/* Kernel timing (tracing).  cf_kernel_timing(1) clears the accumulators and
 * makes every subsequent library launch record a CUDA event pair on its own
 * stream; cf_kernel_timing(0) stops recording.  cf_kernel_timing_read waits
 * for the recorded events and writes a JSON object
 * {"<kernel>": [launches, total_ms], ...} into json (capacity cap bytes,
 * NUL-terminated); *needed receives the full length.  Timing adds one event
 * pair per launch; leave it off outside measurements. */
CF_API cf_status cf_kernel_timing(int32_t enable);
CF_API cf_status cf_kernel_timing_read(char* json, size_t cap, size_t* needed);

/* Thread-local description of the last error on this thread ("" if none). */
CF_API const char* cf_last_error(void);
/* Library version string. */
CF_API const char* cf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CF_H */
