// cf_cic.cu -- counts in cells (section 3.4): the histogram P(N) of each
// count map over the unmasked cells, the mean of that histogram predicted by
// the Poisson-lognormal mixture, and the non-linear transform A*(N) of
// eq. (As).
#include <math.h>

#include "cf_kernels.cuh"

namespace cf {
namespace {

constexpr int kHistMaxBins = 1024;
constexpr int kPredMaxBins = 64;
constexpr int kPredNodes = 512;   // trapezoid nodes over A in [-s^2/2 - 10 s, -s^2/2 + 10 s]

// P(N) = number of cells with f != 0 holding N counts, N < nbins; one block
// row per field, shared-memory bins, one atomic per bin and block.
__global__ void __launch_bounds__(256) k_cic_hist(const int32_t* __restrict__ counts, long long cells,
                                                  const float* __restrict__ f, int nbins, double* __restrict__ hist) {
    __shared__ unsigned int sh[kHistMaxBins];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int32_t* c = counts + (size_t)blockIdx.y * cells;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells;
         i += (long long)gridDim.x * blockDim.x) {
        if (f && f[i] == 0.0f) continue;
        const int32_t n = c[i];
        if (n >= 0 && n < nbins) atomicAdd(&sh[n], 1u);
    }
    __syncthreads();
    double* h = hist + (size_t)blockIdx.y * nbins;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (sh[b]) atomicAdd(&h[b], (double)sh[b]);
}

// <P(N)> = int dA N(A; -s2/2, s2) sum_{f_i != 0} Poisson(N; nbar f_i e^A)
// (the mixture of section 3.4 written with the Poisson probability), by the
// trapezoid rule in A; the Poisson probabilities by the recurrence
// p_{N+1} = p_N mu / (N + 1).  Nodes whose mu exceeds 600 are skipped: there
// Poisson(N; mu) < e^-300 for every N < 64.
__global__ void __launch_bounds__(256) k_cic_pred(const float* __restrict__ f, long long cells, double nbar,
                                                  double s2, int nbins, double* __restrict__ out) {
    double acc[kPredMaxBins];
#pragma unroll
    for (int N = 0; N < kPredMaxBins; ++N) acc[N] = 0.0;
    const double sd = sqrt(s2);
    const double a0 = -0.5 * s2 - 10.0 * sd;
    const double h = 20.0 * sd / (double)(kPredNodes - 1);
    const double norm = h / (sd * sqrt(2.0 * M_PI));
    const long long total = cells * kPredNodes;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / kPredNodes;
        const int q = (int)(t % kPredNodes);
        const double fi = f ? (double)f[i] : 1.0;
        if (fi == 0.0) continue;
        const double A = a0 + h * (double)q;
        const double mu = nbar * fi * exp(A);
        if (mu > 600.0) continue;
        const double z = (A + 0.5 * s2) / sd;
        double p = (q == 0 || q == kPredNodes - 1 ? 0.5 : 1.0) * norm * exp(-0.5 * z * z - mu);
#pragma unroll
        for (int N = 0; N < kPredMaxBins; ++N) {
            acc[N] += p;
            p *= mu / (double)(N + 1);
        }
    }
    __shared__ double red[256 / 32][kPredMaxBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int N = 0; N < kPredMaxBins; ++N) {
        double v = acc[N];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][N] = v;
    }
    __syncthreads();
    for (int N = threadIdx.x; N < nbins; N += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < 256 / 32; ++w) v += red[w][N];
        atomicAdd(&out[N], v);
    }
}

// A*(N) of eq. (As): the root of g(A) = nbar_i s2 e^A + A - s2 (N - 1/2),
// nbar_i = nbar f_i.  g is increasing and convex, so Newton's iteration
// converges from any start (from the left it first overshoots to the right);
// the start is the Lambert-W form A = c - W(k e^c), c = s2 (N - 1/2),
// k = nbar_i s2, with W estimated from ln(k e^c).  Masked cells (f = 0) get 0.
__global__ void k_astar(const int32_t* __restrict__ counts, const float* __restrict__ f, long long cells,
                        long long total, double nbar, double s2, float* __restrict__ out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long cell = idx % cells;
        const double fi = f ? (double)f[cell] : 1.0;
        if (fi == 0.0) {
            out[idx] = 0.0f;
            continue;
        }
        const double c = s2 * ((double)counts[idx] - 0.5);
        const double k = nbar * fi * s2;
        const double lx = log(k) + c;
        double w;
        if (lx < 1.0) {
            const double x = exp(lx);
            w = x / (1.0 + x);
        } else {
            const double l2 = log(lx);
            w = lx - l2 + l2 / lx;
        }
        double A = c - w;
        for (int it = 0; it < 60; ++it) {
            const double e = k * exp(A);
            const double step = (e + A - c) / (e + 1.0);
            A -= step;
            if (fabs(step) <= 1e-15 * (1.0 + fabs(A))) break;
        }
        out[idx] = (float)A;
    }
}

}  // namespace
}  // namespace cf

using namespace cf;

extern "C" cf_status cf_cic_histogram(const int32_t* counts, int64_t cells, int64_t nfields, const float* f,
                                      int32_t nbins, double* hist_out, double* mean, double* cov, cf_stream_t s) {
    clear_error();
    if (!counts || !hist_out) return fail(CF_ERR_ARG, "counts and hist_out are required");
    if (cells < 1 || nfields < 1) return fail(CF_ERR_ARG, "cells and nfields must be >= 1");
    if (nbins < 1 || nbins > kHistMaxBins) return fail(CF_ERR_ARG, "nbins must be in [1, %d]", kHistMaxBins);
    if (nfields > 65535) return fail(CF_ERR_UNSUPPORTED, "at most 65535 fields per call");
    CF_TRY(enter((cudaStream_t)s));
    const cudaStream_t st = (cudaStream_t)s;
    CF_CUDA(cudaMemsetAsync(hist_out, 0, sizeof(double) * (size_t)nfields * nbins, st));
    {
        ScopedKernelTimer kt(st, "cic_hist");
        const int bx = grid_blocks(cells, 256, 152 * 8);
        k_cic_hist<<<dim3((unsigned)bx, (unsigned)nfields), 256, 0, st>>>(counts, cells, f, nbins, hist_out);
        CF_CHECK_LAUNCH();
    }
    return launch_mean_cov(hist_out, nfields, nbins, mean, cov, st);
}

extern "C" cf_status cf_cic_prediction(double sigma2_A, double nbar, const float* f, int64_t cells, int32_t nbins,
                                       double* pred_out, cf_stream_t s) {
    clear_error();
    if (!pred_out) return fail(CF_ERR_ARG, "pred_out is NULL");
    if (!(sigma2_A > 0.0) || !(nbar >= 0.0)) return fail(CF_ERR_ARG, "sigma2_A > 0 and nbar >= 0 required");
    if (cells < 1) return fail(CF_ERR_ARG, "cells must be >= 1");
    if (nbins < 1 || nbins > kPredMaxBins) return fail(CF_ERR_ARG, "nbins must be in [1, %d]", kPredMaxBins);
    CF_TRY(enter((cudaStream_t)s));
    const cudaStream_t st = (cudaStream_t)s;
    CF_CUDA(cudaMemsetAsync(pred_out, 0, sizeof(double) * (size_t)nbins, st));
    ScopedKernelTimer kt(st, "cic_prediction");
    k_cic_pred<<<grid_blocks(cells * kPredNodes, 256, 152 * 4), 256, 0, st>>>(f, cells, nbar, sigma2_A, nbins,
                                                                               pred_out);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

extern "C" cf_status cf_astar(const int32_t* counts, const float* f, int64_t cells, int64_t nfields, double nbar,
                              double sigma2_A, float* out, cf_stream_t s) {
    clear_error();
    if (!counts || !out) return fail(CF_ERR_ARG, "counts and out are required");
    if (!(sigma2_A > 0.0) || !(nbar > 0.0)) return fail(CF_ERR_ARG, "sigma2_A > 0 and nbar > 0 required");
    if (cells < 1 || nfields < 1) return fail(CF_ERR_ARG, "cells and nfields must be >= 1");
    CF_TRY(enter((cudaStream_t)s));
    const cudaStream_t st = (cudaStream_t)s;
    ScopedKernelTimer kt(st, "astar");
    const long long total = cells * nfields;
    k_astar<<<grid_blocks(total, 256), 256, 0, st>>>(counts, f, cells, total, nbar, sigma2_A, out);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// ---------------------------------------------------------------- cumulative information
// Section 3.3, eq. (cuminfo): I(<= b) = sum_{b1, b2 <= b} [C_b^{-1}]_{b1 b2}
// with C_{12} = cov(P1, P2) / (<P1><P2>) restricted to the bins up to b.  With
// the Cholesky factor C = L L^T of the full matrix, the leading b x b block of
// L factors the leading block of C, so I(<= b) = |L_b^{-1} 1|^2 is the
// running sum of y_j^2 for y = L^{-1} 1: one factorisation gives every prefix.
// Bins whose mean is not positive hold no modes and are left out (their
// entry repeats the previous one).  A pivot that is not positive ends the
// factorisation: that bin and all later ones get NaN.
namespace cf {
namespace {
__global__ void __launch_bounds__(256) k_cuminfo(const double* __restrict__ mean, const double* __restrict__ cov,
                                                 int nbins, double* __restrict__ Lm, double* __restrict__ y,
                                                 int* __restrict__ idx, double* __restrict__ info) {
    __shared__ int s_n;
    __shared__ int s_fail;
    __shared__ double s_piv;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int b = 0; b < nbins; ++b)
            if (mean[b] > 0.0) idx[n++] = b;
        s_n = n;
        s_fail = n;
    }
    __syncthreads();
    const int n = s_n;
    // normalised covariance of the kept bins, row-major n x n
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const int bi = idx[i], bj = idx[j];
        Lm[e] = cov[(size_t)bi * nbins + bj] / (mean[bi] * mean[bj]);
    }
    __syncthreads();
    // right-looking Cholesky in place (lower triangle)
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = Lm[(size_t)k * n + k];
            if (!(d > 0.0) && s_fail == n) s_fail = k;
            s_piv = d > 0.0 ? sqrt(d) : 1.0;
            Lm[(size_t)k * n + k] = s_piv;
        }
        __syncthreads();
        const double piv = s_piv;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) Lm[(size_t)i * n + k] /= piv;
        __syncthreads();
        const int m = n - k - 1;
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            if (j <= i) Lm[(size_t)i * n + j] -= Lm[(size_t)i * n + k] * Lm[(size_t)j * n + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // forward solve L y = 1 and running sum of y^2, written at the bins
        double run = 0.0;
        int p = 0;
        for (int b = 0; b < nbins; ++b) {
            if (p < n && idx[p] == b) {
                double v = 1.0;
                for (int j = 0; j < p; ++j) v -= Lm[(size_t)p * n + j] * y[j];
                v /= Lm[(size_t)p * n + p];
                y[p] = v;
                run += v * v;
                ++p;
            }
            info[b] = (p > s_fail) ? __longlong_as_double(0x7ff8000000000000ll) : run;
        }
    }
}
}  // namespace
}  // namespace cf

extern "C" cf_status cf_cumulative_information(const double* mean, const double* cov, int32_t nbins,
                                               double* info_out, void* ws, size_t ws_bytes, cf_stream_t s) {
    clear_error();
    if (!mean || !cov || !info_out) return fail(CF_ERR_ARG, "mean, cov and info_out are required");
    if (nbins < 1 || nbins > 4096) return fail(CF_ERR_ARG, "nbins must be in [1, 4096]");
    const size_t need = sizeof(double) * ((size_t)nbins * nbins + nbins) + sizeof(int) * (size_t)nbins;
    if (!ws || ws_bytes < need) return fail(CF_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, need);
    CF_TRY(enter((cudaStream_t)s));
    double* Lm = (double*)ws;                    // [nbins][nbins]
    double* y = Lm + (size_t)nbins * nbins;      // [nbins]
    int* idx = (int*)(y + nbins);                // [nbins]
    ScopedKernelTimer kt((cudaStream_t)s, "cumulative_information");
    k_cuminfo<<<1, 256, 0, (cudaStream_t)s>>>(mean, cov, nbins, Lm, y, idx, info_out);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// ---------------------------------------------------------------- sub-box copy
// The first n_out[a] cells of every axis of each field (e.g. the survey corner
// of a box-sampled field, section 3.3).
namespace cf {
namespace {
template <typename T>
__global__ void k_copy_corner(const T* __restrict__ in, GridInfo gi, GridInfo go, long long nfields,
                              T* __restrict__ out) {
    const long long total = go.ncell * nfields;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long rem = idx % go.ncell;
        const long long fld = idx / go.ncell;
        long long src = 0, stride = 1;
        for (int a = go.ndim - 1; a >= 0; --a) {
            const long long x = rem % go.n[a];
            rem /= go.n[a];
            src += x * stride;
            stride *= gi.n[a];
        }
        out[idx] = in[fld * gi.ncell + src];
    }
}
}  // namespace
}  // namespace cf

extern "C" cf_status cf_copy_corner(const void* in, cf_dtype dt, const cf_grid* g_in, const cf_grid* g_out,
                                    int64_t nfields, void* out, cf_stream_t s) {
    clear_error();
    if (!in || !out || !g_in || !g_out) return fail(CF_ERR_ARG, "NULL argument");
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d", dt);
    if (g_in->ndim != g_out->ndim || g_in->ndim < 1 || g_in->ndim > 3) return fail(CF_ERR_ARG, "grid dimensions");
    GridInfo gi{}, go{};
    gi.ndim = go.ndim = g_in->ndim;
    gi.ncell = go.ncell = 1;
    for (int a = 0; a < g_in->ndim; ++a) {
        if (g_out->n[a] < 1 || g_out->n[a] > g_in->n[a]) return fail(CF_ERR_ARG, "output larger than input");
        gi.n[a] = g_in->n[a];
        go.n[a] = g_out->n[a];
        gi.ncell *= gi.n[a];
        go.ncell *= go.n[a];
    }
    if (nfields < 1) return fail(CF_ERR_ARG, "nfields must be >= 1");
    CF_TRY(enter((cudaStream_t)s));
    const int blocks = grid_blocks(go.ncell * nfields, 256);
    if (dt == CF_F32)
        k_copy_corner<float><<<blocks, 256, 0, (cudaStream_t)s>>>((const float*)in, gi, go, nfields, (float*)out);
    else
        k_copy_corner<double><<<blocks, 256, 0, (cudaStream_t)s>>>((const double*)in, gi, go, nfields, (double*)out);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

extern "C" cf_status cf_mean_cov(const double* x, int64_t nrows, int32_t ncols, double* mean_or_null,
                                 double* cov_or_null, cf_stream_t s) {
    clear_error();
    if (!x) return fail(CF_ERR_ARG, "x is NULL");
    if (nrows < 1 || ncols < 1) return fail(CF_ERR_ARG, "nrows and ncols must be >= 1");
    CF_TRY(enter((cudaStream_t)s));
    return launch_mean_cov(x, nrows, ncols, mean_or_null, cov_or_null, (cudaStream_t)s);
}
