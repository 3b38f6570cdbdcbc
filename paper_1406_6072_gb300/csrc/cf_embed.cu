// cf_embed.cu -- steps a1-a3: circulant embedding of the two-point function,
// binary64 eigenvalues and the positivity check (section 2, eqs. (grid),
// (Specd), (condition)).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "cf_df.cuh"

namespace cf {

// a1: first row of the circulant, c(m) = xi(|lag(m)|), lag(m_i) = m_i for
// 2 m_i < M_i and m_i - M_i otherwise (for M = 2n the grid of eq. (grid) runs
// -n..n-1).  xi depends on |lag_i| only, so one thread evaluates xi once per
// point of [0, M_0/2] x ... and writes it to the 2^d mirror positions m_i = l_i
// and M_i - l_i (one position when l_i is 0 or M_i/2).
__device__ __forceinline__ double xi_value(int kind, double amp, double scale, double beta, int log1p_xi,
                                           double r2) {
    double v;
    if (kind == CF_XI_GAUSSIAN)
        v = amp * exp(-r2 / (2.0 * scale * scale));
    else if (kind == CF_XI_GEN_CAUCHY)
        v = amp * pow(1.0 + r2 / (scale * scale), -beta);
    else
        v = amp * exp(-sqrt(r2) / scale);
    if (log1p_xi) v = log1p(v);  // eq. (Lncov): Gaussian covariance from the density correlation
    return v;
}

// With equal cell sides h, r^2 = h^2 (l_0^2 + l_1^2 + l_2^2): xi of every
// integer k = sum l_a^2 once (the same binary64 value as the direct
// evaluation when h = 1), which in 3D is far fewer evaluations than lags.
__global__ void k_xi_by_k(int kind, double amp, double scale, double beta, int log1p_xi, double h2, long long kmax,
                          double* __restrict__ tab) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k <= kmax;
         k += (long long)gridDim.x * blockDim.x)
        tab[k] = xi_value(kind, amp, scale, beta, log1p_xi, (double)k * h2);
}

__global__ void k_fill_row(GridInfo g, int kind, double amp, double scale, double beta, int log1p_xi,
                           const double* __restrict__ tab, double* __restrict__ c, C2<double>* __restrict__ z) {
    const long long h0 = g.m[0] / 2, h1 = g.m[1] / 2, h2 = g.m[2] / 2;
    const long long q0 = h0 + 1, q1 = g.ndim > 1 ? h1 + 1 : 1, q2 = g.ndim > 2 ? h2 + 1 : 1;
    const long long total = q0 * q1 * q2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long l2 = t % q2, l1 = (t / q2) % q1, l0 = t / (q1 * q2);
        const long long l[3] = {l0, l1, l2};
        double v;
        if (tab) {
            v = tab[l0 * l0 + l1 * l1 + l2 * l2];
        } else {
            double r2 = 0.0;
            for (int a = 0; a < g.ndim; ++a) {
                const double x = (double)l[a] * g.cell[a];
                r2 += x * x;
            }
            v = xi_value(kind, amp, scale, beta, log1p_xi, r2);
        }
        // mirror positions
        const int na = g.ndim;
        const int nm0 = (l0 == 0 || l0 == h0) ? 1 : 2;
        const int nm1 = (na < 2 || l1 == 0 || l1 == h1) ? 1 : 2;
        const int nm2 = (na < 3 || l2 == 0 || l2 == h2) ? 1 : 2;
        for (int a0 = 0; a0 < nm0; ++a0) {
            const long long m0 = a0 ? g.m[0] - l0 : l0;
            for (int a1 = 0; a1 < nm1; ++a1) {
                const long long m1 = a1 ? g.m[1] - l1 : l1;
                for (int a2 = 0; a2 < nm2; ++a2) {
                    const long long m2 = a2 ? g.m[2] - l2 : l2;
                    const long long idx = (m0 * g.m[1] + m1) * g.m[2] + m2;
                    c[idx] = v;
                    if (z) z[idx] = mk(v, 0.0);
                }
            }
        }
    }
}

__global__ void k_log1p_inplace(double* __restrict__ c, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        c[i] = log1p(c[i]);
}

__global__ void k_real_to_complex(const double* __restrict__ a, double* __restrict__ c_copy,
                                  C2<double>* __restrict__ z, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        if (c_copy) c_copy[i] = v;
        z[i] = mk(v, 0.0);
    }
}

__global__ void k_take_real(const C2<double>* __restrict__ z, double scale, double* __restrict__ out,
                            long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = z[i].x * scale;
}

struct EmbedStats {
    double lmin, lmax, tau, neg_mass, cov_error;
    unsigned long long n_negative, n_zeroed;
};

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

// block-wide reduction helpers (kRedThreads threads)
__device__ __forceinline__ double block_min(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_max(double v, double* sh) { return -block_min(-v, sh); }
__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Order-preserving integer key of a binary64 value (not NaN): the signed
// comparison of keys is the comparison of the values, so minima, maxima and
// threshold tests run on the integer pipes (binary64 throughput is low on
// this GPU).  The map is an involution.
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

__global__ void __launch_bounds__(kRedThreads)
    k_minmax_partial(const double* __restrict__ lam, long long total, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    long long kmn = 0x7fffffffffffffffll, kmx = -0x7fffffffffffffffll - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = order_key(lam[i]);
        kmn = k < kmn ? k : kmn;
        kmx = k > kmx ? k : kmx;
    }
    double mn = key_value(kmn), mx = key_value(kmx);
    mn = block_min(mn, sh);
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = mn;
        part[2 * blockIdx.x + 1] = mx;
    }
}

__global__ void __launch_bounds__(kRedThreads)
    k_minmax_final(const double* __restrict__ part, int nparts, EmbedStats* st) {
    __shared__ double sh[kRedThreads];
    double mn = INFINITY, mx = -INFINITY;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        mn = fmin(mn, part[2 * i]);
        mx = fmax(mx, part[2 * i + 1]);
    }
    mn = block_min(mn, sh);
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) {
        st->lmin = mn;
        st->lmax = mx;
        st->tau = 1e-12 * mx;
        st->neg_mass = 0.0;
        st->cov_error = 0.0;
        st->n_negative = 0;
        st->n_zeroed = 0;
    }
}

// a3: lambda+ = lambda if lambda > tau; 0 if |lambda| <= tau (zeroed); 0 if
// lambda < -tau (negative: counted, its |lambda| summed); s = sqrt(lambda+).
// The binary32 amplitude sqrt(lambda+ / M^d) is formed in binary32 from the
// exactly scaled binary64 value (M^d is a power of two); the binary64
// amplitude is built only when a binary64 sampler needs it (k_s64).
__global__ void __launch_bounds__(kRedThreads)
    k_threshold(const double* __restrict__ lam, long long total, const EmbedStats* __restrict__ st,
                double inv_total, float* __restrict__ s32, double* __restrict__ part,
                unsigned long long* __restrict__ counts) {
    __shared__ double sh[kRedThreads];
    const double tau = st->tau;
    const long long ktau = order_key(tau), kntau = order_key(-tau);
    double neg = 0.0;
    unsigned long long nneg = 0, nzero = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = lam[i];
        const long long k = order_key(l);
        float sv = 0.0f;
        if (k > ktau) {  // l > tau
            sv = sqrtf((float)(l * inv_total));
        } else if (k >= kntau) {  // -tau <= l <= tau
            ++nzero;
        } else {
            ++nneg;
            neg += -l;
        }
        s32[i] = sv;
    }
    neg = block_sum(neg, sh);
    // counts are exact in binary64 (< 2^53): reduce per block, one atomic each
    const double bneg = block_sum((double)nneg, sh);
    const double bzero = block_sum((double)nzero, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = neg;
        if (bneg > 0.0) atomicAdd(&counts[0], (unsigned long long)bneg);
        if (bzero > 0.0) atomicAdd(&counts[1], (unsigned long long)bzero);
    }
}

__global__ void __launch_bounds__(kRedThreads)
    k_threshold_final(const double* __restrict__ part, int nparts, const unsigned long long* counts,
                      EmbedStats* st) {
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        st->neg_mass = s;
        st->n_negative = counts[0];
        st->n_zeroed = counts[1];
    }
}

// realised covariance error max |Re z/M^d - c| over survey lags (|lag_i| < n_i:
// index m_i < n_i or m_i > M_i - n_i on every axis)
__global__ void __launch_bounds__(kRedThreads)
    k_cov_error_partial(const C2<double>* __restrict__ z, const double* __restrict__ c, GridInfo g,
                        double inv_total, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double mx = 0.0;
    int shift[3];  // embedded sides are powers of two: indices by shifts and masks
    for (int a = 0; a < 3; ++a) shift[a] = __ffsll(g.m[a]) - 1;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.mtotal;
         idx += (long long)gridDim.x * blockDim.x) {
        long long rem = idx;
        bool survey = true;
        for (int a = g.ndim - 1; a >= 0; --a) {
            const long long m = rem & (g.m[a] - 1);
            rem >>= shift[a];
            if (m >= g.n[a] && m <= g.m[a] - g.n[a]) survey = false;
        }
        if (survey) mx = fmax(mx, fabs(z[idx].x * inv_total - c[idx]));
    }
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = mx;
}

__global__ void __launch_bounds__(kRedThreads)
    k_cov_error_partial_real(const double* __restrict__ z, const double* __restrict__ c, GridInfo g,
                             double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double mx = 0.0;
    int shift[3];  // embedded sides are powers of two: indices by shifts and masks
    for (int a = 0; a < 3; ++a) shift[a] = __ffsll(g.m[a]) - 1;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.mtotal;
         idx += (long long)gridDim.x * blockDim.x) {
        long long rem = idx;
        bool survey = true;
        for (int a = g.ndim - 1; a >= 0; --a) {
            const long long m = rem & (g.m[a] - 1);
            rem >>= shift[a];
            if (m >= g.n[a] && m <= g.m[a] - g.n[a]) survey = false;
        }
        if (survey) mx = fmax(mx, fabs(z[idx] - c[idx]));
    }
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = mx;
}

__global__ void __launch_bounds__(kRedThreads)
    k_cov_error_final(const double* __restrict__ part, int nparts, EmbedStats* st) {
    __shared__ double sh[kRedThreads];
    double mx = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) mx = fmax(mx, part[i]);
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) st->cov_error = mx;
}


// ---------------------------------------------------------------------------
// DFT of a real array that is even along every axis (x(M - m) = x(m) per
// axis), as the embedded row of an isotropic xi is.  Its DFT is real and even
// along every axis too, so only the non-redundant corner [0, M_a/2]^d is
// transformed and stored (H_a = M_a/2 + 1 per axis); the full result is
// mirrored at the end.  The row pass transforms the rows of the corner's
// leading indices; a column pass rebuilds each line of length M_a from its
// H_a stored values (x(M_a - m) = x(m)) and keeps outputs k <= M_a/2.  Two real
// lines are transformed as the real and imaginary parts of one complex line.
// ---------------------------------------------------------------------------
// S: the arithmetic of the transforms, binary64 or double-float (DF); the
// input x and the output are binary64, the scratch `half` holds S values.
template <typename S>
__device__ __forceinline__ S to_s(double d) {
    if constexpr (sizeof(S) == 8 && __is_same(S, double)) return d;
    else return df_from(d);
}
template <typename S>
__device__ __forceinline__ double from_s(S v) {
    if constexpr (__is_same(S, double)) return v;
    else return df_to(v);
}

// Row r of the corner (nrows = prod of H_a over the leading axes) is full row
// (r / Hm) Mm + r % Hm of in[..][L]: Hm, Mm = H and M of the middle axis in 3D,
// 1 and 1 otherwise.
template <typename S, int L>
__global__ void __launch_bounds__(RowsCfg<S, L>::THREADS, RowsCfg<S, L>::MINB)
    k_even_rows(const double* __restrict__ in, long long nrows, long long Hm, long long Mm, S* __restrict__ out,
                const C2<S>* __restrict__ tw) {
    using Cfg = RowsCfg<S, L>;
    using G = typename Cfg::G;
    constexpr int H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<S>* sm = reinterpret_cast<C2<S>*>(smraw);
    const int line = threadIdx.x / G::TL;
    const int j = threadIdx.x % G::TL;
    const long long pair = (long long)blockIdx.x * Cfg::ROWS + line;
    const long long ra = 2 * pair, rb = ra + 1;
    const bool valid = ra < nrows;
    const bool hasb = rb < nrows;
    const long long fa = valid ? (ra / Hm) * Mm + ra % Hm : 0;
    const long long fb = hasb ? (rb / Hm) * Mm + rb % Hm : 0;
    const double* a = in + (size_t)fa * L;
    const double* b = in + (size_t)fb * L;
    C2<S> v[G::E];
#pragma unroll
    for (int q = 0; q < G::E; ++q) {
        const int x = j + q * (L / G::E);
        v[q] = mk(to_s<S>(a[x]), to_s<S>(hasb ? b[x] : 0.0));
    }
    auto sink = [&](int, int k, C2<S> val) {
        if (!valid || k >= H) return;
        out[(size_t)ra * H + k] = val.x;
        if (hasb) out[(size_t)rb * H + k] = val.y;
    };
    line_fft<S, L, -1, L>(sm, RowLayout<G::PADE, G::PADDED>(), line, j, v, tw, sink);
}

// Columns of in[outer][L/2+1][inner] in pairs (i, i+1), each the stored half
// of an even line of length L: out has the same layout (in place allowed).
template <typename S, int L>
__global__ void __launch_bounds__(ColsCfg<S, L>::THREADS, ColsCfg<S, L>::MINB)
    k_even_cols(const S* in, long long inner, S* out, const C2<S>* __restrict__ tw) {
    using Cfg = ColsCfg<S, L>;
    using G = typename Cfg::G;
    constexpr int H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<S>* sm = reinterpret_cast<C2<S>*>(smraw);
    const int ln = threadIdx.x % Cfg::C;
    const int j = threadIdx.x / Cfg::C;
    const long long ia = 2 * ((long long)blockIdx.x * Cfg::C + ln), ib = ia + 1;
    const long long o = blockIdx.y;
    const bool valid = ia < inner;
    const bool hasb = ib < inner;
    const size_t base = (size_t)o * H * (size_t)inner;
    const S zero = to_s<S>(0.0);
    C2<S> v[G::E];
#pragma unroll
    for (int q = 0; q < G::E; ++q) {
        const int p = j + q * (L / G::E);
        const size_t row = base + (size_t)(p < H ? p : L - p) * (size_t)inner;
        v[q] = mk(valid ? in[row + ia] : zero, hasb ? in[row + ib] : zero);
    }
    auto sink = [&](int, int p, C2<S> val) {
        if (!valid || p >= H) return;
        const size_t row = base + (size_t)p * (size_t)inner;
        out[row + ia] = val.x;
        if (hasb) out[row + ib] = val.y;
    };
    line_fft<S, L, -1, L>(sm, ColLayout<G::E, Cfg::C>(), ln, j, v, tw, sink);
}

// full[M_0]..[M_{d-1}] from the corner half[H_0]..[H_{d-1}] of an array even
// along every axis, times scale (a power of two).  Axes past d have M = H = 1.
template <typename S, bool SCALE>
__global__ void k_even_mirror(const S* __restrict__ half, GridInfo g, double scale, double* __restrict__ full) {
    int sh[3];
    long long M[3], H[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        M[a] = a < g.ndim ? g.m[a] : 1;
        H[a] = M[a] / 2 + 1 < M[a] ? M[a] / 2 + 1 : M[a];
        sh[a] = __ffsll(M[a]) - 1;  // embedded sides are powers of two
    }
    const long long total = g.mtotal;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k2 = t & (M[2] - 1), k1 = (t >> sh[2]) & (M[1] - 1), k0 = t >> (sh[2] + sh[1]);
        const long long c0 = k0 < H[0] ? k0 : M[0] - k0;
        const long long c1 = k1 < H[1] ? k1 : M[1] - k1;
        const long long c2 = k2 < H[2] ? k2 : M[2] - k2;
        const double v = from_s<S>(half[(c0 * H[1] + c1) * H[2] + c2]);
        full[t] = SCALE ? v * scale : v;
    }
}

// lambda+ (threshold tau read on the device) as a real array
__global__ void k_lambda_plus_real(const double* __restrict__ lam, const struct EmbedStats* __restrict__ st,
                                   double* __restrict__ out, long long total) {
    const double tau = st->tau;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = lam[i];
        out[i] = l > tau ? l : 0.0;
    }
}

// lambda+ (threshold tau read on the device) as a complex array, written
// straight into the transform buffer (no in-place real-to-complex widening)
__global__ void k_lambda_plus_complex(const double* __restrict__ lam, const struct EmbedStats* __restrict__ st,
                                      C2<double>* __restrict__ z, long long total) {
    const double tau = st->tau;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = lam[i];
        z[i] = mk(l > tau ? l : 0.0, 0.0);
    }
}

template <typename S, int L>
static cf_status launch_even_rows(const double* in, long long nrows, long long Hm, long long Mm, S* out,
                                  cudaStream_t s) {
    using Cfg = RowsCfg<S, L>;
    auto kern = k_even_rows<S, L>;
    CF_TRY(prepare_smem(kern, Cfg::SMEM));
    const long long pairs = (nrows + 1) / 2;
    ScopedKernelTimer kt(s, sizeof(S) == 8 && __is_same(S, double) ? "even_rows_f64" : "even_rows_df", L);
    kern<<<(unsigned)((pairs + Cfg::ROWS - 1) / Cfg::ROWS), Cfg::THREADS, Cfg::SMEM, s>>>(in, nrows, Hm, Mm, out,
                                                                                     twiddles<S>());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

template <typename S, int L>
static cf_status launch_even_cols(S* data, long long outer, long long inner, cudaStream_t s) {
    using Cfg = ColsCfg<S, L>;
    auto kern = k_even_cols<S, L>;
    CF_TRY(prepare_smem(kern, Cfg::SMEM));
    if (outer > 65535) return fail(CF_ERR_UNSUPPORTED, "even transform with %lld outer slices", outer);
    const long long pairs = (inner + 1) / 2;
    dim3 grid((unsigned)((pairs + Cfg::C - 1) / Cfg::C), (unsigned)outer);
    ScopedKernelTimer kt(s, __is_same(S, double) ? "even_cols_f64" : "even_cols_df", L);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(data, inner, data, twiddles<S>());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// full = scale * DFT(x) for x real and even along every axis; half is scratch
// of prod_a (M_a/2 + 1) values of 8 bytes.  The transforms run in binary64, or
// with CF_EMBED_DF in double-float arithmetic (cf_df.cuh).
template <typename S>
static cf_status even_dft_t(const double* x, const GridInfo& g, double scale, S* half, double* full,
                            cudaStream_t s) {
    const int d = g.ndim;
    long long H[3];
    for (int a = 0; a < d; ++a) H[a] = g.m[a] / 2 + 1;
    long long rows = 1;
    for (int a = 0; a < d - 1; ++a) rows *= H[a];
    const long long Hm = d == 3 ? H[1] : 1, Mm = d == 3 ? g.m[1] : 1;
    CF_TRY(dispatch_line(g.m[d - 1], [&](auto Lc) -> cf_status {
        return launch_even_rows<S, decltype(Lc)::value>(x, rows, Hm, Mm, half, s);
    }));
    for (int a = d - 2; a >= 0; --a) {
        long long inner = 1, outer = 1;
        for (int b2 = a + 1; b2 < d; ++b2) inner *= H[b2];
        for (int b2 = 0; b2 < a; ++b2) outer *= H[b2];
        CF_TRY(dispatch_line(g.m[a], [&](auto Lc) -> cf_status {
            return launch_even_cols<S, decltype(Lc)::value>(half, outer, inner, s);
        }));
    }
    if (scale == 1.0)
        k_even_mirror<S, false><<<grid_blocks(g.mtotal, 256, 4096), 256, 0, s>>>(half, g, scale, full);
    else
        k_even_mirror<S, true><<<grid_blocks(g.mtotal, 256, 4096), 256, 0, s>>>(half, g, scale, full);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

static cf_status even_dft(const double* x, const GridInfo& g, double scale, double* half, double* full,
                          uint32_t flags, cudaStream_t s) {
    if (!(flags & CF_EMBED_DF)) return even_dft_t<double>(x, g, scale, half, full, s);
    static_assert(sizeof(DF) == sizeof(double), "the scratch holds 8-byte values");
    return even_dft_t<DF>(x, g, scale, reinterpret_cast<DF*>(half), full, s);
}

// c (the even row of a parametric xi) on the device: through a table of xi
// by k = sum l_a^2 when the cell sides are equal and the table is smaller
// than a quarter of the lags.
static cf_status fill_even_row(const GridInfo& g, const cf_xi* xi, int log1p_xi, double* c, cudaStream_t s) {
    long long kmax = 0, lags = 1;
    bool equal = true;
    for (int a = 0; a < g.ndim; ++a) {
        kmax += (g.m[a] / 2) * (g.m[a] / 2);
        lags *= g.m[a] / 2 + 1;
        equal = equal && g.cell[a] == g.cell[0];
    }
    double* tab = nullptr;
    if (equal && 4 * (kmax + 1) < lags) {
        if (pool_malloc((void**)&tab, sizeof(double) * (size_t)(kmax + 1), s) != cudaSuccess)
            return fail(CF_ERR_NOMEM, "xi table allocation failed");
        k_xi_by_k<<<grid_blocks(kmax + 1, 256, 1024), 256, 0, s>>>(xi->kind, xi->amp, xi->scale, xi->beta, log1p_xi,
                                                                  g.cell[0] * g.cell[0], kmax, tab);
    }
    k_fill_row<<<grid_blocks(lags, 256, 4096), 256, 0, s>>>(g, xi->kind, xi->amp, xi->scale, xi->beta, log1p_xi,
                                                            tab, c, nullptr);
    if (tab) cudaFreeAsync(tab, s);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// Device buffers of one embedding computation.
struct EmbedScratch {
    C2<double>* z = nullptr;
    double* c = nullptr;
    double* part = nullptr;
    EmbedStats* st = nullptr;
    unsigned long long* counts = nullptr;
    cudaStream_t s = nullptr;
    ~EmbedScratch() {
        if (z) cudaFreeAsync(z, s);
        if (c) cudaFreeAsync(c, s);
        if (part) cudaFreeAsync(part, s);
        if (st) cudaFreeAsync(st, s);
        if (counts) cudaFreeAsync(counts, s);
    }
};

// Common tail: lambda is either in `lam_real` (real, from the even transform)
// or in Re of sc.z (general complex transform); sc.c holds the embedded row
// (target covariance).  Runs a3 and builds the embedding with one host
// synchronisation: the realised-covariance error of the clamped spectrum is
// computed before it (from the device-side threshold) whenever clamping is
// allowed, and reported only if clamping happened.
static cf_status finish_embedding(const GridInfo& gi, EmbedScratch& sc, uint32_t flags, const double* lam_real,
                                  bool even, cf_embedding** out, cf_embed_report* rep) {
    cudaStream_t s = sc.s;
    const long long total = gi.mtotal;
    const int blocks = grid_blocks(total, kRedThreads, kRedBlocks);
    cf_embedding* e = new cf_embedding();
    e->grid = gi;
    CF_CUDA(cudaGetDevice(&e->device));
    e->alloc_stream = s;
    auto cleanup = [&]() { cf_embedding_free(e); };
    // persistent arrays: stream-ordered allocations, released after their last use
    if (pool_malloc((void**)&e->lambda, sizeof(double) * total, s) != cudaSuccess ||
        pool_malloc((void**)&e->s32, sizeof(float) * total, s) != cudaSuccess) {
        cleanup();
        return fail(CF_ERR_NOMEM, "device allocation of the embedding (%lld cells) failed", total);
    }
    const bool want_error = (flags & CF_EMBED_CLAMP) && !(flags & CF_EMBED_SKIP_ERROR);
    {
        ScopedKernelTimer kt(s, "embed_psd");
        if (lam_real)
            CF_CUDA(cudaMemcpyAsync(e->lambda, lam_real, sizeof(double) * total, cudaMemcpyDeviceToDevice, s));
        else
            k_take_real<<<blocks, kRedThreads, 0, s>>>(sc.z, 1.0, e->lambda, total);
        k_minmax_partial<<<blocks, kRedThreads, 0, s>>>(e->lambda, total, sc.part);
        k_minmax_final<<<1, kRedThreads, 0, s>>>(sc.part, blocks, sc.st);
        CF_CUDA(cudaMemsetAsync(sc.counts, 0, 2 * sizeof(unsigned long long), s));
        k_threshold<<<blocks, kRedThreads, 0, s>>>(e->lambda, total, sc.st, 1.0 / (double)total, e->s32, sc.part,
                                                   sc.counts);
        k_threshold_final<<<1, kRedThreads, 0, s>>>(sc.part, blocks, sc.counts, sc.st);
    }
    CF_CHECK_LAUNCH();
    if (want_error) {
        // realised covariance = IDFT(lambda+)/M^d, compared with c on survey lags
        if (even) {
            // lambda+ is real and even: its inverse transform equals its forward one
            double* buf = (double*)sc.z;  // M^d doubles, then scratch for the half spectra
            {
                ScopedKernelTimer kt(s, "embed_cov_error");
                k_lambda_plus_real<<<blocks, kRedThreads, 0, s>>>(e->lambda, sc.st, buf, total);
            }
            CF_CHECK_LAUNCH();
            CF_TRY(even_dft(buf, gi, 1.0 / (double)total, buf + total, buf, flags, s));
            ScopedKernelTimer kt(s, "embed_cov_error");
            k_cov_error_partial_real<<<blocks, kRedThreads, 0, s>>>(buf, sc.c, gi, sc.part);
        } else {
            {
                ScopedKernelTimer kt(s, "embed_cov_error");
                k_lambda_plus_complex<<<blocks, kRedThreads, 0, s>>>(e->lambda, sc.st, sc.z, total);
            }
            CF_CHECK_LAUNCH();
            CF_TRY((fft_nd_inplace<double, +1>(sc.z, gi, s)));
            ScopedKernelTimer kt(s, "embed_cov_error");
            k_cov_error_partial<<<blocks, kRedThreads, 0, s>>>(sc.z, sc.c, gi, 1.0 / (double)total, sc.part);
        }
        k_cov_error_final<<<1, kRedThreads, 0, s>>>(sc.part, blocks, sc.st);
        CF_CHECK_LAUNCH();
    }
    EmbedStats st{};
    CF_TRY(read_back(&st, sc.st, sizeof st, s));
    cf_embed_report r{};
    r.lambda_min = st.lmin;
    r.lambda_max = st.lmax;
    r.tau = st.tau;
    r.neg_mass = st.neg_mass;
    r.n_negative = (int64_t)st.n_negative;
    r.n_zeroed = (int64_t)st.n_zeroed;
    r.clamped = 0;
    r.exact = 1;
    e->tau = st.tau;
    if (!(st.lmax > 0.0)) {
        r.exact = 0;
        if (rep) *rep = r;
        cleanup();
        return fail(CF_ERR_NOT_PSD, "largest eigenvalue %.3e is not positive", st.lmax);
    }
    if (st.n_negative > 0) {
        if (!(flags & CF_EMBED_CLAMP)) {
            r.exact = 0;
            if (rep) *rep = r;
            cleanup();
            return fail(CF_ERR_NOT_PSD,
                        "%llu eigenvalues below -tau (lambda_min/lambda_max = %.3e); set CF_EMBED_CLAMP",
                        st.n_negative, st.lmin / st.lmax);
        }
        r.clamped = 1;
        r.exact = 0;
        if (want_error) r.cov_error = st.cov_error;
    }
    e->report = r;
    if (rep) *rep = r;
    record_use(e, s);
    *out = e;
    return CF_OK;
}

}  // namespace cf

using namespace cf;


static cf_status alloc_scratch(EmbedScratch& sc, long long total) {
    cudaStream_t s = sc.s;
    if (pool_malloc((void**)&sc.z, sizeof(C2<double>) * total, s) != cudaSuccess ||
        pool_malloc((void**)&sc.c, sizeof(double) * total, s) != cudaSuccess ||
        pool_malloc((void**)&sc.part, sizeof(double) * kRedBlocks * 2, s) != cudaSuccess ||
        pool_malloc((void**)&sc.st, sizeof(EmbedStats), s) != cudaSuccess ||
        pool_malloc((void**)&sc.counts, sizeof(unsigned long long) * 2, s) != cudaSuccess)
        return fail(CF_ERR_NOMEM, "device allocation for the embedding of %lld cells failed", total);
    return CF_OK;
}

extern "C" cf_status cf_embed(const cf_grid* g, const cf_xi* xi, uint32_t flags, cf_stream_t stream,
                              cf_embedding** out, cf_embed_report* rep) {
    clear_error();
    if (!out) return fail(CF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!xi) return fail(CF_ERR_ARG, "xi is NULL");
    GridInfo gi;
    CF_TRY(check_grid(g, &gi));
    if (xi->kind < CF_XI_GAUSSIAN || xi->kind > CF_XI_TABLE) return fail(CF_ERR_ARG, "unknown xi kind %d", xi->kind);
    if (xi->kind == CF_XI_TABLE && !xi->table) return fail(CF_ERR_ARG, "CF_XI_TABLE needs a table");
    if (xi->kind != CF_XI_TABLE && !(xi->scale > 0.0)) return fail(CF_ERR_ARG, "xi scale must be > 0");
    CF_TRY(enter((cudaStream_t)stream));
    EmbedScratch sc;
    sc.s = (cudaStream_t)stream;
    CF_TRY(alloc_scratch(sc, gi.mtotal));
    const int blocks = grid_blocks(gi.mtotal, kRedThreads, kRedBlocks);
    const int log1p_xi = (flags & CF_EMBED_LOG1P) ? 1 : 0;
    if (xi->kind == CF_XI_TABLE) {
        if (xi->table_on_device && !log1p_xi) {
            k_real_to_complex<<<blocks, kRedThreads, 0, sc.s>>>(xi->table, sc.c, sc.z, gi.mtotal);
        } else {
            CF_CUDA(cudaMemcpyAsync(sc.c, xi->table, sizeof(double) * gi.mtotal,
                                    xi->table_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sc.s));
            if (log1p_xi) k_log1p_inplace<<<blocks, kRedThreads, 0, sc.s>>>(sc.c, gi.mtotal);
            k_real_to_complex<<<blocks, kRedThreads, 0, sc.s>>>(sc.c, nullptr, sc.z, gi.mtotal);
        }
    } else {
        if (log1p_xi && !(xi->amp > -1.0)) return fail(CF_ERR_ARG, "CF_EMBED_LOG1P needs amp > -1");
        ScopedKernelTimer kt(sc.s, "embed_fill");
        // the row is even: its transform goes through even_dft, which needs
        // no complex copy of it
        CF_TRY(fill_even_row(gi, xi, log1p_xi, sc.c, sc.s));
    }
    CF_CHECK_LAUNCH();
    if (xi->kind != CF_XI_TABLE) {
        // the row depends on |lag| only: even along every axis
        double* full = (double*)sc.z;
        CF_TRY(even_dft(sc.c, gi, 1.0, full + gi.mtotal, full, flags, sc.s));
        return finish_embedding(gi, sc, flags, full, true, out, rep);
    }
    CF_TRY((fft_nd_inplace<double, -1>(sc.z, gi, sc.s)));
    return finish_embedding(gi, sc, flags, nullptr, false, out, rep);
}

// ---------------------------------------------------------------- periodic box (section 3.3)
// Eigenvalues of the k-space (periodic box) sampler of eq. (Periodicboxmodes):
// the box of side B = factor * n carries modes k = 2 pi m / B with variance
// P(k) / cell^d, P the continuous Fourier transform of the covariance, the
// DC mode set to zero.  P is approximated on a fine, large grid `big` (cell
// 1/q, extent o B): lambda_big[o f] / q^d with f the signed frequency.  The
// sampler's embedding grid e has side 2n (factor 1 and 2) or 4n (factor 4);
// for factor 1 the box modes sit on the even frequencies of e with weight
// 2^d (a field with only even frequencies on 2n is n-periodic).
__global__ void k_periodic_lambda(const double* __restrict__ big, GridInfo gbig, GridInfo ge, int factor, int o,
                                  double scale, double* __restrict__ lam) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ge.mtotal;
         idx += (long long)gridDim.x * blockDim.x) {
        long long rem = idx, bidx = 0, bstride = 1;
        bool zero = false, dc = true;
        for (int a = ge.ndim - 1; a >= 0; --a) {
            long long m = rem % ge.m[a];
            rem /= ge.m[a];
            if (factor == 1) {
                if (m & 1) zero = true;
                m >>= 1;
            }
            const long long B = factor == 1 ? ge.m[a] / 2 : ge.m[a];
            const long long f = m < B / 2 ? m : m - B;  // signed box frequency
            if (f != 0) dc = false;
            long long bi = (o * f) % gbig.m[a];
            if (bi < 0) bi += gbig.m[a];
            bidx += bi * bstride;
            bstride *= gbig.m[a];
        }
        lam[idx] = (zero || dc) ? 0.0 : big[bidx] * scale;
    }
}

extern "C" cf_status cf_embed_periodic(const cf_grid* g, const cf_xi* xi, int32_t box_factor, int32_t extent,
                                       int32_t resolution, uint32_t flags, cf_stream_t stream, cf_embedding** out,
                                       cf_embed_report* rep) {
    clear_error();
    if (!out) return fail(CF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !xi) return fail(CF_ERR_ARG, "grid and xi are required");
    if (xi->kind < CF_XI_GAUSSIAN || xi->kind > CF_XI_EXPONENTIAL)
        return fail(CF_ERR_ARG, "the periodic box needs a parametric xi");
    if (!(xi->scale > 0.0)) return fail(CF_ERR_ARG, "xi scale must be > 0");
    if (box_factor != 1 && box_factor != 2 && box_factor != 4) return fail(CF_ERR_ARG, "box_factor must be 1, 2 or 4");
    if (extent < 1 || extent > 16 || (extent & (extent - 1))) return fail(CF_ERR_ARG, "extent must be 1, 2, 4, 8 or 16");
    if (resolution < 1 || resolution > 16 || (resolution & (resolution - 1)))
        return fail(CF_ERR_ARG, "resolution must be 1, 2, 4, 8 or 16");
    GridInfo gs;
    CF_TRY(check_grid(g, &gs));
    for (int a = 0; a < gs.ndim; ++a)
        if (gs.m[a] != 2 * gs.n[a])
            return fail(CF_ERR_UNSUPPORTED, "the periodic box needs power-of-two n and embed_factor 0 or 2");
    const int log1p_xi = (flags & CF_EMBED_LOG1P) ? 1 : 0;
    if (log1p_xi && !(xi->amp > -1.0)) return fail(CF_ERR_ARG, "CF_EMBED_LOG1P needs amp > -1");
    // embedding grid of the sampler and the fine, large grid of the spectrum
    cf_grid ge_in = *g, gb_in = *g;
    for (int a = 0; a < gs.ndim; ++a) {
        ge_in.n[a] = box_factor == 4 ? 2 * g->n[a] : g->n[a];
        gb_in.n[a] = (int64_t)resolution * extent * box_factor * g->n[a] / 2;
        gb_in.cell[a] = g->cell[a] / (double)resolution;
    }
    GridInfo ge, gb;
    CF_TRY(check_grid(&ge_in, &ge));
    CF_TRY(check_grid(&gb_in, &gb));
    CF_TRY(enter((cudaStream_t)stream));
    const cudaStream_t s = (cudaStream_t)stream;
    double* lam_e = nullptr;
    if (pool_malloc((void**)&lam_e, sizeof(double) * (size_t)ge.mtotal, s) != cudaSuccess)
        return fail(CF_ERR_NOMEM, "device allocation of the box eigenvalues failed");
    {
        EmbedScratch bs;
        bs.s = s;
        cf_status st = alloc_scratch(bs, gb.mtotal);
        if (st != CF_OK) {
            cudaFreeAsync(lam_e, s);
            return st;
        }
        const int blocks = grid_blocks(gb.mtotal, kRedThreads, kRedBlocks);
        {
            ScopedKernelTimer kt(s, "embed_fill");
            CF_TRY(fill_even_row(gb, xi, log1p_xi, bs.c, s));
        }
        CF_CHECK_LAUNCH();
        double* full = (double*)bs.z;
        CF_TRY(even_dft(bs.c, gb, 1.0, full + gb.mtotal, full, flags, s));
        double scale = 1.0;
        for (int a = 0; a < gs.ndim; ++a) scale /= (double)resolution;
        if (box_factor == 1) scale *= (double)(1 << gs.ndim);
        k_periodic_lambda<<<grid_blocks(ge.mtotal, 256, 4096), 256, 0, s>>>(full, gb, ge, box_factor, extent, scale,
                                                                            lam_e);
        CF_CHECK_LAUNCH();
    }
    EmbedScratch sc;
    sc.s = s;
    cf_status st = alloc_scratch(sc, ge.mtotal);
    if (st == CF_OK) st = finish_embedding(ge, sc, flags | CF_EMBED_SKIP_ERROR, lam_e, true, out, rep);
    cudaFreeAsync(lam_e, s);
    return st;
}

extern "C" cf_status cf_embed_from_lambda(const cf_grid* g, const double* lambda, uint32_t flags,
                                          cf_stream_t stream, cf_embedding** out, cf_embed_report* rep) {
    clear_error();
    if (!out) return fail(CF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!lambda) return fail(CF_ERR_ARG, "lambda is NULL");
    GridInfo gi;
    CF_TRY(check_grid(g, &gi));
    CF_TRY(enter((cudaStream_t)stream));
    EmbedScratch sc;
    sc.s = (cudaStream_t)stream;
    CF_TRY(alloc_scratch(sc, gi.mtotal));
    const int blocks = grid_blocks(gi.mtotal, kRedThreads, kRedBlocks);
    // target covariance c = IDFT(lambda)/M^d, for the error pass
    k_real_to_complex<<<blocks, kRedThreads, 0, sc.s>>>(lambda, nullptr, sc.z, gi.mtotal);
    CF_CHECK_LAUNCH();
    CF_TRY((fft_nd_inplace<double, +1>(sc.z, gi, sc.s)));
    k_take_real<<<blocks, kRedThreads, 0, sc.s>>>(sc.z, 1.0 / (double)gi.mtotal, sc.c, gi.mtotal);
    k_real_to_complex<<<blocks, kRedThreads, 0, sc.s>>>(lambda, nullptr, sc.z, gi.mtotal);
    CF_CHECK_LAUNCH();
    return finish_embedding(gi, sc, flags, nullptr, false, out, rep);
}
