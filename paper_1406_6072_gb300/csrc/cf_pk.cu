// cf_pk.cu -- step d1: binned power spectrum of real fields or count maps
// (section 3.2, eqs. (Def spec), (Estim)) with its mean and covariance over
// realizations.
//
// Two real fields are transformed at once as z = a + i b along the last axis;
// the row pass separates A = (Z_k + conj Z_{-k})/2 and B = (Z_k - conj Z_{-k})/2i
// into half spectra (k_last in [0, n/2]).  The remaining axes are complex
// column passes; the last one squares, weights (2 for 0 < k_last < n/2, the
// mirror mode -k) and bins in shared memory before one atomic add per bin.
//
// Count maps: delta_g = X/Nhat - I with X = N/f on unmasked cells (0
// elsewhere) and I the unmasked-cell indicator, so for k != 0
// |DFT delta_g|^2 = |DFT X|^2/Nhat^2 - 2 Re(DFT X conj DFT I)/Nhat + |DFT I|^2.
// The transform runs on X (no pre-pass for Nhat): the row pass accumulates
// N_tot per field, the binning pass accumulates |DFT X|^2 and the cross term
// against the mask spectrum DFT I, and the final pass combines them.
#include <math.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "cf_kernels.cuh"

namespace cf {

constexpr int kMaxBins = 512;

// Boxes the cubic power-of-two path below does not take (cf_pk_any.cu):
// 1D, rectangular, sides that are not powers of two, unequal cells.
bool pk_any_needed(const cf_grid* g);
cf_status pk_any_workspace(const cf_grid* g, long long nfields, const cf_bins* b, cf_dtype dt, size_t* bytes);
cf_status pk_any_run(const void* fields, int kind, const float* f, const cf_grid* g, long long nfields,
                     const cf_bins* bins, double* pk_out, int64_t* nmodes_out, double* mean, double* cov, void* ws,
                     size_t ws_bytes, cudaStream_t s);
cf_status pk_bin_edges(const cf_bins* b, double kmax_default, double* e);

struct Edges {
    double e[kMaxBins + 1];
};

enum { PK_FLOAT = 0, PK_DOUBLE = 1, PK_COUNTS = 2, PK_MASK = 3 };

__global__ void k_pk_bintable(Edges ed, int nbins, long long k2max, int16_t* __restrict__ bin_of) {
    for (long long k2 = blockIdx.x * (long long)blockDim.x + threadIdx.x; k2 <= k2max;
         k2 += (long long)gridDim.x * blockDim.x) {
        int b = -1;
        if (k2 > 0) {
            const double kn = sqrt((double)k2);
            if (kn >= ed.e[0] && kn < ed.e[nbins]) {
                b = 0;
                while (!(kn < ed.e[b + 1])) ++b;
            }
        }
        bin_of[k2] = (int16_t)b;
    }
}

// Integer form of the same bins: thr[b] = the least k2 >= 1 with sqrt(k2) >= e_b
// (binary64, correctly rounded, as above; k2max + 1 if none).  sqrt is monotone,
// so bin(k2) = max{b : thr[b] <= k2} for thr[0] <= k2 < thr[nbins], else -1:
// exactly the table's bin, found in shared memory instead of a table read.
// The thresholds are stored after the table (bin_thresholds()).
__global__ void k_pk_thresholds(Edges ed, int nbins, long long k2max, int* __restrict__ thr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbins) return;
    long long lo = 1, hi = k2max + 1;  // first k2 in [lo, hi] with sqrt(k2) >= e_b (hi: none)
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (sqrt((double)mid) >= ed.e[b]) hi = mid; else lo = mid + 1;
    }
    thr[b] = (int)lo;
}

__host__ __device__ inline const int* bin_thresholds(const int16_t* bin_of, long long k2max) {
    return reinterpret_cast<const int*>(reinterpret_cast<const char*>(bin_of) +
                                        ((sizeof(int16_t) * (size_t)(k2max + 1) + 15) & ~(size_t)15));
}
// bytes of the table plus its thresholds
inline size_t bin_table_bytes(long long k2max) {
    return ((sizeof(int16_t) * (size_t)(k2max + 1) + 15) & ~(size_t)15) + sizeof(int) * (kMaxBins + 1);
}

__device__ __forceinline__ long long signed_mode(long long i, long long n) { return i <= n / 2 ? i : i - n; }

#ifndef CF_PKR_E
#define CF_PKR_E 8
#endif
#ifndef CF_PKR_THREADS
#define CF_PKR_THREADS 128
#endif
#ifndef CF_PKR_MINB
#define CF_PKR_MINB 8
#endif
#ifndef CF_PKC_E
#define CF_PKC_E 16
#endif
#ifndef CF_PKC_THREADS
#define CF_PKC_THREADS 256
#endif
#ifndef CF_PKC_MINB
#define CF_PKC_MINB 4
#endif

// Pass 1: pairs of real fields along the last axis -> two half spectra.
template <typename T, int L>
struct PkRowsCfg : TileCfg<T, L, CF_PKR_E, CF_PKR_THREADS, CF_PKR_MINB> {
    static constexpr int ROWS = TileCfg<T, L, CF_PKR_E, CF_PKR_THREADS, CF_PKR_MINB>::LINES;
};
template <typename T, int L>
struct PkColsCfg : TileCfg<T, L, CF_PKC_E, CF_PKC_THREADS, CF_PKC_MINB> {
    static constexpr int C = TileCfg<T, L, CF_PKC_E, CF_PKC_THREADS, CF_PKC_MINB>::LINES;
};

template <typename T, int L, int KIND>
__global__ void __launch_bounds__(PkRowsCfg<T, L>::THREADS, PkRowsCfg<T, L>::MINB)
    k_pk_rows(const void* __restrict__ fields, int kind_unused, const float* __restrict__ f,
              unsigned long long* __restrict__ ntot, double* __restrict__ fsum, long long rows, long long cells,
              long long nfields, long long f0, C2<T>* __restrict__ out, const C2<T>* __restrict__ tw) {
    using Cfg = PkRowsCfg<T, L>;
    constexpr int kind = KIND;  // compile-time: the loads of the loader are not behind branches
    using G = typename Cfg::G;
    constexpr int E = G::E;
    constexpr int STEP = L / E;
    constexpr int H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    const int line = threadIdx.x / G::TL;
    const int j = threadIdx.x % G::TL;
    const long long row = (long long)blockIdx.x * Cfg::ROWS + line;
    const bool valid = row < rows;
    const long long rw = valid ? row : 0;
    const long long fa = f0 + 2ll * blockIdx.y;  // global field index of A
    const long long fb = fa + 1;
    const bool hasb = kind != PK_MASK && fb < nfields;
    // X = N/f (0 where f = 0) for count maps; the indicator of f != 0 for the mask
    unsigned long long na = 0, nb = 0;
    double fs = 0.0;
    auto value = [&](long long fld, long long p, unsigned long long& ncount) -> T {
        const size_t at = (size_t)fld * cells + (size_t)rw * L + p;
        if constexpr (kind == PK_FLOAT) {
            return (T)((const float*)fields)[at];
        } else if constexpr (kind == PK_DOUBLE) {
            return (T)((const double*)fields)[at];
        } else if constexpr (kind == PK_MASK) {
            const float fi = f[rw * L + p];
            if (valid) fs += (double)fi;
            return fi != 0.0f ? (T)1 : (T)0;
        } else {
            const int32_t N = ((const int32_t*)fields)[at];
            if (valid) ncount += (unsigned long long)(long long)N;
            if (!f) return (T)N;
            const T fi = (T)f[rw * L + p];
            return fi != (T)0 ? (T)N / fi : (T)0;
        }
    };
    C2<T> v[E];
    if constexpr (kind == PK_COUNTS) {
        // all loads first (no branch between them), then totals and the mask
        int32_t Na[E], Nb[E];
        const int32_t* ca = (const int32_t*)fields + (size_t)fa * cells + (size_t)rw * L;
        const int32_t* cb = (const int32_t*)fields + (size_t)(hasb ? fb : fa) * cells + (size_t)rw * L;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            Na[q] = ca[j + q * STEP];
            Nb[q] = cb[j + q * STEP];
        }
        if (!hasb) {
#pragma unroll
            for (int q = 0; q < E; ++q) Nb[q] = 0;
        }
        if (valid) {
#pragma unroll
            for (int q = 0; q < E; ++q) {
                na += (unsigned long long)(long long)Na[q];
                nb += (unsigned long long)(long long)Nb[q];
            }
        }
        if (f) {
            float fq[E];
#pragma unroll
            for (int q = 0; q < E; ++q) fq[q] = f[rw * L + j + q * STEP];
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const T fi = (T)fq[q];
                v[q] = fi != (T)0 ? mk((T)Na[q] / fi, (T)Nb[q] / fi) : mk((T)0, (T)0);
            }
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = mk((T)Na[q], (T)Nb[q]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const long long p = j + q * STEP;
            const T va = value(fa, p, na);
            v[q] = mk(va, hasb ? value(fb, p, nb) : (T)0);
        }
    }
    if constexpr (kind == PK_COUNTS || kind == PK_MASK) {
        // totals of the block (all its lines belong to fields fa, fb): warp
        // sums, then one atomic per block and field (not one per warp: the
        // blocks of a field would all queue on one address)
        constexpr int NW = Cfg::THREADS / 32;
        __shared__ unsigned long long s_na[NW], s_nb[NW];
        __shared__ double s_fs[NW];
        for (int o = 16; o > 0; o >>= 1) {
            na += __shfl_down_sync(0xffffffffu, na, o);
            nb += __shfl_down_sync(0xffffffffu, nb, o);
            fs += __shfl_down_sync(0xffffffffu, fs, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_na[threadIdx.x >> 5] = na;
            s_nb[threadIdx.x >> 5] = nb;
            s_fs[threadIdx.x >> 5] = fs;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long ta = 0, tb = 0;
            double tf = 0.0;
            for (int w = 0; w < NW; ++w) {
                ta += s_na[w];
                tb += s_nb[w];
                tf += s_fs[w];
            }
            if (kind == PK_COUNTS) {
                if (ta) atomicAdd(&ntot[fa], ta);
                if (tb) atomicAdd(&ntot[fb], tb);
            } else if (tf != 0.0) {
                atomicAdd(fsum, tf);
            }
        }
    }
    RowLayout<G::PADE, G::PADDED> lay;
    // the spectrum of the line goes back into the exchange buffer
    auto sink = [&](int ln, int p, C2<T> val) { sm[lay(ln, p)] = val; };
    line_fft<T, L, -1, L, true>(sm, lay, line, j, v, tw, sink);
    __syncthreads();
    if (!valid) return;
    const long long la = fa - f0, lb = fb - f0;
    C2<T>* oa = out + ((size_t)la * rows + row) * H;
    C2<T>* ob = out + ((size_t)lb * rows + row) * H;
    const T half = (T)0.5;
    for (int k = j; k < H; k += G::TL) {
        const C2<T> zk = sm[lay(line, k & (L - 1))];
        const C2<T> zm = sm[lay(line, (L - k) & (L - 1))];
        oa[k] = mk(half * (zk.x + zm.x), half * (zk.y - zm.y));
        if (hasb) ob[k] = mk(half * (zk.y + zm.y), half * (zm.x - zk.x));
    }
}

// --------------------------------------------------------------------------
// Binary32 row and binning passes on two lines per thread (CP values, paired
// f32x2 instructions, 16-byte shared-memory exchanges, shared twiddles).
// Rows: lane A carries fields (fa, fa+1) as z = a + i b, lane B fields
// (fa+2, fa+3): four fields per thread.  Binning: lane A field fa, lane B
// field fa+1 at the same column, so both take the same bin decisions.  The
// spectra equal the one-line kernels' up to the rounding of the transform's
// radix order.
// --------------------------------------------------------------------------
template <int L, int TARGET>
struct PkPairCfg {
    static constexpr int E = L < 8 ? L : 8;
    static constexpr int TL = L / E;
    static constexpr int LINES = TL >= TARGET ? 1 : (TARGET / TL > 32 ? 32 : TARGET / TL);
    static constexpr int THREADS = LINES * TL;
    static constexpr int MINB = 1024 / THREADS > 8 ? 8 : (1024 / THREADS > 0 ? 1024 / THREADS : 1);
    static constexpr int PADDED = L + L / E;
    static constexpr size_t SMEM = sizeof(CP) * (size_t)LINES * (size_t)PADDED;
};
#ifndef CF_PKR2_THREADS
#define CF_PKR2_THREADS 128
#endif
#ifndef CF_PKC2_THREADS
#define CF_PKC2_THREADS 256
#endif

template <int L, int KIND>
__global__ void __launch_bounds__(PkPairCfg<L, CF_PKR2_THREADS>::THREADS, PkPairCfg<L, CF_PKR2_THREADS>::MINB)
    k_pk_rows_pair(const void* __restrict__ fields, const float* __restrict__ f, unsigned long long* __restrict__ ntot,
                   long long rows, long long cells, long long nfields, long long f0, long long nchunk,
                   C2<float>* __restrict__ out, const float4* __restrict__ tw) {
    using Cfg = PkPairCfg<L, CF_PKR2_THREADS>;
    constexpr int E = Cfg::E;
    constexpr int STEP = L / E;
    constexpr int H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    CP* sm = reinterpret_cast<CP*>(smraw);
    const int line = threadIdx.x / Cfg::TL;
    const int j = threadIdx.x % Cfg::TL;
    const long long row = (long long)blockIdx.x * Cfg::LINES + line;
    const bool valid = row < rows;
    const long long rw = valid ? row : 0;
    const long long fa = f0 + 4ll * blockIdx.y;  // fields fa .. fa + 3
    // fields of this chunk only: its half spectra hold nchunk fields (a chunk
    // need not be a multiple of four)
    const long long f_end = f0 + nchunk < nfields ? f0 + nchunk : nfields;
    bool has[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) has[q] = fa + q < f_end;
    unsigned long long nsum[4] = {0, 0, 0, 0};
    CP v[E];
    if constexpr (KIND == PK_FLOAT) {
        const float* src[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) src[q] = (const float*)fields + (size_t)(has[q] ? fa + q : fa) * cells + (size_t)rw * L;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int p = j + q * STEP;
            const float a = src[0][p], b = has[1] ? src[1][p] : 0.0f;
            const float c = has[2] ? src[2][p] : 0.0f, d = has[3] ? src[3][p] : 0.0f;
            v[q] = CP{make_float2(a, c), make_float2(b, d)};
        }
    } else {
        const int32_t* src[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            src[q] = (const int32_t*)fields + (size_t)(has[q] ? fa + q : fa) * cells + (size_t)rw * L;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int p = j + q * STEP;
            int32_t n[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) n[k] = has[k] ? src[k][p] : 0;
            if (valid) {
#pragma unroll
                for (int k = 0; k < 4; ++k) nsum[k] += (unsigned long long)(long long)n[k];
            }
            float x[4];
            if (f) {
                const float fi = f[rw * L + p];
#pragma unroll
                for (int k = 0; k < 4; ++k) x[k] = fi != 0.0f ? (float)n[k] / fi : 0.0f;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) x[k] = (float)n[k];
            }
            v[q] = CP{make_float2(x[0], x[2]), make_float2(x[1], x[3])};
        }
        // totals of the block: warp sums, one atomic per block and field
        constexpr int NW = Cfg::THREADS / 32 > 0 ? Cfg::THREADS / 32 : 1;
        __shared__ unsigned long long s_n[4][NW];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) nsum[k] += __shfl_down_sync(0xffffffffu, nsum[k], o);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) s_n[k][threadIdx.x >> 5] = nsum[k];
        __syncthreads();
        if (threadIdx.x < 4 && has[threadIdx.x]) {
            unsigned long long t = 0;
            for (int w = 0; w < NW; ++w) t += s_n[threadIdx.x][w];
            if (t) atomicAdd(&ntot[fa + threadIdx.x], t);
        }
    }
    RowLayout<E, Cfg::PADDED> lay;
    auto to_smem = [&](int ln, int p, CP val) { sm[lay(ln, p)] = val; };
    line_fft_pair<L, -1, L, true>(sm, lay, line, j, v, tw, to_smem);
    __syncthreads();
    if (!valid) return;
    C2<float>* o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = out + ((size_t)(fa + q - f0) * rows + row) * H;
    const float2 half = make_float2(0.5f, 0.5f);
    for (int k = j; k < H; k += Cfg::TL) {
        const CP zk = sm[lay(line, k & (L - 1))];
        const CP zm = sm[lay(line, (L - k) & (L - 1))];
        // lanes: (field fa, fa+2) for the real parts' spectra, (fa+1, fa+3) for the imaginary parts'
        const float2 ar = f2mul(half, f2add(zk.re, zm.re)), ai = f2mul(half, f2sub(zk.im, zm.im));
        const float2 br = f2mul(half, f2add(zk.im, zm.im)), bi = f2mul(half, f2sub(zm.re, zk.re));
        o[0][k] = mk(ar.x, ai.x);
        if (has[1]) o[1][k] = mk(br.x, bi.x);
        if (has[2]) o[2][k] = mk(ar.y, ai.y);
        if (has[3]) o[3][k] = mk(br.y, bi.y);
    }
}

// Binning pass of fields fa = 2 blockIdx.y and fa + 1 of the chunk (no mask
// cross term): the transform along axis 0 of their half spectra, then the
// weighted powers of both, summed per run of equal bins and added to
// shared bins.
template <int L>
__global__ void __launch_bounds__(PkPairCfg<L, CF_PKC2_THREADS>::THREADS, PkPairCfg<L, CF_PKC2_THREADS>::MINB)
    k_pk_cols_pair(const C2<float>* __restrict__ in, long long inner, long long H, long long n_mid, long long n_last,
                   const int16_t* __restrict__ bin_of, long long k2max, int nbins, long long nchunk,
                   double* __restrict__ acc, long long f0, const float4* __restrict__ tw,
                   const int16_t* __restrict__ pbin) {
    using Cfg = PkPairCfg<L, CF_PKC2_THREADS>;
    constexpr int E = Cfg::E;
    constexpr int C = Cfg::LINES;
    extern __shared__ __align__(16) unsigned char smraw[];
    CP* sm = reinterpret_cast<CP*>(smraw);
    float* sbin = reinterpret_cast<float*>(sm + (size_t)C * Cfg::PADDED);  // [2][nbins]
    int* sthr = reinterpret_cast<int*>(sbin + 2 * nbins);
    const int* thr = bin_thresholds(bin_of, k2max);
    for (int b = threadIdx.x; b < 2 * nbins; b += blockDim.x) sbin[b] = 0.0f;
    for (int b = threadIdx.x; b <= nbins; b += blockDim.x) sthr[b] = thr[b];
    const int ln = threadIdx.x % C;
    const int j = threadIdx.x / C;
    const long long i = (long long)blockIdx.x * C + ln;
    const long long oa = 2ll * blockIdx.y, ob = oa + 1;
    const bool valid = i < inner, has_b = ob < nchunk;
    const size_t col = (size_t)(valid ? i : 0);
    const C2<float>* sa = in + (size_t)oa * L * (size_t)inner + col;
    const C2<float>* sb = in + (size_t)(has_b ? ob : oa) * L * (size_t)inner + col;
    CP v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const size_t at = (size_t)(j + q * (L / E)) * (size_t)inner;
        const C2<float> a = sa[at], b = sb[at];
        v[q] = CP{make_float2(a.x, b.x), make_float2(a.y, b.y)};
    }
    ColLayout<E, C> lay;
    auto to_smem = [&](int lnn, int p, CP val) { sm[lay(lnn, p)] = val; };
    line_fft_pair<L, -1, L, true>(sm, lay, ln, j, v, tw, to_smem);
    __syncthreads();
    if (valid && pbin) {
        // this thread's eight consecutive modes p = j E .. j E + 7: their bins
        // in one 16-byte load from the per-mode table
        static_assert(E == 8, "one 16-byte load holds the eight bins of a thread");
        const int il = (int)(i % H);
        const float w = (il == 0 || 2 * (long long)il == n_last) ? 1.0f : 2.0f;
        const float2 ww = make_float2(w, w);
        const uint4 packed = *reinterpret_cast<const uint4*>(pbin + (size_t)i * L + (size_t)j * E);
        const uint32_t words[4] = {packed.x, packed.y, packed.z, packed.w};
        int cur = -1;
        float2 run = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int t = 0; t < E; ++t) {
            const int b = (int)(int16_t)(words[t >> 1] >> (16 * (t & 1)));
            const CP x = sm[lay(ln, j * E + t)];
            if (b != cur) {
                if (cur >= 0) {
                    atomicAdd(&sbin[cur], run.x);
                    atomicAdd(&sbin[nbins + cur], run.y);
                }
                cur = b;
                run = make_float2(0.0f, 0.0f);
            }
            if (b >= 0) run = f2fma(ww, f2fma(x.re, x.re, f2mul(x.im, x.im)), run);
        }
        if (cur >= 0) {
            atomicAdd(&sbin[cur], run.x);
            atomicAdd(&sbin[nbins + cur], run.y);
        }
    } else if (valid) {
        const int il = (int)(i % H);
        const int smid = (int)signed_mode(i / H, n_mid);
        const int c2 = smid * smid + il * il;
        const float w = (il == 0 || 2 * (long long)il == n_last) ? 1.0f : 2.0f;
        const float2 ww = make_float2(w, w);
        const int t_first = sthr[0], t_end = sthr[nbins];
        int cur = -1;
        int lo_t = 0, hi_t = 0;
        float2 run = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int t = 0; t < E; ++t) {
            const int p = j * E + t;
            const CP x = sm[lay(ln, p)];
            const int s0 = p <= L / 2 ? p : p - L;
            const int k2 = s0 * s0 + c2;
            int b = cur;
            if (k2 < lo_t || k2 >= hi_t) {
                if (k2 < t_first || k2 >= t_end) {
                    b = -1;
                    lo_t = hi_t = 0;
                } else {
                    if (cur >= 0) {
                        b = cur;
                        while (k2 >= sthr[b + 1]) ++b;
                        while (k2 < sthr[b]) --b;
                    } else {
                        int lo = 0, hi = nbins;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (sthr[mid] <= k2) lo = mid; else hi = mid;
                        }
                        b = lo;
                    }
                    lo_t = sthr[b];
                    hi_t = sthr[b + 1];
                }
            }
            if (b != cur) {
                if (cur >= 0) {
                    atomicAdd(&sbin[cur], run.x);
                    atomicAdd(&sbin[nbins + cur], run.y);
                }
                cur = b;
                run = make_float2(0.0f, 0.0f);
            }
            if (b >= 0) run = f2fma(ww, f2fma(x.re, x.re, f2mul(x.im, x.im)), run);
        }
        if (cur >= 0) {
            atomicAdd(&sbin[cur], run.x);
            atomicAdd(&sbin[nbins + cur], run.y);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (sbin[b] != 0.0f) atomicAdd(&acc[(size_t)(f0 + oa) * nbins + b], (double)sbin[b]);
        if (has_b && sbin[nbins + b] != 0.0f) atomicAdd(&acc[(size_t)(f0 + ob) * nbins + b], (double)sbin[nbins + b]);
    }
}

// Modes per bin over the full grid, counted on the half spectrum with the
// mirror weights; with a mask spectrum also sum w |DFT I|^2 per bin.
template <typename T>
__global__ void k_pk_nmodes(long long n0, long long n_mid, long long H, long long n_last,
                            const int16_t* __restrict__ bin_of, long long k2max, int nbins,
                            const C2<T>* __restrict__ mask_spec, unsigned long long* __restrict__ nmodes,
                            double* __restrict__ mask_power) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned int* scount = reinterpret_cast<unsigned int*>(smraw);
    double* smask = reinterpret_cast<double*>(scount + ((nbins + 1) & ~1));
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        scount[b] = 0u;
        smask[b] = 0.0;
    }
    __syncthreads();
    const long long inner = n_mid * H;
    const long long total = n0 * inner;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long p = t / inner, i = t - p * inner;
        const long long il = i % H, imid = i / H;
        const long long s0 = signed_mode(p, n0), sm = signed_mode(imid, n_mid);
        const long long k2 = s0 * s0 + sm * sm + il * il;
        const int b = k2 <= k2max ? bin_of[k2] : -1;
        if (b < 0) continue;
        const unsigned int w = (il == 0 || 2 * il == n_last) ? 1u : 2u;
        if (nmodes) atomicAdd(&scount[b], w);
        if (mask_spec) {
            const C2<T> m = mask_spec[t];
            atomicAdd(&smask[b], (double)w * ((double)m.x * m.x + (double)m.y * m.y));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (nmodes && scount[b]) atomicAdd(&nmodes[b], (unsigned long long)scount[b]);
        if (mask_spec && smask[b] != 0.0) atomicAdd(&mask_power[b], smask[b]);
    }
}

// Last pass: FFT along axis 0, then binning from shared memory.  Thread
// (column ln, j) walks the E consecutive k0 of its column; neighbouring k0
// mostly share a bin, so the weighted powers are summed in registers and
// added to the shared bins once per run of equal bins.  With a mask
// spectrum the cross term Re(X conj I) is binned the same way.
template <typename T, int L>
__global__ void __launch_bounds__(PkColsCfg<T, L>::THREADS, PkColsCfg<T, L>::MINB)
    k_pk_cols(const C2<T>* __restrict__ in, long long inner, long long H, long long n_mid, long long n_last,
              const int16_t* __restrict__ bin_of, long long k2max, int nbins, double* __restrict__ acc,
              double* __restrict__ acc_cross, const C2<T>* __restrict__ mask_spec, long long f0,
              const C2<T>* __restrict__ tw) {
    using Cfg = PkColsCfg<T, L>;
    using G = typename Cfg::G;
    constexpr int E = G::E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    T* sbin = reinterpret_cast<T*>(sm + (size_t)Cfg::C * G::PADDED);
    T* scross = sbin + nbins;
    int* sthr = reinterpret_cast<int*>(scross + nbins);
    const int* thr = bin_thresholds(bin_of, k2max);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        sbin[b] = (T)0;
        scross[b] = (T)0;
    }
    for (int b = threadIdx.x; b <= nbins; b += blockDim.x) sthr[b] = thr[b];
    const int ln = threadIdx.x % Cfg::C;
    const int j = threadIdx.x / Cfg::C;
    const long long i = (long long)blockIdx.x * Cfg::C + ln;
    const long long o = blockIdx.y;
    const bool valid = i < inner;
    const C2<T>* src = in + (size_t)o * L * (size_t)inner + (size_t)(valid ? i : 0);
    C2<T> v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = src[(size_t)(j + q * (L / E)) * (size_t)inner];
    ColLayout<E, Cfg::C> lay;
    auto sink = [&](int lnn, int p, C2<T> val) { sm[lay(lnn, p)] = val; };
    line_fft<T, L, -1, L, true>(sm, lay, ln, j, v, tw, sink);
    __syncthreads();
    if (valid) {
        // 32-bit mode arithmetic: k2 <= k2max < 2^31
        const int il = (int)(i % H);
        const int smid = (int)signed_mode(i / H, n_mid);
        const int c2 = smid * smid + il * il;
        const T w = (il == 0 || 2 * (long long)il == n_last) ? (T)1 : (T)2;
        const int t_first = sthr[0], t_end = sthr[nbins];  // (t_first >= 1: the DC mode has no bin)
        int cur = -1;
        int lo_t = 0, hi_t = 0;  // [thr[cur], thr[cur + 1]) while cur >= 0, else empty
        T run = (T)0, runx = (T)0;
#pragma unroll 4
        for (int t = 0; t < E; ++t) {
            const int p = j * E + t;
            const C2<T> x = sm[lay(ln, p)];
            const int s0 = p <= L / 2 ? p : p - L;
            const int k2 = s0 * s0 + c2;
            int b = cur;
            if (k2 < lo_t || k2 >= hi_t) {
                if (k2 < t_first || k2 >= t_end) {
                    b = -1;
                    lo_t = hi_t = 0;
                } else {
                    if (cur >= 0) {
                        // neighbouring modes sit in the same or a nearby bin
                        b = cur;
                        while (k2 >= sthr[b + 1]) ++b;
                        while (k2 < sthr[b]) --b;
                    } else {
                        int lo = 0, hi = nbins;  // sthr[lo] <= k2 < sthr[hi]
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (sthr[mid] <= k2) lo = mid; else hi = mid;
                        }
                        b = lo;
                    }
                    lo_t = sthr[b];
                    hi_t = sthr[b + 1];
                }
            }
            if (b != cur) {
                if (cur >= 0) {
                    atomicAdd(&sbin[cur], run);
                    if (mask_spec) atomicAdd(&scross[cur], runx);
                }
                cur = b;
                run = (T)0;
                runx = (T)0;
            }
            if (b >= 0) {
                run += w * (x.x * x.x + x.y * x.y);
                if (mask_spec) {
                    const C2<T> m = mask_spec[(size_t)p * inner + i];
                    runx += w * (x.x * m.x + x.y * m.y);
                }
            }
        }
        if (cur >= 0) {
            atomicAdd(&sbin[cur], run);
            if (mask_spec) atomicAdd(&scross[cur], runx);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const size_t at = (size_t)(f0 + o) * nbins + b;
        if (sbin[b] != (T)0) atomicAdd(&acc[at], (double)sbin[b]);
        if (mask_spec && scross[b] != (T)0) atomicAdd(&acc_cross[at], (double)scross[b]);
    }
}

// pk = cell^d/(prod n) * S/N_b; for count maps S = acc/Nhat^2 - 2 cross/Nhat + mask_power
// with Nhat = N_tot/sum f (0 when there are no counts).
__global__ void k_pk_finalize(const double* __restrict__ acc, const double* __restrict__ acc_cross,
                              const double* __restrict__ mask_power, const unsigned long long* __restrict__ ntot,
                              const double* __restrict__ fsum_dev, double fsum_host,
                              const unsigned long long* __restrict__ nmodes, long long nfields, int nbins,
                              double volfac, double* __restrict__ pk, int64_t* __restrict__ nmodes_out) {
    const long long total = nfields * nbins;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(idx % nbins);
        const long long fld = idx / nbins;
        const unsigned long long nm = nmodes[b];
        double S = acc[idx];
        if (ntot) {
            const double fsum = fsum_dev ? fsum_dev[0] : fsum_host;
            const double nhat = fsum > 0.0 ? (double)ntot[fld] / fsum : 0.0;
            if (nhat > 0.0) {
                S = S / (nhat * nhat);
                if (acc_cross) S += -2.0 * acc_cross[idx] / nhat + mask_power[b];
            } else {
                S = 0.0;
            }
        }
        pk[idx] = nm ? volfac * S / (double)nm : 0.0;
        if (idx < nbins && nmodes_out) nmodes_out[idx] = (int64_t)nmodes[idx];
    }
}

// mean over fields: one block per bin, threads over fields
__global__ void k_pk_mean(const double* __restrict__ pk, long long nfields, int nbins, double* __restrict__ mean) {
    __shared__ double sh[256];
    const int b = blockIdx.x;
    double s = 0.0;
    for (long long f = threadIdx.x; f < nfields; f += blockDim.x) s += pk[f * nbins + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[b] = nfields > 0 ? sh[0] / (double)nfields : 0.0;
}

// unbiased covariance: one warp per bin pair (a, b >= a), blockIdx.y = a and
// warp blockIdx.x * 8 + w gives b - a; lanes over fields with a warp-shuffle
// sum (short dependent chains: binary64 latency is long on this part)
__global__ void __launch_bounds__(256) k_pk_cov(const double* __restrict__ pk, const double* __restrict__ mean,
                                                long long nfields, int nbins, double* __restrict__ cov) {
    const int a = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double ma = mean[a];
    const int b = a + (int)blockIdx.x * 8 + warp;
    if (b < nbins) {
        const double mb = mean[b];
        double s = 0.0;
        for (long long f = lane; f < nfields; f += 32) s += (pk[f * nbins + a] - ma) * (pk[f * nbins + b] - mb);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double c = nfields > 1 ? s / (double)(nfields - 1) : 0.0;
            cov[(size_t)a * nbins + b] = c;
            cov[(size_t)b * nbins + a] = c;
        }
    }
}

// ----------------------------------------------------------------- host side
// Bin edges e[0..nbins] of a cf_bins (kmax <= 0: kmax_default).
cf_status pk_bin_edges(const cf_bins* b, double kmax_default, double* e) {
    const double kmax = b->kmax > 0.0 ? b->kmax : kmax_default;
    const double kmin = b->kmin;
    for (int i = 0; i <= b->nbins; ++i) {
        if (b->kind == CF_BINS_LINEAR)
            e[i] = kmin + (double)i * ((kmax - kmin) / (double)b->nbins);
        else if (b->kind == CF_BINS_LOG) {
            if (!(kmin > 0.0)) return fail(CF_ERR_ARG, "log bins need kmin > 0");
            e[i] = kmin * exp((double)i * (log(kmax / kmin) / (double)b->nbins));
        } else if (b->kind == CF_BINS_EDGES) {
            if (!b->edges) return fail(CF_ERR_ARG, "CF_BINS_EDGES needs edges");
            e[i] = b->edges[i];
        } else
            return fail(CF_ERR_ARG, "unknown bins kind %d", b->kind);
        if (i > 0 && !(e[i] > e[i - 1])) return fail(CF_ERR_ARG, "bin edges must increase");
    }
    return CF_OK;
}

// pk = volfac * acc / N_b per field and bin, then the mean and unbiased
// covariance over fields (scratch: nbins doubles for the mean when only the
// covariance is wanted).
cf_status pk_finish(const double* acc, const unsigned long long* nmodes, long long nfields, int nbins,
                    double volfac, double* pk_out, int64_t* nmodes_out, double* mean, double* cov, double* scratch,
                    cudaStream_t s);

struct PkPlan {
    GridInfo g;         // survey grid (n used as the transform sizes)
    int nbins;
    Edges edges;
    long long k2max;
    long long H;        // n_last/2 + 1
    long long rows;     // prod of leading axes
    size_t elem;
    long long chunk;    // fields per chunk (even)
    size_t off_bin, off_nmodes, off_acc, off_cross, off_mpow, off_ntot, off_fsum, off_mask, off_half, total;
};

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static cf_status make_plan(const cf_grid* grid, long long nfields, const cf_bins* b, size_t elem, PkPlan* P) {
    if (!grid) return fail(CF_ERR_ARG, "grid is NULL");
    if (!b) return fail(CF_ERR_ARG, "bins is NULL");
    if (grid->ndim < 2 || grid->ndim > 3)
        return fail(grid->ndim == 1 ? CF_ERR_UNSUPPORTED : CF_ERR_ARG, "power spectrum needs ndim 2 or 3");
    GridInfo& g = P->g;
    g.ndim = grid->ndim;
    g.ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < g.ndim) {
            g.n[a] = grid->n[a];
            g.cell[a] = grid->cell[a];
            if (g.n[a] < 2 || !is_pow2(g.n[a]) || g.n[a] > kMaxLine)
                return fail(CF_ERR_UNSUPPORTED, "power spectrum needs power-of-two sizes 2..%lld (n[%d] = %lld)",
                            kMaxLine, a, g.n[a]);
            if (g.n[a] != grid->n[0]) return fail(CF_ERR_UNSUPPORTED, "power spectrum needs equal sizes on all axes");
            if (!(g.cell[a] > 0.0)) return fail(CF_ERR_ARG, "cell must be > 0");
        } else {
            g.n[a] = 1;
            g.cell[a] = 1.0;
        }
        g.m[a] = g.n[a];
        g.ncell *= g.n[a];
    }
    g.mtotal = g.ncell;
    if (b->nbins < 1 || b->nbins > kMaxBins) return fail(CF_ERR_ARG, "nbins must be 1..%d", kMaxBins);
    P->nbins = b->nbins;
    CF_TRY(pk_bin_edges(b, (double)(g.n[0] / 2), P->edges.e));
    P->k2max = 0;
    for (int a = 0; a < g.ndim; ++a) P->k2max += (g.n[a] / 2) * (g.n[a] / 2);
    const long long nl = g.n[g.ndim - 1];
    P->H = nl / 2 + 1;
    P->rows = g.ncell / nl;
    P->elem = elem;
    const size_t per_field = elem * (size_t)P->rows * (size_t)P->H;
    static const size_t target = [] {
        const char* e = getenv("CF_PK_CHUNK_MB");  // half spectra per chunk (measured: large is faster)
        long mb = e ? atol(e) : 1024;
        return (size_t)(mb < 1 ? 1 : mb) << 20;
    }();
    long long chunk = (long long)(target / (per_field ? per_field : 1));
    if (chunk < 2) chunk = 2;
    chunk &= ~1ll;
    if (chunk > 65534) chunk = 65534;
    const long long nf_even = (nfields + 1) & ~1ll;
    if (chunk > nf_even) chunk = nf_even < 2 ? 2 : nf_even;
    P->chunk = chunk;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    P->off_bin = take(bin_table_bytes(P->k2max));
    P->off_nmodes = take(sizeof(unsigned long long) * P->nbins);
    P->off_acc = take(sizeof(double) * (size_t)nfields * P->nbins);
    P->off_cross = take(sizeof(double) * (size_t)nfields * P->nbins);
    P->off_mpow = take(sizeof(double) * P->nbins);
    P->off_ntot = take(sizeof(unsigned long long) * (size_t)nfields);
    P->off_fsum = take(sizeof(double));
    P->off_mask = take(per_field);
    P->off_half = take(per_field * (size_t)chunk);
    P->total = o;
    return CF_OK;
}

// Bin tables and mode counts depend only on (device, grid, edges): they are
// built once per key on the first call's stream and kept for the life of the
// process (at most kBinCacheMax keys; beyond that they are rebuilt per call
// in the workspace).  Later calls on other streams wait on the build event.
struct BinCacheEntry {
    int device;
    int ndim;
    long long n0;
    int nbins;
    std::vector<double> edges;
    int16_t* bin_of;
    unsigned long long* nmodes;
    int16_t* pbin;  // bin of every (half-spectrum column, axis-0 mode), or null
    cudaEvent_t ready;
};
constexpr size_t kBinCacheMax = 32;
static std::mutex g_bin_mu;
static std::vector<BinCacheEntry> g_bin_cache;

static cf_status build_bins(const PkPlan& P, int16_t* bin_of, unsigned long long* nmodes, cudaStream_t s) {
    const GridInfo& g = P.g;
    const int d = g.ndim;
    const long long n_mid = d == 3 ? g.n[1] : 1;
    const long long inner = n_mid * P.H;
    k_pk_bintable<<<grid_blocks(P.k2max + 1, 256, 1024), 256, 0, s>>>(P.edges, P.nbins, P.k2max, bin_of);
    k_pk_thresholds<<<(P.nbins + 1 + 127) / 128, 128, 0, s>>>(P.edges, P.nbins, P.k2max,
                                                           const_cast<int*>(bin_thresholds(bin_of, P.k2max)));
    CF_CUDA(cudaMemsetAsync(nmodes, 0, sizeof(unsigned long long) * P.nbins, s));
    const size_t smem = (size_t)((P.nbins + 1) & ~1) * sizeof(unsigned int) + (size_t)P.nbins * sizeof(double);
    k_pk_nmodes<float><<<grid_blocks(g.n[0] * inner, 256, 256), 256, smem, s>>>(
        g.n[0], n_mid, P.H, g.n[d - 1], bin_of, P.k2max, P.nbins, nullptr, nmodes, nullptr);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// The bin of every mode the paired binning pass visits: pbin[i n0 + p] for
// half-spectrum column i (3D: axis-1 mode i / H, last-axis mode i % H) and
// axis-0 mode p, from bin_of (-1: no bin).  The pass then reads a thread's
// eight bins with one 16-byte load instead of searching the thresholds per
// mode.
__global__ void k_pk_pbin(long long n0, long long n_mid, long long H, const int16_t* __restrict__ bin_of,
                          long long k2max, int16_t* __restrict__ pbin) {
    const long long total = n_mid * H * n0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / n0, p = e - i * n0;
        const long long il = i % H, sm = signed_mode(i / H, n_mid), s0 = signed_mode(p, n0);
        const long long k2 = s0 * s0 + sm * sm + il * il;
        pbin[e] = k2 <= k2max ? bin_of[k2] : (int16_t)-1;
    }
}

// pbin tables up to this size (bytes) are kept with the cached bins
constexpr size_t kPbinMaxBytes = (size_t)32 << 20;

// Returns the cached tables for P (building them on stream s if needed), or
// the workspace copies when the cache is full (then without pbin).
static cf_status get_bins(const PkPlan& P, char* ws, cudaStream_t s, const int16_t** bin_of,
                          const unsigned long long** nmodes, const int16_t** pbin = nullptr) {
    if (pbin) *pbin = nullptr;
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    std::vector<double> edges(P.edges.e, P.edges.e + P.nbins + 1);
    std::lock_guard<std::mutex> lk(g_bin_mu);
    for (auto& c : g_bin_cache) {
        if (c.device == dev && c.ndim == P.g.ndim && c.n0 == P.g.n[0] && c.nbins == P.nbins && c.edges == edges) {
            // a capturing stream may only wait on an event from outside the
            // capture as an external dependency (an event-wait node)
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CF_CUDA(cudaStreamIsCapturing(s, &cs));
            CF_CUDA(cudaStreamWaitEvent(s, c.ready, cs == cudaStreamCaptureStatusNone ? 0 : cudaEventWaitExternal));
            *bin_of = c.bin_of;
            *nmodes = c.nmodes;
            if (pbin) *pbin = c.pbin;
            return CF_OK;
        }
    }
    if (g_bin_cache.size() >= kBinCacheMax) {
        int16_t* b = (int16_t*)(ws + P.off_bin);
        unsigned long long* nm = (unsigned long long*)(ws + P.off_nmodes);
        CF_TRY(build_bins(P, b, nm, s));
        *bin_of = b;
        *nmodes = nm;
        return CF_OK;
    }
    BinCacheEntry c{dev, P.g.ndim, P.g.n[0], P.nbins, edges, nullptr, nullptr, nullptr, nullptr};
    CF_CUDA(cudaMalloc((void**)&c.bin_of, bin_table_bytes(P.k2max)));
    CF_CUDA(cudaMalloc((void**)&c.nmodes, sizeof(unsigned long long) * P.nbins));
    CF_CUDA(cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming));
    CF_TRY(build_bins(P, c.bin_of, c.nmodes, s));
    const long long n_mid = P.g.ndim == 3 ? P.g.n[1] : 1;
    const size_t pbin_bytes = sizeof(int16_t) * (size_t)n_mid * (size_t)P.H * (size_t)P.g.n[0];
    if (P.g.ndim >= 2 && pbin_bytes <= kPbinMaxBytes) {
        CF_CUDA(cudaMalloc((void**)&c.pbin, pbin_bytes));
        k_pk_pbin<<<grid_blocks((long long)(pbin_bytes / sizeof(int16_t)), 256, 2048), 256, 0, s>>>(
            P.g.n[0], n_mid, P.H, c.bin_of, P.k2max, c.pbin);
        CF_CHECK_LAUNCH();
    }
    CF_CUDA(cudaEventRecord(c.ready, s));
    g_bin_cache.push_back(c);
    *bin_of = c.bin_of;
    *nmodes = c.nmodes;
    if (pbin) *pbin = c.pbin;
    return CF_OK;
}

template <typename T, int L>
static cf_status launch_pk_rows(const void* fields, int kind, const float* f, unsigned long long* ntot,
                                double* fsum, const PkPlan& P, long long nfields, long long f0, long long nchunk,
                                C2<T>* out, cudaStream_t s) {
    using Cfg = PkRowsCfg<T, L>;
    using Kern = decltype(&k_pk_rows<T, L, sizeof(T) == 8 ? PK_DOUBLE : PK_FLOAT>);
    Kern kern = nullptr;
    if constexpr (sizeof(T) == 8) {
        if (kind == PK_DOUBLE) kern = k_pk_rows<T, L, PK_DOUBLE>;
    } else {
        if (kind == PK_FLOAT) kern = k_pk_rows<T, L, PK_FLOAT>;
        else if (kind == PK_COUNTS) kern = k_pk_rows<T, L, PK_COUNTS>;
        else if (kind == PK_MASK) kern = k_pk_rows<T, L, PK_MASK>;
    }
    if (!kern) return fail(CF_ERR_UNSUPPORTED, "power-spectrum input kind %d with this precision", kind);
    CF_TRY(prepare_smem(kern, Cfg::SMEM));
    dim3 grid((unsigned)((P.rows + Cfg::ROWS - 1) / Cfg::ROWS), (unsigned)((nchunk + 1) / 2));
    ScopedKernelTimer kt(s, sizeof(T) == 4 ? "pk_rows_f32" : "pk_rows_f64", L);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(fields, kind, f, ntot, fsum, P.rows, P.g.ncell, nfields, f0, out,
                                               twiddles<T>());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

template <typename T, int L>
static cf_status launch_pk_cols(const C2<T>* in, long long inner, long long n_mid, const PkPlan& P,
                                const int16_t* bin_of, double* acc, double* cross, const C2<T>* mask_spec, long long f0,
                                long long nchunk, cudaStream_t s) {
    using Cfg = PkColsCfg<T, L>;
    auto kern = k_pk_cols<T, L>;
    const size_t smem = Cfg::SMEM + 2 * sizeof(T) * (size_t)P.nbins + sizeof(int) * (size_t)(P.nbins + 1);
    CF_TRY(prepare_smem(kern, smem));
    dim3 grid((unsigned)((inner + Cfg::C - 1) / Cfg::C), (unsigned)nchunk);
    ScopedKernelTimer kt(s, sizeof(T) == 4 ? "pk_cols_f32" : "pk_cols_f64", L);
    kern<<<grid, Cfg::THREADS, smem, s>>>(in, inner, P.H, n_mid, P.g.n[P.g.ndim - 1], bin_of, P.k2max, P.nbins, acc,
                                          cross, mask_spec, f0, twiddles<T>());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// The paired binary32 row and binning passes (off with CF_PK_PAIR=0 in the
// environment); the masked count maps' cross term keeps the one-line kernels.
static bool pk_pair() {
    static const bool on = [] {
        const char* e = getenv("CF_PK_PAIR");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <int L>
static cf_status launch_pk_rows_pair(const void* fields, int kind, const float* f, unsigned long long* ntot,
                                     const PkPlan& P, long long nfields, long long f0, long long nchunk,
                                     C2<float>* out, cudaStream_t s) {
    using Cfg = PkPairCfg<L, CF_PKR2_THREADS>;
    auto kern = kind == PK_COUNTS ? k_pk_rows_pair<L, PK_COUNTS> : k_pk_rows_pair<L, PK_FLOAT>;
    CF_TRY(prepare_smem(kern, Cfg::SMEM));
    dim3 grid((unsigned)((P.rows + Cfg::LINES - 1) / Cfg::LINES), (unsigned)((nchunk + 3) / 4));
    ScopedKernelTimer kt(s, "pk_rows_f32", L);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(fields, f, ntot, P.rows, P.g.ncell, nfields, f0, nchunk, out,
                                               twiddles_f32x2());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

template <int L>
static cf_status launch_pk_cols_pair(const C2<float>* in, long long inner, long long n_mid, const PkPlan& P,
                                     const int16_t* bin_of, double* acc, long long f0, long long nchunk,
                                     cudaStream_t s, const int16_t* pbin) {
    using Cfg = PkPairCfg<L, CF_PKC2_THREADS>;
    auto kern = k_pk_cols_pair<L>;
    const size_t smem = Cfg::SMEM + 2 * sizeof(float) * (size_t)P.nbins + sizeof(int) * (size_t)(P.nbins + 1);
    CF_TRY(prepare_smem(kern, smem));
    dim3 grid((unsigned)((inner + Cfg::LINES - 1) / Cfg::LINES), (unsigned)((nchunk + 1) / 2));
    ScopedKernelTimer kt(s, "pk_cols_f32", L);
    kern<<<grid, Cfg::THREADS, smem, s>>>(in, inner, P.H, n_mid, P.g.n[P.g.ndim - 1], bin_of, P.k2max, P.nbins,
                                          nchunk, acc, f0, twiddles_f32x2(), pbin);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// Transform along the remaining axes of half spectra [nc][rows][H] in place
// except the first axis (3D: axis 1).
template <typename T>
static cf_status pk_middle_axis(const PkPlan& P, C2<T>* half, long long nc, cudaStream_t s) {
    if (P.g.ndim != 3) return CF_OK;
    FieldEpi<T> none{};
    return launch_cols<T, -1, 0>(P.g.n[1], half, nc * P.g.n[0], P.H, half, 0, none, s);
}

template <typename T>
static cf_status pk_impl(const void* fields, int kind, const float* f, const PkPlan& P, long long nfields,
                         double* pk_out, int64_t* nmodes_out, double* mean, double* cov, char* ws, cudaStream_t s) {
    const GridInfo& g = P.g;
    const int16_t* bin_of = nullptr;
    const int16_t* pbin = nullptr;
    const unsigned long long* nmodes = nullptr;
    double* acc = (double*)(ws + P.off_acc);
    double* cross = (double*)(ws + P.off_cross);
    double* mpow = (double*)(ws + P.off_mpow);
    unsigned long long* ntot = (unsigned long long*)(ws + P.off_ntot);
    double* fsum = (double*)(ws + P.off_fsum);
    C2<T>* mask_spec = (C2<T>*)(ws + P.off_mask);
    C2<T>* half = (C2<T>*)(ws + P.off_half);
    const bool counts = kind == PK_COUNTS;
    const bool masked = counts && f != nullptr;
    const int d = g.ndim;
    const long long nl = g.n[d - 1];
    const long long inner = (d == 3 ? g.n[1] : 1) * P.H;
    const long long n_mid = d == 3 ? g.n[1] : 1;
    {
        ScopedKernelTimer kt(s, "pk_setup");
        CF_TRY(get_bins(P, ws, s, &bin_of, &nmodes, &pbin));
        // zero the accumulators (acc .. mask spectrum)
        CF_CUDA(cudaMemsetAsync(ws + P.off_acc, 0, P.off_half - P.off_acc, s));
    }
    CF_CHECK_LAUNCH();
    if (masked) {
        // spectrum of the unmasked-cell indicator (and sum f) through the same passes
        CF_TRY(dispatch_line(nl, [&](auto Lc) -> cf_status {
            return launch_pk_rows<T, decltype(Lc)::value>(nullptr, PK_MASK, f, ntot, fsum, P, 1, 0, 1, mask_spec, s);
        }));
        CF_TRY(pk_middle_axis<T>(P, mask_spec, 1, s));
        FieldEpi<T> none{};
        CF_TRY((launch_cols<T, -1, 0>(g.n[0], mask_spec, 1, inner, mask_spec, 0, none, s)));
    }
    if (masked) {
        ScopedKernelTimer kt(s, "pk_setup");
        const size_t smem = (size_t)((P.nbins + 1) & ~1) * sizeof(unsigned int) + (size_t)P.nbins * sizeof(double);
        k_pk_nmodes<T><<<grid_blocks(g.n[0] * inner, 256, 256), 256, smem, s>>>(
            g.n[0], n_mid, P.H, nl, bin_of, P.k2max, P.nbins, mask_spec, nullptr, mpow);
    }
    CF_CHECK_LAUNCH();
    const bool paired = sizeof(T) == 4 && pk_pair() && (kind == PK_FLOAT || kind == PK_COUNTS);
    for (long long f0 = 0; f0 < nfields; f0 += P.chunk) {
        const long long nc = (nfields - f0) < P.chunk ? (nfields - f0) : P.chunk;
        CF_TRY(dispatch_line(nl, [&](auto Lc) -> cf_status {
            constexpr int LL = decltype(Lc)::value;
            if constexpr (sizeof(T) == 4 && LL >= 16) {
                if (paired)
                    return launch_pk_rows_pair<LL>(fields, kind, f, ntot, P, nfields, f0, nc, (C2<float>*)half, s);
            }
            return launch_pk_rows<T, LL>(fields, kind, f, ntot, fsum, P, nfields, f0, nc, half, s);
        }));
        CF_TRY(pk_middle_axis<T>(P, half, nc, s));
        CF_TRY(dispatch_line(g.n[0], [&](auto Lc) -> cf_status {
            constexpr int LL = decltype(Lc)::value;
            if constexpr (sizeof(T) == 4 && LL >= 16) {
                if (paired && !masked)
                    return launch_pk_cols_pair<LL>((const C2<float>*)half, inner, n_mid, P, bin_of, acc, f0, nc, s,
                                                   LL == g.n[0] ? pbin : nullptr);
            }
            return launch_pk_cols<T, LL>(half, inner, n_mid, P, bin_of, acc, masked ? cross : nullptr,
                                         masked ? mask_spec : nullptr, f0, nc, s);
        }));
    }
    double volfac = 1.0;
    for (int a = 0; a < d; ++a) volfac *= g.cell[a] / (double)g.n[a];
    {
        ScopedKernelTimer kt(s, "pk_finalize");
        k_pk_finalize<<<grid_blocks(nfields * P.nbins, 256, 1024), 256, 0, s>>>(
            acc, masked ? cross : nullptr, mpow, counts ? ntot : nullptr, masked ? fsum : nullptr, (double)g.ncell,
            nmodes, nfields, P.nbins, volfac, pk_out, nmodes_out);
        if (mean || cov) {
            double* mu = mean ? mean : cross;  // scratch when only the covariance is wanted
            k_pk_mean<<<P.nbins, 256, 0, s>>>(pk_out, nfields, P.nbins, mu);
            if (cov) k_pk_cov<<<dim3((P.nbins + 7) / 8, P.nbins), 256, 0, s>>>(pk_out, mu, nfields, P.nbins, cov);
        }
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// Spectra of F real fields of a 2D square grid whose transform along one
// axis is done already (the sampler's fused column pass): half[F][n][n/2+1],
// the transformed axis last.  The binning pass transforms the other axis and
// bins with the mirror weights of the half axis (k^2 is symmetric in the two
// axes), then the final pass, mean and covariance.  acc_ws holds
// pk_halves_acc_bytes() bytes.
size_t pk_halves_acc_bytes(const cf_grid* grid, long long F, const cf_bins* bins) {
    PkPlan P;
    if (make_plan(grid, F, bins, sizeof(C2<float>), &P) != CF_OK) return 0;
    return align256(P.off_half);
}

cf_status pk_from_halves_f32(const cf_grid* grid, long long F, const cf_bins* bins, const C2<float>* half,
                             double* pk_out, int64_t* nmodes_out, double* mean, double* cov, char* acc_ws,
                             cudaStream_t s) {
    PkPlan P;
    CF_TRY(make_plan(grid, F, bins, sizeof(C2<float>), &P));
    if (P.g.ndim != 2) return fail(CF_ERR_UNSUPPORTED, "fused spectra are 2D");
    const int16_t* bin_of = nullptr;
    const unsigned long long* nmodes = nullptr;
    double* acc = (double*)(acc_ws + P.off_acc);
    double* mpow = (double*)(acc_ws + P.off_mpow);
    {
        ScopedKernelTimer kt(s, "pk_setup");
        CF_TRY(get_bins(P, acc_ws, s, &bin_of, &nmodes));
        CF_CUDA(cudaMemsetAsync(acc_ws + P.off_acc, 0, P.off_half - P.off_acc, s));
    }
    CF_TRY(dispatch_line(P.g.n[0], [&](auto Lc) -> cf_status {
        return launch_pk_cols<float, decltype(Lc)::value>(half, P.H, 1, P, bin_of, acc, nullptr, nullptr, 0, F, s);
    }));
    const double volfac = P.g.cell[0] / (double)P.g.n[0] * P.g.cell[1] / (double)P.g.n[1];
    {
        ScopedKernelTimer kt(s, "pk_finalize");
        k_pk_finalize<<<grid_blocks(F * P.nbins, 256, 1024), 256, 0, s>>>(acc, nullptr, mpow, nullptr, nullptr,
                                                                          (double)P.g.ncell, nmodes, F, P.nbins,
                                                                          volfac, pk_out, nmodes_out);
        if (mean || cov) {
            double* mu = mean ? mean : (double*)(acc_ws + P.off_cross);
            k_pk_mean<<<P.nbins, 256, 0, s>>>(pk_out, F, P.nbins, mu);
            if (cov) k_pk_cov<<<dim3((P.nbins + 7) / 8, P.nbins), 256, 0, s>>>(pk_out, mu, F, P.nbins, cov);
        }
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}

cf_status pk_finish(const double* acc, const unsigned long long* nmodes, long long nfields, int nbins,
                    double volfac, double* pk_out, int64_t* nmodes_out, double* mean, double* cov, double* scratch,
                    cudaStream_t s) {
    ScopedKernelTimer kt(s, "pk_finalize");
    k_pk_finalize<<<grid_blocks(nfields * nbins, 256, 1024), 256, 0, s>>>(acc, nullptr, nullptr, nullptr, nullptr, 1.0,
                                                                          nmodes, nfields, nbins, volfac, pk_out,
                                                                          nmodes_out);
    if (mean || cov) {
        double* mu = mean ? mean : scratch;
        k_pk_mean<<<nbins, 256, 0, s>>>(pk_out, nfields, nbins, mu);
        if (cov) k_pk_cov<<<dim3((nbins + 7) / 8, nbins), 256, 0, s>>>(pk_out, mu, nfields, nbins, cov);
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// Mean over rows and unbiased covariance of x [nrows][ncols] (binary64); used
// for the power spectra and for the counts-in-cells histograms.
cf_status launch_mean_cov(const double* x, long long nrows, int ncols, double* mean, double* cov, cudaStream_t s) {
    if (!mean && !cov) return CF_OK;
    double* mu = mean;
    if (!mu && pool_malloc((void**)&mu, sizeof(double) * (size_t)ncols, s) != cudaSuccess)
        return fail(CF_ERR_NOMEM, "scratch for the mean failed");
    k_pk_mean<<<ncols, 256, 0, s>>>(x, nrows, ncols, mu);
    if (cov) k_pk_cov<<<dim3((ncols + 7) / 8, ncols), 256, 0, s>>>(x, mu, nrows, ncols, cov);
    if (!mean) cudaFreeAsync(mu, s);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

}  // namespace cf

using namespace cf;

extern "C" cf_status cf_power_spectrum_workspace_size(const cf_grid* g, int64_t nfields, const cf_bins* b, cf_dtype dt,
                                                      size_t* bytes) {
    clear_error();
    if (!bytes) return fail(CF_ERR_ARG, "bytes is NULL");
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d", dt);
    if (pk_any_needed(g)) return pk_any_workspace(g, nfields, b, dt, bytes);
    PkPlan P;
    CF_TRY(make_plan(g, nfields, b, dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>), &P));
    *bytes = P.total;
    return CF_OK;
}

static cf_status pk_common(const void* fields, int kind, cf_dtype dt, const float* f, const cf_grid* g, int64_t nfields,
                           const cf_bins* bins, double* pk_out, int64_t* nmodes_out, double* mean, double* cov,
                           void* ws, size_t ws_bytes, cf_stream_t s) {
    clear_error();
    if (!fields || !pk_out) return fail(CF_ERR_ARG, "fields and pk_out are required");
    if (nfields < 1) return fail(CF_ERR_ARG, "nfields must be >= 1");
    if (nfields > 65535) return fail(CF_ERR_UNSUPPORTED, "at most 65535 fields per call");
    if (pk_any_needed(g)) {
        CF_TRY(enter((cudaStream_t)s));
        const int any_kind = kind == PK_COUNTS ? 2 : (dt == CF_F64 ? 1 : 0);
        return pk_any_run(fields, any_kind, f, g, nfields, bins, pk_out, nmodes_out, mean, cov, ws, ws_bytes,
                          (cudaStream_t)s);
    }
    const size_t elem = dt == CF_F64 ? sizeof(C2<double>) : sizeof(C2<float>);
    PkPlan P;
    CF_TRY(make_plan(g, nfields, bins, elem, &P));
    if (!ws || ws_bytes < P.total) return fail(CF_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, P.total);
    CF_TRY(enter((cudaStream_t)s));
    if (dt == CF_F64)
        return pk_impl<double>(fields, kind, f, P, nfields, pk_out, nmodes_out, mean, cov, (char*)ws, (cudaStream_t)s);
    return pk_impl<float>(fields, kind, f, P, nfields, pk_out, nmodes_out, mean, cov, (char*)ws, (cudaStream_t)s);
}

extern "C" cf_status cf_power_spectrum(const void* fields, cf_dtype dt, const cf_grid* g, int64_t nfields,
                                       const cf_bins* bins, double* pk_out, int64_t* nmodes_out, double* mean_or_null,
                                       double* cov_or_null, void* ws, size_t ws_bytes, cf_stream_t s) {
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d", dt);
    return pk_common(fields, dt == CF_F32 ? PK_FLOAT : PK_DOUBLE, dt, nullptr, g, nfields, bins, pk_out, nmodes_out,
                     mean_or_null, cov_or_null, ws, ws_bytes, s);
}

extern "C" cf_status cf_power_spectrum_counts(const int32_t* counts, const float* f_or_null, const cf_grid* g,
                                              int64_t nfields, const cf_bins* bins, double* pk_out,
                                              int64_t* nmodes_out, double* mean_or_null, double* cov_or_null,
                                              void* ws, size_t ws_bytes, cf_stream_t s) {
    return pk_common(counts, PK_COUNTS, CF_F32, f_or_null, g, nfields, bins, pk_out, nmodes_out, mean_or_null,
                     cov_or_null, ws, ws_bytes, s);
}
