// cf_kernels.cuh -- transform-pass kernels shared by the embedding, the
// sampler and the power spectrum, and the compile-time dispatch over the line
// length.
#pragma once
#include <stdio.h>

#include <type_traits>
#include <utility>

#include "cf_fft.cuh"
#include "cf_internal.h"

namespace cf {

// --------------------------------------------------------------------------
// Fused field epilogue of the last inverse-transform pass: split W into the
// Re/Im fields and (binary32) apply the lognormal transform and the Poisson
// draw of section 3.1 to both fields of the survey cell.
// --------------------------------------------------------------------------
// Per-realization parameters of a batched launch (realizations of several
// requests of one grid shape in one launch): the request's amplitudes, noise
// key and realization index, its output arrays and lognormal/Poisson step.
struct RealDesc {
    const float* s;         // sqrt(lambda+/M^d) of the request's embedding (amplitude 1)
    float* fields;          // [2][cells] of this realization
    int32_t* counts;        // [2][cells] or null
    double half_sigma2, nbar;
    float amp_scale;        // sqrt(amp)
    float half_sigma2_f, nbar_f;
    uint32_t r;             // realization index (noise counter and Poisson field pair)
    uint32_t key0, key1;    // noise key
    uint32_t pkey0, pkey1;  // Poisson key
};

template <typename T>
struct FieldEpi {
    T* fields;          // [chunk][2][cells] or null
    int32_t* counts;    // [chunk][2][cells] or null (no lognormal/Poisson step)
    float* delta;       // [chunk][2][cells] or null
    const float* f;     // [cells] or null (f = 1)
    double half_sigma2;
    float half_sigma2_f;
    double nbar;
    float nbar_f;
    uint32_t pkey0, pkey1;
    uint32_t r0;        // global index of the chunk's first realization
    long long cells;
    const RealDesc* desc;  // batched launch: per-realization parameters (else null)
    PoissonDefer defer;    // inconclusive binary32 decisions (null items: decide in place)

    __device__ __forceinline__ int32_t count(int32_t* dst, float G, double half_sigma2_d, float half_sigma2_ff,
                                             double nbar_d, float nbar_ff, float fi, unsigned long long ub) const {
        const int j = poisson_count_try(G, half_sigma2_ff, nbar_ff, fi, ub);
        return j >= 0 ? j : poisson_defer(defer, dst, G, half_sigma2_d, nbar_d, fi, ub);
    }

    __device__ __forceinline__ void operator()(int rl, long long cell, C2<T> w) const {
        if (desc) {
            batched(desc[rl], cell, w);
            return;
        }
        const size_t base = (size_t)rl * 2 * (size_t)cells + (size_t)cell;
        if (fields) {
            fields[base] = w.x;
            fields[base + cells] = w.y;
        }
        if (counts) {
            const float g0 = (float)w.x, g1 = (float)w.y;
            const uint4 x = poisson_words((unsigned long long)cell, r0 + (uint32_t)rl, pkey0, pkey1);
            const float fi = f ? f[cell] : 1.0f;
            counts[base] = count(counts + base, g0, half_sigma2, half_sigma2_f, nbar, nbar_f, fi, bits53(x.x, x.y));
            counts[base + cells] =
                count(counts + base + cells, g1, half_sigma2, half_sigma2_f, nbar, nbar_f, fi, bits53(x.z, x.w));
            if (delta) {
                delta[base] = expf(g0 - half_sigma2_f) - 1.0f;
                delta[base + cells] = expf(g1 - half_sigma2_f) - 1.0f;
            }
        }
    }

    __device__ __forceinline__ void batched(const RealDesc& d, long long cell, C2<T> w) const {
        const float g0 = (float)w.x, g1 = (float)w.y;
        d.fields[cell] = g0;
        d.fields[cell + cells] = g1;
        if (d.counts) {
            const uint4 x = poisson_words((unsigned long long)cell, d.r, d.pkey0, d.pkey1);
            d.counts[cell] = count(d.counts + cell, g0, d.half_sigma2, d.half_sigma2_f, d.nbar, d.nbar_f, 1.0f,
                                   bits53(x.x, x.y));
            d.counts[cell + cells] = count(d.counts + cell + cells, g1, d.half_sigma2, d.half_sigma2_f, d.nbar,
                                           d.nbar_f, 1.0f, bits53(x.z, x.w));
        }
    }
};

// --------------------------------------------------------------------------
// Column pass: FFT along the middle axis of in[outer][L][inner] for a tile of
// C consecutive inner indices per CTA.  Outputs with point index < keep
// (keep <= KEEP, which is L/2 or L at compile time) are produced.  mode 0:
// complex output out[outer][keep][inner] (in place allowed when keep == L);
// mode 1: field epilogue with realization = outer index and cell =
// point*inner + i.
// --------------------------------------------------------------------------
// Build-time tunables of the CTA shapes, per kernel family: binary32 points
// per thread (E), threads per CTA, and the minimum number of resident CTAs per
// SM given to the register allocator.  Families: COLS (column passes:
// sampler, embedding, power spectrum 3D middle axis), ROWS (in-place row
// transforms), SROWS (noise-fused sampler rows), PKR / PKC (power spectrum
// row and binning passes).
#ifndef CF_COLS_E
#define CF_COLS_E 8
#endif
#ifndef CF_COLS_THREADS
#define CF_COLS_THREADS 256
#endif
#ifndef CF_COLS_MINB
#define CF_COLS_MINB 4
#endif
// SCOLS: the sampler's binary32 inverse column passes on lines of at least
// CF_SCOLS_MIN_L points: 16 points per thread and 512 threads, i.e. 8
// adjacent columns of 1024 points per CTA (64-byte row segments per load),
// measured 35 % faster for the fused column pass than the COLS shape (2
// columns of 1024 per CTA).  Forward passes keep the COLS shape (16 points
// per thread spill there).
#ifndef CF_SCOLS_E
#define CF_SCOLS_E 16
#endif
#ifndef CF_SCOLS_THREADS
#define CF_SCOLS_THREADS 512
#endif
#ifndef CF_SCOLS_MINB
#define CF_SCOLS_MINB 2
#endif
#ifndef CF_SCOLS_MIN_L
#define CF_SCOLS_MIN_L 256
#endif
#ifndef CF_ROWS_E
#define CF_ROWS_E 8
#endif
#ifndef CF_ROWS_THREADS
#define CF_ROWS_THREADS 256
#endif
#ifndef CF_ROWS_MINB
#define CF_ROWS_MINB 4
#endif

// binary32 uses the family's E, binary64 the global CF_E64
template <typename T, int E32>
struct FamilyE {
    static constexpr int value = sizeof(T) == 4 ? E32 : CF_E64;
};

template <typename T, int L, int E32, int THREADS_, int MINB_>
struct TileCfg {
    using G = LineGeom<T, L, FamilyE<T, E32>::value>;
    // lines per CTA
    static constexpr int LINES = G::TL >= THREADS_ ? 1 : ((THREADS_ / G::TL) > 32 ? 32 : (THREADS_ / G::TL));
    static constexpr int THREADS = LINES * G::TL;
    // resident CTAs promised to the register allocator: at most 1024 threads
    // per SM in total, i.e. at least 64 registers per thread (a line longer
    // than one CTA's default thread count otherwise got 32 and spilled)
    static constexpr int MINB = THREADS * MINB_ <= 1024 ? MINB_ : (1024 / THREADS > 0 ? 1024 / THREADS : 1);
    static constexpr size_t SMEM = sizeof(C2<T>) * (size_t)LINES * (size_t)G::PADDED;
};

// WIDE: the SCOLS shape (binary32 sampler columns), else COLS.
template <typename T, int L, bool WIDE = false>
struct ColsShape {
    static constexpr bool W = WIDE && sizeof(T) == 4 && L >= CF_SCOLS_MIN_L;
    static constexpr int E = W ? CF_SCOLS_E : CF_COLS_E;
    static constexpr int THREADS = W ? CF_SCOLS_THREADS : CF_COLS_THREADS;
    static constexpr int MINB = W ? CF_SCOLS_MINB : CF_COLS_MINB;
};

template <typename T, int L, bool WIDE = false>
struct ColsCfg : TileCfg<T, L, ColsShape<T, L, WIDE>::E, ColsShape<T, L, WIDE>::THREADS, ColsShape<T, L, WIDE>::MINB> {
    static constexpr int C =
        TileCfg<T, L, ColsShape<T, L, WIDE>::E, ColsShape<T, L, WIDE>::THREADS, ColsShape<T, L, WIDE>::MINB>::LINES;
};

// The body of one block of k_cols: column tile bx of outer slice o (a
// persistent kernel calls it for several tiles in turn).
template <typename T, int L, int SIGN, int KEEP_HALF>
__device__ __forceinline__ void cols_block(long long bx, long long o, const C2<T>* in, long long inner, int keep,
                                           C2<T>* out, int mode, const FieldEpi<T>& epi,
                                           const C2<T>* __restrict__ tw) {
    using Cfg = ColsCfg<T, L, (SIGN > 0 && KEEP_HALF)>;
    using G = typename Cfg::G;
    constexpr int KEEP = KEEP_HALF ? L / 2 : L;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    const int ln = threadIdx.x % Cfg::C;
    const int j = threadIdx.x / Cfg::C;
    const long long i = bx * Cfg::C + ln;
    const bool valid = i < inner;
    const C2<T>* src = in + (size_t)o * L * (size_t)inner + (size_t)(valid ? i : 0);
    C2<T> v[G::E];
#pragma unroll
    for (int q = 0; q < G::E; ++q) v[q] = src[(size_t)(j + q * (L / G::E)) * (size_t)inner];
    const ColLayout<G::E, Cfg::C> lay;
    if (mode == 0) {
        auto sink = [&](int, int p, C2<T> val) {
            if (valid && p < keep) out[((size_t)o * keep + p) * (size_t)inner + i] = val;
        };
        line_fft<T, L, SIGN, KEEP>(sm, lay, ln, j, v, tw, sink);
        return;
    }
    // field epilogue: the kept outputs go to shared memory first, and the
    // epilogue (split, lognormal, Poisson) runs after the transform, when
    // the line's registers are free again
    auto to_smem = [&](int, int p, C2<T> val) {
        if (p < keep) sm[lay(ln, p)] = val;
    };
    line_fft<T, L, SIGN, KEEP, true>(sm, lay, ln, j, v, tw, to_smem);
    __syncthreads();
    if (valid) {
#pragma unroll 1
        for (int p = j; p < keep; p += G::TL) epi((int)o, (long long)p * inner + i, sm[lay(ln, p)]);
    }
    __syncthreads();  // the exchange buffer is free for the next tile
}

template <typename T, int L, int SIGN, int KEEP_HALF>
__global__ void __launch_bounds__(ColsCfg<T, L, (SIGN > 0 && KEEP_HALF)>::THREADS,
                                  ColsCfg<T, L, (SIGN > 0 && KEEP_HALF)>::MINB)
    k_cols(const C2<T>* in, long long inner, int keep, C2<T>* out, int mode, FieldEpi<T> epi,
           const C2<T>* __restrict__ tw) {
    cols_block<T, L, SIGN, KEEP_HALF>(blockIdx.x, blockIdx.y, in, inner, keep, out, mode, epi, tw);
}

// --------------------------------------------------------------------------
// Row pass on contiguous lines: in-place complex FFT of rows of length L.
// --------------------------------------------------------------------------
template <typename T, int L>
struct RowsCfg : TileCfg<T, L, CF_ROWS_E, CF_ROWS_THREADS, CF_ROWS_MINB> {
    static constexpr int ROWS = TileCfg<T, L, CF_ROWS_E, CF_ROWS_THREADS, CF_ROWS_MINB>::LINES;
};

template <typename T, int L, int SIGN>
__global__ void __launch_bounds__(RowsCfg<T, L>::THREADS, RowsCfg<T, L>::MINB)
    k_rows_c2c(C2<T>* data, long long nrows, const C2<T>* __restrict__ tw) {
    using Cfg = RowsCfg<T, L>;
    using G = typename Cfg::G;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    const int line = threadIdx.x / G::TL;
    const int j = threadIdx.x % G::TL;
    const long long row = (long long)blockIdx.x * Cfg::ROWS + line;
    const bool valid = row < nrows;
    C2<T>* base = data + (size_t)(valid ? row : 0) * L;
    C2<T> v[G::E];
#pragma unroll
    for (int q = 0; q < G::E; ++q) v[q] = base[j + q * (L / G::E)];
    auto sink = [&](int, int p, C2<T> val) {
        if (valid) base[p] = val;
    };
    line_fft<T, L, SIGN, L>(sm, RowLayout<G::PADE, G::PADDED>(), line, j, v, tw, sink);
}

// --------------------------------------------------------------------------
// Launch helpers.
// --------------------------------------------------------------------------
template <class K>
inline cf_status prepare_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail(CF_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    return CF_OK;
}

// Calls f(std::integral_constant<int, L>{}) for the runtime line length L.
template <class F>
inline cf_status dispatch_line(long long L, F&& f) {
    switch (L) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 128: return f(std::integral_constant<int, 128>{});
    case 256: return f(std::integral_constant<int, 256>{});
    case 512: return f(std::integral_constant<int, 512>{});
    case 1024: return f(std::integral_constant<int, 1024>{});
    case 2048: return f(std::integral_constant<int, 2048>{});
    case 4096: return f(std::integral_constant<int, 4096>{});
    default: return fail(CF_ERR_UNSUPPORTED, "transform length %lld not supported", L);
    }
}

template <typename T>
inline const C2<T>* twiddles();
template <>
inline const C2<float>* twiddles<float>() { return twiddles_f32(); }
template <>
inline const C2<double>* twiddles<double>() { return twiddles_f64(); }

// Column pass launch over in[outer][L][inner]; keep = 0 keeps L/2 outputs
// (KEEP_HALF) or L.
template <typename T, int SIGN, int KEEP_HALF>
inline cf_status launch_cols(long long L, const C2<T>* in, long long outer, long long inner, C2<T>* out,
                             int mode, const FieldEpi<T>& epi, cudaStream_t s, long long keep = 0) {
    if (outer > 65535) return fail(CF_ERR_UNSUPPORTED, "column pass with %lld outer slices", outer);
    const long long full = KEEP_HALF ? L / 2 : L;
    if (keep == 0) keep = full;
    if (keep < 1 || keep > full) return fail(CF_ERR_ARG, "column pass keeps %lld of %lld outputs", keep, L);
    return dispatch_line(L, [&](auto Lc) -> cf_status {
        constexpr int LL = decltype(Lc)::value;
        using Cfg = ColsCfg<T, LL, (SIGN > 0 && KEEP_HALF)>;
        auto kern = k_cols<T, LL, SIGN, KEEP_HALF>;
        CF_TRY(prepare_smem(kern, Cfg::SMEM));
        dim3 grid((unsigned)((inner + Cfg::C - 1) / Cfg::C), (unsigned)outer);
        const char* name = SIGN > 0 ? (mode == 1 ? (epi.counts ? "icols_fields_lp" : "icols_fields") : "icols")
                                    : "fcols";
        char full[64];
        snprintf(full, sizeof full, "%s_%s", name, sizeof(T) == 4 ? "f32" : "f64");
        ScopedKernelTimer kt(s, full, LL);
        kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(in, inner, (int)keep, out, mode, epi, twiddles<T>());
        CF_CHECK_LAUNCH();
        return CF_OK;
    });
}

template <typename T, int SIGN>
inline cf_status launch_rows_c2c(long long L, C2<T>* data, long long nrows, cudaStream_t s) {
    return dispatch_line(L, [&](auto Lc) -> cf_status {
        constexpr int LL = decltype(Lc)::value;
        using Cfg = RowsCfg<T, LL>;
        auto kern = k_rows_c2c<T, LL, SIGN>;
        CF_TRY(prepare_smem(kern, Cfg::SMEM));
        dim3 grid((unsigned)((nrows + Cfg::ROWS - 1) / Cfg::ROWS));
        ScopedKernelTimer kt(s, SIGN > 0 ? (sizeof(T) == 4 ? "irows_f32" : "irows_f64")
                                         : (sizeof(T) == 4 ? "frows_f32" : "frows_f64"), LL);
        kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(data, nrows, twiddles<T>());
        CF_CHECK_LAUNCH();
        return CF_OK;
    });
}

// In-place N-D complex transform (unnormalised) of data[m0][m1][m2].
template <typename T, int SIGN>
inline cf_status fft_nd_inplace(C2<T>* data, const GridInfo& g, cudaStream_t s) {
    const int d = g.ndim;
    long long total = g.mtotal;
    CF_TRY((launch_rows_c2c<T, SIGN>(g.m[d - 1], data, total / g.m[d - 1], s)));
    for (int a = d - 2; a >= 0; --a) {
        long long inner = 1, outer = 1;
        for (int b = a + 1; b < d; ++b) inner *= g.m[b];
        for (int b = 0; b < a; ++b) outer *= g.m[b];
        FieldEpi<T> none{};
        CF_TRY((launch_cols<T, SIGN, 0>(g.m[a], data, outer, inner, data, 0, none, s)));
    }
    return CF_OK;
}

inline int grid_blocks(long long n, int threads, int cap = 152 * 16) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

}  // namespace cf
