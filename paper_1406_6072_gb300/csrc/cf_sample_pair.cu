// cf_sample_pair.cu -- the binary32 sampler passes with two lines per thread
// (section 2, eq. (Papos2) and the closing paragraph: noise, scaling and the
// pruned inverse transform; section 3.1 in the field epilogue).
//
// Each value holds the same point of two lines (CP: two realizations, or two
// slabs of the 3D middle pass), so the noise's polynomials, the scaling and
// every transform stage run as paired binary32 instructions (f32x2), the
// twiddles are shared by both lines and every shared-memory exchange moves
// 16 bytes per access.  E = 8 points per line and thread.  The draws are
// bit-identical to the one-line kernels' (the same operations per lane); the
// transform's rounding differs from theirs only by its radix order.
//
// CTA shapes: `shape` 0, 1, 2 aims at 128, 256 or 512 threads per CTA in the
// row pass and 512, 256 or 1024 in the column pass (as many whole lines as
// fit).  Every shape computes every output with the same operations, so the
// choice changes no result bit; the sampler's autotuner (cf_tune_sample)
// picks the fastest per grid.
#include "cf_kernels.cuh"

namespace cf {

// Threads aimed at per CTA for each shape.
__host__ __device__ constexpr int pair_rows_threads(int shape) { return shape == 1 ? 256 : (shape == 2 ? 512 : 128); }
__host__ __device__ constexpr int pair_cols_threads(int shape) { return shape == 1 ? 256 : (shape == 2 ? 1024 : 512); }

template <int L, int TARGET>
struct PairCfg {
    static constexpr int E = L < 8 ? L : 8;
    static constexpr int TL = L / E;  // threads per line
    static constexpr int LINES = TL >= TARGET ? 1 : (TARGET / TL > 32 ? 32 : TARGET / TL);
    static constexpr int THREADS = LINES * TL;
    // at most 1024 resident threads per SM: 64 registers per thread
    static constexpr int MINB = 1024 / THREADS > 8 ? 8 : (1024 / THREADS > 0 ? 1024 / THREADS : 1);
    static constexpr int PADDED = L + L / E;
    static constexpr size_t SMEM = sizeof(CP) * (size_t)LINES * (size_t)PADDED;
};

// Row pass: rows of realizations ra = 2 blockIdx.y and rb = ra + 1 of the
// chunk (rb absent in an odd tail); lane A draws realization ra's noise, lane
// B rb's (each with its own amplitudes and key in a batched launch), scales
// it by sqrt(lambda+/M^d), transforms the row and keeps the first `keep`
// outputs: intermediate [chunk][nrows][keep].
template <int L, bool DESC, int LW>
__global__ void __launch_bounds__(PairCfg<L, LW>::THREADS, PairCfg<L, LW>::MINB)
    k_sample_rows_pair(const float* __restrict__ s, float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                       long long nrows, int keep, int chunk, C2<float>* __restrict__ out,
                       const float4* __restrict__ tw, const RealDesc* __restrict__ desc) {
    using Cfg = PairCfg<L, LW>;
    constexpr int E = Cfg::E;
    constexpr int STEP = L / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    CP* sm = reinterpret_cast<CP*>(smraw);
    const int line = threadIdx.x / Cfg::TL;
    const int j = threadIdx.x % Cfg::TL;
    const long long row = (long long)blockIdx.x * Cfg::LINES + line;
    const int ra = 2 * blockIdx.y, rb = ra + 1;
    const bool valid = row < nrows, valid_b = rb < chunk;
    const long long rw = valid ? row : 0;
    const float* sa_row = s + (size_t)rw * L;
    const float* sb_row = sa_row;
    float amp_a = amp_scale, amp_b = amp_scale;
    uint32_t ka0 = key0, ka1 = key1, kb0 = key0, kb1 = key1, r_a = r0 + (uint32_t)ra, r_b = r0 + (uint32_t)rb;
    if constexpr (DESC) {
        const RealDesc& da = desc[ra];
        const RealDesc& db = desc[valid_b ? rb : ra];
        sa_row = da.s + (size_t)rw * L;
        sb_row = db.s + (size_t)rw * L;
        amp_a = da.amp_scale;
        amp_b = db.amp_scale;
        ka0 = da.key0;
        ka1 = da.key1;
        kb0 = db.key0;
        kb1 = db.key1;
        r_a = da.r;
        r_b = db.r;
    }
    CP v[E];
    // binary32 noise pairs columns c and c + L/2 in one Philox call: points
    // j + q STEP and j + (q + E/2) STEP of this thread
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
        const int col = j + q * STEP;
        const float sal = __fmul_rn(__ldg(sa_row + col), amp_a);
        const float sah = __fmul_rn(__ldg(sa_row + col + L / 2), amp_a);
        float sbl = sal, sbh = sah;
        if constexpr (DESC) {
            sbl = __fmul_rn(__ldg(sb_row + col), amp_b);
            sbh = __fmul_rn(__ldg(sb_row + col + L / 2), amp_b);
        }
        // where sqrt(lambda+) is zero (a clamped or zeroed eigenvalue) the
        // scaled draw is zero whatever the noise: a warp whose amplitudes of
        // a half are all zero skips that half's Box-Muller, and the Philox
        // call when both halves are zero (every other draw is unchanged:
        // the generator is counter-based)
        const bool need_lo = __any_sync(0xffffffffu, sal != 0.0f || sbl != 0.0f);
        const bool need_hi = __any_sync(0xffffffffu, sah != 0.0f || sbh != 0.0f);
        CP lo = CP{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}, hi = lo;
        if (need_lo || need_hi) {
            const unsigned long long pc = (unsigned long long)rw * (L / 2) + col;
            const uint4 xa = philox4x32_10(make_uint4((uint32_t)pc, (uint32_t)(pc >> 32), r_a, 0u), ka0, ka1);
            const uint4 xb = philox4x32_10(make_uint4((uint32_t)pc, (uint32_t)(pc >> 32), r_b, 0u), kb0, kb1);
            if (need_lo) {
                const CP e = box_muller_f32x2(xa.x, xa.y, xb.x, xb.y);
                const float2 fl = make_float2(sal, sbl);
                lo = CP{f2mul(e.re, fl), f2mul(e.im, fl)};
            }
            if (need_hi) {
                const CP e = box_muller_f32x2(xa.z, xa.w, xb.z, xb.w);
                const float2 fh = make_float2(sah, sbh);
                hi = CP{f2mul(e.re, fh), f2mul(e.im, fh)};
            }
        }
        v[q] = lo;
        v[q + E / 2] = hi;
    }
    C2<float>* oa = out + ((size_t)ra * nrows + row) * keep;
    C2<float>* ob = out + ((size_t)rb * nrows + row) * keep;
    auto sink = [&](int, int p, CP val) {
        if (!valid || p >= keep) return;
        oa[p] = mk(val.re.x, val.im.x);
        if (valid_b) ob[p] = mk(val.re.y, val.im.y);
    };
    line_fft_pair<L, +1, L / 2>(sm, RowLayout<E, Cfg::PADDED>(), line, j, v, tw, sink);
}

// Column pass: lines o = 2 blockIdx.y and o + 1 of in[outer][L][inner], the
// CTA's columns adjacent.  MODE 0: complex output out[outer][keep][inner];
// MODE 1: the field epilogue with realization = outer index.
template <int L, int MODE, int LW>
__global__ void __launch_bounds__(PairCfg<L, LW>::THREADS, PairCfg<L, LW>::MINB)
    k_cols_pair(const C2<float>* __restrict__ in, long long outer, long long inner, int keep,
                C2<float>* __restrict__ out, FieldEpi<float> epi, const float4* __restrict__ tw) {
    using Cfg = PairCfg<L, LW>;
    constexpr int E = Cfg::E;
    constexpr int STEP = L / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    CP* sm = reinterpret_cast<CP*>(smraw);
    const int ln = threadIdx.x % Cfg::LINES;
    const int j = threadIdx.x / Cfg::LINES;
    const long long i = (long long)blockIdx.x * Cfg::LINES + ln;
    const long long oa = 2ll * blockIdx.y, ob = oa + 1;
    const bool valid = i < inner, valid_b = ob < outer;
    const size_t col = (size_t)(valid ? i : 0);
    const C2<float>* sa = in + (size_t)oa * L * (size_t)inner + col;
    const C2<float>* sb = in + (size_t)(valid_b ? ob : oa) * L * (size_t)inner + col;
    CP v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const size_t at = (size_t)(j + q * STEP) * (size_t)inner;
        const C2<float> a = sa[at], b = sb[at];
        v[q] = CP{make_float2(a.x, b.x), make_float2(a.y, b.y)};
    }
    auto sink = [&](int, int p, CP val) {
        if (!valid || p >= keep) return;
        if constexpr (MODE == 0) {
            out[((size_t)oa * keep + p) * (size_t)inner + (size_t)i] = mk(val.re.x, val.im.x);
            if (valid_b) out[((size_t)ob * keep + p) * (size_t)inner + (size_t)i] = mk(val.re.y, val.im.y);
        } else {
            // one copy of the epilogue for both lines (its code is long)
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                if (h && !valid_b) break;
                epi((int)(oa + h), (long long)p * inner + i, h ? mk(val.re.y, val.im.y) : mk(val.re.x, val.im.x));
            }
        }
    };
    line_fft_pair<L, +1, L / 2>(sm, ColLayout<E, Cfg::LINES>(), ln, j, v, tw, sink);
}

// Calls f(std::integral_constant<int, TARGET>{}) for the shape: the three
// shapes exist for lines of 256 points or more (where they differ in
// occupancy and load width), the default alone below.
template <bool ROWS, int L, class F>
static cf_status dispatch_shape(int shape, F&& f) {
    if constexpr (L >= 256) {
        switch (shape) {
        case 1: return f(std::integral_constant<int, ROWS ? pair_rows_threads(1) : pair_cols_threads(1)>{});
        case 2: return f(std::integral_constant<int, ROWS ? pair_rows_threads(2) : pair_cols_threads(2)>{});
        default: break;
        }
    }
    return f(std::integral_constant<int, ROWS ? pair_rows_threads(0) : pair_cols_threads(0)>{});
}

cf_status launch_rows_pair(long long L, int keep, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                           int chunk, long long nrows, C2<float>* out, cudaStream_t st, const RealDesc* desc,
                           int shape) {
    return dispatch_line(L, [&](auto Lc) -> cf_status {
        constexpr int LL = decltype(Lc)::value;
        if constexpr (LL < 16) {
            return fail(CF_ERR_UNSUPPORTED, "paired rows need 16 points or more");
        } else {
            return dispatch_shape<true, LL>(shape, [&](auto Wc) -> cf_status {
                constexpr int LW = decltype(Wc)::value;
                using Cfg = PairCfg<LL, LW>;
                auto kern = desc ? k_sample_rows_pair<LL, true, LW> : k_sample_rows_pair<LL, false, LW>;
                CF_TRY(prepare_smem(kern, Cfg::SMEM));
                dim3 grid((unsigned)((nrows + Cfg::LINES - 1) / Cfg::LINES), (unsigned)((chunk + 1) / 2));
                ScopedKernelTimer kt(st, "sample_rows_f32", LL);
                kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(s, amp_scale, (uint32_t)seed, (uint32_t)(seed >> 32), r0,
                                                            nrows, keep, chunk, out, twiddles_f32x2(), desc);
                CF_CHECK_LAUNCH();
                return CF_OK;
            });
        }
    });
}

cf_status launch_cols_pair(long long L, const C2<float>* in, long long outer, long long inner, C2<float>* out,
                           int mode, const FieldEpi<float>& epi, cudaStream_t st, long long keep, int shape) {
    if (outer > 2 * 65535ll) return fail(CF_ERR_UNSUPPORTED, "column pass with %lld outer slices", outer);
    if (keep < 1 || keep > L / 2) return fail(CF_ERR_ARG, "column pass keeps %lld of %lld outputs", keep, L);
    return dispatch_line(L, [&](auto Lc) -> cf_status {
        constexpr int LL = decltype(Lc)::value;
        if constexpr (LL < 16) {
            return fail(CF_ERR_UNSUPPORTED, "paired columns need 16 points or more");
        } else {
            return dispatch_shape<false, LL>(shape, [&](auto Wc) -> cf_status {
                constexpr int LW = decltype(Wc)::value;
                using Cfg = PairCfg<LL, LW>;
                auto kern = mode ? k_cols_pair<LL, 1, LW> : k_cols_pair<LL, 0, LW>;
                CF_TRY(prepare_smem(kern, Cfg::SMEM));
                dim3 grid((unsigned)((inner + Cfg::LINES - 1) / Cfg::LINES), (unsigned)((outer + 1) / 2));
                ScopedKernelTimer kt(st, mode ? (epi.counts ? "icols_fields_lp_f32" : "icols_fields_f32") : "icols_f32",
                                     LL);
                kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(in, outer, inner, (int)keep, out, epi, twiddles_f32x2());
                CF_CHECK_LAUNCH();
                return CF_OK;
            });
        }
    });
}

}  // namespace cf
