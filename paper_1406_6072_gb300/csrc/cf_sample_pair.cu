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
#include <cooperative_groups.h>

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

// Row pass (block (bx, by)): rows of realizations ra = 2 by and rb = ra + 1
// of the chunk (rb absent in an odd tail); lane A draws realization ra's noise, lane
// B rb's (each with its own amplitudes and key in a batched launch), scales
// it by sqrt(lambda+/M^d), transforms the row and keeps the first `keep`
// outputs: intermediate [chunk][nrows][keep].
template <int L, bool DESC, int LW>
__device__ __forceinline__ void rows_pair_block(long long bx, long long by, const float* __restrict__ s,
                                                float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                                                long long nrows, int keep, int chunk, C2<float>* __restrict__ out,
                                                const float4* __restrict__ tw, const RealDesc* __restrict__ desc) {
    using Cfg = PairCfg<L, LW>;
    constexpr int E = Cfg::E;
    constexpr int STEP = L / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    CP* sm = reinterpret_cast<CP*>(smraw);
    const int line = threadIdx.x / Cfg::TL;
    const int j = threadIdx.x % Cfg::TL;
    const long long row = bx * Cfg::LINES + line;
    const int ra = 2 * (int)by, rb = ra + 1;
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
        CP lo, hi;
        const unsigned long long pc = (unsigned long long)rw * (L / 2) + col;
        noise_pair_f32x2(pc, r_a, ka0, ka1, pc, r_b, kb0, kb1, lo, hi);
        const float2 fl = make_float2(sal, sbl), fh = make_float2(sah, sbh);
        v[q] = CP{f2mul(lo.re, fl), f2mul(lo.im, fl)};
        v[q + E / 2] = CP{f2mul(hi.re, fh), f2mul(hi.im, fh)};
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

template <int L, bool DESC, int LW>
__global__ void __launch_bounds__(PairCfg<L, LW>::THREADS, PairCfg<L, LW>::MINB)
    k_sample_rows_pair(const float* __restrict__ s, float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                       long long nrows, int keep, int chunk, C2<float>* __restrict__ out,
                       const float4* __restrict__ tw, const RealDesc* __restrict__ desc) {
    // one-dimensional grid, the realization pairs of a row block adjacent:
    // blocks resident together read the same rows of sqrt(lambda+), so an
    // amplitude array larger than L2 leaves DRAM once per launch
    const unsigned pairs = (unsigned)(chunk + 1) / 2;
    rows_pair_block<L, DESC, LW>(blockIdx.x / pairs, blockIdx.x % pairs, s, amp_scale, key0, key1, r0, nrows, keep,
                                 chunk, out, tw, desc);
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
                const long long blocks = (nrows + Cfg::LINES - 1) / Cfg::LINES * (long long)((chunk + 1) / 2);
                if (blocks > 0x7fffffffll) return fail(CF_ERR_UNSUPPORTED, "row pass of %lld blocks", blocks);
                ScopedKernelTimer kt(st, "sample_rows_f32", LL);
                kern<<<(unsigned)blocks, Cfg::THREADS, Cfg::SMEM, st>>>(s, amp_scale, (uint32_t)seed,
                                                                        (uint32_t)(seed >> 32), r0, nrows, keep,
                                                                        chunk, out, twiddles_f32x2(), desc);
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

// --------------------------------------------------------------------------
// The whole binary32 sampler of one chunk in one cooperative launch, for the
// small grids where launch and dependency overheads weigh most (2D embedded
// sides of 64 or 128, 3D of 64 or 128): the blocks stay resident and walk the
// tiles of the row pass, then (after a grid-wide barrier) those of the
// column passes, then the deferred binary64 Poisson decisions.  Every tile
// runs the same code as the separate kernels (rows_pair_block, cols_block),
// so the results are identical bit for bit.  256 threads per block: the row
// pass with the 256-thread shape, the column passes with their default shape
// for lines of at most 128 points.
// --------------------------------------------------------------------------
namespace cgp = cooperative_groups;

struct PersistArgs {
    const float* s;
    float amp_scale;
    uint32_t key0, key1, r0;
    int chunk;
    const RealDesc* desc;
    long long m0, m1, n0, n1, n2;  // 2D: m1 = M_last, n2 unused
    C2<float>* buf1;
    C2<float>* buf2;
    FieldEpi<float> epi;
    PoissonDefer defer;
};

constexpr int kPersistThreads = 256;

// LL: last axis (rows), LM: middle axis (3D; 0 in 2D), L0: axis 0.
template <int LL, int LM, int L0, bool DESC>
__global__ void __launch_bounds__(kPersistThreads, 2)
    k_sample_persistent(PersistArgs a, const float4* __restrict__ tw4, const C2<float>* __restrict__ tw) {
    cgp::grid_group grid = cgp::this_grid();
    static_assert(PairCfg<LL, kPersistThreads>::THREADS == kPersistThreads, "row shape");
    static_assert(ColsCfg<float, L0, true>::THREADS == kPersistThreads, "column shape");
    const bool three = LM > 0;
    const long long nrows = three ? a.m0 * a.m1 : a.m0;
    const int keep_last = (int)(three ? a.n2 : a.n1);
    {
        using RC = PairCfg<LL, kPersistThreads>;
        const long long nbx = (nrows + RC::LINES - 1) / RC::LINES, nby = (a.chunk + 1) / 2;
        for (long long it = blockIdx.x; it < nbx * nby; it += gridDim.x) {
            rows_pair_block<LL, DESC, kPersistThreads>(it % nbx, it / nbx, a.s, a.amp_scale, a.key0, a.key1, a.r0,
                                                       nrows, keep_last, a.chunk, a.buf1, tw4, a.desc);
            __syncthreads();
        }
    }
    grid.sync();
    if constexpr (LM > 0) {
        static_assert(ColsCfg<float, LM, true>::THREADS == kPersistThreads, "middle shape");
        // axis 1 of [chunk M0][M1][n2] -> [chunk M0][n1][n2]
        using CC = ColsCfg<float, LM, true>;
        const long long tiles = (a.n2 + CC::C - 1) / CC::C, outer = (long long)a.chunk * a.m0;
        for (long long it = blockIdx.x; it < tiles * outer; it += gridDim.x) {
            cols_block<float, LM, +1, 1>(it % tiles, it / tiles, a.buf1, a.n2, (int)a.n1, a.buf2, 0, a.epi, tw);
            __syncthreads();
        }
        grid.sync();
    }
    {
        // axis 0 with the field epilogue
        using CC = ColsCfg<float, L0, true>;
        const long long inner = three ? a.n1 * a.n2 : a.n1;
        const long long tiles = (inner + CC::C - 1) / CC::C;
        const C2<float>* in = three ? a.buf2 : a.buf1;
        for (long long it = blockIdx.x; it < tiles * a.chunk; it += gridDim.x) {
            cols_block<float, L0, +1, 1>(it % tiles, it / tiles, in, inner, (int)a.n0, nullptr, 1, a.epi, tw);
            __syncthreads();
        }
    }
    if (a.defer.items) {
        grid.sync();
        const unsigned int n = *a.defer.count < a.defer.capacity ? *a.defer.count : a.defer.capacity;
        for (unsigned int i = blockIdx.x * kPersistThreads + threadIdx.x; i < n; i += gridDim.x * kPersistThreads) {
            const PoissonTodo t = a.defer.items[i];
            *t.dst = poisson_count_f64(t.G, t.half_sigma2, t.nbar, t.f, t.ubits);
        }
    }
}

// Grids the persistent kernel takes: binary32, 2D with embedded sides 64 or
// 128 on both axes, 3D with 64 or 128 on all three.
bool persistent_ok(const GridInfo& g) {
    auto ok = [](long long m) { return m == 64 || m == 128; };
    if (g.ndim == 2) return ok(g.m[0]) && ok(g.m[1]);
    if (g.ndim == 3) return ok(g.m[0]) && ok(g.m[1]) && ok(g.m[2]);
    return false;
}

template <int LL, int LM, int L0, bool DESC>
static cf_status launch_persistent_t(PersistArgs& a, cudaStream_t st) {
    auto kern = k_sample_persistent<LL, LM, L0, DESC>;
    const size_t smem = std::max(PairCfg<LL, kPersistThreads>::SMEM,
                                 std::max(ColsCfg<float, L0, true>::SMEM, LM > 0 ? ColsCfg<float, (LM > 0 ? LM : 64), true>::SMEM : (size_t)0));
    CF_TRY(prepare_smem(kern, smem));
    int per_sm = 0, dev = 0, sms = 0;
    CF_CUDA(cudaGetDevice(&dev));
    CF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistThreads, smem));
    if (per_sm < 1) return fail(CF_ERR_UNSUPPORTED, "persistent sampler does not fit an SM");
    // as many blocks as the largest phase has tiles, at most all resident ones
    const long long nrows = LM > 0 ? a.m0 * a.m1 : a.m0;
    long long want = ((nrows + PairCfg<LL, kPersistThreads>::LINES - 1) / PairCfg<LL, kPersistThreads>::LINES) *
                     ((a.chunk + 1) / 2);
    const long long cap = (long long)per_sm * sms;
    const unsigned blocks = (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
    const float4* tw4 = twiddles_f32x2();
    const C2<float>* tw = twiddles_f32();
    void* args[] = {(void*)&a, (void*)&tw4, (void*)&tw};
    ScopedKernelTimer kt(st, "sample_persistent_f32", LL);
    CF_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kPersistThreads), args, smem, st));
    CF_CHECK_LAUNCH();
    return CF_OK;
}

template <bool DESC>
static cf_status launch_persistent_d(const GridInfo& g, PersistArgs& a, cudaStream_t st) {
    if (g.ndim == 2) {
        if (g.m[0] == 64 && g.m[1] == 64) return launch_persistent_t<64, 0, 64, DESC>(a, st);
        if (g.m[0] == 64 && g.m[1] == 128) return launch_persistent_t<128, 0, 64, DESC>(a, st);
        if (g.m[0] == 128 && g.m[1] == 64) return launch_persistent_t<64, 0, 128, DESC>(a, st);
        if (g.m[0] == 128 && g.m[1] == 128) return launch_persistent_t<128, 0, 128, DESC>(a, st);
    } else if (g.ndim == 3 && g.m[0] == g.m[1] && g.m[1] == g.m[2]) {
        if (g.m[0] == 64) return launch_persistent_t<64, 64, 64, DESC>(a, st);
        if (g.m[0] == 128) return launch_persistent_t<128, 128, 128, DESC>(a, st);
    }
    return fail(CF_ERR_UNSUPPORTED, "no persistent sampler for this grid");
}

// One chunk of nr realizations through the persistent kernel: buf1 / buf2 as
// in the separate passes; the deferred-decision list's counter is cleared on
// st before the launch (as the separate passes do).
cf_status launch_sample_persistent(const GridInfo& g, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                                   int nr, C2<float>* buf1, C2<float>* buf2, const FieldEpi<float>& epi,
                                   const PoissonDefer& defer, const RealDesc* desc, cudaStream_t st) {
    if (!persistent_ok(g)) return fail(CF_ERR_UNSUPPORTED, "no persistent sampler for this grid");
    PersistArgs a{};
    a.s = s;
    a.amp_scale = amp_scale;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.r0 = r0;
    a.chunk = nr;
    a.desc = desc;
    a.m0 = g.m[0];
    a.m1 = g.ndim == 3 ? g.m[1] : g.m[1];
    a.n0 = g.n[0];
    a.n1 = g.n[1];
    a.n2 = g.ndim == 3 ? g.n[2] : 1;
    a.buf1 = buf1;
    a.buf2 = buf2;
    a.epi = epi;
    a.defer = defer;
    if (defer.items) CF_CUDA(cudaMemsetAsync(defer.count, 0, sizeof(unsigned int), st));
    return desc ? launch_persistent_d<true>(g, a, st) : launch_persistent_d<false>(g, a, st);
}

}  // namespace cf
