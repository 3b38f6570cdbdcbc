// cf_sample.cu -- steps b1-b4 (and c1-c2 fused): per-realization exact
// Gaussian fields by the pruned inverse transform of scaled complex noise
// (section 2, eq. (Papos2) and the closing paragraph), plus the stand-alone
// noise draw.
#include "cf_kernels.cuh"

#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>

namespace cf {

#ifndef CF_SROWS_E
#define CF_SROWS_E 16
#endif
#ifndef CF_SROWS_THREADS
#define CF_SROWS_THREADS 128
#endif
#ifndef CF_SROWS_MINB
#define CF_SROWS_MINB 8
#endif
// Rows of at most this length read all their amplitudes before drawing the
// noise (measured: 7 % faster for 256-point rows, 3 % slower for 1024)
#ifndef CF_SROWS_PREFETCH_MAX_L
#define CF_SROWS_PREFETCH_MAX_L 256
#endif

template <typename T, int L>
struct SRowsCfg : TileCfg<T, L, CF_SROWS_E, CF_SROWS_THREADS, CF_SROWS_MINB> {
    static constexpr int ROWS = TileCfg<T, L, CF_SROWS_E, CF_SROWS_THREADS, CF_SROWS_MINB>::LINES;
};

// --------------------------------------------------------------------------
// Pass 1: rows along the last axis.  Each thread draws the noise of its E
// first-stage points (Philox stream 0), scales it by sqrt(lambda+)/sqrt(M^d),
// runs the inverse line transform, and keeps the first `keep` outputs (the
// survey's n <= L/2 points).  Output: complex intermediate
// [chunk][nrows][keep] (EPI false), or for a one-dimensional grid the fields
// (and counts) directly (EPI true; a separate instantiation, so that the
// multi-dimensional row pass carries no epilogue code and registers).
// --------------------------------------------------------------------------
template <typename T, int L, bool EPI>
__global__ void __launch_bounds__(SRowsCfg<T, L>::THREADS, SRowsCfg<T, L>::MINB)
    k_sample_rows(const T* __restrict__ s, T amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                  long long nrows, int keep, C2<T>* __restrict__ out, FieldEpi<T> epi,
                  const C2<T>* __restrict__ tw, const RealDesc* __restrict__ desc) {
    using Cfg = SRowsCfg<T, L>;
    using G = typename Cfg::G;
    constexpr int E = G::E;
    constexpr int STEP = L / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    const int line = threadIdx.x / G::TL;
    const int j = threadIdx.x % G::TL;
    const long long row = (long long)blockIdx.x * Cfg::ROWS + line;
    const int rl = blockIdx.y;
    uint32_t r = r0 + (uint32_t)rl;
    if constexpr (sizeof(T) == 4) {
        if (desc) {  // batched launch: this realization's request
            const RealDesc& d = desc[rl];
            s = (const T*)d.s;
            amp_scale = (T)d.amp_scale;
            key0 = d.key0;
            key1 = d.key1;
            r = d.r;
        }
    }
    const bool valid = row < nrows;
    const long long rw = valid ? row : 0;
    const T* srow = s + (size_t)rw * L;
    C2<T> v[E];
    if constexpr (sizeof(T) == 4) {
        // binary32: columns c and c + L/2 share one Philox call (pair index
        // row*L/2 + c); first-stage points j + q*STEP and j + (q + E/2)*STEP
        // are exactly such a pair.
        if constexpr (L <= CF_SROWS_PREFETCH_MAX_L) {
            // the amplitudes first (L2 reads), the noise while they arrive
            float sa[E / 2], sb[E / 2];
#pragma unroll
            for (int q = 0; q < E / 2; ++q) {
                sa[q] = __ldg(srow + j + q * STEP);
                sb[q] = __ldg(srow + j + q * STEP + L / 2);
            }
#pragma unroll
            for (int q = 0; q < E / 2; ++q) {
                const int col = j + q * STEP;
                C2<float> lo, hi;
                noise_pair_f32((unsigned long long)rw * (L / 2) + col, r, key0, key1, lo, hi);
                v[q] = cscale(lo, sa[q] * amp_scale);
                v[q + E / 2] = cscale(hi, sb[q] * amp_scale);
            }
        } else if constexpr (E >= 4) {
            // two cell pairs of this thread at once: the paired Box-Muller
            // (the same draws, its polynomials in f32x2 instructions)
#pragma unroll
            for (int q = 0; q < E / 2; q += 2) {
                const int ca = j + q * STEP, cb = ca + STEP;
                CP lo, hi;
                noise_pair_f32x2((unsigned long long)rw * (L / 2) + ca, r, key0, key1,
                                 (unsigned long long)rw * (L / 2) + cb, r, key0, key1, lo, hi);
                v[q] = cscale(mk(lo.re.x, lo.im.x), srow[ca] * amp_scale);
                v[q + 1] = cscale(mk(lo.re.y, lo.im.y), srow[cb] * amp_scale);
                v[q + E / 2] = cscale(mk(hi.re.x, hi.im.x), srow[ca + L / 2] * amp_scale);
                v[q + 1 + E / 2] = cscale(mk(hi.re.y, hi.im.y), srow[cb + L / 2] * amp_scale);
            }
        } else {
#pragma unroll
            for (int q = 0; q < E / 2; ++q) {
                const int col = j + q * STEP;
                C2<float> lo, hi;
                noise_pair_f32((unsigned long long)rw * (L / 2) + col, r, key0, key1, lo, hi);
                v[q] = cscale(lo, srow[col] * amp_scale);
                v[q + E / 2] = cscale(hi, srow[col + L / 2] * amp_scale);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int col = j + q * STEP;
            const C2<double> e = noise_f64((unsigned long long)rw * L + col, r, key0, key1);
            v[q] = cscale(e, srow[col] * amp_scale);
        }
    }
    auto sink = [&](int, int p, C2<T> val) {
        if (!valid || p >= keep) return;
        if constexpr (EPI)
            epi(rl, (long long)row * keep + p, val);
        else
            out[((size_t)rl * nrows + row) * keep + p] = val;
    };
    line_fft<T, L, +1, L / 2>(sm, RowLayout<G::PADE, G::PADDED>(), line, j, v, tw, sink);
}

// Paired binary32 passes (cf_sample_pair.cu): two realizations (or two
// slabs) per thread in f32x2 instructions; `shape` picks the CTA shape
// (0 = default; all shapes give identical results).
constexpr int kPairShapes = 3;
cf_status launch_rows_pair(long long L, int keep, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                           int chunk, long long nrows, C2<float>* out, cudaStream_t st, const RealDesc* desc,
                           int shape);
cf_status launch_cols_pair(long long L, const C2<float>* in, long long outer, long long inner, C2<float>* out,
                           int mode, const FieldEpi<float>& epi, cudaStream_t st, long long keep, int shape);
// The whole binary32 sampler of a chunk in one cooperative launch (small
// grids, persistent_ok).
bool persistent_ok(const GridInfo& g);
cf_status launch_sample_persistent(const GridInfo& g, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                                   int nr, C2<float>* buf1, C2<float>* buf2, const FieldEpi<float>& epi,
                                   const PoissonDefer& defer, const RealDesc* desc, cudaStream_t st);

// Binary32 row pass of 256- and 1024-point rows with P = sqrt(L) lanes per
// row (cf_sample_warp.cu; CF_SROWS_WARP=0 in the environment turns it off).
bool warp_rows_len(long long L);
cf_status launch_rows_warp(long long L, int keep, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                           int chunk, long long nrows, C2<float>* out, cudaStream_t st, const RealDesc* desc,
                           int shape);
static bool warp_rows() {
    static const bool on = [] {
        const char* e = getenv("CF_SROWS_WARP");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Binary32 row pass with two realizations per thread (CF_SROWS_PAIR=0 in the
// environment turns it off).
static bool pair_rows() {
    static const bool on = [] {
        const char* e = getenv("CF_SROWS_PAIR");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Paired column passes of the binary32 sampler: off unless CF_SCOLS_PAIR=1
// in the environment.  Measured slower than k_cols on the 512^2 workload
// (0.327 against 0.296 ms per step): the column pass is bound by its
// lognormal + Poisson epilogue, which runs per line, and 8 points per thread
// take one more exchange stage than k_cols's 16.  Its fields differ from
// k_cols's (and from the fused spectra path's) in rounding only.
static bool pair_cols() {
    static const bool on = [] {
        const char* e = getenv("CF_SCOLS_PAIR");
        return e && e[0] == '1';
    }();
    return on;
}

// Column pass of the sampler over in[outer][L][inner] keeping `keep` < = L/2
// outputs: the paired kernel in binary32 (lines of 16 points or more), else
// k_cols.
template <typename T>
static cf_status launch_sampler_cols(long long L, const C2<T>* in, long long outer, long long inner, C2<T>* out,
                                     int mode, const FieldEpi<T>& epi, cudaStream_t st, long long keep,
                                     int shape = 0) {
    if constexpr (sizeof(T) == 4) {
        if (L >= 16 && pair_cols()) return launch_cols_pair(L, in, outer, inner, out, mode, epi, st, keep, shape);
    }
    return launch_cols<T, +1, 1>(L, in, outer, inner, out, mode, epi, st, keep);
}

template <typename T>
static cf_status launch_sample_rows(long long L, int keep, const T* s, T amp_scale, uint64_t seed, uint32_t r0,
                                    int chunk, long long nrows, C2<T>* out, int mode, const FieldEpi<T>& epi,
                                    cudaStream_t st, const RealDesc* desc = nullptr, int shape = 0) {
    if constexpr (sizeof(T) == 4) {
        if (mode == 0 && warp_rows_len(L) && warp_rows())
            return launch_rows_warp(L, keep, s, amp_scale, seed, r0, chunk, nrows, out, st, desc, shape);
        if (mode == 0 && L >= 16 && pair_rows())
            return launch_rows_pair(L, keep, s, amp_scale, seed, r0, chunk, nrows, out, st, desc, shape);
    }
    return dispatch_line(L, [&](auto Lc) -> cf_status {
        constexpr int LL = decltype(Lc)::value;
        using Cfg = SRowsCfg<T, LL>;
        auto kern = mode ? k_sample_rows<T, LL, true> : k_sample_rows<T, LL, false>;
        CF_TRY(prepare_smem(kern, Cfg::SMEM));
        dim3 grid((unsigned)((nrows + Cfg::ROWS - 1) / Cfg::ROWS), (unsigned)chunk);
        ScopedKernelTimer kt(st, sizeof(T) == 4 ? "sample_rows_f32" : "sample_rows_f64", LL);
        kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(s, amp_scale, (uint32_t)seed, (uint32_t)(seed >> 32), r0,
                                                     nrows, keep, out, epi, twiddles<T>(), desc);
        CF_CHECK_LAUNCH();
        return CF_OK;
    });
}

// --------------------------------------------------------------------------
// Last sampler pass of a 2D square grid (L = M0 = 2n) fused with the first
// axis of the fields' power spectrum (section 3.2, eq. (Def spec)): the CTA's
// C columns are transformed back, cropped and passed to the field epilogue
// as in k_cols, and the cropped columns W (Re = field 2r, Im = field 2r+1)
// are kept in shared memory and transformed forward along axis 0 (length
// n).  The two real fields' spectra separate per column:
// A(k) = (Z(k) + conj Z(-k))/2, B(k) = (Z(k) - conj Z(-k))/2i, k in [0, n/2],
// written as half[field][column][k] -- the layout of the power spectrum's
// half spectra with the two axes swapped, which for a square grid its
// binning pass takes as it is.
// --------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(ColsCfg<float, L, true>::THREADS, ColsCfg<float, L, true>::MINB)
    k_cols_spec(const C2<float>* __restrict__ in, FieldEpi<float> epi, C2<float>* __restrict__ half,
                long long half_f0, const C2<float>* __restrict__ tw) {
    using Cfg = ColsCfg<float, L, true>;
    using G = typename Cfg::G;
    constexpr int C = Cfg::C;
    constexpr int N = L / 2;                    // survey side
    constexpr int HN = N / 2 + 1;               // half spectrum length
    using GF = LineGeom<float, N, 8>;           // forward lines: C lines of N points
    static_assert(C * GF::TL == Cfg::THREADS, "forward transform must use every thread");
    static_assert(C * GF::PADDED <= C * G::PADDED, "forward lines must fit the exchange buffer");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<float>* sm = reinterpret_cast<C2<float>*>(smraw);
    const int ln = threadIdx.x % C;
    const int j = threadIdx.x / C;
    const long long col0 = (long long)blockIdx.x * C;
    const long long o = blockIdx.y;
    const C2<float>* src = in + (size_t)o * L * (size_t)N + (size_t)(col0 + ln);
    C2<float> v[G::E];
#pragma unroll
    for (int q = 0; q < G::E; ++q) v[q] = src[(size_t)(j + q * (L / G::E)) * (size_t)N];
    RowLayout<GF::PADE, GF::PADDED> lf;
    auto sink = [&](int lnn, int p, C2<float> val) {
        epi((int)o, (long long)p * N + col0 + lnn, val);
        sm[lf(lnn, p)] = val;  // after the last stage's barrier: the buffer is free
    };
    line_fft<float, L, +1, L / 2, true>(sm, ColLayout<G::E, C>(), ln, j, v, tw, sink);
    __syncthreads();
    // forward transform of the C cropped columns
    const int lineF = threadIdx.x / GF::TL, jF = threadIdx.x % GF::TL;
    C2<float> w[GF::E];
#pragma unroll
    for (int q = 0; q < GF::E; ++q) w[q] = sm[lf(lineF, jF + q * (N / GF::E))];
    auto sinkF = [&](int lnn, int p, C2<float> val) { sm[lf(lnn, p)] = val; };
    line_fft<float, N, -1, N, true>(sm, lf, lineF, jF, w, tw, sinkF);
    __syncthreads();
    const long long fa = half_f0 + 2 * o, fb = fa + 1;
    for (int t = threadIdx.x; t < C * HN; t += Cfg::THREADS) {
        const int l = t / HN, k = t % HN;
        const C2<float> z = sm[lf(l, k)];
        const C2<float> zm = sm[lf(l, (N - k) & (N - 1))];
        const size_t c = (size_t)(col0 + l);
        half[((size_t)fa * N + c) * HN + k] = mk(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        half[((size_t)fb * N + c) * HN + k] = mk(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
    }
}

template <int L>
static cf_status launch_cols_spec(const C2<float>* in, int nr, const FieldEpi<float>& epi, C2<float>* half,
                                  long long half_f0, cudaStream_t st) {
    using Cfg = ColsCfg<float, L, true>;
    auto kern = k_cols_spec<L>;
    CF_TRY(prepare_smem(kern, Cfg::SMEM));
    dim3 grid((unsigned)((L / 2) / Cfg::C), (unsigned)nr);
    ScopedKernelTimer kt(st, epi.counts ? "icols_fields_lp_spec_f32" : "icols_fields_spec_f32", L);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(in, epi, half, half_f0, twiddles<float>());
    CF_CHECK_LAUNCH();
    return CF_OK;
}

static cf_status launch_cols_spec_any(long long L, const C2<float>* in, int nr, const FieldEpi<float>& epi,
                                      C2<float>* half, long long half_f0, cudaStream_t st) {
    switch (L) {
    case 256: return launch_cols_spec<256>(in, nr, epi, half, half_f0, st);
    case 512: return launch_cols_spec<512>(in, nr, epi, half, half_f0, st);
    case 1024: return launch_cols_spec<1024>(in, nr, epi, half, half_f0, st);
    case 2048: return launch_cols_spec<2048>(in, nr, epi, half, half_f0, st);
    case 4096: return launch_cols_spec<4096>(in, nr, epi, half, half_f0, st);
    default: return fail(CF_ERR_UNSUPPORTED, "fused spectra need embedded sides 256..4096 (got %lld)", L);
    }
}

// Intermediate bytes of one realization.
static size_t per_realization_bytes(const GridInfo& g, size_t elem) {
    if (g.ndim == 1) return 0;
    if (g.ndim == 2) return elem * (size_t)g.m[0] * (size_t)g.n[1];
    return elem * ((size_t)g.m[0] * g.m[1] * g.n[2] + (size_t)g.m[0] * g.n[1] * g.n[2]);
}

// Target bytes of one chunk's intermediates: large launches (measured faster
// than L2-sized chunks whose intermediate stays in L2); CF_CHUNK_MB overrides.
static size_t chunk_target_bytes() {
    static size_t v = [] {
        const char* e = getenv("CF_CHUNK_MB");
        long mb = e ? atol(e) : 1024;
        if (mb < 1) mb = 1;
        return (size_t)mb << 20;
    }();
    return v;
}

// Spectra from the fused column pass's half spectra (cf_pk.cu).
size_t pk_halves_acc_bytes(const cf_grid* grid, long long F, const cf_bins* bins);
cf_status pk_from_halves_f32(const cf_grid* grid, long long F, const cf_bins* bins, const C2<float>* half,
                             double* pk_out, int64_t* nmodes_out, double* mean, double* cov, char* acc_ws,
                             cudaStream_t s);

// Tensor-core modes (cf_tc.cu).
cf_status tc_check_grid(const GridInfo& g);
size_t tc_bytes_per_realization(const GridInfo& g);
size_t tc_header_bytes();
cf_status sample_tc(const cf_embedding* e, bool bf16, uint64_t seed, uint64_t r0, int R, float* fields, void* ws,
                    size_t ws_bytes, int chunk, double amp_scale, cudaStream_t st);

// Tuned schedule per (device, grid shape, element size), set by
// cf_tune_sample: realizations per launch and the CTA shapes of the paired
// binary32 row and column passes (0: not tuned / default).
struct SamplerTuning {
    int chunk = 0;
    int rows_shape = 0;
    int cols_shape = 0;
    int persistent = 0;  // one cooperative launch per chunk (small binary32 grids)
};
static std::mutex g_tune_mu;
static std::map<std::string, SamplerTuning> g_tuned;

static std::string tune_key(const GridInfo& g, size_t elem) {
    int dev = 0;
    cudaGetDevice(&dev);
    char b[128];
    snprintf(b, sizeof b, "%d:%d:%lld:%lld:%lld:%zu", dev, g.ndim, g.m[0], g.m[1], g.m[2], elem);
    return b;
}

static SamplerTuning tuned_of(const GridInfo& g, size_t elem) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(g, elem));
    return it == g_tuned.end() ? SamplerTuning{} : it->second;
}

static int tuned_chunk(const GridInfo& g, size_t elem) { return tuned_of(g, elem).chunk; }

// Binary32 workspaces end with the list of Poisson decisions left to the
// binary64 walk (a counter, then entries; about 4e-4 of the counts at
// nbar = 2, room for 1/256 of them): the fix-up kernel decides them after the
// column pass, with full warps.  Without room for the list the epilogue
// decides in place.
constexpr size_t kDeferHead = 256;
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static size_t defer_entries(const GridInfo& g) { return (size_t)(2 * g.ncell) / 256 + 16; }
static size_t defer_bytes(const GridInfo& g, size_t elem) {
    return elem == sizeof(C2<float>) ? sizeof(PoissonTodo) * defer_entries(g) : 0;
}

// Workspace bytes of a chunk of c realizations: intermediates, then the list.
static size_t chunk_bytes(const GridInfo& g, size_t elem, size_t c) {
    const size_t list = defer_bytes(g, elem);
    return align256(c * per_realization_bytes(g, elem)) + (list ? kDeferHead + c * list : 0);
}

static int pick_chunk(const GridInfo& g, size_t elem, int R, size_t ws_bytes) {
    const size_t per = per_realization_bytes(g, elem);
    if (per == 0) return R < 65535 ? R : 65535;  // grid.y bound
    const int tuned = tuned_chunk(g, elem);
    size_t c = tuned > 0 ? (size_t)tuned : chunk_target_bytes() / per;
    if (c < 1) c = 1;
    if (c > (size_t)R) c = (size_t)R;
    if (c > 65535) c = 65535;
    // the most realizations whose intermediates and list fit, else the most
    // whose intermediates alone fit
    const size_t list = defer_bytes(g, elem);
    size_t by_ws = ws_bytes / (per + list);
    if (by_ws > c) by_ws = c;
    while (by_ws > 0 && chunk_bytes(g, elem, by_ws) > ws_bytes) --by_ws;
    if (by_ws == 0) by_ws = ws_bytes / per;
    if (c > by_ws) c = by_ws;
    return (int)c;
}

// The list inside a workspace holding `chunk` realizations (null items when
// it does not fit).
static PoissonDefer defer_list(const GridInfo& g, size_t elem, int chunk, void* ws, size_t ws_bytes) {
    PoissonDefer d{};
    if (!ws || !defer_bytes(g, elem) || chunk_bytes(g, elem, (size_t)chunk) > ws_bytes) return d;
    unsigned char* t = (unsigned char*)ws + align256((size_t)chunk * per_realization_bytes(g, elem));
    const size_t cap = (size_t)chunk * defer_entries(g);
    d.count = (unsigned int*)t;
    d.items = (PoissonTodo*)(t + kDeferHead);
    d.capacity = cap > 0xffffffffull ? 0xffffffffu : (unsigned int)cap;
    return d;
}

// Decides the listed counts in binary64 (one thread per entry).  One warp per
// block, eight blocks per SM: the walks are bound by the binary64 pipe, which
// the warps of an SM share, so the entries are spread over as many SMs as they
// fill instead of four warps to each.
constexpr int kFixupThreads = 32;
constexpr int kFixupBlocksPerSm = 8;
__global__ void __launch_bounds__(kFixupThreads) k_poisson_fixup(PoissonDefer d) {
    const unsigned int n = *d.count < d.capacity ? *d.count : d.capacity;
    for (unsigned int i = blockIdx.x * (unsigned)kFixupThreads + threadIdx.x; i < n;
         i += gridDim.x * (unsigned)kFixupThreads) {
        const PoissonTodo t = d.items[i];
        *t.dst = poisson_count_f64(t.G, t.half_sigma2, t.nbar, t.f, t.ubits);
    }
}

static cf_status defer_begin(const PoissonDefer& d, cudaStream_t st) {
    if (d.items) CF_CUDA(cudaMemsetAsync(d.count, 0, sizeof(unsigned int), st));
    return CF_OK;
}

static cf_status defer_end(const PoissonDefer& d, cudaStream_t st) {
    if (!d.items) return CF_OK;
    int dev = 0, sms = 0;
    CF_CUDA(cudaGetDevice(&dev));
    CF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ScopedKernelTimer kt(st, "poisson_fixup");
    k_poisson_fixup<<<(sms > 0 ? sms : 1) * kFixupBlocksPerSm, kFixupThreads, 0, st>>>(d);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// spec_half (binary32, 2D square grids): also the first axis of the fields'
// power spectrum, half[2R][n][n/2+1] (k_cols_spec).
template <typename T>
static cf_status sample_impl(const cf_embedding* e, uint64_t seed, uint64_t r0, int R, void* fields,
                             const cf_lp_params* lp, void* ws, size_t ws_bytes, double amp_scale,
                             cudaStream_t st, C2<float>* spec_half = nullptr) {
    const GridInfo& g = e->grid;
    const size_t elem = sizeof(C2<T>);
    const SamplerTuning tn = tuned_of(g, elem);
    const int chunk = pick_chunk(g, elem, R, ws_bytes);
    if (chunk < 1) return fail(CF_ERR_NOMEM, "workspace of %zu bytes holds no realization (%zu needed)", ws_bytes,
                               per_realization_bytes(g, elem));
    if (sizeof(T) == 8) CF_TRY(ensure_s64(const_cast<cf_embedding*>(e), st));
    const T* s = sizeof(T) == 4 ? (const T*)(const void*)e->s32 : (const T*)(const void*)e->s64;
    const long long cells = g.ncell;
    const int d = g.ndim;
    C2<T>* buf1 = (C2<T>*)ws;
    C2<T>* buf2 = nullptr;
    if (d == 3) buf2 = buf1 + (size_t)chunk * g.m[0] * g.m[1] * g.n[2];
    const PoissonDefer defer = lp ? defer_list(g, elem, chunk, ws, ws_bytes) : PoissonDefer{};
    for (int c0 = 0; c0 < R; c0 += chunk) {
        const int nr = (R - c0) < chunk ? (R - c0) : chunk;
        FieldEpi<T> epi{};
        epi.defer = defer;
        epi.fields = fields ? (T*)fields + (size_t)c0 * 2 * cells : nullptr;
        epi.cells = cells;
        epi.r0 = (uint32_t)(r0 + (uint64_t)c0);
        if (lp) {
            epi.counts = lp->counts_out + (size_t)c0 * 2 * cells;
            epi.delta = lp->delta_out ? lp->delta_out + (size_t)c0 * 2 * cells : nullptr;
            epi.f = lp->f;
            epi.half_sigma2 = 0.5 * lp->sigma2;
            epi.half_sigma2_f = (float)(0.5 * lp->sigma2);
            epi.nbar = lp->nbar;
            epi.nbar_f = (float)lp->nbar;
            epi.pkey0 = (uint32_t)lp->seed;
            epi.pkey1 = (uint32_t)(lp->seed >> 32);
        }
        const uint32_t rr0 = (uint32_t)(r0 + (uint64_t)c0);
        const long long Ml = g.m[d - 1];
        const long long nrows = g.mtotal / Ml;
        if constexpr (sizeof(T) == 4) {
            if (tn.persistent && !spec_half && persistent_ok(g)) {
                CF_TRY(launch_sample_persistent(g, s, (float)amp_scale, seed, rr0, nr, buf1, buf2, epi, defer, nullptr,
                                                st));
                continue;
            }
        }
        CF_TRY(defer_begin(defer, st));
        if (d == 1) {
            CF_TRY(launch_sample_rows<T>(Ml, (int)g.n[d - 1], s, (T)amp_scale, seed, rr0, nr, nrows, nullptr, 1, epi, st));
        } else if (d == 2) {
            CF_TRY(launch_sample_rows<T>(Ml, (int)g.n[d - 1], s, (T)amp_scale, seed, rr0, nr, nrows, buf1, 0, epi, st, nullptr,
                                             tn.rows_shape));
            // pass 2: columns of [chunk][M0][N1], keep N0, fields epilogue
            if constexpr (sizeof(T) == 4) {
                if (spec_half) {
                    CF_TRY(launch_cols_spec_any(g.m[0], buf1, nr, epi, spec_half, 2 * (long long)c0, st));
                    CF_TRY(defer_end(defer, st));
                    continue;
                }
            }
            CF_TRY(launch_sampler_cols<T>(g.m[0], buf1, nr, g.n[1], nullptr, 1, epi, st, g.n[0], tn.cols_shape));
        } else {
            CF_TRY(launch_sample_rows<T>(Ml, (int)g.n[d - 1], s, (T)amp_scale, seed, rr0, nr, nrows, buf1, 0, epi, st, nullptr,
                                             tn.rows_shape));
            // pass 2: axis 1 of [chunk*M0][M1][N2] -> [chunk*M0][N1][N2]
            CF_TRY(launch_sampler_cols<T>(g.m[1], buf1, (long long)nr * g.m[0], g.n[2], buf2, 0, epi, st, g.n[1],
                                          tn.cols_shape));
            // pass 3: axis 0 of [chunk][M0][N1*N2] -> fields
            CF_TRY(launch_sampler_cols<T>(g.m[0], buf2, nr, g.n[1] * g.n[2], nullptr, 1, epi, st, g.n[0],
                                          tn.cols_shape));
        }
        CF_TRY(defer_end(defer, st));
    }
    record_use(const_cast<cf_embedding*>(e), st);
    return CF_OK;
}

static bool is_tc(cf_dtype dt) { return dt == CF_BF16_TC || dt == CF_F16_TC; }

static cf_status check_sample_args(const cf_embedding* e, uint64_t r0, int32_t R, cf_dtype dt, bool tc_ok = false) {
    if (!e) return fail(CF_ERR_ARG, "embedding is NULL");
    if (R < 0) return fail(CF_ERR_ARG, "R must be >= 0");
    if (is_tc(dt)) {
        if (!tc_ok) return fail(CF_ERR_UNSUPPORTED, "dtype %d is available in cf_sample only", dt);
        CF_TRY(tc_check_grid(e->grid));
    } else if (dt != CF_F32 && dt != CF_F64) {
        return fail(CF_ERR_UNSUPPORTED, "dtype %d not supported by this call", dt);
    }
    if (r0 + (uint64_t)R > (1ull << 32)) return fail(CF_ERR_ARG, "realization index exceeds 32 bits");
    return CF_OK;
}

// ----------------------------------------------------------------- noise draw
__global__ void k_noise_f32(uint32_t key0, uint32_t key1, uint32_t r0, long long ncells, long long m_last,
                            C2<float>* __restrict__ out) {
    const long long half = m_last / 2;
    const long long npairs = ncells / 2;
    const uint32_t r = r0 + blockIdx.y;
    C2<float>* o = out + (size_t)blockIdx.y * ncells;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npairs;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / half, c = p % half;
        C2<float> lo, hi;
        noise_pair_f32((unsigned long long)p, r, key0, key1, lo, hi);
        o[row * m_last + c] = lo;
        o[row * m_last + c + half] = hi;
    }
}

__global__ void k_noise_f64(uint32_t key0, uint32_t key1, uint32_t r0, long long ncells, C2<double>* __restrict__ out) {
    const uint32_t r = r0 + blockIdx.y;
    C2<double>* o = out + (size_t)blockIdx.y * ncells;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ncells;
         k += (long long)gridDim.x * blockDim.x)
        o[k] = noise_f64((unsigned long long)k, r, key0, key1);
}

// Batched binary32 sampler (serving): nreal realizations described by
// desc (device array) on grid g, all writing fields (and counts) through their
// descriptors; ws holds the chunk intermediates.
cf_status sample_batch_f32(const GridInfo& g, const RealDesc* desc, int nreal, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    const size_t elem = sizeof(C2<float>);
    const SamplerTuning tn = tuned_of(g, elem);
    const int chunk = pick_chunk(g, elem, nreal, ws_bytes);
    if (chunk < 1) return fail(CF_ERR_NOMEM, "batch workspace too small");
    const long long cells = g.ncell;
    const int d = g.ndim;
    C2<float>* buf1 = (C2<float>*)ws;
    C2<float>* buf2 = d == 3 ? buf1 + (size_t)chunk * g.m[0] * g.m[1] * g.n[2] : nullptr;
    const long long Ml = g.m[d - 1];
    const long long nrows = g.mtotal / Ml;
    const PoissonDefer defer = defer_list(g, elem, chunk, ws, ws_bytes);
    for (int c0 = 0; c0 < nreal; c0 += chunk) {
        const int nr = (nreal - c0) < chunk ? (nreal - c0) : chunk;
        FieldEpi<float> epi{};
        epi.cells = cells;
        epi.desc = desc + c0;
        epi.defer = defer;
        if (tn.persistent && persistent_ok(g)) {
            CF_TRY(launch_sample_persistent(g, nullptr, 1.0f, 0, 0, nr, buf1, buf2, epi, defer, desc + c0, st));
            continue;
        }
        CF_TRY(defer_begin(defer, st));
        if (d == 1) {
            CF_TRY(launch_sample_rows<float>(Ml, (int)g.n[d - 1], nullptr, 1.0f, 0, 0, nr, nrows, nullptr, 1, epi, st, desc + c0));
        } else if (d == 2) {
            CF_TRY(launch_sample_rows<float>(Ml, (int)g.n[d - 1], nullptr, 1.0f, 0, 0, nr, nrows, buf1, 0, epi, st, desc + c0,
                                             tn.rows_shape));
            CF_TRY(launch_sampler_cols<float>(g.m[0], buf1, nr, g.n[1], nullptr, 1, epi, st, g.n[0], tn.cols_shape));
        } else {
            CF_TRY(launch_sample_rows<float>(Ml, (int)g.n[d - 1], nullptr, 1.0f, 0, 0, nr, nrows, buf1, 0, epi, st, desc + c0,
                                             tn.rows_shape));
            CF_TRY(launch_sampler_cols<float>(g.m[1], buf1, (long long)nr * g.m[0], g.n[2], buf2, 0, epi, st, g.n[1],
                                              tn.cols_shape));
            CF_TRY(launch_sampler_cols<float>(g.m[0], buf2, nr, g.n[1] * g.n[2], nullptr, 1, epi, st, g.n[0],
                                              tn.cols_shape));
        }
        CF_TRY(defer_end(defer, st));
    }
    return CF_OK;
}

size_t sample_chunk_bytes(const GridInfo& g, int nreal) {
    const size_t elem = sizeof(C2<float>);
    return chunk_bytes(g, elem, (size_t)pick_chunk(g, elem, nreal < 1 ? 1 : nreal, (size_t)-1));
}

// Entry for cf_sample_noalloc (cf_noalloc.cu): the binary32 sampler into a
// given workspace, and the intermediate bytes one realization needs.
cf_status sample_f32_into(const cf_embedding* e, uint64_t seed, uint64_t r0, int R, void* fields, void* ws,
                          size_t ws_bytes, cudaStream_t st) {
    return sample_impl<float>(e, seed, r0, R, fields, nullptr, ws, ws_bytes, 1.0, st);
}

size_t sample_bytes_per_realization(const cf_embedding* e, cf_dtype dt) {
    return per_realization_bytes(e->grid, dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>));
}

}  // namespace cf

using namespace cf;

extern "C" cf_status cf_sample_workspace_size(const cf_embedding* e, int32_t R, cf_dtype dt, size_t* bytes) {
    clear_error();
    if (!e || !bytes) return fail(CF_ERR_ARG, "NULL argument");
    if (is_tc(dt)) {
        CF_TRY(tc_check_grid(e->grid));
        const int chunk = pick_chunk(e->grid, 4, R < 1 ? 1 : R, (size_t)-1);
        *bytes = tc_header_bytes() + tc_bytes_per_realization(e->grid) * (size_t)(chunk < 1 ? 1 : chunk);
        return CF_OK;
    }
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d not supported by this call", dt);
    const size_t elem = dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>);
    int chunk = pick_chunk(e->grid, elem, R < 1 ? 1 : R, (size_t)-1);
    *bytes = chunk_bytes(e->grid, elem, (size_t)(chunk < 1 ? 1 : chunk));
    return CF_OK;
}

extern "C" cf_status cf_sample(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, cf_dtype dt,
                               void* fields_out, void* ws, size_t ws_bytes, cf_stream_t s) {
    clear_error();
    CF_TRY(check_sample_args(e, r0, R, dt, true));
    if (!fields_out) return fail(CF_ERR_ARG, "fields_out is NULL");
    if (R == 0) return CF_OK;
    CF_TRY(enter_with(e, (cudaStream_t)s));
    if (is_tc(dt)) {
        const size_t head = tc_header_bytes();
        const int chunk = ws && ws_bytes > head ? pick_chunk(e->grid, 4, R, ws_bytes - head) : 0;
        if (chunk < 1)
            return fail(CF_ERR_NOMEM, "workspace of %zu bytes holds no realization (%zu needed)", ws_bytes,
                        head + tc_bytes_per_realization(e->grid));
        CF_TRY(sample_tc(e, dt == CF_BF16_TC, seed, r0, R, (float*)fields_out, ws, ws_bytes, chunk, 1.0,
                         (cudaStream_t)s));
        record_use(const_cast<cf_embedding*>(e), (cudaStream_t)s);
        return CF_OK;
    }
    if (dt == CF_F32) return sample_impl<float>(e, seed, r0, R, fields_out, nullptr, ws, ws_bytes, 1.0, (cudaStream_t)s);
    return sample_impl<double>(e, seed, r0, R, fields_out, nullptr, ws, ws_bytes, 1.0, (cudaStream_t)s);
}

extern "C" cf_status cf_sample_lp(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, cf_dtype dt,
                                  void* fields_out, const cf_lp_params* lp, void* ws, size_t ws_bytes,
                                  cf_stream_t s) {
    clear_error();
    CF_TRY(check_sample_args(e, r0, R, dt));
    if (dt != CF_F32) return fail(CF_ERR_UNSUPPORTED, "the fused lognormal/Poisson epilogue is binary32 only");
    if (!lp || !lp->counts_out) return fail(CF_ERR_ARG, "lp and lp->counts_out are required");
    if (!(lp->nbar >= 0.0)) return fail(CF_ERR_ARG, "nbar must be >= 0");
    if (R == 0) return CF_OK;
    CF_TRY(enter_with(e, (cudaStream_t)s));
    return sample_impl<float>(e, seed, r0, R, fields_out, lp, ws, ws_bytes, 1.0, (cudaStream_t)s);
}

// Time of sample_impl on R realizations under tuning t (one warm-up run,
// then the mean of two), or a negative status.
static cf_status time_schedule(const cf_embedding* e, cf_dtype dt, int32_t R, void* ws, size_t ws_bytes,
                               void* fields, const std::string& key, SamplerTuning t, cudaStream_t st,
                               cudaEvent_t a, cudaEvent_t b, float* ms) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = t;
    }
    cf_status r = CF_OK;
    for (int rep = 0; rep < 3 && r == CF_OK; ++rep) {
        if (rep == 1) CF_CUDA(cudaEventRecord(a, st));
        r = dt == CF_F32 ? sample_impl<float>(e, 1, 0, R, fields, nullptr, ws, ws_bytes, 1.0, st)
                         : sample_impl<double>(e, 1, 0, R, fields, nullptr, ws, ws_bytes, 1.0, st);
    }
    if (r != CF_OK) return r;
    CF_CUDA(cudaEventRecord(b, st));
    CF_CUDA(cudaEventSynchronize(b));
    CF_CUDA(cudaEventElapsedTime(ms, a, b));
    *ms *= 0.5f;
    return CF_OK;
}

extern "C" cf_status cf_tune_sample(const cf_embedding* e, cf_dtype dt, int32_t R, void* ws, size_t ws_bytes,
                                    void* fields_scratch, cf_stream_t s, int32_t* chunk_out, double* ms_out) {
    clear_error();
    CF_TRY(check_sample_args(e, 0, R, dt));
    if (R < 1 || !fields_scratch) return fail(CF_ERR_ARG, "R >= 1 and fields_scratch are required");
    CF_TRY(enter_with(e, (cudaStream_t)s));
    const cudaStream_t st = (cudaStream_t)s;
    const size_t elem = dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>);
    const size_t per = per_realization_bytes(e->grid, elem);
    const std::string key = tune_key(e->grid, elem);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned.erase(key);
    }
    cudaEvent_t a, b;
    CF_CUDA(cudaEventCreate(&a));
    CF_CUDA(cudaEventCreate(&b));
    auto done = [&](cf_status r) {
        if (r != CF_OK) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned.erase(key);
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return r;
    };
    SamplerTuning best{};
    float best_ms = 1e30f;
    // 1. realizations per launch, default CTA shapes
    for (int c = 1; c <= R; c *= 2) {
        if (per > 0 && per * (size_t)c > ws_bytes) break;
        SamplerTuning t{};
        t.chunk = c;
        float ms = 0.f;
        const cf_status r = time_schedule(e, dt, R, ws, ws_bytes, fields_scratch, key, t, st, a, b, &ms);
        if (r != CF_OK) return done(r);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
        if (per == 0) break;  // one-dimensional grids have no intermediate
    }
    // 2. CTA shapes of the paired binary32 passes at that chunk (lines of
    // 256 points or more have three shapes each; every shape gives the same
    // results bit for bit)
    bool shaped = false;
    for (int a2 = 0; a2 < e->grid.ndim; ++a2) shaped = shaped || e->grid.m[a2] >= 256;
    if (dt == CF_F32 && e->grid.ndim >= 2 && shaped && (pair_rows() || pair_cols())) {
        const SamplerTuning base = best;
        const int ncs = pair_cols() ? kPairShapes : 1;
        for (int rs = 0; rs < (pair_rows() ? kPairShapes : 1); ++rs)
            for (int cs = 0; cs < ncs; ++cs) {
                if (rs == 0 && cs == 0) continue;
                SamplerTuning t = base;
                t.rows_shape = rs;
                t.cols_shape = cs;
                float ms = 0.f;
                const cf_status r = time_schedule(e, dt, R, ws, ws_bytes, fields_scratch, key, t, st, a, b, &ms);
                if (r != CF_OK) return done(r);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
    }
    // 3. the whole chunk in one persistent cooperative launch (small binary32 grids)
    if (dt == CF_F32 && persistent_ok(e->grid)) {
        SamplerTuning t = best;
        t.persistent = 1;
        float ms = 0.f;
        const cf_status r = time_schedule(e, dt, R, ws, ws_bytes, fields_scratch, key, t, st, a, b, &ms);
        if (r != CF_OK) return done(r);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    if (chunk_out) *chunk_out = best.chunk;
    if (ms_out) *ms_out = (double)best_ms / (double)R;
    return done(CF_OK);
}

extern "C" cf_status cf_tune_set(const cf_embedding* e, cf_dtype dt, int32_t chunk, int32_t rows_shape,
                                 int32_t cols_shape, int32_t persistent) {
    clear_error();
    if (!e) return fail(CF_ERR_ARG, "embedding is NULL");
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d", dt);
    if (chunk < 0 || chunk > 65535) return fail(CF_ERR_ARG, "chunk must be 0..65535");
    if (rows_shape < 0 || rows_shape >= kPairShapes || cols_shape < 0 || cols_shape >= kPairShapes)
        return fail(CF_ERR_ARG, "shapes must be 0..%d", kPairShapes - 1);
    if (persistent != 0 && persistent != 1) return fail(CF_ERR_ARG, "persistent must be 0 or 1");
    if (persistent && (dt != CF_F32 || !persistent_ok(e->grid)))
        return fail(CF_ERR_UNSUPPORTED, "the persistent sampler takes binary32 grids with embedded sides 64 or 128");
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) CF_CUDA(cudaSetDevice(e->device));
    const std::string key = tune_key(e->grid, dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>));
    if (dev != e->device) CF_CUDA(cudaSetDevice(dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (chunk == 0 && rows_shape == 0 && cols_shape == 0 && persistent == 0)
        g_tuned.erase(key);
    else
        g_tuned[key] = SamplerTuning{chunk, rows_shape, cols_shape, persistent};
    return CF_OK;
}

extern "C" cf_status cf_tune_info(const cf_embedding* e, cf_dtype dt, int32_t* chunk, int32_t* rows_shape,
                                  int32_t* cols_shape, int32_t* persistent) {
    clear_error();
    if (!e) return fail(CF_ERR_ARG, "embedding is NULL");
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d", dt);
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) CF_CUDA(cudaSetDevice(e->device));
    const SamplerTuning t = tuned_of(e->grid, dt == CF_F32 ? sizeof(C2<float>) : sizeof(C2<double>));
    if (dev != e->device) CF_CUDA(cudaSetDevice(dev));
    if (chunk) *chunk = t.chunk;
    if (rows_shape) *rows_shape = t.rows_shape;
    if (cols_shape) *cols_shape = t.cols_shape;
    if (persistent) *persistent = t.persistent;
    return CF_OK;
}

extern "C" cf_status cf_draw_noise(uint64_t seed, uint64_t r0, int32_t R, int64_t ncells, int64_t m_last,
                                   cf_dtype dt, void* out, cf_stream_t s) {
    clear_error();
    if (!out) return fail(CF_ERR_ARG, "out is NULL");
    if (R < 0 || ncells < 0) return fail(CF_ERR_ARG, "negative size");
    if (R > 65535) return fail(CF_ERR_UNSUPPORTED, "at most 65535 realizations per call");
    if (r0 + (uint64_t)R > (1ull << 32)) return fail(CF_ERR_ARG, "realization index exceeds 32 bits");
    if (dt != CF_F32 && dt != CF_F64) return fail(CF_ERR_UNSUPPORTED, "dtype %d not supported by this call", dt);
    if (dt == CF_F32 && (m_last < 2 || (m_last & 1) || ncells % m_last))
        return fail(CF_ERR_ARG, "m_last must be even and divide ncells");
    if (R == 0 || ncells == 0) return CF_OK;
    CF_TRY(enter((cudaStream_t)s));
    const dim3 grid((unsigned)grid_blocks(dt == CF_F32 ? ncells / 2 : ncells, 256, 2048), (unsigned)R);
    ScopedKernelTimer kt((cudaStream_t)s, dt == CF_F32 ? "noise_f32" : "noise_f64");
    if (dt == CF_F32) {
        k_noise_f32<<<grid, 256, 0, (cudaStream_t)s>>>((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)r0, ncells,
                                                      m_last, (C2<float>*)out);
    } else if (dt == CF_F64) {
        k_noise_f64<<<grid, 256, 0, (cudaStream_t)s>>>((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)r0, ncells,
                                                      (C2<double>*)out);
    } else {
        return fail(CF_ERR_UNSUPPORTED, "dtype %d not supported by this call", dt);
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}

// ------------------------------------------------------------- fused spectra
static cf_status spectra_layout(const cf_embedding* e, int32_t R, const cf_bins* bins, cf_grid* grid, size_t* acc,
                                size_t* half) {
    const GridInfo& g = e->grid;
    if (g.ndim != 2 || g.n[0] != g.n[1] || g.m[0] != 2 * g.n[0] || g.m[1] != 2 * g.n[1] || g.m[0] < 256 ||
        g.m[0] > 4096)
        return fail(CF_ERR_UNSUPPORTED, "fused spectra need a square 2D survey of side 128..2048 embedded in 2n");
    if (g.cell[0] != g.cell[1]) return fail(CF_ERR_UNSUPPORTED, "fused spectra need equal cell sides");
    if (R < 1 || 2ll * R > 65535) return fail(CF_ERR_ARG, "R must be 1..32767");
    *grid = cf_grid{};
    grid->ndim = 2;
    grid->embed_factor = 2;
    for (int a = 0; a < 2; ++a) {
        grid->n[a] = g.n[a];
        grid->cell[a] = g.cell[a];
    }
    *acc = pk_halves_acc_bytes(grid, 2ll * R, bins);
    if (*acc == 0) return fail(CF_ERR_ARG, "invalid bins for the power spectrum");
    *half = sizeof(C2<float>) * 2 * (size_t)R * (size_t)g.n[0] * (size_t)(g.n[1] / 2 + 1);
    return CF_OK;
}

extern "C" cf_status cf_sample_spectra_workspace_size(const cf_embedding* e, int32_t R, const cf_bins* bins,
                                                      size_t* pk_ws_bytes) {
    clear_error();
    if (!e || !bins || !pk_ws_bytes) return fail(CF_ERR_ARG, "NULL argument");
    cf_grid grid;
    size_t acc = 0, half = 0;
    CF_TRY(spectra_layout(e, R, bins, &grid, &acc, &half));
    *pk_ws_bytes = acc + half;
    return CF_OK;
}

extern "C" cf_status cf_sample_spectra(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R, float* fields_out,
                                       const cf_lp_params* lp, const cf_bins* bins, double* pk_out,
                                       int64_t* nmodes_out, double* mean_or_null, double* cov_or_null, void* ws,
                                       size_t ws_bytes, void* pk_ws, size_t pk_ws_bytes, cf_event_t sampled,
                                       cf_stream_t s) {
    clear_error();
    CF_TRY(check_sample_args(e, r0, R, CF_F32));
    if (!fields_out || !bins || !pk_out || !nmodes_out) return fail(CF_ERR_ARG, "fields, bins, pk and nmodes are required");
    if (lp && !lp->counts_out) return fail(CF_ERR_ARG, "lp->counts_out is required");
    if (lp && !(lp->nbar >= 0.0)) return fail(CF_ERR_ARG, "nbar must be >= 0");
    cf_grid grid;
    size_t acc = 0, half = 0;
    CF_TRY(spectra_layout(e, R, bins, &grid, &acc, &half));
    if (!pk_ws || pk_ws_bytes < acc + half)
        return fail(CF_ERR_NOMEM, "spectra workspace of %zu bytes, %zu needed", pk_ws_bytes, acc + half);
    const cudaStream_t st = (cudaStream_t)s;
    CF_TRY(enter_with(e, st));
    C2<float>* halves = (C2<float>*)((char*)pk_ws + acc);
    CF_TRY(sample_impl<float>(e, seed, r0, R, fields_out, lp, ws, ws_bytes, 1.0, st, halves));
    if (sampled) CF_CUDA(cudaEventRecord((cudaEvent_t)sampled, st));
    return pk_from_halves_f32(&grid, 2ll * R, bins, halves, pk_out, nmodes_out, mean_or_null, cov_or_null,
                              (char*)pk_ws, st);
}
