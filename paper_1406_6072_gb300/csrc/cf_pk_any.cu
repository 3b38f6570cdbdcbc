// cf_pk_any.cu -- step d1 on any survey box: rectangular grids and sides that
// are not powers of two, in one to three dimensions (section 3.2, eq.
// (Def spec); the estimator has no shape restriction).
//
// Mode m of a box with sides L_d = n_d cell_d has wavevector k_d = 2 pi s_d /
// L_d (s_d the signed index).  |k| is measured in units of the fundamental
// 2 pi / L_ref of the longest side: q = sqrt(sum_d (s_d r_d)^2), r_d = L_ref /
// L_d, every operation rounded in binary64 in this order, so a mode's bin is
// the same bit-exact decision on the host-side reference and here (for a cube
// r_d = 1 and q is the integer index length of the cubic path in cf_pk.cu).
//
// Two real fields travel as one complex array z = a + i b through full
// complex transforms along every axis; the binning pass separates
// A_k = (Z_k + conj Z_-k)/2 and B_k = (Z_k - conj Z_-k)/2i at each mode and
// bins |A|^2, |B|^2 through a per-mode bin table (cached per grid and edges).
// A power-of-two side runs the Stockham line transform directly; any other
// side N runs Bluestein's chirp-z algorithm (1968): with c_n = e^{-pi i n^2/N},
// X_k = c_k sum_n (x_n c_n) conj(c_{k-n}), a convolution done as two
// power-of-two transforms of length P >= 2N - 1 with the transform of the
// chirp precomputed in binary64.
#include <math.h>

#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "cf_kernels.cuh"

namespace cf {

constexpr int kAnyMaxBins = 512;

struct AnyEdges {
    double e[kAnyMaxBins + 1];
};

// CTA shape of the any-length line passes: 8 points per thread, 256 threads.
template <typename T, int P>
struct AnyCfg : TileCfg<T, P, 8, 256, 4> {};

// Transform of every line of length N along the middle axis of
// data[outer][N][inner] (in place).  COLS: the CTA takes LINES consecutive
// inner indices of one outer slice (coalesced loads across the lines); else
// LINES consecutive rows (inner == 1).  BLUE: Bluestein through length P;
// otherwise N == P.
template <typename T, int P, bool BLUE, bool COLS>
__global__ void __launch_bounds__(AnyCfg<T, P>::THREADS, AnyCfg<T, P>::MINB)
    k_any_lines(C2<T>* data, long long outer, long long inner, int N, const C2<T>* __restrict__ chirp,
                const C2<T>* __restrict__ bhat, const C2<T>* __restrict__ tw) {
    using Cfg = AnyCfg<T, P>;
    using G = typename Cfg::G;
    constexpr int E = G::E;
    constexpr int LINES = Cfg::LINES;
    constexpr int STEP = P / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
    int line, j;
    long long o, i;
    bool valid;
    if constexpr (COLS) {
        line = threadIdx.x % LINES;
        j = threadIdx.x / LINES;
        const long long tiles = (inner + LINES - 1) / LINES;
        o = (long long)blockIdx.x / tiles;
        i = ((long long)blockIdx.x % tiles) * LINES + line;
        valid = i < inner;
    } else {
        line = threadIdx.x / G::TL;
        j = threadIdx.x % G::TL;
        o = (long long)blockIdx.x * LINES + line;
        i = 0;
        valid = o < outer;
    }
    C2<T>* base = data + (size_t)(valid ? o : 0) * (size_t)N * (size_t)inner + (size_t)(valid ? i : 0);
    using Lay = typename std::conditional<COLS, ColLayout<E, LINES>, RowLayout<G::PADE, G::PADDED>>::type;
    const Lay lay;
    C2<T> v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int p = j + q * STEP;
        C2<T> x = mk((T)0, (T)0);
        if (p < N) {
            x = base[(size_t)p * (size_t)inner];
            if constexpr (BLUE) x = cmul(x, chirp[p]);
        }
        v[q] = x;
    }
    if constexpr (BLUE) {
        auto to_smem = [&](int ln, int p, C2<T> val) { sm[lay(ln, p)] = val; };
        line_fft<T, P, -1, P, true>(sm, lay, line, j, v, tw, to_smem);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int p = j + q * STEP;
            v[q] = cmul(sm[lay(line, p)], bhat[p]);
        }
        auto sink = [&](int, int p, C2<T> val) {
            if (valid && p < N) base[(size_t)p * (size_t)inner] = cmul(val, chirp[p]);
        };
        line_fft<T, P, +1, P>(sm, lay, line, j, v, tw, sink);
    } else {
        auto sink = [&](int, int p, C2<T> val) {
            if (valid) base[(size_t)p * (size_t)inner] = val;
        };
        line_fft<T, P, -1, P>(sm, lay, line, j, v, tw, sink);
    }
}

// Box geometry for the kernels below.
struct AnyGrid {
    int ndim;
    long long n[3];
    long long cells;
};

__device__ __forceinline__ long long any_signed(long long i, long long n) { return 2 * i <= n ? i : i - n; }

// Bin of every mode (int16, -1: not binned) and the modes per bin.
__global__ void k_any_modebins(AnyGrid g, double r0, double r1, double r2, AnyEdges ed, int nbins,
                               int16_t* __restrict__ bin_of, unsigned long long* __restrict__ nmodes) {
    const double r[3] = {r0, r1, r2};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.cells;
         t += (long long)gridDim.x * blockDim.x) {
        long long rem = t;
        long long sv[3] = {0, 0, 0};
        for (int d = g.ndim - 1; d >= 0; --d) {
            const long long idx = rem % g.n[d];
            rem /= g.n[d];
            sv[d] = any_signed(idx, g.n[d]);
        }
        double q2 = 0.0;
        for (int d = 0; d < g.ndim; ++d) {
            const double x = __dmul_rn((double)sv[d], r[d]);
            q2 = __dadd_rn(q2, __dmul_rn(x, x));
        }
        int b = -1;
        if (q2 != 0.0) {
            const double kn = __dsqrt_rn(q2);
            if (kn >= ed.e[0] && kn < ed.e[nbins]) {
                b = 0;
                while (!(kn < ed.e[b + 1])) ++b;
            }
        }
        bin_of[t] = (int16_t)b;
        if (b >= 0) atomicAdd(&nmodes[b], 1ull);
    }
}

// Count totals per field (the N_tot of eq. (Estim)) and, for field 0's
// block row, the sum of the surface fraction.
__global__ void k_any_totals(const int32_t* __restrict__ counts, const float* __restrict__ f, long long cells,
                             long long f0, unsigned long long* __restrict__ ntot, double* __restrict__ fsum) {
    const long long fld = f0 + blockIdx.y;
    const int32_t* c = counts + (size_t)fld * (size_t)cells;
    unsigned long long n = 0;
    double fs = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells;
         i += (long long)gridDim.x * blockDim.x) {
        n += (unsigned long long)(long long)c[i];
        if (blockIdx.y == 0 && f0 == 0) fs += f ? (double)f[i] : 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_down_sync(0xffffffffu, n, o);
        fs += __shfl_down_sync(0xffffffffu, fs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n) atomicAdd(&ntot[fld], n);
        if (blockIdx.y == 0 && f0 == 0) atomicAdd(fsum, fs);
    }
}

enum { ANY_FLOAT = 0, ANY_DOUBLE = 1, ANY_COUNTS = 2 };

// z[pair][cells] = a + i b for fields (f0 + 2 pair, f0 + 2 pair + 1); count
// maps become delta_g = (N/f - Nhat)/Nhat on f != 0 (0 elsewhere).
template <typename T, int KIND>
__global__ void k_any_pack(const void* __restrict__ fields, const float* __restrict__ f, long long cells,
                           long long nfields, long long f0, const unsigned long long* __restrict__ ntot,
                           const double* __restrict__ fsum, C2<T>* __restrict__ z) {
    const long long fa = f0 + 2ll * blockIdx.y, fb = fa + 1;
    const bool hasb = fb < nfields;
    double nha = 0.0, nhb = 0.0;
    if constexpr (KIND == ANY_COUNTS) {
        const double fs = *fsum;
        nha = fs > 0.0 ? (double)ntot[fa] / fs : 0.0;
        nhb = (hasb && fs > 0.0) ? (double)ntot[fb] / fs : 0.0;
    }
    C2<T>* out = z + (size_t)blockIdx.y * (size_t)cells;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells;
         i += (long long)gridDim.x * blockDim.x) {
        T a = (T)0, b = (T)0;
        if constexpr (KIND == ANY_FLOAT) {
            const float* x = (const float*)fields;
            a = (T)x[(size_t)fa * cells + i];
            if (hasb) b = (T)x[(size_t)fb * cells + i];
        } else if constexpr (KIND == ANY_DOUBLE) {
            const double* x = (const double*)fields;
            a = (T)x[(size_t)fa * cells + i];
            if (hasb) b = (T)x[(size_t)fb * cells + i];
        } else {
            const int32_t* x = (const int32_t*)fields;
            const double fi = f ? (double)f[i] : 1.0;
            if (fi != 0.0) {
                if (nha > 0.0) a = (T)(((double)x[(size_t)fa * cells + i] / fi - nha) / nha);
                if (hasb && nhb > 0.0) b = (T)(((double)x[(size_t)fb * cells + i] / fi - nhb) / nhb);
            }
        }
        out[i] = mk(a, b);
    }
}

// Binning: for pair p of the chunk, A and B at every mode t (and its mirror
// -t), |A|^2 and |B|^2 summed per bin in shared memory, then one atomic add
// per bin and field into acc[field][bin].
template <typename T>
__global__ void k_any_bin(const C2<T>* __restrict__ z, AnyGrid g, const int16_t* __restrict__ bin_of, int nbins,
                          long long nfields, long long f0, double* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* sa = reinterpret_cast<double*>(smraw);
    double* sb = sa + nbins;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        sa[b] = 0.0;
        sb[b] = 0.0;
    }
    __syncthreads();
    const long long fa = f0 + 2ll * blockIdx.y, fb = fa + 1;
    const bool hasb = fb < nfields;
    const C2<T>* zp = z + (size_t)blockIdx.y * (size_t)g.cells;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.cells;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = bin_of[t];
        if (b < 0) continue;
        long long rem = t, tm = 0, stride = 1;
        for (int d = g.ndim - 1; d >= 0; --d) {
            const long long idx = rem % g.n[d];
            rem /= g.n[d];
            tm += (idx == 0 ? 0 : g.n[d] - idx) * stride;
            stride *= g.n[d];
        }
        const C2<T> Z = zp[t], Zm = zp[tm];
        const double ax = 0.5 * ((double)Z.x + (double)Zm.x), ay = 0.5 * ((double)Z.y - (double)Zm.y);
        atomicAdd(&sa[b], ax * ax + ay * ay);
        if (hasb) {
            const double bx = 0.5 * ((double)Z.y + (double)Zm.y), by = 0.5 * ((double)Zm.x - (double)Z.x);
            atomicAdd(&sb[b], bx * bx + by * by);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (sa[b] != 0.0) atomicAdd(&acc[(size_t)fa * nbins + b], sa[b]);
        if (hasb && sb[b] != 0.0) atomicAdd(&acc[(size_t)fb * nbins + b], sb[b]);
    }
}

// ----------------------------------------------------------------- host side
static size_t any_align(size_t v) { return (v + 255) & ~(size_t)255; }

// Bluestein length for side N (N itself for powers of two).
static long long blue_length(long long N) {
    if (is_pow2(N)) return N;
    long long P = 1;
    while (P < 2 * N - 1) P <<= 1;
    return P;
}

bool pk_any_needed(const cf_grid* g) {
    if (!g || g->ndim < 1 || g->ndim > 3) return false;
    if (g->ndim == 1) return true;
    for (int a = 0; a < g->ndim; ++a)
        if (g->n[a] != g->n[0] || !is_pow2(g->n[a]) || g->cell[a] != g->cell[0]) return true;
    return false;
}

struct AnyPlan {
    AnyGrid g;
    double cell[3];
    double r[3];
    int nbins;
    AnyEdges edges;
    size_t elem;
    long long pairs_chunk;
    size_t off_bin, off_nmodes, off_mu, off_acc, off_ntot, off_fsum, off_z, total;
};

cf_status pk_bin_edges(const cf_bins* b, double kmax_default, double* e);

static cf_status any_plan(const cf_grid* grid, long long nfields, const cf_bins* b, size_t elem, AnyPlan* P) {
    if (!grid) return fail(CF_ERR_ARG, "grid is NULL");
    if (!b) return fail(CF_ERR_ARG, "bins is NULL");
    if (grid->ndim < 1 || grid->ndim > 3) return fail(CF_ERR_ARG, "ndim must be 1, 2 or 3");
    if (b->nbins < 1 || b->nbins > kAnyMaxBins) return fail(CF_ERR_ARG, "nbins must be 1..%d", kAnyMaxBins);
    AnyGrid& g = P->g;
    g.ndim = grid->ndim;
    g.cells = 1;
    double lref = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (a < g.ndim) {
            g.n[a] = grid->n[a];
            P->cell[a] = grid->cell[a];
            if (g.n[a] < 1) return fail(CF_ERR_ARG, "n[%d] must be >= 1", a);
            if (!(P->cell[a] > 0.0)) return fail(CF_ERR_ARG, "cell must be > 0");
            if (is_pow2(g.n[a]) ? g.n[a] > kMaxLine : g.n[a] > kMaxLine / 2)
                return fail(CF_ERR_UNSUPPORTED,
                            "power spectrum sides up to %lld (powers of two) or %lld (other sizes); n[%d] = %lld",
                            kMaxLine, kMaxLine / 2, a, g.n[a]);
            const double L = (double)g.n[a] * P->cell[a];
            if (L > lref) lref = L;
        } else {
            g.n[a] = 1;
            P->cell[a] = 1.0;
        }
        g.cells *= g.n[a];
    }
    double kmax_default = 0.0;
    for (int a = 0; a < 3; ++a) {
        P->r[a] = a < g.ndim ? lref / ((double)g.n[a] * P->cell[a]) : 1.0;
        if (a < g.ndim) {
            const double nyq = 0.5 * (double)g.n[a] * P->r[a];
            if (a == 0 || nyq < kmax_default) kmax_default = nyq;
        }
    }
    P->nbins = b->nbins;
    CF_TRY(pk_bin_edges(b, kmax_default, P->edges.e));
    P->elem = elem;
    const size_t per_pair = elem * (size_t)g.cells;
    long long pc = (long long)((size_t)(512ull << 20) / (per_pair ? per_pair : 1));
    const long long pairs = (nfields + 1) / 2;
    if (pc < 1) pc = 1;
    if (pc > pairs) pc = pairs;
    if (pc > 65535) pc = 65535;
    P->pairs_chunk = pc;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = any_align(o + bytes);
        return at;
    };
    P->off_bin = take(sizeof(int16_t) * (size_t)g.cells);
    P->off_nmodes = take(sizeof(unsigned long long) * P->nbins);
    P->off_mu = take(sizeof(double) * P->nbins);
    P->off_acc = take(sizeof(double) * (size_t)nfields * P->nbins);
    P->off_ntot = take(sizeof(unsigned long long) * (size_t)nfields);
    P->off_fsum = take(sizeof(double));
    P->off_z = take(per_pair * (size_t)pc);
    P->total = o;
    return CF_OK;
}

// Bluestein tables per (device, N, precision): chirp c_n (N values) and
// bhat = DFT_P(b)/P, b_m = conj(c_|m|) placed circularly, both from binary64
// arithmetic on the host (long double angles).  Kept for the process.
struct BlueTables {
    void* chirp = nullptr;
    void* bhat = nullptr;
    cudaEvent_t ready = nullptr;
    std::vector<unsigned char> staging;  // host copy read by the asynchronous upload
};
static std::mutex g_blue_mu;
static std::map<std::tuple<int, long long, size_t>, BlueTables*> g_blue;

static void host_fft(std::vector<std::complex<double>>& a) {  // forward, unnormalised, radix 2
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L / (long double)len;
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w((double)cosl(ang * (long double)k), (double)sinl(ang * (long double)k));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

template <typename T>
static cf_status blue_tables(long long N, cudaStream_t s, const C2<T>** chirp, const C2<T>** bhat) {
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_blue_mu);
    const auto key = std::make_tuple(dev, N, sizeof(T));
    auto it = g_blue.find(key);
    if (it == g_blue.end()) {
        const long long P = blue_length(N);
        std::vector<std::complex<double>> c(N), b(P, 0.0);
        for (long long n = 0; n < N; ++n) {
            const long long m = (n * n) % (2 * N);  // e^{-pi i n^2/N} has period 2N in n^2
            const long double ang = -3.141592653589793238462643383279502884L * (long double)m / (long double)N;
            c[n] = std::complex<double>((double)cosl(ang), (double)sinl(ang));
        }
        for (long long m = 0; m < N; ++m) {
            b[m] = std::conj(c[m]);
            if (m) b[P - m] = std::conj(c[m]);
        }
        host_fft(b);
        BlueTables* t = new BlueTables();
        std::vector<C2<T>> tab(N + P);
        for (long long n = 0; n < N; ++n) {
            tab[n].x = (T)c[n].real();
            tab[n].y = (T)c[n].imag();
        }
        for (long long p = 0; p < P; ++p) {
            tab[N + p].x = (T)(b[p].real() / (double)P);
            tab[N + p].y = (T)(b[p].imag() / (double)P);
        }
        t->staging.assign(reinterpret_cast<const unsigned char*>(tab.data()),
                          reinterpret_cast<const unsigned char*>(tab.data() + tab.size()));
        void* d = nullptr;
        if (cudaMalloc(&d, sizeof(C2<T>) * (size_t)(N + P)) != cudaSuccess) {
            delete t;
            return fail(CF_ERR_NOMEM, "device allocation of the Bluestein tables failed");
        }
        CF_CUDA(cudaMemcpyAsync(d, t->staging.data(), t->staging.size(), cudaMemcpyHostToDevice, s));
        CF_CUDA(cudaEventCreateWithFlags(&t->ready, cudaEventDisableTiming));
        CF_CUDA(cudaEventRecord(t->ready, s));
        t->chirp = d;
        t->bhat = (C2<T>*)d + N;
        it = g_blue.emplace(key, t).first;
    } else {
        CF_CUDA(cudaStreamWaitEvent(s, it->second->ready, 0));
    }
    *chirp = (const C2<T>*)it->second->chirp;
    *bhat = (const C2<T>*)it->second->bhat;
    return CF_OK;
}

// Transform of z[outer][N][inner] along its middle axis.
template <typename T>
static cf_status any_axis(C2<T>* z, long long outer, long long N, long long inner, cudaStream_t s) {
    if (N == 1) return CF_OK;
    const long long P = blue_length(N);
    const C2<T>* chirp = nullptr;
    const C2<T>* bhat = nullptr;
    if (P != N) CF_TRY(blue_tables<T>(N, s, &chirp, &bhat));
    return dispatch_line(P, [&](auto Pc) -> cf_status {
        constexpr int PP = decltype(Pc)::value;
        using Cfg = AnyCfg<T, PP>;
        auto launch = [&](auto kern) -> cf_status {
            CF_TRY(prepare_smem(kern, Cfg::SMEM));
            const long long blocks = inner == 1 ? (outer + Cfg::LINES - 1) / Cfg::LINES
                                                : outer * ((inner + Cfg::LINES - 1) / Cfg::LINES);
            if (blocks > 0x7fffffffll) return fail(CF_ERR_UNSUPPORTED, "%lld transform blocks", blocks);
            ScopedKernelTimer kt(s, sizeof(T) == 4 ? "pk_any_lines_f32" : "pk_any_lines_f64", PP);
            kern<<<(unsigned)blocks, Cfg::THREADS, Cfg::SMEM, s>>>(z, outer, inner, (int)N, chirp, bhat,
                                                                  twiddles<T>());
            CF_CHECK_LAUNCH();
            return CF_OK;
        };
        if (P != N)
            return inner == 1 ? launch(k_any_lines<T, PP, true, false>) : launch(k_any_lines<T, PP, true, true>);
        return inner == 1 ? launch(k_any_lines<T, PP, false, false>) : launch(k_any_lines<T, PP, false, true>);
    });
}

// Mode-bin tables cached per (device, grid, cells, edges).
struct AnyBinEntry {
    int device;
    int ndim;
    long long n[3];
    double cell[3];
    std::vector<double> edges;
    int16_t* bin_of;
    unsigned long long* nmodes;
    cudaEvent_t ready;
};
static std::mutex g_anybin_mu;
static std::vector<AnyBinEntry> g_anybin;
constexpr size_t kAnyBinMax = 32;

static cf_status any_build_bins(const AnyPlan& P, int16_t* bin_of, unsigned long long* nmodes, cudaStream_t s) {
    CF_CUDA(cudaMemsetAsync(nmodes, 0, sizeof(unsigned long long) * P.nbins, s));
    k_any_modebins<<<grid_blocks(P.g.cells, 256, 1024), 256, 0, s>>>(P.g, P.r[0], P.r[1], P.r[2], P.edges, P.nbins,
                                                                     bin_of, nmodes);
    CF_CHECK_LAUNCH();
    return CF_OK;
}

static cf_status any_get_bins(const AnyPlan& P, char* ws, cudaStream_t s, const int16_t** bin_of,
                              const unsigned long long** nmodes) {
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    std::vector<double> edges(P.edges.e, P.edges.e + P.nbins + 1);
    std::lock_guard<std::mutex> lk(g_anybin_mu);
    for (auto& c : g_anybin) {
        bool same = c.device == dev && c.ndim == P.g.ndim && c.edges == edges;
        for (int a = 0; a < 3 && same; ++a) same = c.n[a] == P.g.n[a] && c.cell[a] == P.cell[a];
        if (same) {
            CF_CUDA(cudaStreamWaitEvent(s, c.ready, 0));
            *bin_of = c.bin_of;
            *nmodes = c.nmodes;
            return CF_OK;
        }
    }
    if (g_anybin.size() >= kAnyBinMax) {
        int16_t* b = (int16_t*)(ws + P.off_bin);
        unsigned long long* nm = (unsigned long long*)(ws + P.off_nmodes);
        CF_TRY(any_build_bins(P, b, nm, s));
        *bin_of = b;
        *nmodes = nm;
        return CF_OK;
    }
    AnyBinEntry c{dev, P.g.ndim, {P.g.n[0], P.g.n[1], P.g.n[2]}, {P.cell[0], P.cell[1], P.cell[2]}, edges,
                  nullptr, nullptr, nullptr};
    CF_CUDA(cudaMalloc((void**)&c.bin_of, sizeof(int16_t) * (size_t)P.g.cells));
    CF_CUDA(cudaMalloc((void**)&c.nmodes, sizeof(unsigned long long) * P.nbins));
    CF_CUDA(cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming));
    CF_TRY(any_build_bins(P, c.bin_of, c.nmodes, s));
    CF_CUDA(cudaEventRecord(c.ready, s));
    g_anybin.push_back(c);
    *bin_of = c.bin_of;
    *nmodes = c.nmodes;
    return CF_OK;
}

// Shared with cf_pk.cu: the final normalisation, mean and covariance.
cf_status pk_finish(const double* acc, const unsigned long long* nmodes, long long nfields, int nbins,
                    double volfac, double* pk_out, int64_t* nmodes_out, double* mean, double* cov, double* scratch,
                    cudaStream_t s);

template <typename T>
static cf_status any_impl(const void* fields, int kind, const float* f, const AnyPlan& P, long long nfields,
                          double* pk_out, int64_t* nmodes_out, double* mean, double* cov, char* ws, cudaStream_t s) {
    const AnyGrid& g = P.g;
    const int16_t* bin_of = nullptr;
    const unsigned long long* nmodes = nullptr;
    double* acc = (double*)(ws + P.off_acc);
    unsigned long long* ntot = (unsigned long long*)(ws + P.off_ntot);
    double* fsum = (double*)(ws + P.off_fsum);
    C2<T>* z = (C2<T>*)(ws + P.off_z);
    {
        ScopedKernelTimer kt(s, "pk_setup");
        CF_TRY(any_get_bins(P, ws, s, &bin_of, &nmodes));
        CF_CUDA(cudaMemsetAsync(ws + P.off_acc, 0, P.off_z - P.off_acc, s));
    }
    if (kind == ANY_COUNTS) {
        for (long long f0 = 0; f0 < nfields; f0 += 65535) {
            const long long nf = nfields - f0 < 65535 ? nfields - f0 : 65535;
            k_any_totals<<<dim3(grid_blocks(g.cells, 256, 64), (unsigned)nf), 256, 0, s>>>(
                (const int32_t*)fields, f, g.cells, f0, ntot, fsum);
        }
        CF_CHECK_LAUNCH();
    }
    const long long pairs = (nfields + 1) / 2;
    for (long long p0 = 0; p0 < pairs; p0 += P.pairs_chunk) {
        const long long np = pairs - p0 < P.pairs_chunk ? pairs - p0 : P.pairs_chunk;
        const dim3 pg((unsigned)grid_blocks(g.cells, 256, 512), (unsigned)np);
        if (kind == ANY_FLOAT)
            k_any_pack<T, ANY_FLOAT><<<pg, 256, 0, s>>>(fields, f, g.cells, nfields, 2 * p0, ntot, fsum, z);
        else if (kind == ANY_DOUBLE)
            k_any_pack<T, ANY_DOUBLE><<<pg, 256, 0, s>>>(fields, f, g.cells, nfields, 2 * p0, ntot, fsum, z);
        else
            k_any_pack<T, ANY_COUNTS><<<pg, 256, 0, s>>>(fields, f, g.cells, nfields, 2 * p0, ntot, fsum, z);
        CF_CHECK_LAUNCH();
        for (int a = g.ndim - 1; a >= 0; --a) {
            long long outer = np, inner = 1;
            for (int b = 0; b < a; ++b) outer *= g.n[b];
            for (int b = a + 1; b < g.ndim; ++b) inner *= g.n[b];
            CF_TRY(any_axis<T>(z, outer, g.n[a], inner, s));
        }
        const size_t smem = 2 * sizeof(double) * (size_t)P.nbins;
        k_any_bin<T><<<pg, 256, smem, s>>>(z, g, bin_of, P.nbins, nfields, 2 * p0, acc);
        CF_CHECK_LAUNCH();
    }
    double volfac = 1.0;
    for (int a = 0; a < g.ndim; ++a) volfac *= P.cell[a] / (double)g.n[a];
    return pk_finish(acc, nmodes, nfields, P.nbins, volfac, pk_out, nmodes_out, mean, cov, (double*)(ws + P.off_mu), s);
}

cf_status pk_any_workspace(const cf_grid* g, long long nfields, const cf_bins* b, cf_dtype dt, size_t* bytes) {
    AnyPlan P;
    CF_TRY(any_plan(g, nfields, b, dt == CF_F64 ? sizeof(C2<double>) : sizeof(C2<float>), &P));
    *bytes = P.total;
    return CF_OK;
}

// kind: 0 binary32 fields, 1 binary64 fields, 2 count maps (binary32 transforms).
cf_status pk_any_run(const void* fields, int kind, const float* f, const cf_grid* g, long long nfields,
                     const cf_bins* bins, double* pk_out, int64_t* nmodes_out, double* mean, double* cov, void* ws,
                     size_t ws_bytes, cudaStream_t s) {
    const bool f64 = kind == ANY_DOUBLE;
    AnyPlan P;
    CF_TRY(any_plan(g, nfields, bins, f64 ? sizeof(C2<double>) : sizeof(C2<float>), &P));
    if (!ws || ws_bytes < P.total) return fail(CF_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, P.total);
    if (f64) return any_impl<double>(fields, kind, f, P, nfields, pk_out, nmodes_out, mean, cov, (char*)ws, s);
    return any_impl<float>(fields, kind, f, P, nfields, pk_out, nmodes_out, mean, cov, (char*)ws, s);
}

}  // namespace cf
