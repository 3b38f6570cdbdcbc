// cf_tc.cu -- the per-realization inverse transforms of section 2 (closing
// paragraph: the field is the inverse DFT of sqrt(lambda) times white noise)
// run as DFT-matrix GEMMs on the fifth-generation tensor cores:
// cf_dtype CF_BF16_TC and CF_F16_TC.
//
// A line of L = 16^S points is transformed in S radix-16 stages.  With
// n = n_0 + 16 n_1 (+ 256 n_2) and k = k_0 + 16 k_1 (+ 256 k_2), stage s is the
// 16-point DFT over the most significant untransformed digit, written as a
// real GEMM: A rows are the other digits (L/16 rows per line), A columns the
// 16 complex inputs interleaved as (re, im) (K = 32); B is the real 32 x 32
// form of the 16-point DFT matrix; D (binary32, in tensor memory) holds the 16
// complex outputs of each row.  Between stages the epilogue multiplies by the
// twiddle factors w_L^{u k} in binary32, rounds to the 16-bit input type and
// scatters into the next stage's A.  The DFT matrix is split into a 16-bit
// head and a 16-bit remainder (two MMAs accumulate A*B_hi + A*B_lo), so its
// entries act at nearly binary32 accuracy; the data are rounded to 16 bits
// at every stage, which sets the error of these modes.
//
// 2D: pass 1 draws the noise of one embedded row per line (the same binary32
// noise as CF_F32), scales it and transforms the last axis, keeping n1
// outputs (16-bit complex intermediate [M0][n1]); pass 2 transforms the
// columns, keeping n0 outputs, and writes the Re/Im fields in binary32.  3D
// adds a middle pass: the column kernel per slab along axis 1, writing the
// next 16-bit intermediate [M0][n1][n2].
// The inputs are pre-scaled by a power of two alpha chosen from sum(s^2)
// (computed once per embedding) so the intermediate has unit mean square
// (range of fp16); the fields are multiplied by 1/alpha at the end.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "cf_device.cuh"
#include "cf_kernels.cuh"
#include "cf_tc.cuh"

namespace cf {
namespace {

constexpr int kCtaRows = 2048;               // A rows per block and stage (all warpgroups)
// A: the 4 core matrices of a row group (K = 32) are contiguous (LBO = 128),
// row groups 528 bytes apart (16 bytes of padding shift rows r and r + 8 by
// four banks).  Every descriptor's reach stays inside the operand whichever
// of the two strides is taken along K.
constexpr int kLBO = 128;                    // K-direction core-matrix stride
constexpr int kSBO = 4 * 128 + 16;           // row-direction core-matrix stride
constexpr int kBBytes = 32 * 32 * 2;         // one 32 x 32 16-bit matrix
constexpr uint32_t kTmemCols = 512;          // (kCtaRows / 128) tiles x 32 columns

// Geometry of a block of WGS warpgroups: each owns kWgRows rows of A (its
// lines), kTiles M = 128 tiles and kTiles x 32 tensor-memory columns.  The
// warpgroups' operands are kABytes + 16 apart, so that the same offset in two
// of them falls four banks apart.
template <int WGS>
struct Geo {
    static constexpr int kWgRows = kCtaRows / WGS;
    static constexpr int kTiles = kWgRows / 128;
    static constexpr int kABytes = (kWgRows / 8) * kSBO;
    static constexpr int kAStride = kABytes + 16;
    static constexpr int kThreads = 128 * WGS;
    static constexpr int kBOff = WGS * kAStride;
    static constexpr int kBarOff = kBOff + 2 * kBBytes;
    static constexpr int kSmem = kBarOff + 8 * WGS + 16;
};
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per tensor-core wait

__device__ unsigned int g_tc_faults;         // waits that ran out of time

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase; a wait that runs out is counted.
__device__ __forceinline__ void wait_phase(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > kWaitNs) {
            atomicAdd(&g_tc_faults, 1u);
            return;
        }
    }
}

// Input scale alpha = 2^-round(log2(sqrt(sum(s^2) * factor))), factor =
// 2 L1 amp^2 / M^d: the mean square of the row-transformed intermediate is
// 2 L1 amp^2 sum(s^2) / M^d (E|eps|^2 = 2, the row transform multiplies the
// mean square by L1), so alpha brings it to about 1.  inverse: 1/alpha.
__device__ __forceinline__ float input_scale(const double* __restrict__ sumsq, double factor, bool inverse) {
    const double ms = sumsq[0] * factor;
    int e = ms > 0.0 ? (int)lrint(-0.5 * log2(ms)) : 0;
    e = e < -60 ? -60 : (e > 60 ? 60 : e);
    return ldexpf(1.0f, inverse ? -e : e);
}

__device__ __forceinline__ uint32_t a_off(int r, int kappa) {
    return (uint32_t)((r >> 3) * kSBO + (kappa >> 3) * kLBO + (r & 7) * 16 + (kappa & 7) * 2);
}

// B (N = 32 rows n, K = 32): core matrices of a row group contiguous (LBO =
// 128), row groups 512 bytes apart.
__device__ __forceinline__ uint32_t b_off(int n, int kappa) {
    return (uint32_t)((n >> 3) * 512 + (kappa >> 3) * 128 + (n & 7) * 16 + (kappa & 7) * 2);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float re, float im) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(re, im);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

template <bool BF16>
__device__ __forceinline__ uint16_t round16(float v, float& back) {
    if constexpr (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        back = __bfloat162float(h);
        return *reinterpret_cast<const uint16_t*>(&h);
    } else {
        const __half h = __float2half_rn(v);
        back = __half2float(h);
        return *reinterpret_cast<const uint16_t*>(&h);
    }
}

__device__ __forceinline__ C2<float> cmulf(C2<float> a, C2<float> b) {
    return mk(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Real 32 x 32 form of the 16-point inverse DFT matrix, head and remainder:
// B(2j + pj, 2k + pk) from w16^{jk} = c + i s: (c, s; -s, c).
template <bool BF16>
__device__ void build_dft16(unsigned char* bhi, unsigned char* blo, const C2<float>* __restrict__ tw) {
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int kappa = e & 31, n = e >> 5;
        const int j = kappa >> 1, pj = kappa & 1, k = n >> 1, pk = n & 1;
        const C2<float> w = tw[((j * k) & 15) * (TWN / 16)];
        const float v = pj == 0 ? (pk == 0 ? w.x : w.y) : (pk == 0 ? -w.y : w.x);
        float back;
        const uint16_t h = round16<BF16>(v, back);
        float unused;
        const uint16_t l = round16<BF16>(v - back, unused);
        *reinterpret_cast<uint16_t*>(bhi + b_off(n, kappa)) = h;
        *reinterpret_cast<uint16_t*>(blo + b_off(n, kappa)) = l;
    }
}

// One stage of the warpgroup's tiles: D_t = A_t * (B_hi + B_lo), N outputs.
template <int N, bool BF16, int TILES>
__device__ __forceinline__ void issue_stage(uint32_t a_addr, uint32_t bhi, uint32_t blo, uint32_t tmem,
                                            uint32_t bar) {
    constexpr uint32_t idesc = tc::idesc_f16(128, N, BF16);
    tc::fence_after_sync();
#pragma unroll 1
    for (int t = 0; t < TILES; ++t) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint64_t ad = tc::sdesc(a_addr + (uint32_t)(t * 16 * kSBO + c * 2 * kLBO), kLBO, kSBO);
            tc::mma_f16(tmem + 32 * t, ad, tc::sdesc(bhi + c * 256, 128, 512), idesc, c > 0 ? 1u : 0u);
            tc::mma_f16(tmem + 32 * t, ad, tc::sdesc(blo + c * 256, 128, 512), idesc, 1u);
        }
    }
    tc::mma_commit(bar);
}

// Twiddle w_L^{u k}, k = 0..15, applied to the 16 outputs of one row and
// scattered into the next stage's A (row dst0 + dstride k, column pair kk).
template <bool BF16>
__device__ __forceinline__ void twiddle_scatter(const uint32_t (&r)[32], const C2<float>* __restrict__ tw, int step,
                                                unsigned char* A, int dst0, int dstride, int kk) {
    const C2<float> w1 = tw[step & (TWN - 1)];
    const C2<float> w4 = tw[(4 * step) & (TWN - 1)];
    const C2<float> w2 = cmulf(w1, w1), w3 = cmulf(w2, w1);
    const C2<float> w8 = cmulf(w4, w4), w12 = cmulf(w8, w4);
    const C2<float> wb[4] = {mk(1.0f, 0.0f), w1, w2, w3};
    const C2<float> wa[4] = {mk(1.0f, 0.0f), w4, w8, w12};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * a + b;
            const C2<float> w = (a == 0) ? wb[b] : (b == 0 ? wa[a] : cmulf(wa[a], wb[b]));
            const C2<float> y = cmulf(mk(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1])), w);
            *reinterpret_cast<uint32_t*>(A + a_off(dst0 + dstride * k, kk)) = pack2<BF16>(y.x, y.y);
        }
    }
}

// Epilogue of stage `stage` (< S) for local A row `row` of this warpgroup.
template <int S, int stage, bool BF16>
__device__ __forceinline__ void stage_epilogue(const uint32_t (&r)[32], int row, const C2<float>* __restrict__ tw,
                                               unsigned char* A) {
    constexpr int L = S == 3 ? 4096 : 256;
    constexpr int RPL = L / 16;
    const int line = row / RPL, lrow = row % RPL;
    const int base = line * RPL;
    if constexpr (S == 3 && stage == 1) {
        // rows (n0, n1) -> next rows (n0, k0), column n1; twiddle w^{(n0 + 16 n1) k0}
        twiddle_scatter<BF16>(r, tw, lrow * (TWN / L), A, base + (lrow & 15), 16, 2 * (lrow >> 4));
    } else if constexpr (S == 3 && stage == 2) {
        // rows (n0, k0) -> next rows (k0, k1), column n0; twiddle w^{16 n0 k1}
        twiddle_scatter<BF16>(r, tw, 16 * (lrow & 15) * (TWN / L), A, base + (lrow >> 4), 16, 2 * (lrow & 15));
    } else {
        // S == 2: rows n0 -> next rows k0, column n0; twiddle w^{n0 k0}
        twiddle_scatter<BF16>(r, tw, lrow * (TWN / L), A, base, 1, 2 * lrow);
    }
}

// Kept output points of the last stage: row (k0[, k1]) holds k = row + (L/16) k_last, k_last < 8.
template <int S>
__device__ __forceinline__ int out_point(int lrow, int klast) {
    return lrow + (S == 3 ? 256 : 16) * klast;
}

// Runs the S stages of one warpgroup on its A (loaded, fenced, synchronised),
// calling sink(line, point, re, im) for every kept output.
template <int S, bool BF16, int WGS, class Sink>
__device__ __forceinline__ void run_stages(unsigned char* A, uint32_t a_addr, uint32_t bhi, uint32_t blo,
                                           uint32_t tmem, uint32_t bar, uint32_t& phase,
                                           const C2<float>* __restrict__ tw, int wg, Sink&& sink) {
    constexpr int kTiles = Geo<WGS>::kTiles;
    constexpr int L = S == 3 ? 4096 : 256;
    constexpr int RPL = L / 16;
    const int wtid = threadIdx.x & 127;
    const int warp = wtid >> 5, lane = wtid & 31;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
#pragma unroll 1
    for (int stage = 1; stage <= S; ++stage) {
        const bool last = stage == S;
        if (wtid == 0) {
            if (last)
                issue_stage<16, BF16, kTiles>(a_addr, bhi, blo, tmem, bar);
            else
                issue_stage<32, BF16, kTiles>(a_addr, bhi, blo, tmem, bar);
        }
        wait_phase(bar, phase);
        phase ^= 1u;
        __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the per-thread wait
        tc::fence_after_sync();
#pragma unroll 1
        for (int t = 0; t < kTiles; ++t) {
            const int row = 128 * t + 32 * warp + lane;
            uint32_t r[32];
            const uint32_t taddr = tmem + lane_base + 32 * t;
            if (last)
                tc::tmem_ld16(taddr, r);
            else
                tc::tmem_ld32(taddr, r);
            tc::tmem_ld_wait(r);
            if (last) {
                const int line = row / RPL, lrow = row % RPL;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    sink(line, out_point<S>(lrow, k), __uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
            } else if (stage == 1) {
                stage_epilogue<S, 1, BF16>(r, row, tw, A);
            } else {
                stage_epilogue<S, 2, BF16>(r, row, tw, A);
            }
        }
        tc::fence_before_sync();
        if (!last) tc::fence_proxy_async_smem();
        tc::bar_sync(1 + wg, 128);
    }
}

struct TcShared {
    unsigned char* A;     // this warpgroup's operand
    uint32_t a_addr, bhi, blo, tmem, bar;
};

// Common prologue: barriers, tensor memory, DFT matrices.  Returns this
// warpgroup's view.
template <bool BF16, int WGS>
__device__ __forceinline__ TcShared tc_prologue(unsigned char* smraw, const C2<float>* __restrict__ tw, int wg) {
    using Gm = Geo<WGS>;
    unsigned char* Bh = smraw + Gm::kBOff;
    unsigned char* Bl = Bh + kBBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + Gm::kBarOff);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + WGS);
    if (threadIdx.x == 0) {
        for (int w = 0; w < WGS; ++w) tc::mbar_init(tc::smem_u32(&bars[w]), 1);
        tc::fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tc::smem_u32(tslot), kTmemCols);
        tc::tmem_relinquish();
    }
    build_dft16<BF16>(Bh, Bl, tw);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TcShared s;
    s.A = smraw + wg * Gm::kAStride;
    s.a_addr = tc::smem_u32(s.A);
    s.bhi = tc::smem_u32(Bh);
    s.blo = tc::smem_u32(Bl);
    s.tmem = *tslot + (uint32_t)(Gm::kTiles * 32 * wg);
    s.bar = tc::smem_u32(&bars[wg]);
    return s;
}

template <int WGS>
__device__ __forceinline__ void tc_epilogue(unsigned char* smraw) {
    const uint32_t* tslot = reinterpret_cast<const uint32_t*>(smraw + Geo<WGS>::kBarOff + 8 * WGS);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(*tslot, kTmemCols);
    }
}

// ---------------------------------------------------------------- first radix
// Lines of L = RF * LS points with RF in {2, 4, 8} (LS = 256) start with a
// radix-RF decimation-in-frequency stage in binary32: for each n' < LS the
// inputs x[n' + LS j], j < RF, give y_k = sum_j x_j w_RF^{jk}, multiplied by
// w_L^{n' k}, which is point n' of sub-line k; the tensor-core stages then
// transform the RF sub-lines of LS points, and output p' of sub-line k is
// X[k + RF p'].  Keeping the first L/2 outputs keeps p' < LS/2 of every
// sub-line.
template <int RF>
__device__ __forceinline__ void first_radix(C2<float> (&x)[RF], int np, const C2<float>* __restrict__ tw) {
    if constexpr (RF > 1) {
        dftR<RF, +1>(x);
        constexpr int L = RF * 256;
#pragma unroll
        for (int k = 1; k < RF; ++k) x[k] = cmulf(x[k], tw[(np * k * (TWN / L)) & (TWN - 1)]);
    }
}

template <bool BF16>
__device__ __forceinline__ C2<float> unpack2(uint32_t u) {
    if constexpr (BF16) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
        return mk(f.x, f.y);
    } else {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
        return mk(f.x, f.y);
    }
}

// ---------------------------------------------------------------- pass 1
// Rows of the embedded grid (L = M1 = RF * LS): noise, scale, transform, keep
// n1 = L/2.  Block: WGS * LPW consecutive rows of realization r0 + blockIdx.x,
// LPW per warpgroup (RF sub-lines each).
template <int S, int RF, bool BF16, int WGS>
__global__ void __launch_bounds__(Geo<WGS>::kThreads, 1)
    k_tc_rows(const float* __restrict__ s, float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
              long long nrows, uint32_t* __restrict__ inter, const double* __restrict__ sumsq, double factor,
              const C2<float>* __restrict__ tw) {
    constexpr int LS = S == 3 ? 4096 : 256;
    constexpr int L = RF * LS;
    constexpr int RPL = LS / 16;
    constexpr int SLPW = Geo<WGS>::kWgRows / RPL;  // sub-lines per warpgroup
    constexpr int LPW = SLPW / RF;                  // lines per warpgroup
    static_assert(LPW >= 1, "line does not fit a warpgroup");
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ float s_alpha;
    // the input scale in binary64 once per block (the prologue's barrier
    // publishes it): per thread it kept the slow binary64 pipe busy
    if (threadIdx.x == 0) s_alpha = input_scale(sumsq, factor, false);
    const int wg = threadIdx.x >> 7, wtid = threadIdx.x & 127;
    const TcShared sh = tc_prologue<BF16, WGS>(tc_smem, tw, wg);
    const float alpha = s_alpha;
    // blockIdx.x: realization, blockIdx.y: block of rows, so that the blocks
    // running at the same time read the same rows of sqrt(lambda) (L2 hits)
    const uint32_t r = r0 + blockIdx.x;
    const long long row0 = (long long)blockIdx.y * (WGS * LPW) + wg * LPW;
    if constexpr (RF == 1) {
        // columns col and col + L/2 share one Philox call.  Within a warp,
        // lanes take rows j + (lane & 7) of one row group and column groups
        // (lane >> 3) + 4 b of the A operand (col = row + RPL * group): 32 banks.
        // tasks t and t + 128 of this thread draw their noise together (paired
        // Box-Muller, the same draws as one at a time)
        static_assert((LPW * (L / 2)) % 256 == 0, "tasks come in pairs");
#pragma unroll 1
        for (int t0 = wtid; t0 < LPW * (L / 2); t0 += 256) {
            int gq[2], rrq[2], grpq[2], colq[2];
            long long rowq[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = t0 + 128 * h;
                const int g = t / (L / 2), e = t % (L / 2);
                const int lane = e & 31, w = e >> 5;
                gq[h] = g;
                rrq[h] = (lane & 7) + 8 * (w % (RPL / 8));
                grpq[h] = (lane >> 3) + 4 * (w / (RPL / 8));
                colq[h] = rrq[h] + RPL * grpq[h];
                rowq[h] = row0 + g;
            }
            CP lo, hi;
            noise_pair_f32x2((unsigned long long)rowq[0] * (L / 2) + colq[0], r, key0, key1,
                             (unsigned long long)rowq[1] * (L / 2) + colq[1], r, key0, key1, lo, hi);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float* srow = s + (size_t)rowq[h] * L;
                const C2<float> l = h ? mk(lo.re.y, lo.im.y) : mk(lo.re.x, lo.im.x);
                const C2<float> u = h ? mk(hi.re.y, hi.im.y) : mk(hi.re.x, hi.im.x);
                const C2<float> xl = cscale(cscale(l, srow[colq[h]] * amp_scale), alpha);
                const C2<float> xh = cscale(cscale(u, srow[colq[h] + L / 2] * amp_scale), alpha);
                *reinterpret_cast<uint32_t*>(sh.A + a_off(gq[h] * RPL + rrq[h], 2 * grpq[h])) = pack2<BF16>(xl.x, xl.y);
                *reinterpret_cast<uint32_t*>(sh.A + a_off(gq[h] * RPL + rrq[h], 2 * (grpq[h] + 8))) =
                    pack2<BF16>(xh.x, xh.y);
            }
        }
    } else {
        // task (line g, point n' of the sub-lines): the RF inputs n' + LS j;
        // inputs j and j + RF/2 are a Philox pair (their columns differ by L/2)
#pragma unroll 1
        for (int t = wtid; t < LPW * LS; t += 128) {
            const int g = t / LS, e = t % LS;
            const int lane = e & 31, w = e >> 5;
            const int np = (lane & 7) + 8 * (w & 1) + 16 * ((lane >> 3) + 4 * (w >> 1));
            const long long row = row0 + g;
            const float* srow = s + (size_t)row * L;
            C2<float> x[RF];
#pragma unroll
            for (int j = 0; j < RF / 2; ++j) {
                const int col = np + LS * j;
                C2<float> lo, hi;
                noise_pair_f32((unsigned long long)row * (L / 2) + col, r, key0, key1, lo, hi);
                x[j] = cscale(cscale(lo, srow[col] * amp_scale), alpha);
                x[j + RF / 2] = cscale(cscale(hi, srow[col + L / 2] * amp_scale), alpha);
            }
            first_radix<RF>(x, np, tw);
#pragma unroll
            for (int k = 0; k < RF; ++k)
                *reinterpret_cast<uint32_t*>(sh.A + a_off((g * RF + k) * RPL + np % RPL, 2 * (np / RPL))) =
                    pack2<BF16>(x[k].x, x[k].y);
        }
    }
    tc::fence_proxy_async_smem();
    tc::bar_sync(1 + wg, 128);
    uint32_t phase = 0;
    uint32_t* out = inter + ((size_t)blockIdx.x * nrows + row0) * (L / 2);
    run_stages<S, BF16, WGS>(sh.A, sh.a_addr, sh.bhi, sh.blo, sh.tmem, sh.bar, phase, tw, wg,
                             [&](int sl, int p, float re, float im) {
                                 const int g = sl / RF, q = sl % RF + RF * p;
                                 out[(size_t)g * (L / 2) + q] = pack2<BF16>(re, im);
                             });
    tc_epilogue<WGS>(tc_smem);
}

// ---------------------------------------------------------------- pass 2
// Columns of the intermediate [M0][n1] (L = M0 = RF * LS): transform, keep
// n0 = L/2, write field 2r (Re) and 2r + 1 (Im) times 1/alpha.  Block:
// LC = WGS * LPW adjacent columns, loaded by the whole block.
template <int S, int RF, bool BF16, int WGS, bool OUT16>
__global__ void __launch_bounds__(Geo<WGS>::kThreads, 1)
    k_tc_cols(const uint32_t* __restrict__ inter, long long n1, float* __restrict__ fields, long long cells,
              uint32_t* __restrict__ out16, const double* __restrict__ sumsq, double factor,
              const C2<float>* __restrict__ tw) {
    constexpr int LS = S == 3 ? 4096 : 256;
    constexpr int L = RF * LS;
    constexpr int RPL = LS / 16;
    constexpr int SLPW = Geo<WGS>::kWgRows / RPL;
    constexpr int LPW = SLPW / RF;
    constexpr int LC = WGS * LPW;
    static_assert(LPW >= 1, "line does not fit a warpgroup");
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ float s_inv_alpha;
    if (threadIdx.x == 0) s_inv_alpha = input_scale(sumsq, factor, true);
    const int wg = threadIdx.x >> 7;
    const TcShared sh = tc_prologue<BF16, WGS>(tc_smem, tw, wg);
    const float inv_alpha = s_inv_alpha;
    const long long cta0 = (long long)blockIdx.x * LC;
    const uint32_t* in = inter + (size_t)blockIdx.y * L * n1;
    if constexpr (RF == 1 && LC == 8) {
        // lane & 7 -> column (warpgroup operand 4 banks apart), lane >> 3 ->
        // point group: 32 banks per store, 32-byte row segments per load
#pragma unroll 4
        for (int t = threadIdx.x; t < LC * L; t += Geo<WGS>::kThreads) {
            const int li = t & 7, j = t >> 3;
            const int grp = (j & 3) + 4 * (j / (4 * RPL));
            const int n = RPL * grp + ((j >> 2) % RPL);
            const uint32_t v = in[(size_t)n * n1 + cta0 + li];
            unsigned char* A = tc_smem + (li / LPW) * Geo<WGS>::kAStride;
            *reinterpret_cast<uint32_t*>(A + a_off((li % LPW) * RPL + n % RPL, 2 * (n / RPL))) = v;
        }
    } else if constexpr (RF == 1) {
#pragma unroll 4
        for (int t = threadIdx.x; t < LC * L; t += Geo<WGS>::kThreads) {
            const int li = t % LC, n = t / LC;
            const uint32_t v = in[(size_t)n * n1 + cta0 + li];
            unsigned char* A = tc_smem + (li / LPW) * Geo<WGS>::kAStride;
            *reinterpret_cast<uint32_t*>(A + a_off((li % LPW) * RPL + n % RPL, 2 * (n / RPL))) = v;
        }
    } else {
        // task (column li, point n'): the RF inputs n' + LS j of the column
#pragma unroll 2
        for (int t = threadIdx.x; t < LC * LS; t += Geo<WGS>::kThreads) {
            const int li = t % LC, np = t / LC;
            C2<float> x[RF];
#pragma unroll
            for (int j = 0; j < RF; ++j) x[j] = unpack2<BF16>(in[(size_t)(np + LS * j) * n1 + cta0 + li]);
            first_radix<RF>(x, np, tw);
            unsigned char* A = tc_smem + (li / LPW) * Geo<WGS>::kAStride;
#pragma unroll
            for (int k = 0; k < RF; ++k)
                *reinterpret_cast<uint32_t*>(A + a_off(((li % LPW) * RF + k) * RPL + np % RPL, 2 * (np / RPL))) =
                    pack2<BF16>(x[k].x, x[k].y);
        }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    uint32_t phase = 0;
    // the last stage's outputs go to this warpgroup's operand buffer (its MMAs
    // have completed): stage[sl][p], p < LS/2, as (re, im) ...
    float2* stage = reinterpret_cast<float2*>(sh.A);
    run_stages<S, BF16, WGS>(sh.A, sh.a_addr, sh.bhi, sh.blo, sh.tmem, sh.bar, phase, tw, wg,
                             [&](int sl, int p, float re, float im) {
                                 stage[sl * (LS / 2) + p] = make_float2(re, im);
                             });
    __syncthreads();
    // ... then the block writes rows q < L/2 of its LC adjacent columns: the
    // Re/Im fields times 1/alpha, or (OUT16, an inner axis of a 3D grid) the
    // next 16-bit intermediate [slab][L/2][n1]
    float* f0 = OUT16 ? nullptr : fields + (size_t)blockIdx.y * 2 * cells;
    uint32_t* o16 = OUT16 ? out16 + (size_t)blockIdx.y * (L / 2) * n1 : nullptr;
#pragma unroll 4
    for (int t = threadIdx.x; t < LC * (L / 2); t += Geo<WGS>::kThreads) {
        const int li = t % LC, q = t / LC;
        const int sl = (li % LPW) * RF + q % RF, p = q / RF;
        const float2* st = reinterpret_cast<const float2*>(tc_smem + (li / LPW) * Geo<WGS>::kAStride);
        const float2 v = st[sl * (LS / 2) + p];
        const size_t o = (size_t)q * n1 + cta0 + li;
        if constexpr (OUT16) {
            o16[o] = pack2<BF16>(v.x, v.y);
        } else {
            f0[o] = v.x * inv_alpha;
            f0[o + cells] = v.y * inv_alpha;
        }
    }
    tc_epilogue<WGS>(tc_smem);
}

#ifndef CF_TC_WGS
#define CF_TC_WGS 8  // warpgroups per block (2, 4 or 8): build-time tunable
#endif

template <bool BF16, int S, int RF>
cf_status launch_tc_shape(bool rows, dim3 grid, cudaStream_t st, const float* s, float amp, uint32_t key0,
                          uint32_t key1, uint32_t r0, long long nrows, uint32_t* inter, long long n1, float* fields,
                          long long cells, uint32_t* out16, const double* sumsq, double factor) {
    constexpr int WGS = CF_TC_WGS;
    using Gm = Geo<WGS>;
    constexpr int L = RF * (S == 3 ? 4096 : 256);
    const C2<float>* tw = twiddles_f32();
    if (rows) {
        auto kern = k_tc_rows<S, RF, BF16, WGS>;
        CF_TRY(prepare_smem(kern, Gm::kSmem));
        ScopedKernelTimer kt(st, BF16 ? "tc_rows_bf16" : "tc_rows_f16", L);
        kern<<<grid, Gm::kThreads, Gm::kSmem, st>>>(s, amp, key0, key1, r0, nrows, inter, sumsq, factor, tw);
    } else {
        auto kern = out16 ? k_tc_cols<S, RF, BF16, WGS, true> : k_tc_cols<S, RF, BF16, WGS, false>;
        CF_TRY(prepare_smem(kern, Gm::kSmem));
        ScopedKernelTimer kt(st, BF16 ? "tc_cols_bf16" : "tc_cols_f16", L);
        kern<<<grid, Gm::kThreads, Gm::kSmem, st>>>(inter, n1, fields, cells, out16, sumsq, factor, tw);
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}

template <bool BF16>
cf_status launch_tc(long long L, bool rows, dim3 grid, cudaStream_t st, const float* s, float amp, uint32_t key0,
                    uint32_t key1, uint32_t r0, long long nrows, uint32_t* inter, long long n1, float* fields,
                    long long cells, uint32_t* out16, const double* sumsq, double factor) {
    switch (L) {
    case 4096: return launch_tc_shape<BF16, 3, 1>(rows, grid, st, s, amp, key0, key1, r0, nrows, inter, n1, fields,
                                                  cells, out16, sumsq, factor);
    case 2048: return launch_tc_shape<BF16, 2, 8>(rows, grid, st, s, amp, key0, key1, r0, nrows, inter, n1, fields,
                                                  cells, out16, sumsq, factor);
    case 1024: return launch_tc_shape<BF16, 2, 4>(rows, grid, st, s, amp, key0, key1, r0, nrows, inter, n1, fields,
                                                  cells, out16, sumsq, factor);
    case 512: return launch_tc_shape<BF16, 2, 2>(rows, grid, st, s, amp, key0, key1, r0, nrows, inter, n1, fields,
                                                 cells, out16, sumsq, factor);
    case 256: return launch_tc_shape<BF16, 2, 1>(rows, grid, st, s, amp, key0, key1, r0, nrows, inter, n1, fields,
                                                 cells, out16, sumsq, factor);
    default: return fail(CF_ERR_UNSUPPORTED, "tensor-core line length %lld", L);
    }
}

bool tc_length_ok(long long L) { return L == 256 || L == 512 || L == 1024 || L == 2048 || L == 4096; }

}  // namespace

// Lines per block of a pass with line length L (all warpgroups): the block
// holds kCtaRows A rows, L/16 per line.
static long long tc_lines_per_block(long long L) { return kCtaRows / (L / 16); }

cf_status tc_check_grid(const GridInfo& g) {
    bool ok = g.ndim == 2 || g.ndim == 3;
    for (int a = 0; ok && a < g.ndim; ++a) ok = tc_length_ok(g.m[a]) && g.m[a] == 2 * g.n[a];
    if (!ok)
        return fail(CF_ERR_UNSUPPORTED,
                    "tensor-core modes need a 2D or 3D grid with embedded sides 2n = 256..4096");
    return CF_OK;
}

size_t tc_bytes_per_realization(const GridInfo& g) {
    if (g.ndim == 2) return 4 * (size_t)g.m[0] * (size_t)g.n[1];
    return 4 * ((size_t)g.m[0] * g.m[1] * g.n[2] + (size_t)g.m[0] * g.n[1] * g.n[2]);
}
size_t tc_header_bytes() { return 0; }

// Fields [R][2][n0][n1] (binary32) of realizations r0.. through the tensor
// cores; ws: header + chunk intermediates.
cf_status sample_tc(const cf_embedding* e, bool bf16, uint64_t seed, uint64_t r0, int R, float* fields, void* ws,
                    size_t ws_bytes, int chunk, double amp_scale, cudaStream_t st) {
    const GridInfo& g = e->grid;
    CF_TRY(tc_check_grid(g));
    CF_TRY(ensure_sumsq(const_cast<cf_embedding*>(e), st));
    const double* sumsq = e->sumsq;
    const int d = g.ndim;
    const double factor = 2.0 * (double)g.m[d - 1] * amp_scale * amp_scale / (double)g.mtotal;
    if (d == 3 && (long long)chunk * g.m[0] > 65535) chunk = (int)(65535 / g.m[0]);
    uint32_t* inter = (uint32_t*)ws;
    const long long cells = g.ncell;
    auto launch = [&](long long L, bool rows, dim3 grid, uint32_t rr, long long nrows, uint32_t* in, long long ncols,
                      float* f, uint32_t* out16) -> cf_status {
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        return bf16 ? launch_tc<true>(L, rows, grid, st, e->s32, (float)amp_scale, k0, k1, rr, nrows, in, ncols, f,
                                      cells, out16, sumsq, factor)
                    : launch_tc<false>(L, rows, grid, st, e->s32, (float)amp_scale, k0, k1, rr, nrows, in, ncols, f,
                                       cells, out16, sumsq, factor);
    };
    for (int c0 = 0; c0 < R; c0 += chunk) {
        const int nr = (R - c0) < chunk ? (R - c0) : chunk;
        const uint32_t rr = (uint32_t)(r0 + (uint64_t)c0);
        float* f = fields + (size_t)c0 * 2 * (size_t)cells;
        if (d == 2) {
            // rows (noise, axis 1) -> [M0][n1]; columns (axis 0) -> fields
            const dim3 g1((unsigned)nr, (unsigned)(g.m[0] / tc_lines_per_block(g.m[1])));
            const dim3 g2((unsigned)(g.n[1] / tc_lines_per_block(g.m[0])), (unsigned)nr);
            CF_TRY(launch(g.m[1], true, g1, rr, g.m[0], inter, g.n[1], nullptr, nullptr));
            CF_TRY(launch(g.m[0], false, g2, 0, 0, inter, g.n[1], f, nullptr));
        } else {
            // rows (noise, axis 2) -> [M0 M1][n2]; axis 1 per slab -> [M0][n1][n2];
            // axis 0 -> fields
            uint32_t* inter2 = inter + (size_t)nr * g.m[0] * g.m[1] * g.n[2];
            const long long rows = g.m[0] * g.m[1];
            const dim3 g1((unsigned)nr, (unsigned)(rows / tc_lines_per_block(g.m[2])));
            const dim3 g2((unsigned)(g.n[2] / tc_lines_per_block(g.m[1])), (unsigned)(nr * g.m[0]));
            const dim3 g3((unsigned)(g.n[1] * g.n[2] / tc_lines_per_block(g.m[0])), (unsigned)nr);
            CF_TRY(launch(g.m[2], true, g1, rr, rows, inter, g.n[2], nullptr, nullptr));
            CF_TRY(launch(g.m[1], false, g2, 0, 0, inter, g.n[2], nullptr, inter2));
            CF_TRY(launch(g.m[0], false, g3, 0, 0, inter2, g.n[1] * g.n[2], f, nullptr));
        }
    }
    return CF_OK;
}

}  // namespace cf

extern "C" cf_status cf_tc_faults(cf_stream_t s, uint32_t* count) {
    using namespace cf;
    clear_error();
    if (!count) return fail(CF_ERR_ARG, "count is NULL");
    CF_TRY(enter((cudaStream_t)s));
    CF_CUDA(cudaStreamSynchronize((cudaStream_t)s));
    unsigned int v = 0, zero = 0;
    CF_CUDA(cudaMemcpyFromSymbol(&v, g_tc_faults, sizeof v));
    CF_CUDA(cudaMemcpyToSymbol(g_tc_faults, &zero, sizeof zero));
    *count = v;
    return CF_OK;
}
