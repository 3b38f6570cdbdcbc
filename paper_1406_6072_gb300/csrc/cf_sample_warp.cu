// cf_sample_warp.cu -- the binary32 noise row pass of the sampler for rows
// of L = P^2 points (P = 32: 1024 points, one row per warp; P = 16: 256
// points, two rows per warp), section 2, eq. (Papos2) and the closing
// paragraph: noise, scaling by sqrt(lambda+/M^d) and the pruned inverse
// transform along the last axis.
//
// A row is held by P lanes, split as n = g + P n2 (lane g holds the P points
// n2 = 0..P-1) and k = k2 + P k1, so that
//   X[k2 + P k1] = sum_g wP^(g k1) [ wL^(g k2) sum_n2 x[g + P n2] wP^(n2 k2) ]
// (w_N = exp(+2 pi i / N), the inverse transform's sign): a P-point transform
// in registers per lane, one twiddle per point, one transpose through the
// lane group's own tile of shared memory (synchronised by the warp alone: no
// CTA barrier on the path), and a second P-point transform in registers of
// which only the outputs k1 < P/2 (k < L/2, the kept half) are formed.
// Every lane has P independent points in each stage, which hides the
// latencies that bound the shared-memory exchanges of the radix-8 line
// transforms; the noise's Box-Muller runs two cell pairs of the lane at a
// time in paired binary32 instructions.
//
// The draws are the specification's (the same Philox counters and operations
// as every other sampler kernel, bit for bit); the transform's rounding
// differs from the radix-8 kernels' only by its order.  Warps are independent,
// so the CTA shape (8, 4 or 16 warps) changes no result bit.
#include "cf_kernels.cuh"
#include "cf_warpfft.cuh"

namespace cf {

// P lanes per row and P points per lane: rows of L = P^2 points, 32 / P rows
// per warp (P = 32: one row per warp; P = 16: two rows of 256 points).
__host__ __device__ constexpr int warp_rows_warps(int shape) { return shape == 1 ? 4 : (shape == 2 ? 16 : 8); }

template <int P, int W>
struct WarpRowsCfg {
    static constexpr int L = P * P;
    static constexpr int RPW = 32 / P;  // rows per warp
    static constexpr int PAD = P + 1;   // transpose tile row stride (complex values)
    static constexpr int THREADS = 32 * W;
    // 20 resident warps per SM for 32-point lanes (102 registers per thread)
    static constexpr int MINB = P == 32 ? (20 / W > 0 ? 20 / W : 1) : (32 / W > 0 ? 32 / W : 1);
    static constexpr size_t SMEM = sizeof(C2<float>) * ((size_t)P * P + (size_t)W * RPW * P * PAD);
};

// Block b of the one-dimensional grid covers realization rl = b mod chunk
// and row block bx = b / chunk (realizations adjacent, so that the blocks
// resident together read the same rows of sqrt(lambda+) and a 3D amplitude
// array larger than L2 leaves DRAM once per launch, not once per
// realization); lane group `lane / P` of warp `threadIdx.x / 32` transforms
// row (bx W + warp) RPW + lane / P of realization rl: intermediate
// out[chunk][nrows][keep], keep <= L/2.
template <int P, bool DESC, int W>
__global__ void __launch_bounds__(WarpRowsCfg<P, W>::THREADS, WarpRowsCfg<P, W>::MINB)
    k_sample_rows_warp(const float* __restrict__ s, float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                       long long nrows, int keep, int chunk, C2<float>* __restrict__ out,
                       const C2<float>* __restrict__ tw, const RealDesc* __restrict__ desc) {
    using Cfg = WarpRowsCfg<P, W>;
    constexpr int L = Cfg::L;
    constexpr int PAD = Cfg::PAD;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<float>* twl = reinterpret_cast<C2<float>*>(smraw);  // twl[k2 * P + g] = w_L^(g k2)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % P, sub = lane / P;
    C2<float>* tile = twl + P * P + ((size_t)warp * Cfg::RPW + sub) * P * PAD;
    for (int i = threadIdx.x; i < P * P; i += Cfg::THREADS) {
        const int k2 = i / P, l = i % P;
        twl[i] = tw[((l * k2) & (L - 1)) * (TWN / L)];
    }
    __syncthreads();
    const int rl = (int)(blockIdx.x % (unsigned)chunk);
    const long long bx = blockIdx.x / (unsigned)chunk;
    const long long row = (bx * W + warp) * Cfg::RPW + sub;
    // the warp's lane groups stay together to the end (warp-wide exchange);
    // a group past the last row works on row 0 and stores nothing
    if ((bx * W + warp) * Cfg::RPW >= nrows) return;
    const bool valid = row < nrows;
    const long long rw = valid ? row : 0;
    const float* srow = s + (size_t)rw * L;
    float amp = amp_scale;
    uint32_t k0 = key0, k1 = key1, r = r0 + (uint32_t)rl;
    if constexpr (DESC) {
        const RealDesc& d = desc[rl];
        srow = d.s + (size_t)rw * L;
        amp = d.amp_scale;
        k0 = d.key0;
        k1 = d.key1;
        r = d.r;
    }
    C2<float> v[P];
    // noise: one Philox call per cell pair (c, c + L/2), c = g + P n2 for
    // n2 < P/2 (points n2 and n2 + P/2 of this lane); two pairs per paired
    // Box-Muller
    const unsigned long long pbase = (unsigned long long)rw * (L / 2) + (unsigned long long)g;
#pragma unroll
    for (int n2 = 0; n2 < P / 2; n2 += 2) {
        const int ca = g + P * n2, cb = ca + P;
        CP lo, hi;
        noise_pair_f32x2(pbase + P * n2, r, k0, k1, pbase + P * (n2 + 1), r, k0, k1, lo, hi);
        const float sa = __fmul_rn(__ldg(srow + ca), amp), sb = __fmul_rn(__ldg(srow + cb), amp);
        const float sah = __fmul_rn(__ldg(srow + ca + L / 2), amp), sbh = __fmul_rn(__ldg(srow + cb + L / 2), amp);
        v[n2] = mk(__fmul_rn(lo.re.x, sa), __fmul_rn(lo.im.x, sa));
        v[n2 + 1] = mk(__fmul_rn(lo.re.y, sb), __fmul_rn(lo.im.y, sb));
        v[n2 + P / 2] = mk(__fmul_rn(hi.re.x, sah), __fmul_rn(hi.im.x, sah));
        v[n2 + 1 + P / 2] = mk(__fmul_rn(hi.re.y, sbh), __fmul_rn(hi.im.y, sbh));
    }
    // first stage: y[k2] = sum_n2 v[n2] w_P^(n2 k2), times w_L^(g k2), stored
    // to the group's tile as row g
    C2<float> y[P];
    RegFft<P, +1, false>::template run<1>(v, y);
    tile[g * PAD] = y[0];
#pragma unroll
    for (int k2 = 1; k2 < P; ++k2) tile[g * PAD + k2] = cmul(y[k2], twl[k2 * P + g]);
    __syncwarp();
    // second stage: g = k2 now; column k2 of the tile over l
#pragma unroll
    for (int l = 0; l < P; ++l) v[l] = tile[l * PAD + g];
    RegFft<P, +1, true>::template run<1>(v, y);
    if (!valid) return;
    C2<float>* o = out + ((size_t)rl * (size_t)nrows + (size_t)row) * (size_t)keep;
#pragma unroll
    for (int k1 = 0; k1 < P / 2; ++k1) {
        const int k = g + P * k1;
        if (k < keep) o[k] = y[k1];
    }
}

// Rows of 256 or 1024 points.
bool warp_rows_len(long long L) { return L == 256 || L == 1024; }

cf_status launch_rows_warp(long long L, int keep, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                           int chunk, long long nrows, C2<float>* out, cudaStream_t st, const RealDesc* desc,
                           int shape) {
    if (!warp_rows_len(L)) return fail(CF_ERR_UNSUPPORTED, "warp row pass for rows of 256 or 1024 points only");
    if (keep < 1 || keep > L / 2) return fail(CF_ERR_ARG, "row pass keeps %d of %lld outputs", keep, L);
    if (chunk < 1 || chunk > 65535) return fail(CF_ERR_ARG, "row pass over %d realizations", chunk);
    auto go = [&](auto Pc, auto Wc) -> cf_status {
        constexpr int P = decltype(Pc)::value;
        constexpr int W = decltype(Wc)::value;
        using Cfg = WarpRowsCfg<P, W>;
        auto kern = desc ? k_sample_rows_warp<P, true, W> : k_sample_rows_warp<P, false, W>;
        CF_TRY(prepare_smem(kern, Cfg::SMEM));
        const long long per_block = (long long)W * Cfg::RPW;
        const long long blocks = (nrows + per_block - 1) / per_block * (long long)chunk;
        if (blocks > 0x7fffffffll) return fail(CF_ERR_UNSUPPORTED, "row pass of %lld blocks", blocks);
        ScopedKernelTimer kt(st, "sample_rows_f32", Cfg::L);
        kern<<<(unsigned)blocks, Cfg::THREADS, Cfg::SMEM, st>>>(s, amp_scale, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                                r0, nrows, keep, chunk, out, twiddles_f32(), desc);
        CF_CHECK_LAUNCH();
        return CF_OK;
    };
    auto with_w = [&](auto Pc) -> cf_status {
        switch (warp_rows_warps(shape)) {
            case 4: return go(Pc, std::integral_constant<int, 4>());
            case 16: return go(Pc, std::integral_constant<int, 16>());
            default: return go(Pc, std::integral_constant<int, 8>());
        }
    };
    return L == 1024 ? with_w(std::integral_constant<int, 32>()) : with_w(std::integral_constant<int, 16>());
}

}  // namespace cf
