// cf_sample_warp.cu -- the binary32 noise row pass of the sampler for rows
// of 1024 points with one warp per row (section 2, eq. (Papos2) and the
// closing paragraph: noise, scaling by sqrt(lambda+/M^d) and the pruned
// inverse transform along the last axis).
//
// The row is split as n = l + 32 n2 (lane l holds the 32 points n2 = 0..31)
// and k = k2 + 32 k1, so that
//   X[k2 + 32 k1] = sum_l w32^(l k1) [ w1024^(l k2) sum_n2 x[l + 32 n2] w32^(n2 k2) ]
// (w_N = exp(+2 pi i / N), the inverse transform's sign): a 32-point
// transform in registers per lane, one twiddle per point, one transpose
// through the warp's own tile of shared memory (synchronised by the warp
// alone: no CTA barrier on the path), and a second 32-point transform in
// registers of which only the outputs k1 < 16 (k < 512, the kept half) are
// formed.  Every lane has 32 independent points in each stage, which hides
// the latencies that bound the shared-memory exchanges of the radix-8 line
// transforms; the noise's Box-Muller runs two cell pairs of the lane at a
// time in paired binary32 instructions.
//
// The draws are the specification's (the same Philox counters and operations
// as every other sampler kernel, bit for bit); the transform's rounding
// differs from the radix-8 kernels' only by its order.  Warps are independent,
// so the CTA shape (8, 4 or 16 warps) changes no result bit.
#include "cf_kernels.cuh"

namespace cf {

// cos(pi m / 16) for m = 0..8
__host__ __device__ constexpr double cos_pi16_base(int m) {
    return m == 0   ? 1.0
           : m == 1 ? 0.98078528040323044913
           : m == 2 ? 0.92387953251128675613
           : m == 3 ? 0.83146961230254523708
           : m == 4 ? 0.70710678118654752440
           : m == 5 ? 0.55557023301960222474
           : m == 6 ? 0.38268343236508977173
           : m == 7 ? 0.19509032201612826785
                    : 0.0;
}
// cos and sin of pi m / 16 for m = 0..15 (the powers of w32 in the upper
// half-plane)
__host__ __device__ constexpr double cos_pi16(int m) { return m <= 8 ? cos_pi16_base(m) : -cos_pi16_base(16 - m); }
__host__ __device__ constexpr double sin_pi16(int m) { return m <= 8 ? cos_pi16_base(8 - m) : cos_pi16_base(m - 8); }

// w_N^(SIGN k) o for N dividing 32 and k < N/2 (compile-time after unrolling):
// the trivial factors 1 and SIGN i without multiplications
template <int N, int SIGN>
__device__ __forceinline__ C2<float> rot_const(int k, C2<float> o) {
    const int m = (32 / N) * k;  // w_N^k = w_32^m
    if (m == 0) return o;
    if (m == 8) return mul_si<SIGN>(o);
    const float c = (float)cos_pi16(m), s = SIGN > 0 ? (float)sin_pi16(m) : -(float)sin_pi16(m);
    return mk(o.x * c - o.y * s, o.x * s + o.y * c);
}

// Radix-2 decimation-in-time transform of N points x[0], x[S], ..., x[(N-1) S]
// in registers: y[k] = sum_n x[n S] w_N^(SIGN n k); HALF: only k < N/2.
template <int N, int SIGN, bool HALF>
struct RegFft {
    template <int S>
    static __device__ __forceinline__ void run(const C2<float>* x, C2<float>* y) {
        if constexpr (N == 1) {
            y[0] = x[0];
        } else {
            C2<float> e[N / 2], o[N / 2];
            RegFft<N / 2, SIGN, false>::template run<2 * S>(x, e);
            RegFft<N / 2, SIGN, false>::template run<2 * S>(x + S, o);
#pragma unroll
            for (int k = 0; k < N / 2; ++k) {
                const C2<float> t = rot_const<N, SIGN>(k, o[k]);
                y[k] = e[k] + t;
                if constexpr (!HALF) y[k + N / 2] = e[k] - t;
            }
        }
    }
};

constexpr int kWarpRowL = 1024;
constexpr int kWarpRowPad = 33;  // transpose tile row stride (complex values)

__host__ __device__ constexpr int warp_rows_warps(int shape) { return shape == 1 ? 4 : (shape == 2 ? 16 : 8); }

template <int W>
struct WarpRowsCfg {
    static constexpr int THREADS = 32 * W;
    // 20 resident warps per SM: 102 registers per thread
    static constexpr int MINB = 20 / W > 0 ? 20 / W : 1;
    static constexpr size_t SMEM = sizeof(C2<float>) * (32 * 32 + (size_t)W * 32 * kWarpRowPad);
};

// Warp `threadIdx.x / 32` of block (bx, rl) transforms row bx W + warp of
// realization rl of the chunk: intermediate out[chunk][nrows][keep], keep <= 512.
template <bool DESC, int W>
__global__ void __launch_bounds__(WarpRowsCfg<W>::THREADS, WarpRowsCfg<W>::MINB)
    k_sample_rows_warp(const float* __restrict__ s, float amp_scale, uint32_t key0, uint32_t key1, uint32_t r0,
                       long long nrows, int keep, C2<float>* __restrict__ out, const C2<float>* __restrict__ tw,
                       const RealDesc* __restrict__ desc) {
    constexpr int L = kWarpRowL;
    constexpr int P = 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<float>* twl = reinterpret_cast<C2<float>*>(smraw);  // twl[k2 * 32 + l] = w1024^(l k2)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C2<float>* tile = twl + 32 * 32 + warp * 32 * kWarpRowPad;
    for (int i = threadIdx.x; i < 32 * 32; i += WarpRowsCfg<W>::THREADS) {
        const int k2 = i >> 5, l = i & 31;
        twl[i] = tw[((l * k2) & (L - 1)) * (TWN / L)];
    }
    __syncthreads();
    const long long row = (long long)blockIdx.x * W + warp;
    if (row >= nrows) return;
    const int rl = blockIdx.y;
    const float* srow = s + (size_t)row * L;
    float amp = amp_scale;
    uint32_t k0 = key0, k1 = key1, r = r0 + (uint32_t)rl;
    if constexpr (DESC) {
        const RealDesc& d = desc[rl];
        srow = d.s + (size_t)row * L;
        amp = d.amp_scale;
        k0 = d.key0;
        k1 = d.key1;
        r = d.r;
    }
    C2<float> v[P];
    // noise: one Philox call per cell pair (c, c + L/2), c = lane + 32 n2 for
    // n2 < 16 (points n2 and n2 + 16 of this lane); two pairs per paired
    // Box-Muller
    const unsigned long long pbase = (unsigned long long)row * (L / 2) + (unsigned long long)lane;
#pragma unroll
    for (int n2 = 0; n2 < P / 2; n2 += 2) {
        const int ca = lane + 32 * n2, cb = ca + 32;
        CP lo, hi;
        noise_pair_f32x2(pbase + 32 * n2, r, k0, k1, pbase + 32 * (n2 + 1), r, k0, k1, lo, hi);
        const float sa = __fmul_rn(__ldg(srow + ca), amp), sb = __fmul_rn(__ldg(srow + cb), amp);
        const float sah = __fmul_rn(__ldg(srow + ca + L / 2), amp), sbh = __fmul_rn(__ldg(srow + cb + L / 2), amp);
        v[n2] = mk(__fmul_rn(lo.re.x, sa), __fmul_rn(lo.im.x, sa));
        v[n2 + 1] = mk(__fmul_rn(lo.re.y, sb), __fmul_rn(lo.im.y, sb));
        v[n2 + P / 2] = mk(__fmul_rn(hi.re.x, sah), __fmul_rn(hi.im.x, sah));
        v[n2 + 1 + P / 2] = mk(__fmul_rn(hi.re.y, sbh), __fmul_rn(hi.im.y, sbh));
    }
    // first stage: y[k2] = sum_n2 v[n2] w32^(n2 k2), times w1024^(lane k2),
    // stored to the tile as row `lane`
    C2<float> y[P];
    RegFft<P, +1, false>::template run<1>(v, y);
    tile[lane * kWarpRowPad] = y[0];
#pragma unroll
    for (int k2 = 1; k2 < P; ++k2) tile[lane * kWarpRowPad + k2] = cmul(y[k2], twl[k2 * 32 + lane]);
    __syncwarp();
    // second stage: lane = k2 now; column k2 of the tile over l
#pragma unroll
    for (int l = 0; l < P; ++l) v[l] = tile[l * kWarpRowPad + lane];
    RegFft<P, +1, true>::template run<1>(v, y);
    C2<float>* o = out + ((size_t)rl * (size_t)nrows + (size_t)row) * (size_t)keep;
#pragma unroll
    for (int k1 = 0; k1 < P / 2; ++k1) {
        const int k = lane + 32 * k1;
        if (k < keep) o[k] = y[k1];
    }
}

cf_status launch_rows_warp(long long L, int keep, const float* s, float amp_scale, uint64_t seed, uint32_t r0,
                           int chunk, long long nrows, C2<float>* out, cudaStream_t st, const RealDesc* desc,
                           int shape) {
    if (L != kWarpRowL) return fail(CF_ERR_UNSUPPORTED, "warp row pass for rows of %d points only", kWarpRowL);
    if (keep < 1 || keep > L / 2) return fail(CF_ERR_ARG, "row pass keeps %d of %lld outputs", keep, L);
    if (chunk < 1 || chunk > 65535) return fail(CF_ERR_ARG, "row pass over %d realizations", chunk);
    auto go = [&](auto Wc) -> cf_status {
        constexpr int W = decltype(Wc)::value;
        using Cfg = WarpRowsCfg<W>;
        auto kern = desc ? k_sample_rows_warp<true, W> : k_sample_rows_warp<false, W>;
        CF_TRY(prepare_smem(kern, Cfg::SMEM));
        dim3 grid((unsigned)((nrows + W - 1) / W), (unsigned)chunk);
        ScopedKernelTimer kt(st, "sample_rows_f32", kWarpRowL);
        kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(s, amp_scale, (uint32_t)seed, (uint32_t)(seed >> 32), r0, nrows,
                                                     keep, out, twiddles_f32(), desc);
        CF_CHECK_LAUNCH();
        return CF_OK;
    };
    switch (warp_rows_warps(shape)) {
        case 8: return go(std::integral_constant<int, 8>());
        case 16: return go(std::integral_constant<int, 16>());
        default: return go(std::integral_constant<int, 4>());
    }
}

}  // namespace cf
