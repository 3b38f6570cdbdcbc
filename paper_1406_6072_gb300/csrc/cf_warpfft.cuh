// cf_warpfft.cuh -- a radix-2 transform of up to 32 points held in one
// thread's registers, with compile-time twiddles (the per-lane stages of the
// warp row pass, cf_sample_warp.cu).
#pragma once
#include "cf_device.cuh"

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

// One radix-2 butterfly with the twiddle w_N^(SIGN k): y0 = e + w o and, when
// y1 is wanted, y1 = e - w o.  A non-trivial twiddle is folded into two fused
// multiply-adds per component, e.x + o.x c - o.y s, and the difference is
// formed as 2 e - y0 (one fused multiply-add, exact product), six
// instructions where a separate product and two sums take eight; the trivial
// twiddles 1 and SIGN i take additions only.
template <int N, int SIGN, bool Y1>
__device__ __forceinline__ void butterfly_const(int k, C2<float> e, C2<float> o, C2<float>& y0, C2<float>& y1) {
    const int m = (32 / N) * k;  // w_N^k = w_32^m
    if (m == 0 || m == 8) {
        const C2<float> t = m == 0 ? o : mul_si<SIGN>(o);
        y0 = e + t;
        if constexpr (Y1) y1 = e - t;
        return;
    }
    const float c = (float)cos_pi16(m), s = SIGN > 0 ? (float)sin_pi16(m) : -(float)sin_pi16(m);
    y0 = mk(__fmaf_rn(o.x, c, __fmaf_rn(-o.y, s, e.x)), __fmaf_rn(o.x, s, __fmaf_rn(o.y, c, e.y)));
    if constexpr (Y1) y1 = mk(__fmaf_rn(2.0f, e.x, -y0.x), __fmaf_rn(2.0f, e.y, -y0.y));
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
                if constexpr (HALF) {
                    C2<float> unused;
                    butterfly_const<N, SIGN, false>(k, e[k], o[k], y[k], unused);
                } else {
                    butterfly_const<N, SIGN, true>(k, e[k], o[k], y[k], y[k + N / 2]);
                }
            }
        }
    }
};

}  // namespace cf
