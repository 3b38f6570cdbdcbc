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

}  // namespace cf
