// cf_fft.cuh -- CTA-level line FFTs for sm_103a.
//
// A CTA transforms several lines of length L (a power of two, 2..4096) at
// once.  Each line is handled by TL = L/E threads that hold E points each in
// registers (E = 16 in binary32, 8 in binary64).  The transform is a Stockham
// autosort FFT: every stage applies radix-R butterflies (R = E, the last stage
// R = L / E^k) entirely in registers, and consecutive stages exchange data
// through shared memory (one write + one read per stage boundary), padded by
// one slot every E points so that the stride-R accesses of the early stages
// hit distinct banks.  The first stage's inputs come from the caller
// (generated noise or global loads) and the last stage's outputs go to a
// caller functor (global stores with cropping, or a fused epilogue), so a
// transform costs (#stages - 1) shared-memory round trips and no global
// traffic beyond its input and output.
#pragma once
#include "cf_device.cuh"

namespace cf {

constexpr int TWN = 8192;  // twiddle table length: w[j] = exp(+2 pi i j / TWN)

// Points held per thread (build-time tunables; powers of two, 2..16).
#ifndef CF_E32
#define CF_E32 16
#endif
#ifndef CF_E64
#define CF_E64 8
#endif

template <typename T>
struct FftE;
template <>
struct FftE<float> {
    static constexpr int value = CF_E32;
};
template <>
struct FftE<double> {
    static constexpr int value = CF_E64;
};

template <typename T, int L, int EMAX = FftE<T>::value>
struct LineGeom {
    static constexpr int E = L < EMAX ? L : EMAX;  // points per thread
    static constexpr int TL = L / E;               // threads per line
    static constexpr int PADDED = L + L / E;       // padded line length (line stride)
    // padding granularity of the row layout: one slot per E points, except
    // one per 16 for 8-byte elements with E = 8 (there a slot per 8 points
    // shifts 16 consecutive lanes over 17 slots and every contiguous access
    // of a warp takes 3 shared-memory wavefronts instead of 2)
    static constexpr int PADE = (sizeof(T) == 4 && E == 8) ? 16 : E;
};

// padded shared-memory slot of point p
template <int E>
__device__ __forceinline__ int padp(int p) { return p + p / E; }

// Lines stored one after the other (row tiles).
template <int E, int STRIDE>
struct RowLayout {
    __device__ __forceinline__ int operator()(int line, int p) const { return line * STRIDE + padp<E>(p); }
};
// Lines interleaved point-major (column tiles of C lines).
template <int E, int C>
struct ColLayout {
    __device__ __forceinline__ int operator()(int line, int p) const { return padp<E>(p) * C + line; }
};

// ---------------------------------------------------------------- radix kernels
// Scalar type of the constants of a value type (C2<T>: T; CP: float).
template <typename V>
struct VScalar;
template <typename T>
struct VScalar<C2<T>> {
    using type = T;
};
template <>
struct VScalar<CP> {
    using type = float;
};

template <int SIGN, typename V>
__device__ __forceinline__ void dft2(V& a, V& b) {
    const V t = a;
    a = t + b;
    b = t - b;
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
    const C2<T> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = mul_si<SIGN>(a1 - a3);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}
// paired lines: the product by SIGN i is folded into the additions
template <int SIGN>
__device__ __forceinline__ void dft4(CP& a0, CP& a1, CP& a2, CP& a3) {
    const CP t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, d = a1 - a3;
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = add_si<SIGN>(t1, d);
    a3 = sub_si<SIGN>(t1, d);
}

// multiply by exp(SIGN i theta) given (cos theta, sin theta)
template <int SIGN, typename T>
__device__ __forceinline__ C2<T> rot(C2<T> a, T c, T s) {
    return cmul(a, mk(c, SIGN > 0 ? s : -s));
}
template <int SIGN>
__device__ __forceinline__ CP rot(CP a, float c, float s) {
    return cmul_cs(a, c, SIGN > 0 ? s : -s);
}

template <int SIGN, typename V>
__device__ __forceinline__ void dft8(V* v) {
    using T = typename VScalar<V>::type;
    dft4<SIGN>(v[0], v[2], v[4], v[6]);
    dft4<SIGN>(v[1], v[3], v[5], v[7]);
    const T h = (T)0.70710678118654752440;
    const V o0 = v[1];
    const V o1 = rot<SIGN>(v[3], h, h);
    const V o2 = v[5];  // times SIGN i, folded into the additions below
    const V o3 = rot<SIGN>(v[7], -h, h);
    const V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + o1;
    v[5] = e1 - o1;
    v[2] = add_si<SIGN>(e2, o2);
    v[6] = sub_si<SIGN>(e2, o2);
    v[3] = e3 + o3;
    v[7] = e3 - o3;
}

template <int SIGN, typename T>
__device__ __forceinline__ void dft16(C2<T>* v) {
    // four length-4 DFTs over n1 (stride 4), twiddles w16^{n2 k1}, four more over n2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<SIGN>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
    const T h = (T)0.70710678118654752440;
    v[5] = rot<SIGN>(v[5], c1, s1);      // n2=1,k1=1: w^1
    v[9] = rot<SIGN>(v[9], h, h);        // n2=1,k1=2: w^2
    v[13] = rot<SIGN>(v[13], s1, c1);    // n2=1,k1=3: w^3
    v[6] = rot<SIGN>(v[6], h, h);        // n2=2,k1=1: w^2
    v[10] = mul_si<SIGN>(v[10]);         // n2=2,k1=2: w^4
    v[14] = rot<SIGN>(v[14], -h, h);     // n2=2,k1=3: w^6
    v[7] = rot<SIGN>(v[7], s1, c1);      // n2=3,k1=1: w^3
    v[11] = rot<SIGN>(v[11], -h, h);     // n2=3,k1=2: w^6
    v[15] = rot<SIGN>(v[15], -c1, -s1);  // n2=3,k1=3: w^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4x4 block
    C2<T> t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, int SIGN, typename V>
__device__ __forceinline__ void dftR(V* v) {
    if constexpr (R == 2) {
        dft2<SIGN>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft8<SIGN>(v);
    } else if constexpr (R == 16) {
        dft16<SIGN>(v);
    }
}

template <int SIGN, typename T>
__device__ __forceinline__ C2<T> twiddle(const C2<T>* __restrict__ tw, int idx) {
    const C2<T> w = tw[idx];
    return SIGN > 0 ? w : mk(w.x, -w.y);
}
// broadcast table of the paired lines: (cos, cos, sin, sin)
template <int SIGN>
__device__ __forceinline__ float4 twiddle(const float4* __restrict__ tw, int idx) {
    const float4 w = tw[idx];
    return SIGN > 0 ? w : make_float4(w.x, w.y, -w.z, -w.w);
}

// ---------------------------------------------------------------- Stockham stages
// v holds this thread's inputs of the stage with sub-transform size NS:
// butterfly b (jb = j + b*TL) takes points jb + q*(L/R), q < R, in v[b*R + q].
// KEEP: only outputs with point index < KEEP are produced (KEEP = L or L/2).
// out(line, point, value) receives each kept output of the last stage.
// SYNC_OUT: barrier before the last stage emits its outputs, so that out()
// may write into the exchange buffer sm itself.
template <typename V, typename TW, int L, int E, int SIGN, int KEEP, int NS, bool SYNC_OUT, class Lay, class Out>
__device__ __forceinline__ void fft_stage(V* sm, const Lay& lay, int line, int j, V (&v)[E],
                                          const TW* __restrict__ tw, Out& out) {
    constexpr int R = (E < L / NS) ? E : (L / NS);
    constexpr int TL = L / E;
    constexpr int B = E / R;
    constexpr int STRIDE = L / R;
    if constexpr (NS > 1) {
        constexpr int TWS = TWN / (NS * R);
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int k = (j + b * TL) & (NS - 1);
#pragma unroll
            for (int q = 1; q < R; ++q)
                v[b * R + q] = cmul(v[b * R + q], twiddle<SIGN>(tw, (q * k * TWS) & (TWN - 1)));
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) dftR<R, SIGN>(&v[b * R]);
    if constexpr (NS * R == L) {
        if constexpr (SYNC_OUT) __syncthreads();
#pragma unroll
        for (int b = 0; b < B; ++b)
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (q * STRIDE < KEEP) out(line, j + b * TL + q * STRIDE, v[b * R + q]);
    } else {
        __syncthreads();
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int jb = j + b * TL;
            const int base = (jb / NS) * (NS * R) + (jb & (NS - 1));
#pragma unroll
            for (int q = 0; q < R; ++q) sm[lay(line, base + q * NS)] = v[b * R + q];
        }
        __syncthreads();
        constexpr int NS2 = NS * R;
        constexpr int R2 = (E < L / NS2) ? E : (L / NS2);
        constexpr int B2 = E / R2;
        constexpr int STRIDE2 = L / R2;
#pragma unroll
        for (int b = 0; b < B2; ++b)
#pragma unroll
            for (int q = 0; q < R2; ++q) v[b * R2 + q] = sm[lay(line, j + b * TL + q * STRIDE2)];
        fft_stage<V, TW, L, E, SIGN, KEEP, NS2, SYNC_OUT>(sm, lay, line, j, v, tw, out);
    }
}

// Full transform of a line whose first-stage inputs v[q] = x[j + q*L/E] are
// already in registers.  Every thread of the CTA must call this (it contains
// __syncthreads); threads without a valid line pass dummy data.
template <typename T, int L, int SIGN, int KEEP, bool SYNC_OUT = false, int E, class Lay, class Out>
__device__ __forceinline__ void line_fft(C2<T>* sm, const Lay& lay, int line, int j, C2<T> (&v)[E],
                                         const C2<T>* __restrict__ tw, Out& out) {
    fft_stage<C2<T>, C2<T>, L, E, SIGN, KEEP, 1, SYNC_OUT>(sm, lay, line, j, v, tw, out);
}

// The same for two lines at once (CP values, broadcast twiddle table).
template <int L, int SIGN, int KEEP, bool SYNC_OUT = false, int E, class Lay, class Out>
__device__ __forceinline__ void line_fft_pair(CP* sm, const Lay& lay, int line, int j, CP (&v)[E],
                                              const float4* __restrict__ tw, Out& out) {
    fft_stage<CP, float4, L, E, SIGN, KEEP, 1, SYNC_OUT>(sm, lay, line, j, v, tw, out);
}

}  // namespace cf
