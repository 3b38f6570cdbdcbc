// cf_df.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two binary32 numbers with |lo| <= ulp(hi)/2, about 48 bits of
// significand.  The operations are the error-free transformations of Knuth
// (two-sum) and Dekker (fast two-sum; the exact product through a fused
// multiply-add), composed as in the double-double algorithms of Hida, Li and
// Bailey (QD library paper, 2001): addition with both low parts propagated
// (relative error about 2^-47), multiplication with the cross terms (about
// 2^-47).  Every operation is a fixed sequence of round-to-nearest _rn
// intrinsics, so the compiler neither contracts nor reorders it.
//
// Used for the embedding's transforms: binary64 throughput is a small
// fraction of binary32 throughput on this GPU, and 48 bits keep the
// eigenvalues well inside their 1e-12 lambda_max tolerance.
#pragma once
#include "cf_kernels.cuh"

namespace cf {

struct DF {
    float hi, lo;
    DF() = default;
    // hi = fl32(d), lo = fl32(d - hi) (folded at compile time for literals)
    __host__ __device__ constexpr DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF(s, e);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }

__device__ __forceinline__ DF operator*(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// binary64 <-> double-float (run time)
__device__ __forceinline__ DF df_from(double d) {
    const float h = __double2float_rn(d);
    return DF(h, __double2float_rn(__dsub_rn(d, (double)h)));
}
__device__ __forceinline__ double df_to(DF a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// the transforms' geometry: 8 points per thread, as for binary64
template <>
struct FftE<DF> {
    static constexpr int value = CF_E64;
};

// twiddle table of the current device (TWN entries, the binary64 table split)
const C2<DF>* twiddles_df();
template <>
inline const C2<DF>* twiddles<DF>() { return twiddles_df(); }

}  // namespace cf
