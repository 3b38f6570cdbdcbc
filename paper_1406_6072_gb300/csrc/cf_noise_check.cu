// cf_noise_check.cu -- self-check of the binary32 noise arithmetic (section 2,
// eq. (Papos2): the draws are the specification's only if every operation
// rounds as specified).  The noise kernels form the logarithm's quotient and
// the Box-Muller square root with short sequences (noise_quotient,
// noise_sqrt in cf_device.cuh); these kernels compare them with the IEEE
// correctly rounded quotient and square root over every binary32 input the
// noise can give them.
#include "cf_internal.h"
#include "cf_kernels.cuh"

namespace cf {

// Quotient inputs: every binary32 m from sqrt(1/2) to sqrt(2) (bit patterns
// lo .. hi), a = m - 1, b = m + 1 as the logarithm forms them.
__global__ void k_check_quotient(uint32_t lo, uint32_t hi, unsigned long long* bad, uint32_t* example) {
    const unsigned long long n = (unsigned long long)(hi - lo) + 1;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float m = __uint_as_float(lo + (uint32_t)i);
        const float a = __fsub_rn(m, 1.0f), b = __fadd_rn(m, 1.0f);
        if (__float_as_uint(noise_quotient(a, b)) != __float_as_uint(__fdiv_rn(a, b))) {
            if (atomicAdd(bad, 1ull) == 0ull) *example = __float_as_uint(m);
        }
    }
}

// Square-root inputs: +0, -0 and every binary32 x from 2^-24 to 34 (the
// smallest nonzero -2 ln u is about 2^-23, the largest 33.3).
__global__ void k_check_sqrt(uint32_t lo, uint32_t hi, unsigned long long* bad, uint32_t* example) {
    const unsigned long long n = (unsigned long long)(hi - lo) + 1;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n + 2;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t bits = i < n ? lo + (uint32_t)i : (i == n ? 0x00000000u : 0x80000000u);
        const float x = __uint_as_float(bits);
        if (__float_as_uint(noise_sqrt(x)) != __float_as_uint(__fsqrt_rn(x))) {
            if (atomicAdd(bad, 1ull) == 0ull) *example = bits;
        }
    }
}

}  // namespace cf

using namespace cf;

extern "C" cf_status cf_noise_selfcheck(uint64_t* mismatches, uint32_t* examples) {
    clear_error();
    if (!mismatches) return fail(CF_ERR_ARG, "mismatches is NULL");
    CF_TRY(enter(nullptr));
    unsigned long long* d = nullptr;
    CF_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long) + 2 * sizeof(uint32_t)));
    uint32_t* ex = reinterpret_cast<uint32_t*>(d + 2);
    cf_status st = CF_OK;
    if (cudaMemset(d, 0, 2 * sizeof(unsigned long long) + 2 * sizeof(uint32_t)) != cudaSuccess) {
        st = fail(CF_ERR_CUDA, "cudaMemset failed");
    } else {
        // sqrt(1/2) rounded down and sqrt(2) rounded up, as binary32 bit patterns
        k_check_quotient<<<1024, 256>>>(0x3F3504F3u, 0x3FB504F4u, d, ex);
        k_check_sqrt<<<4096, 256>>>(0x33800000u, 0x42080000u, d + 1, ex + 1);
        unsigned long long h[2] = {0, 0};
        uint32_t hx[2] = {0, 0};
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(hx, ex, sizeof(hx), cudaMemcpyDeviceToHost) != cudaSuccess) {
            st = fail(CF_ERR_CUDA, "noise self-check kernels failed");
        } else {
            mismatches[0] = h[0];
            mismatches[1] = h[1];
            if (examples) {
                examples[0] = hx[0];
                examples[1] = hx[1];
            }
        }
    }
    cudaFree(d);
    return st;
}
