// cf_lp.cu -- steps c1-c2 stand-alone: lognormal transform and Poisson
// sampling of given Gaussian fields (section 3.1, eqs. (Lncov), (sampling)).
#include "cf_kernels.cuh"

namespace cf {

template <typename T>
__global__ void k_lognormal_poisson(const T* __restrict__ G, long long cells, long long nfields, double half_sigma2,
                                    float half_sigma2_f, double nbar, const float* __restrict__ f, uint32_t key0,
                                    uint32_t key1, unsigned long long field0, float* __restrict__ delta,
                                    int32_t* __restrict__ counts) {
    const long long total = cells * nfields;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long jf = idx / cells;
        const long long i = idx - jf * cells;
        const unsigned long long field = field0 + (unsigned long long)jf;
        const uint4 x = poisson_words((unsigned long long)i, (uint32_t)(field >> 1), key0, key1);
        const unsigned long long ub = (field & 1) ? bits53(x.z, x.w) : bits53(x.x, x.y);
        const float fi = f ? f[i] : 1.0f;
        const T g = G[idx];
        int n;
        if constexpr (sizeof(T) == 4) {
            n = poisson_count_fast(g, half_sigma2, half_sigma2_f, nbar, (float)nbar, fi, ub);
            if (delta) delta[idx] = expf(g - half_sigma2_f) - 1.0f;
        } else {
            const double rho = exp(g - half_sigma2);
            const double U = __dmul_rn(__ull2double_rn(ub), 0x1p-53);
            n = poisson_icdf_f64(U, nbar * (double)fi * rho);
            if (delta) delta[idx] = (float)(rho - 1.0);
        }
        counts[idx] = n;
    }
}

}  // namespace cf

using namespace cf;

extern "C" cf_status cf_lognormal_poisson(const void* G, cf_dtype dt, int64_t cells_per_field, int64_t nfields,
                                          double sigma2, double nbar, const float* f_or_null, uint64_t seed,
                                          uint64_t field0, float* delta_out_or_null, int32_t* counts_out,
                                          cf_stream_t s) {
    clear_error();
    if (!G || !counts_out) return fail(CF_ERR_ARG, "G and counts_out are required");
    if (cells_per_field < 0 || nfields < 0) return fail(CF_ERR_ARG, "negative size");
    if (!(nbar >= 0.0)) return fail(CF_ERR_ARG, "nbar must be >= 0");
    if (((field0 + (uint64_t)nfields) >> 1) > 0xffffffffull) return fail(CF_ERR_ARG, "field index exceeds 33 bits");
    const long long total = (long long)cells_per_field * nfields;
    if (total == 0) return CF_OK;
    CF_TRY(enter((cudaStream_t)s));
    const int blocks = grid_blocks(total, 256, 152 * 32);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    ScopedKernelTimer kt((cudaStream_t)s, dt == CF_F32 ? "lognormal_poisson_f32" : "lognormal_poisson_f64");
    if (dt == CF_F32) {
        k_lognormal_poisson<float><<<blocks, 256, 0, (cudaStream_t)s>>>(
            (const float*)G, cells_per_field, nfields, 0.5 * sigma2, (float)(0.5 * sigma2), nbar, f_or_null, k0, k1,
            field0, delta_out_or_null, counts_out);
    } else if (dt == CF_F64) {
        k_lognormal_poisson<double><<<blocks, 256, 0, (cudaStream_t)s>>>(
            (const double*)G, cells_per_field, nfields, 0.5 * sigma2, (float)(0.5 * sigma2), nbar, f_or_null, k0, k1,
            field0, delta_out_or_null, counts_out);
    } else {
        return fail(CF_ERR_UNSUPPORTED, "dtype %d not supported", dt);
    }
    CF_CHECK_LAUNCH();
    return CF_OK;
}
