// cf_plan.cu -- the per-realization path of one embedding recorded once as a
// CUDA graph and replayed: a small kernel advances the device-side
// realization counter and writes the per-realization descriptors, then the
// descriptor-driven binary32 sampler (noise, transforms, field split and the
// optional lognormal + Poisson step) and the optional power spectra of the
// fields and of the count maps with their mean and covariance.  Replays
// need no host work beyond one graph launch, and no realization is drawn
// twice: launch k draws [r0 + kR, r0 + (k+1)R).
#include "cf_kernels.cuh"

namespace cf {
cf_status sample_batch_f32(const GridInfo& g, const RealDesc* desc, int nreal, void* ws, size_t ws_bytes,
                           cudaStream_t st);
size_t sample_chunk_bytes(const GridInfo& g, int nreal);
}  // namespace cf

using namespace cf;

struct cf_plan {
    int device = 0;
    int R = 0;
    GridInfo g{};
    const cf_embedding* e = nullptr;
    RealDesc* desc = nullptr;             // [R] device descriptors
    unsigned long long* ctr = nullptr;    // device: next realization index
    void* ws = nullptr;                   // sampler intermediates
    size_t ws_bytes = 0;
    void* pk_ws = nullptr;
    size_t pk_ws_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// desc[i].r = counter + i for the R realizations of this launch; counter += R.
__global__ void k_plan_advance(RealDesc* __restrict__ desc, int R, unsigned long long* __restrict__ ctr) {
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = *ctr;
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) desc[i].r = (uint32_t)(base + (unsigned long long)i);
    __syncthreads();
    if (threadIdx.x == 0) *ctr = base + (unsigned long long)R;
}

void plan_release(cf_plan* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->desc) cudaFree(p->desc);
    if (p->ctr) cudaFree(p->ctr);
    if (p->ws) cudaFree(p->ws);
    if (p->pk_ws) cudaFree(p->pk_ws);
    delete p;
}

struct PlanArgs {
    const cf_lp_params* lp;
    const cf_bins* bins;
    float* fields;
    double *pk, *mean, *cov, *pkc, *meanc, *covc;
    int64_t* nmodes;
};

// The work of one launch, enqueued on st (eagerly, or while st captures).
cf_status plan_body(cf_plan* p, const PlanArgs& a, cudaStream_t st) {
    k_plan_advance<<<1, 256, 0, st>>>(p->desc, p->R, p->ctr);
    CF_CHECK_LAUNCH();
    CF_TRY(sample_batch_f32(p->g, p->desc, p->R, p->ws, p->ws_bytes, st));
    if (a.bins) {
        cf_grid grid{};
        grid.ndim = p->g.ndim;
        for (int d = 0; d < p->g.ndim; ++d) {
            grid.n[d] = p->g.n[d];
            grid.cell[d] = p->g.cell[d];
        }
        const int64_t F = 2 * (int64_t)p->R;
        CF_TRY(cf_power_spectrum(a.fields, CF_F32, &grid, F, a.bins, a.pk, a.nmodes, a.mean, a.cov, p->pk_ws,
                                 p->pk_ws_bytes, (cf_stream_t)st));
        if (a.lp && a.pkc)
            CF_TRY(cf_power_spectrum_counts(a.lp->counts_out, nullptr, &grid, F, a.bins, a.pkc, a.nmodes, a.meanc,
                                            a.covc, p->pk_ws, p->pk_ws_bytes, (cf_stream_t)st));
    }
    return CF_OK;
}

}  // namespace

extern "C" cf_status cf_plan_create(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R,
                                    const cf_lp_params* lp, const cf_bins* bins, float* fields_out, double* pk_out,
                                    int64_t* nmodes_out, double* mean_or_null, double* cov_or_null,
                                    double* pk_counts_out, double* mean_counts_or_null, double* cov_counts_or_null,
                                    cf_stream_t s, cf_plan** out) {
    clear_error();
    if (!out) return fail(CF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!e || !fields_out) return fail(CF_ERR_ARG, "embedding and fields_out are required");
    if (R < 1) return fail(CF_ERR_ARG, "R must be >= 1");
    if (r0 > (1ull << 32)) return fail(CF_ERR_ARG, "realization index exceeds 32 bits");
    if (lp && (!lp->counts_out || lp->f || lp->delta_out))
        return fail(CF_ERR_UNSUPPORTED, "plans take counts_out only (no mask, no delta output)");
    if (bins && (!pk_out || !nmodes_out)) return fail(CF_ERR_ARG, "bins need pk_out and nmodes_out");
    if (pk_counts_out && !(bins && lp)) return fail(CF_ERR_ARG, "pk_counts_out needs bins and lp");
    CF_TRY(enter_with(e, (cudaStream_t)s));
    const cudaStream_t st = (cudaStream_t)s;
    cf_plan* p = new cf_plan();
    auto bail = [&](cf_status code) {
        plan_release(p);
        return code;
    };
#define PLAN_CUDA(call)                                                                    \
    do {                                                                                   \
        const cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return bail(fail(CF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)
    PLAN_CUDA(cudaGetDevice(&p->device));
    p->R = R;
    p->g = e->grid;
    p->e = e;
    // descriptors: every field but the realization index is fixed
    std::vector<RealDesc> hd((size_t)R);
    const long long cells = p->g.ncell;
    for (int i = 0; i < R; ++i) {
        RealDesc& d = hd[(size_t)i];
        d = RealDesc{};
        d.s = e->s32;
        d.fields = fields_out + (size_t)i * 2 * (size_t)cells;
        d.counts = lp ? lp->counts_out + (size_t)i * 2 * (size_t)cells : nullptr;
        d.half_sigma2 = lp ? 0.5 * lp->sigma2 : 0.0;
        d.nbar = lp ? lp->nbar : 0.0;
        d.amp_scale = 1.0f;
        d.half_sigma2_f = lp ? (float)(0.5 * lp->sigma2) : 0.0f;
        d.nbar_f = lp ? (float)lp->nbar : 0.0f;
        d.r = 0;
        d.key0 = (uint32_t)seed;
        d.key1 = (uint32_t)(seed >> 32);
        d.pkey0 = lp ? (uint32_t)lp->seed : 0u;
        d.pkey1 = lp ? (uint32_t)(lp->seed >> 32) : 0u;
    }
    if (cudaMalloc((void**)&p->desc, sizeof(RealDesc) * (size_t)R) != cudaSuccess ||
        cudaMalloc((void**)&p->ctr, sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(CF_ERR_NOMEM, "plan allocation failed"));
    p->ws_bytes = sample_chunk_bytes(p->g, R);
    if (p->ws_bytes && cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess)
        return bail(fail(CF_ERR_NOMEM, "plan workspace allocation failed"));
    if (bins) {
        cf_grid grid{};
        grid.ndim = p->g.ndim;
        for (int d = 0; d < p->g.ndim; ++d) {
            grid.n[d] = p->g.n[d];
            grid.cell[d] = p->g.cell[d];
        }
        cf_status stt = cf_power_spectrum_workspace_size(&grid, 2 * (int64_t)R, bins, CF_F32, &p->pk_ws_bytes);
        if (stt != CF_OK) return bail(stt);
        if (cudaMalloc(&p->pk_ws, p->pk_ws_bytes) != cudaSuccess)
            return bail(fail(CF_ERR_NOMEM, "plan power-spectrum workspace allocation failed"));
    }
    PLAN_CUDA(cudaMemcpyAsync(p->desc, hd.data(), sizeof(RealDesc) * (size_t)R, cudaMemcpyHostToDevice, st));
    const PlanArgs a{lp, bins, fields_out, pk_out, mean_or_null, cov_or_null, pk_counts_out, mean_counts_or_null,
                     cov_counts_or_null, nmodes_out};
    // one eager pass fills the library's caches (bin tables), so that the
    // captured pass performs launches only; then the counter is set to r0
    {
        const unsigned long long zero = 0;
        PLAN_CUDA(cudaMemcpyAsync(p->ctr, &zero, sizeof zero, cudaMemcpyHostToDevice, st));
        cf_status stt = plan_body(p, a, st);
        if (stt != CF_OK) return bail(stt);
        PLAN_CUDA(cudaStreamSynchronize(st));
    }
    cudaStream_t cap = nullptr;
    PLAN_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    {
        const cudaError_t eb = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (eb != cudaSuccess) {
            cudaStreamDestroy(cap);
            return bail(fail(CF_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(eb)));
        }
    }
    const cf_status body = plan_body(p, a, cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (body != CF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return bail(body);
    }
    if (ec != cudaSuccess) return bail(fail(CF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec)));
    p->graph = graph;
    if (cudaGraphInstantiate(&p->exec, graph, 0) != cudaSuccess)
        return bail(fail(CF_ERR_CUDA, "graph instantiation failed"));
    const unsigned long long start = r0;
    PLAN_CUDA(cudaMemcpy(p->ctr, &start, sizeof start, cudaMemcpyHostToDevice));
    *out = p;
    return CF_OK;
#undef PLAN_CUDA
}

extern "C" cf_status cf_plan_launch(cf_plan* p, cf_stream_t s) {
    clear_error();
    if (!p) return fail(CF_ERR_ARG, "plan is NULL");
    CF_TRY(enter((cudaStream_t)s));
    ScopedKernelTimer kt((cudaStream_t)s, "plan_launch");
    CF_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)s));
    record_use(const_cast<cf_embedding*>(p->e), (cudaStream_t)s);
    return CF_OK;
}

extern "C" cf_status cf_plan_seek(cf_plan* p, uint64_t r0, cf_stream_t s) {
    clear_error();
    if (!p) return fail(CF_ERR_ARG, "plan is NULL");
    if (r0 > (1ull << 32)) return fail(CF_ERR_ARG, "realization index exceeds 32 bits");
    CF_TRY(enter((cudaStream_t)s));
    // the value is copied from the host before the call returns (pageable source)
    const unsigned long long v = r0;
    CF_CUDA(cudaMemcpyAsync(p->ctr, &v, sizeof v, cudaMemcpyHostToDevice, (cudaStream_t)s));
    CF_CUDA(cudaStreamSynchronize((cudaStream_t)s));
    return CF_OK;
}

extern "C" cf_status cf_plan_destroy(cf_plan* p) {
    if (!p) return CF_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    plan_release(p);
    return CF_OK;
}
