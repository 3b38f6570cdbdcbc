// cf_noalloc.cu -- cf_sample_noalloc: the binary32 sampler with its
// workspace in a fixed array inside the library instead of caller memory.
//
// For callers that cannot allocate device memory where they call the sampler:
// code that runs while another thread captures a CUDA graph in global capture
// mode (a cudaMalloc there is an error), and programs whose device memory is
// reserved up front by a fixed budget or another allocator.  They still pass
// the embedding and the output array; nothing here allocates device memory.
//
// The array below exists once on every device that loads this library and
// stays allocated until the process exits.  Host code must not use its name
// as an address (in host code it is only a stand-in object): the device
// address comes from cudaGetSymbolAddress, looked up once per device, with
// that device current, during the first call on the device.
#include <mutex>

#include "cf_kernels.cuh"

namespace cf {

// Largest intermediate one realization may need (see the header).
constexpr size_t kNoAllocScratchBytes = 16ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    void* scratch = nullptr;   // device address of g_noalloc_scratch
    cudaEvent_t order = nullptr;
};
static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc[64];

// One-time set-up on the current device: the scratch address and the event
// that orders successive calls.
static cf_status noalloc_setup(int dev, NoAllocDevice** out) {
    NoAllocDevice& d = g_noalloc[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(CF_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        e = cudaEventCreateWithFlags(&d.order, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(CF_ERR_CUDA, "cudaEventCreate failed: %s", cudaGetErrorString(e));
        d.scratch = p;
        d.ready = true;
    }
    *out = &d;
    return CF_OK;
}

// Defined in cf_sample.cu (shared with cf_sample).
cf_status sample_f32_into(const cf_embedding* e, uint64_t seed, uint64_t r0, int R, void* fields, void* ws,
                          size_t ws_bytes, cudaStream_t st);
size_t sample_bytes_per_realization(const cf_embedding* e, cf_dtype dt);

}  // namespace cf

using namespace cf;

extern "C" cf_status cf_sample_noalloc(const cf_embedding* e, uint64_t seed, uint64_t r0, int32_t R,
                                       void* fields_out, cf_stream_t s) {
    clear_error();
    if (!e || !fields_out) return fail(CF_ERR_ARG, "embedding and fields_out are required");
    if (R < 0) return fail(CF_ERR_ARG, "R must be >= 0");
    if (r0 + (uint64_t)R > (1ull << 32)) return fail(CF_ERR_ARG, "realization index exceeds 32 bits");
    const size_t per = sample_bytes_per_realization(e, CF_F32);
    if (per > kNoAllocScratchBytes)
        return fail(CF_ERR_UNSUPPORTED,
                    "one realization of this grid needs %zu bytes of scratch; the static scratch holds %zu bytes "
                    "(use cf_sample with a caller workspace)",
                    per, kNoAllocScratchBytes);
    if (R == 0) return CF_OK;
    const cudaStream_t st = (cudaStream_t)s;
    CF_TRY(enter_with(e, st));
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CF_ERR_UNSUPPORTED, "device index %d", dev);
    // The host lock and the device event keep successive calls from
    // overlapping on the GPU: they all share the one scratch array.
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice* d = nullptr;
    CF_TRY(noalloc_setup(dev, &d));
    CF_CUDA(cudaStreamWaitEvent(st, d->order, 0));
    const cf_status r = sample_f32_into(e, seed, r0, R, fields_out, d->scratch, kNoAllocScratchBytes, st);
    CF_CUDA(cudaEventRecord(d->order, st));
    return r;
}
