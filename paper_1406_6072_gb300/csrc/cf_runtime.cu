// cf_runtime.cu -- error state, per-device set-up (twiddle tables), grid
// validation and embedding accessors.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

#include "cf_df.cuh"
#include "cf_internal.h"

namespace cf {

static thread_local std::string g_last_error;

cf_status fail(cf_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

// Twiddle tables, one copy per device that loads the library.
__device__ C2<float> g_tw32[TWN];
__device__ C2<double> g_tw64[TWN];
__device__ C2<DF> g_twdf[TWN];
__device__ float4 g_tw32x2[TWN];  // (cos, cos, sin, sin): the paired-lines table

__global__ void k_init_twiddles(C2<float>* tw32, C2<double>* tw64, C2<DF>* twdf, float4* tw32x2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= TWN) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)TWN, &s, &c);
    tw64[j] = mk(c, s);
    tw32[j] = mk((float)c, (float)s);
    twdf[j] = mk(df_from(c), df_from(s));
    tw32x2[j] = make_float4((float)c, (float)c, (float)s, (float)s);
}

static constexpr int kMaxDevices = 64;
static std::mutex g_init_mu;
static bool g_inited[kMaxDevices];
static C2<float>* g_tw32_ptr[kMaxDevices];
static C2<double>* g_tw64_ptr[kMaxDevices];
static C2<DF>* g_twdf_ptr[kMaxDevices];
static float4* g_tw32x2_ptr[kMaxDevices];
// Library memory pool per device: stream-ordered allocations of embeddings,
// scratch and served results.  Freed blocks stay in the pool (release
// threshold: unlimited), so that repeated embeddings do not map and unmap
// device memory at every synchronisation.
static cudaMemPool_t g_pool[kMaxDevices];

static int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

cf_status ensure_device_init() {
    int dev = 0;
    CF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CF_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (g_inited[dev]) return CF_OK;
    void* p32 = nullptr;
    void* p64 = nullptr;
    void* pdf = nullptr;
    void* p32x2 = nullptr;
    CF_CUDA(cudaGetSymbolAddress(&p32x2, g_tw32x2));
    CF_CUDA(cudaGetSymbolAddress(&p32, g_tw32));
    CF_CUDA(cudaGetSymbolAddress(&p64, g_tw64));
    CF_CUDA(cudaGetSymbolAddress(&pdf, g_twdf));
    k_init_twiddles<<<(TWN + 255) / 256, 256>>>((C2<float>*)p32, (C2<double>*)p64, (C2<DF>*)pdf, (float4*)p32x2);
    CF_CHECK_LAUNCH();
    CF_CUDA(cudaDeviceSynchronize());
    g_tw32_ptr[dev] = (C2<float>*)p32;
    g_tw64_ptr[dev] = (C2<double>*)p64;
    g_twdf_ptr[dev] = (C2<DF>*)pdf;
    g_tw32x2_ptr[dev] = (float4*)p32x2;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    CF_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
    uint64_t keep = ~0ull;
    CF_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    g_inited[dev] = true;
    return CF_OK;
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
    return cudaMallocFromPoolAsync(p, bytes, g_pool[current_device()], s);
}

// ---------------------------------------------------------------- read-back
namespace {
constexpr int kSlots = 64;
constexpr size_t kSlotBytes = 256;
std::mutex g_slot_mu;
unsigned char* g_slots = nullptr;  // kSlots * kSlotBytes, pinned, mapped, portable
bool g_slot_used[kSlots];

__global__ void k_store_bytes(const unsigned long long* __restrict__ src, unsigned long long* dst, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

int slot_acquire() {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    if (!g_slots && cudaHostAlloc((void**)&g_slots, kSlots * kSlotBytes,
                                  cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        g_slots = nullptr;
        cudaGetLastError();
        return -1;
    }
    for (int i = 0; i < kSlots; ++i)
        if (!g_slot_used[i]) {
            g_slot_used[i] = true;
            return i;
        }
    return -1;
}

void slot_release(int i) {
    std::lock_guard<std::mutex> lk(g_slot_mu);
    g_slot_used[i] = false;
}
}  // namespace

cf_status read_back(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    const int words = (int)((bytes + 7) / 8);
    const int i = bytes <= kSlotBytes && ((uintptr_t)src & 7) == 0 ? slot_acquire() : -1;
    if (i < 0) {  // no slot free: an ordinary copy
        CF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        CF_CUDA(cudaStreamSynchronize(s));
        return CF_OK;
    }
    unsigned char* host = g_slots + (size_t)i * kSlotBytes;
    void* dev = nullptr;
    cudaError_t e = cudaHostGetDevicePointer(&dev, host, 0);
    if (e == cudaSuccess) {
        k_store_bytes<<<1, 32, 0, s>>>((const unsigned long long*)src, (unsigned long long*)dev, words);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) memcpy(dst, host, bytes);
    slot_release(i);
    if (e != cudaSuccess) return fail(CF_ERR_CUDA, "read-back: %s", cudaGetErrorString(e));
    return CF_OK;
}

bool sync_check_enabled() {
    static const bool on = [] {
        const char* e = getenv("CF_SYNC_CHECK");
        return e && e[0] == '1';
    }();
    return on;
}

cf_status enter(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return ensure_device_init();  // a capturing stream may not be queried; it is the current device's
    if (s) {
        int dev = -1;
        cudaError_t e = cudaStreamGetDevice(s, &dev);
        if (e != cudaSuccess) return fail(CF_ERR_CUDA, "cudaStreamGetDevice: %s", cudaGetErrorString(e));
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != dev) CF_CUDA(cudaSetDevice(dev));
    }
    return ensure_device_init();
}

cf_status enter_with(const cf_embedding* e, cudaStream_t s) {
    CF_TRY(enter(s));
    int cur = -1;
    CF_CUDA(cudaGetDevice(&cur));
    if (e->device != cur)
        return fail(CF_ERR_ARG, "the embedding was built on device %d but the stream belongs to device %d", e->device,
                    cur);
    return CF_OK;
}

const C2<float>* twiddles_f32() { return g_tw32_ptr[current_device()]; }
const C2<double>* twiddles_f64() { return g_tw64_ptr[current_device()]; }
const C2<DF>* twiddles_df() { return g_twdf_ptr[current_device()]; }
const float4* twiddles_f32x2() { return g_tw32x2_ptr[current_device()]; }

cf_status check_grid(const cf_grid* g, GridInfo* gi) {
    if (!g) return fail(CF_ERR_ARG, "grid is NULL");
    if (g->ndim < 1 || g->ndim > 3) return fail(CF_ERR_ARG, "ndim must be 1, 2 or 3 (got %d)", g->ndim);
    const int p = g->embed_factor == 0 ? 2 : g->embed_factor;
    if (p != 2 && p != 4 && p != 8) return fail(CF_ERR_ARG, "embed_factor must be 0, 2, 4 or 8 (got %d)", p);
    gi->ndim = g->ndim;
    gi->factor = p;
    gi->ncell = 1;
    gi->mtotal = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < g->ndim) {
            const long long n = (long long)g->n[a];
            if (n < 1) return fail(CF_ERR_ARG, "n[%d] = %lld must be >= 1", a, n);
            long long m = 1;  // the smallest power of two >= p n
            while (m < p * n && m <= kMaxLine) m <<= 1;
            if (m > kMaxLine)
                return fail(CF_ERR_UNSUPPORTED, "embedding size for n[%d] = %lld at factor %d exceeds %lld", a, n,
                            p, kMaxLine);
            const double c = g->cell[a];
            if (!(c > 0.0)) return fail(CF_ERR_ARG, "cell[%d] must be > 0", a);
            gi->n[a] = n;
            gi->m[a] = m;
            gi->cell[a] = c;
            gi->ncell *= n;
            gi->mtotal *= m;
        } else {
            gi->n[a] = 1;
            gi->m[a] = 1;
            gi->cell[a] = 1.0;
        }
    }
    return CF_OK;
}

}  // namespace cf

using namespace cf;

extern "C" const char* cf_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* cf_version(void) { return "cf 0.1 (sm_103a)"; }

namespace cf {

// One non-blocking stream per device on which embeddings are released.
static cudaStream_t g_free_stream[kMaxDevices];
static std::mutex g_free_mu;

void record_use(cf_embedding* e, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(e->mu);
    for (auto& u : e->uses) {
        if (u.first == s) {
            cudaEventRecord(u.second, s);
            return;
        }
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
    cudaEventRecord(ev, s);
    e->uses.emplace_back(s, ev);
}

__global__ void k_s64(const double* __restrict__ lam, double tau, double inv_total, double* __restrict__ s64,
                      long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = lam[i];
        s64[i] = l > tau ? sqrt(l * inv_total) : 0.0;
    }
}

cf_status ensure_s64(cf_embedding* e, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->s64) {
        CF_CUDA(cudaStreamWaitEvent(s, e->s64_ready, 0));
        return CF_OK;
    }
    const long long total = e->grid.mtotal;
    double* p = nullptr;
    if (pool_malloc((void**)&p, sizeof(double) * total, s) != cudaSuccess)
        return fail(CF_ERR_NOMEM, "device allocation of the binary64 amplitudes failed");
    const int blocks = (int)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256);
    k_s64<<<blocks, 256, 0, s>>>(e->lambda, e->tau, 1.0 / (double)total, p, total);
    CF_CHECK_LAUNCH();
    CF_CUDA(cudaEventCreateWithFlags(&e->s64_ready, cudaEventDisableTiming));
    CF_CUDA(cudaEventRecord(e->s64_ready, s));
    e->s64 = p;
    return CF_OK;
}

// sum of s^2 over the embedding: per-block partial sums, then one block
__global__ void __launch_bounds__(256) k_sumsq_partial(const float* __restrict__ s, long long total,
                                                       double* __restrict__ part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < total; i += (long long)gridDim.x * 256)
        acc += (double)s[i] * (double)s[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) k_sumsq_final(const double* __restrict__ part, int n, double* out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

cf_status ensure_sumsq(cf_embedding* e, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->sumsq) {
        CF_CUDA(cudaStreamWaitEvent(s, e->sumsq_ready, 0));
        return CF_OK;
    }
    constexpr int kParts = 1024;
    double* p = nullptr;
    if (pool_malloc((void**)&p, sizeof(double) * (kParts + 1), s) != cudaSuccess)
        return fail(CF_ERR_NOMEM, "device allocation of the amplitude sum failed");
    k_sumsq_partial<<<kParts, 256, 0, s>>>(e->s32, e->grid.mtotal, p + 1);
    k_sumsq_final<<<1, 256, 0, s>>>(p + 1, kParts, p);
    CF_CHECK_LAUNCH();
    CF_CUDA(cudaEventCreateWithFlags(&e->sumsq_ready, cudaEventDisableTiming));
    CF_CUDA(cudaEventRecord(e->sumsq_ready, s));
    e->sumsq = p;
    return CF_OK;
}

}  // namespace cf

// Stream-ordered release: a library-owned stream waits for the last recorded
// use on every stream, then frees; no host-side wait.
extern "C" cf_status cf_embedding_free(cf_embedding* e) {
    if (!e) return CF_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e->device);
    cudaStream_t fs = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_free_mu);
        if (!g_free_stream[e->device]) cudaStreamCreateWithFlags(&g_free_stream[e->device], cudaStreamNonBlocking);
        fs = g_free_stream[e->device];
    }
    {
        std::lock_guard<std::mutex> lk(e->mu);
        for (auto& u : e->uses) {
            cudaStreamWaitEvent(fs, u.second, 0);
            cudaEventDestroy(u.second);
        }
        e->uses.clear();
    }
    if (e->lambda) cudaFreeAsync(e->lambda, fs);
    if (e->s64) cudaFreeAsync(e->s64, fs);
    if (e->sumsq) cudaFreeAsync(e->sumsq, fs);
    if (e->s64_ready) cudaEventDestroy(e->s64_ready);
    if (e->sumsq_ready) cudaEventDestroy(e->sumsq_ready);
    if (e->s32) cudaFreeAsync(e->s32, fs);
    cudaSetDevice(prev);
    delete e;
    return CF_OK;
}

extern "C" cf_status cf_embedding_lambda(const cf_embedding* e, double* dst, cf_stream_t s) {
    if (!e || !dst) return fail(CF_ERR_ARG, "NULL argument");
    CF_CUDA(cudaMemcpyAsync(dst, e->lambda, sizeof(double) * (size_t)e->grid.mtotal,
                            cudaMemcpyDeviceToDevice, (cudaStream_t)s));
    record_use(const_cast<cf_embedding*>(e), (cudaStream_t)s);
    return CF_OK;
}

__global__ void k_sqrt_lambda_plus(const double* __restrict__ lam, double tau, double* __restrict__ dst,
                                   long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = lam[i];
        dst[i] = l > tau ? sqrt(l) : 0.0;
    }
}

extern "C" cf_status cf_embedding_sqrt_lambda(const cf_embedding* e, double* dst, cf_stream_t s) {
    if (!e || !dst) return fail(CF_ERR_ARG, "NULL argument");
    const long long total = e->grid.mtotal;
    const int blocks = (int)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256);
    k_sqrt_lambda_plus<<<blocks, 256, 0, (cudaStream_t)s>>>(e->lambda, e->tau, dst, total);
    CF_CHECK_LAUNCH();
    record_use(const_cast<cf_embedding*>(e), (cudaStream_t)s);
    return CF_OK;
}

extern "C" cf_status cf_embedding_info(const cf_embedding* e, cf_grid* g, cf_embed_report* rep) {
    if (!e) return fail(CF_ERR_ARG, "NULL embedding");
    if (g) {
        g->ndim = e->grid.ndim;
        g->embed_factor = e->grid.factor;
        for (int a = 0; a < 3; ++a) {
            g->n[a] = e->grid.n[a];
            g->cell[a] = e->grid.cell[a];
        }
    }
    if (rep) *rep = e->report;
    return CF_OK;
}

// ----------------------------------------------------------------- kernel timing
#include <map>
#include <vector>

namespace cf {
namespace {
struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;
std::map<std::string, std::pair<long long, double>> g_acc;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

ScopedKernelTimer::ScopedKernelTimer(cudaStream_t s, const char* name, long long variant) : s_(s) {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;  // graph capture
    if (variant >= 0)
        snprintf(name_, sizeof name_, "%s<%lld>", name, variant);
    else
        snprintf(name_, sizeof name_, "%s", name);
    a_ = take_event();
    b_ = take_event();
    cudaEventRecord(a_, s_);
}

ScopedKernelTimer::~ScopedKernelTimer() {
    if (!a_) return;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(g_tmu);
    g_pending.push_back({name_, a_, b_});
}

static void drain_pending() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& acc = g_acc[p.name];
        acc.first += 1;
        acc.second += ms;
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace cf

extern "C" cf_status cf_kernel_timing(int32_t enable) {
    std::lock_guard<std::mutex> lk(cf::g_tmu);
    cf::drain_pending();
    if (enable) cf::g_acc.clear();
    cf::g_timing = enable != 0;
    return CF_OK;
}

extern "C" cf_status cf_kernel_timing_read(char* json, size_t cap, size_t* needed) {
    std::lock_guard<std::mutex> lk(cf::g_tmu);
    cf::drain_pending();
    std::string out = "{";
    bool first = true;
    for (auto& kv : cf::g_acc) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
                 kv.second.second);
        out += buf;
        first = false;
    }
    out += "}";
    if (needed) *needed = out.size() + 1;
    if (json && cap > 0) {
        size_t n = out.size() < cap - 1 ? out.size() : cap - 1;
        memcpy(json, out.data(), n);
        json[n] = 0;
    }
    return CF_OK;
}
