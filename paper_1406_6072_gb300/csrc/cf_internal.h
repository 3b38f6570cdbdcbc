// cf_internal.h -- host-side declarations shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/cf.h"
#include "cf_device.cuh"

namespace cf {

// thread-local error message; returns st for tail calls
cf_status fail(cf_status st, const char* fmt, ...);
void clear_error();

#define CF_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::cf::fail(CF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// After a launch: reports launch errors; with CF_SYNC_CHECK=1 in the
// environment also waits for the device and reports execution errors at the
// launch that caused them (a debugging aid; off by default).
#define CF_CHECK_LAUNCH()                                                                  \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ == cudaSuccess && ::cf::sync_check_enabled()) e_ = cudaDeviceSynchronize(); \
        if (e_ != cudaSuccess)                                                             \
            return ::cf::fail(CF_ERR_CUDA, "kernel launch failed at %s:%d: %s", __FILE__,  \
                              __LINE__, cudaGetErrorString(e_));                           \
    } while (0)

#define CF_TRY(expr)                       \
    do {                                   \
        cf_status st_ = (expr);            \
        if (st_ != CF_OK) return st_;      \
    } while (0)

bool sync_check_enabled();

// One-time per-device set-up (twiddle tables).  Synchronises the device the
// first time it runs on a device.
cf_status ensure_device_init();
// Stream-ordered allocation from the library's pool on the current device
// (release with cudaFreeAsync).
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);

// Small results the host waits for (the embedding statistics) are stored by a
// kernel into pinned, device-mapped host memory: the wait then ends when the
// kernel does, instead of queueing its read-back behind bulk transfers on a
// copy engine.  read_back() copies `bytes` (<= 256) from device memory `src`
// into `dst` on the host, synchronising stream s.
cf_status read_back(void* dst, const void* src, size_t bytes, cudaStream_t s);
// Mean over rows and unbiased covariance (1/(nrows-1)) of x [nrows][ncols]; either output may be null.
cf_status launch_mean_cov(const double* x, long long nrows, int ncols, double* mean, double* cov, cudaStream_t s);
// Entry-point prologue: makes the device of stream s current (the legacy
// default stream keeps the current device) and runs the one-time set-up.
cf_status enter(cudaStream_t s);
// enter(s), then refuses an embedding that lives on another device than the
// stream's (its arrays would be another GPU's memory to the kernels).
cf_status enter_with(const cf_embedding* e, cudaStream_t s);
const C2<float>* twiddles_f32();   // current device, TWN entries exp(+2 pi i j/TWN)
const C2<double>* twiddles_f64();
const float4* twiddles_f32x2();    // current device, (cos, cos, sin, sin) of the same angles

inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
inline int log2i(long long v) {
    int r = 0;
    while ((1ll << r) < v) ++r;
    return r;
}

constexpr long long kMaxLine = 4096;  // longest supported transform line

// Per-launch CUDA-event timing (see cf_kernel_timing).  Constructed right
// before a launch and destroyed right after it on the same stream.
class ScopedKernelTimer {
  public:
    ScopedKernelTimer(cudaStream_t s, const char* name, long long variant = -1);
    ~ScopedKernelTimer();
    ScopedKernelTimer(const ScopedKernelTimer&) = delete;
    ScopedKernelTimer& operator=(const ScopedKernelTimer&) = delete;

  private:
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    char name_[96];
};

// Validates a survey grid for the sampler; fills M and totals.
struct GridInfo {
    int ndim;
    int factor;        // embedded side / survey side (M = factor * n per axis)
    long long n[3];
    long long m[3];
    double cell[3];
    long long ncell;   // prod n
    long long mtotal;  // prod m
};
cf_status check_grid(const cf_grid* g, GridInfo* gi);

}  // namespace cf

struct cf_embedding {
    cf::GridInfo grid;
    double* lambda = nullptr;    // raw eigenvalues [mtotal]
    double* s64 = nullptr;       // sqrt(lambda+ / mtotal) [mtotal], built on first binary64 use
    float* s32 = nullptr;        // sqrt(lambda+ / mtotal) in binary32 [mtotal]
    double* sumsq = nullptr;     // sum of s32^2 (tensor-core input scaling), built on first use
    cudaEvent_t s64_ready = nullptr, sumsq_ready = nullptr;  // completion of the lazy builds
    double tau = 0.0;
    cf_embed_report report{};
    int device = 0;
    cudaStream_t alloc_stream = nullptr;
    std::mutex mu;                                           // guards s64 and uses
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;  // last use per stream
};

namespace cf {
// Records that work enqueued on stream s reads embedding e (the free waits for it).
void record_use(cf_embedding* e, cudaStream_t s);
// Builds e->s64 (on stream s) if it does not exist yet; s waits for the build.
cf_status ensure_s64(cf_embedding* e, cudaStream_t s);
// Builds e->sumsq (on stream s) if it does not exist yet; s waits for the build.
cf_status ensure_sumsq(cf_embedding* e, cudaStream_t s);
}  // namespace cf
