// cf_serve.cu -- CUDA backend of the serving loop and its C ABI.
//
// Each slot is one stream with its own descriptor staging buffers and
// completion event; embeddings are built (by the scheduler's embedding
// thread) on a stream of the highest priority.  A batch is one chunked, descriptor-driven sampler launch
// (cf_sample.cu: sample_batch_f32) covering the realizations of all its
// requests, followed by the optional host copies; results stay in
// stream-ordered device allocations until the client releases them.
#include <math.h>

#include <memory>

#include "cf_kernels.cuh"
#include "cf_serve_core.h"

namespace cf {
cf_status sample_batch_f32(const GridInfo& g, const RealDesc* desc, int nreal, void* ws, size_t ws_bytes,
                           cudaStream_t st);
size_t sample_chunk_bytes(const GridInfo& g, int nreal);
}  // namespace cf

using namespace cf;

namespace {

struct CudaSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    RealDesc* host_desc = nullptr;   // pinned staging
    RealDesc* dev_desc = nullptr;
    void* ws = nullptr;
    int capacity = 0;
};

class CudaBackend : public cfserve::Backend {
  public:
    // nslots streams; with `priority_last`, the last one (the slot reserved
    // for small requests) has the highest priority
    CudaBackend(int device, int nslots, int max_real, bool priority_last)
        : device_(device), max_real_(max_real) {
        cudaSetDevice(device_);
        // spectra are built on the highest-priority stream: a request that
        // waits for its embedding then does not also wait for the blocks of
        // large batches already queued on the device
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        ok_ = cudaStreamCreateWithPriority(&embed_stream_, cudaStreamNonBlocking, greatest) == cudaSuccess;
        slots_.resize(nslots);
        for (int i = 0; i < nslots; ++i) {
            CudaSlot& s = slots_[i];
            const int prio = (priority_last && i == nslots - 1) ? greatest : least;
            ok_ = ok_ && cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio) == cudaSuccess;
            ok_ = ok_ && cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess;
            ok_ = ok_ && cudaMallocHost((void**)&s.host_desc, sizeof(RealDesc) * (size_t)max_real) == cudaSuccess;
            ok_ = ok_ && cudaMalloc((void**)&s.dev_desc, sizeof(RealDesc) * (size_t)max_real) == cudaSuccess;
            s.capacity = max_real;
        }
    }

    // every stream, event and descriptor buffer was created
    bool ok() const { return ok_; }

    ~CudaBackend() override {
        cudaSetDevice(device_);
        cudaDeviceSynchronize();
        for (auto& s : slots_) {
            if (s.ws) cudaFree(s.ws);
            if (s.dev_desc) cudaFree(s.dev_desc);
            if (s.host_desc) cudaFreeHost(s.host_desc);
            if (s.done) cudaEventDestroy(s.done);
            if (s.stream) cudaStreamDestroy(s.stream);
        }
        if (embed_stream_) cudaStreamDestroy(embed_stream_);
    }

    static GridInfo grid_of(const cf_request& r) {
        GridInfo g{};
        check_grid(&r.grid, &g);
        return g;
    }

    size_t embed_bytes(const cf_request& r) override {
        const GridInfo g = grid_of(r);
        // kept: lambda (8 B) + binary32 amplitudes (4 B); transient scratch while built: 24 B
        return (size_t)g.mtotal * (8 + 4 + 24);
    }

    cf_status embed(const cf_request& r, void** handle, cf_embed_report* rep) override {
        cudaSetDevice(device_);
        cf_embedding* e = nullptr;
        const cf_status st = cf_embed(&r.grid, &r.xi, r.embed_flags, (cf_stream_t)embed_stream_, &e, rep);
        *handle = e;
        return st;
    }

    void free_embedding(void* h) override { cf_embedding_free((cf_embedding*)h); }

    size_t result_bytes(const cf_request& r) override {
        const GridInfo g = grid_of(r);
        const size_t cells = (size_t)g.ncell * 2 * (size_t)r.R;
        return cells * sizeof(float) + (r.want_counts ? cells * sizeof(int32_t) : 0);
    }

    size_t batch_bytes(const std::vector<cfserve::Job*>& jobs) override {
        int n = 0;
        for (auto* j : jobs) n += j->req.R;
        return sample_chunk_bytes(grid_of(jobs[0]->req), n);
    }

    cf_status alloc_result(int slot, cfserve::Job* j) override {
        cudaSetDevice(device_);
        const GridInfo g = grid_of(j->req);
        const size_t cells = (size_t)g.ncell * 2 * (size_t)j->req.R;
        cudaStream_t s = slots_[slot].stream;
        if (pool_malloc(&j->dev_fields, cells * sizeof(float), s) != cudaSuccess)
            return fail(CF_ERR_NOMEM, "result allocation failed");
        if (j->req.want_counts && pool_malloc(&j->dev_counts, cells * sizeof(int32_t), s) != cudaSuccess)
            return fail(CF_ERR_NOMEM, "result allocation failed");
        result_stream_[j] = s;
        return CF_OK;
    }

    void free_result(cfserve::Job* j) override {
        cudaSetDevice(device_);
        cudaStream_t s = slots_[0].stream;
        auto it = result_stream_.find(j);
        if (it != result_stream_.end()) {
            s = it->second;
            result_stream_.erase(it);
        }
        if (j->dev_fields) cudaFreeAsync(j->dev_fields, s);
        if (j->dev_counts) cudaFreeAsync(j->dev_counts, s);
        j->dev_fields = nullptr;
        j->dev_counts = nullptr;
    }

    cf_status launch(int slot, const std::vector<cfserve::Job*>& jobs) override {
        cudaSetDevice(device_);
        CudaSlot& sl = slots_[slot];
        const GridInfo g = grid_of(jobs[0]->req);
        int n = 0;
        for (auto* j : jobs) n += j->req.R;
        if (n > sl.capacity) return fail(CF_ERR_ARG, "batch larger than the descriptor capacity");
        // the previous batch of this slot has finished (retired), so the
        // staging buffer is free
        int k = 0;
        for (auto* j : jobs) {
            const cf_embedding* e = (const cf_embedding*)j->emb->handle;
            const cf_request& r = j->req;
            for (int i = 0; i < r.R; ++i, ++k) {
                RealDesc& d = sl.host_desc[k];
                d.s = e->s32;
                d.fields = (float*)j->dev_fields + (size_t)i * 2 * (size_t)g.ncell;
                d.counts = r.want_counts ? (int32_t*)j->dev_counts + (size_t)i * 2 * (size_t)g.ncell : nullptr;
                d.half_sigma2 = 0.5 * r.sigma2;
                d.nbar = r.nbar;
                d.amp_scale = (float)sqrt(r.xi.amp);
                d.half_sigma2_f = (float)(0.5 * r.sigma2);
                d.nbar_f = (float)r.nbar;
                d.r = (uint32_t)(r.r0 + (uint64_t)i);
                d.key0 = (uint32_t)r.seed;
                d.key1 = (uint32_t)(r.seed >> 32);
                d.pkey0 = (uint32_t)r.lp_seed;
                d.pkey1 = (uint32_t)(r.lp_seed >> 32);
            }
        }
        CF_CUDA(cudaMemcpyAsync(sl.dev_desc, sl.host_desc, sizeof(RealDesc) * (size_t)n, cudaMemcpyHostToDevice,
                                sl.stream));
        const size_t wsb = sample_chunk_bytes(g, n);
        if (wsb && pool_malloc(&sl.ws, wsb, sl.stream) != cudaSuccess)
            return fail(CF_ERR_NOMEM, "batch workspace allocation failed");
        CF_TRY(sample_batch_f32(g, sl.dev_desc, n, sl.ws, wsb, sl.stream));
        for (auto* j : jobs) {
            const size_t cells = (size_t)g.ncell * 2 * (size_t)j->req.R;
            if (j->req.host_fields)
                CF_CUDA(cudaMemcpyAsync(j->req.host_fields, j->dev_fields, cells * sizeof(float),
                                        cudaMemcpyDeviceToHost, sl.stream));
            if (j->req.want_counts && j->req.host_counts)
                CF_CUDA(cudaMemcpyAsync(j->req.host_counts, j->dev_counts, cells * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, sl.stream));
            // the embedding is read by this stream's work
            record_use((cf_embedding*)j->emb->handle, sl.stream);
        }
        CF_CUDA(cudaEventRecord(sl.done, sl.stream));
        return CF_OK;
    }

    bool done(int slot) override {
        cudaSetDevice(device_);
        return cudaEventQuery(slots_[slot].done) == cudaSuccess;
    }

    void finish(int slot) override {
        CudaSlot& sl = slots_[slot];
        if (sl.ws) {
            cudaFreeAsync(sl.ws, sl.stream);
            sl.ws = nullptr;
        }
    }

  private:
    int device_;
    int max_real_;
    bool ok_ = false;
    cudaStream_t embed_stream_ = nullptr;
    std::vector<CudaSlot> slots_;
    std::map<cfserve::Job*, cudaStream_t> result_stream_;
};

}  // namespace

struct cf_server {
    std::unique_ptr<CudaBackend> backend;
    std::unique_ptr<cfserve::Scheduler> sched;
};

extern "C" cf_status cf_serve_create(const cf_serve_cfg* cfg, cf_server** out) {
    clear_error();
    if (!cfg || !out) return fail(CF_ERR_ARG, "cfg and out are required");
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->queue_capacity < 1 || cfg->cache_entries < 1 ||
        cfg->max_batch_realizations < 1 || cfg->hbm_budget == 0 || cfg->small_request_cells < 0)
        return fail(CF_ERR_ARG, "cfg fields must be positive");
    int ndev = 0;
    CF_CUDA(cudaGetDeviceCount(&ndev));
    if (cfg->device < 0 || cfg->device >= ndev) return fail(CF_ERR_ARG, "device %d does not exist", cfg->device);
    CF_CUDA(cudaSetDevice(cfg->device));
    CF_TRY(ensure_device_init());
    cf_server* sv = new cf_server();
    const bool reserved = cfg->small_request_cells > 0;
    sv->backend.reset(new CudaBackend(cfg->device, cfg->max_inflight + (reserved ? 1 : 0),
                                      cfg->max_batch_realizations, reserved));
    if (!sv->backend->ok()) {
        delete sv;
        cudaGetLastError();
        return fail(CF_ERR_NOMEM, "serving streams or descriptor buffers could not be created");
    }
    sv->sched.reset(new cfserve::Scheduler(*cfg, sv->backend.get()));
    *out = sv;
    return CF_OK;
}

extern "C" cf_status cf_serve_submit(cf_server* sv, const cf_request* req, uint64_t* ticket) {
    if (!sv || !req || !ticket) return fail(CF_ERR_ARG, "NULL argument");
    GridInfo g;
    CF_TRY(check_grid(&req->grid, &g));
    const cf_status st = sv->sched->submit(*req, ticket);
    if (st == CF_ERR_ARG)
        return fail(st, "invalid request (1 <= R <= max_batch_realizations, amp > 0, scale > 0, parametric xi "
                        "required, no CF_EMBED_LOG1P)");
    if (st == CF_ERR_BUSY) return fail(st, "queue full or server stopping");
    return st;
}

extern "C" cf_status cf_serve_poll(cf_server* sv, uint64_t ticket, cf_result* res) {
    if (!sv) return fail(CF_ERR_ARG, "NULL server");
    return sv->sched->poll(ticket, res);
}

extern "C" cf_status cf_serve_wait(cf_server* sv, uint64_t ticket, int64_t timeout_us, cf_result* res) {
    if (!sv) return fail(CF_ERR_ARG, "NULL server");
    return sv->sched->wait(ticket, timeout_us, res);
}

extern "C" cf_status cf_serve_release(cf_server* sv, uint64_t ticket) {
    if (!sv) return fail(CF_ERR_ARG, "NULL server");
    return sv->sched->release(ticket);
}

extern "C" cf_status cf_serve_stats(cf_server* sv, cf_serve_statistics* st) {
    if (!sv || !st) return fail(CF_ERR_ARG, "NULL argument");
    sv->sched->stats(st);
    return CF_OK;
}

extern "C" cf_status cf_serve_destroy(cf_server* sv) {
    if (!sv) return CF_OK;
    sv->sched->stop();
    sv->sched.reset();
    sv->backend.reset();
    delete sv;
    return CF_OK;
}
