// cf_serve_core.h -- scheduling core of the serving loop, free of CUDA.
//
// Requests wait in a FIFO queue; a worker thread admits, while a slot is free
// and device memory fits the budget, the first queued request whose spectrum
// is resident, batches queued requests of the same grid shape with it (up to
// max_batch_realizations), keeps the embeddings of recent spectra in an LRU
// cache (at amplitude 1; the request's amplitude is applied at sampling) and
// retires finished batches.  A spectrum that is not resident is built by a
// second thread (the binary64 embedding with its positivity report takes
// milliseconds and waits on the device); requests waiting for it are passed
// over meanwhile, so a build never holds up requests whose spectra are ready,
// nor the retiring of finished batches.  All device work goes through a
// Backend: the CUDA one lives in cf_serve.cu; the tests drive this core with
// a fake one on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cf.h"

namespace cfserve {

enum JobState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct CacheEntry;

struct Job {
    uint64_t ticket = 0;
    cf_request req{};
    JobState state = QUEUED;
    cf_status status = CF_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    int cache_hit = 0;
    bool built_for = false;       // its spectrum was missing and built for it (a cache miss)
    cf_embed_report rep{};
    CacheEntry* emb = nullptr;
    size_t result_bytes = 0;
    void* dev_fields = nullptr;   // backend-owned result memory
    void* dev_counts = nullptr;
};

struct CacheEntry {
    std::string key;
    void* handle = nullptr;       // backend embedding (null when the spectrum failed)
    size_t bytes = 0;
    int refs = 0;                 // running jobs using it (+1 while it is built)
    bool building = false;        // queued for or in the embedding thread
    uint64_t last_use = 0;
    cf_status status = CF_OK;
    cf_embed_report rep_unit{};   // report at amplitude 1
};

class Backend {
  public:
    virtual ~Backend() {}
    // Bytes the embedding of this request's spectrum will hold (and need while built).
    virtual size_t embed_bytes(const cf_request& r) = 0;
    // Builds the embedding of r's spectrum at amplitude 1 (blocking; called
    // from the scheduler's embedding thread, concurrently with the others).
    virtual cf_status embed(const cf_request& r, void** handle, cf_embed_report* rep) = 0;
    virtual void free_embedding(void* handle) = 0;
    virtual size_t result_bytes(const cf_request& r) = 0;
    // Device temporaries of one batched launch of these jobs.
    virtual size_t batch_bytes(const std::vector<Job*>& jobs) = 0;
    virtual cf_status alloc_result(int slot, Job* j) = 0;
    virtual void free_result(Job* j) = 0;
    // Enqueues the batch on the slot (asynchronous).
    virtual cf_status launch(int slot, const std::vector<Job*>& jobs) = 0;
    virtual bool done(int slot) = 0;
    virtual void finish(int slot) = 0;
};

inline double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Shape key: requests with equal keys can share one launch.
inline std::string shape_key(const cf_request& r) {
    char b[160];
    snprintf(b, sizeof b, "%d:%lld:%lld:%lld:%d:%d", r.grid.ndim, (long long)r.grid.n[0],
             (long long)(r.grid.ndim > 1 ? r.grid.n[1] : 1), (long long)(r.grid.ndim > 2 ? r.grid.n[2] : 1),
             r.grid.embed_factor == 0 ? 2 : r.grid.embed_factor, r.want_counts ? 1 : 0);
    return b;
}

// Spectrum key: everything lambda depends on except the amplitude.
inline std::string spectrum_key(const cf_request& r) {
    char b[320];
    const int d = r.grid.ndim;
    snprintf(b, sizeof b, "%d:%lld:%lld:%lld:%d:%.17g:%.17g:%.17g:%d:%.17g:%.17g:%u", d, (long long)r.grid.n[0],
             (long long)(d > 1 ? r.grid.n[1] : 1), (long long)(d > 2 ? r.grid.n[2] : 1),
             r.grid.embed_factor == 0 ? 2 : r.grid.embed_factor, r.grid.cell[0],
             d > 1 ? r.grid.cell[1] : 1.0, d > 2 ? r.grid.cell[2] : 1.0, r.xi.kind, r.xi.scale,
             r.xi.kind == CF_XI_GEN_CAUCHY ? r.xi.beta : 0.0, r.embed_flags);
    return b;
}

inline cf_embed_report scale_report(const cf_embed_report& u, double amp) {
    cf_embed_report r = u;
    r.lambda_min *= amp;
    r.lambda_max *= amp;
    r.tau *= amp;
    r.neg_mass *= amp;
    r.cov_error *= amp;
    return r;
}

class Scheduler {
  public:
    Scheduler(const cf_serve_cfg& cfg, Backend* be) : cfg_(cfg), be_(be) {
        if (cfg_.max_inflight < 1) cfg_.max_inflight = 1;
        if (cfg_.queue_capacity < 1) cfg_.queue_capacity = 1;
        if (cfg_.cache_entries < 1) cfg_.cache_entries = 1;
        if (cfg_.max_batch_realizations < 1) cfg_.max_batch_realizations = 1;
        if (cfg_.small_request_cells < 0) cfg_.small_request_cells = 0;
        // slots [0, max_inflight) take any request; slot max_inflight (if
        // small_request_cells > 0) only small ones
        slots_.resize(cfg_.max_inflight + (cfg_.small_request_cells > 0 ? 1 : 0));
        worker_ = std::thread([this] { run(); });
        embedder_ = std::thread([this] { build_loop(); });
    }

    ~Scheduler() { stop(); }

    cf_status submit(const cf_request& r, uint64_t* ticket) {
        if (r.grid.ndim < 1 || r.grid.ndim > 3 || r.R < 1 || !(r.xi.amp > 0.0) || !(r.xi.scale > 0.0) ||
            r.xi.kind < CF_XI_GAUSSIAN || r.xi.kind > CF_XI_EXPONENTIAL || (r.want_counts && !(r.nbar >= 0.0)))
            return CF_ERR_ARG;
        for (int a = 0; a < r.grid.ndim; ++a)
            if (r.grid.n[a] < 1) return CF_ERR_ARG;
        if (r.r0 + (uint64_t)r.R > (1ull << 32)) return CF_ERR_ARG;
        if (r.R > cfg_.max_batch_realizations) return CF_ERR_ARG;  // a request runs in one launch
        if (r.embed_flags & CF_EMBED_LOG1P) return CF_ERR_ARG;      // not linear in the amplitude
        std::lock_guard<std::mutex> lk(mu_);
        if (stopping_) return CF_ERR_BUSY;
        if ((int)queue_.size() >= cfg_.queue_capacity) {
            ++rejected_;
            return CF_ERR_BUSY;
        }
        Job* j = new Job();
        j->ticket = ++next_ticket_;
        j->req = r;
        j->t_submit = now_s();
        if (first_submit_ == 0) first_submit_ = j->t_submit;
        jobs_[j->ticket] = j;
        queue_.push_back(j);
        ++submitted_;
        *ticket = j->ticket;
        cv_work_.notify_one();
        return CF_OK;
    }

    cf_status poll(uint64_t t, cf_result* res) {
        std::lock_guard<std::mutex> lk(mu_);
        return poll_locked(t, res);
    }

    cf_status wait(uint64_t t, int64_t timeout_us, cf_result* res) {
        std::unique_lock<std::mutex> lk(mu_);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
        for (;;) {
            const cf_status s = poll_locked(t, res);
            if (s != CF_ERR_BUSY) return s;
            if (timeout_us < 0) {
                cv_done_.wait(lk);
            } else if (cv_done_.wait_until(lk, deadline) == std::cv_status::timeout) {
                const cf_status s2 = poll_locked(t, res);
                return s2 == CF_ERR_BUSY ? CF_ERR_TIMEOUT : s2;
            }
        }
    }

    cf_status release(uint64_t t) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return CF_ERR_NOT_FOUND;
        Job* j = it->second;
        if (j->state != DONE) return CF_ERR_BUSY;
        if (j->dev_fields || j->dev_counts) be_->free_result(j);
        in_use_ -= j->result_bytes;
        jobs_.erase(it);
        delete j;
        cv_work_.notify_one();
        return CF_OK;
    }

    void stats(cf_serve_statistics* s) {
        std::lock_guard<std::mutex> lk(mu_);
        memset(s, 0, sizeof *s);
        s->submitted = submitted_;
        s->completed = completed_;
        s->failed = failed_;
        s->rejected = rejected_;
        s->queued = (int64_t)queue_.size();
        int64_t inflight = 0;
        for (auto& sl : slots_) inflight += (int64_t)sl.jobs.size();
        s->inflight = inflight;
        s->cache_hits = cache_hits_;
        s->cache_misses = cache_misses_;
        s->cache_evictions = cache_evictions_;
        s->batches = batches_;
        s->batched_requests = batched_requests_;
        s->realizations = realizations_;
        s->bytes_in_use = in_use_;
        s->bytes_peak = peak_;
        s->budget = cfg_.hbm_budget;
        if (!latencies_.empty()) {
            std::vector<double> v = latencies_;
            std::sort(v.begin(), v.end());
            auto pct = [&](double q) {
                const double pos = q * (double)(v.size() - 1);
                const size_t lo = (size_t)pos;
                const size_t hi = std::min(lo + 1, v.size() - 1);
                return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
            };
            s->p50_ms = pct(0.50);
            s->p99_ms = pct(0.99);
            double sum = 0;
            for (double x : v) sum += x;
            s->mean_ms = sum / (double)v.size();
        }
        if (last_done_ > first_submit_ && first_submit_ > 0)
            s->realizations_per_s = (double)done_realizations_ / (last_done_ - first_submit_);
    }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stopped_) return;
            stopping_ = true;
            cv_work_.notify_all();
        }
        if (worker_.joinable()) worker_.join();
        {
            // the build in progress ends; pending ones are dropped
            std::lock_guard<std::mutex> lk(mu_);
            builds_stop_ = true;
            cv_build_.notify_all();
        }
        if (embedder_.joinable()) embedder_.join();
        std::lock_guard<std::mutex> lk(mu_);
        for (auto& kv : jobs_) {
            Job* j = kv.second;
            if (j->dev_fields || j->dev_counts) be_->free_result(j);
            delete j;
        }
        jobs_.clear();
        queue_.clear();
        for (auto& e : cache_)
            if (e.handle) be_->free_embedding(e.handle);
        cache_.clear();
        stopped_ = true;
        cv_done_.notify_all();
    }

  private:
    struct Slot {
        std::vector<Job*> jobs;
        size_t bytes = 0;
    };

    cf_status poll_locked(uint64_t t, cf_result* res) {
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return CF_ERR_NOT_FOUND;
        Job* j = it->second;
        if (j->state != DONE) return CF_ERR_BUSY;
        if (res) {
            memset(res, 0, sizeof *res);
            res->status = j->status;
            res->cache_hit = j->cache_hit;
            res->queue_ms = j->t_start > 0 ? 1e3 * (j->t_start - j->t_submit) : 0.0;
            res->run_ms = j->t_start > 0 ? 1e3 * (j->t_done - j->t_start) : 0.0;
            res->latency_ms = 1e3 * (j->t_done - j->t_submit);
            res->dev_fields = (const float*)j->dev_fields;
            res->dev_counts = (const int32_t*)j->dev_counts;
            res->embed = j->rep;
        }
        return CF_OK;
    }

    void complete(Job* j, cf_status st, double t) {
        j->state = DONE;
        j->status = st;
        j->t_done = t;
        if (st == CF_OK) {
            ++completed_;
            latencies_.push_back(1e3 * (t - j->t_submit));
            done_realizations_ += (uint64_t)j->req.R;
            last_done_ = std::max(last_done_, t);
        } else {
            ++failed_;
        }
        cv_done_.notify_all();
    }

    CacheEntry* find_entry(const std::string& key) {
        for (auto& e : cache_)
            if (e.key == key) return &e;
        return nullptr;
    }

    // Frees least recently used unreferenced embeddings until `need` bytes
    // fit or none is left to evict; true when they fit.
    bool make_room(size_t need) {
        while (in_use_ + need > cfg_.hbm_budget) {
            auto victim = cache_.end();
            for (auto it = cache_.begin(); it != cache_.end(); ++it)
                if (it->refs == 0 && (victim == cache_.end() || it->last_use < victim->last_use)) victim = it;
            if (victim == cache_.end()) return false;
            if (victim->handle) be_->free_embedding(victim->handle);
            in_use_ -= victim->bytes;
            cache_.erase(victim);
            ++cache_evictions_;
        }
        return true;
    }

    bool anything_in_flight() const {
        for (auto& sl : slots_)
            if (!sl.jobs.empty()) return true;
        return false;
    }

    // Retires finished batches; true if any finished.
    bool retire() {
        bool any = false;
        for (int i = 0; i < (int)slots_.size(); ++i) {
            Slot& sl = slots_[i];
            if (sl.jobs.empty() || !be_->done(i)) continue;
            be_->finish(i);
            const double t = now_s();
            for (Job* j : sl.jobs) {
                j->emb->refs -= 1;
                complete(j, CF_OK, t);
            }
            in_use_ -= sl.bytes;
            sl.jobs.clear();
            sl.bytes = 0;
            any = true;
        }
        return any;
    }

    // Starts building the spectrum of queued job j on the embedding thread
    // (its bytes reserved, the entry pinned while it is built); returns the
    // new entry, or null if the budget has no room for it yet (*rejected:
    // never, even with nothing else in memory).
    CacheEntry* start_build(Job* j, bool* rejected) {
        *rejected = false;
        const size_t need = be_->embed_bytes(j->req);
        if (!make_room(need)) {
            if (!anything_in_flight() && builds_in_progress() == 0 && need > cfg_.hbm_budget) *rejected = true;
            return nullptr;
        }
        while ((int)cache_.size() >= cfg_.cache_entries) {
            auto victim = cache_.end();
            for (auto it = cache_.begin(); it != cache_.end(); ++it)
                if (it->refs == 0 && (victim == cache_.end() || it->last_use < victim->last_use)) victim = it;
            if (victim == cache_.end()) break;
            if (victim->handle) be_->free_embedding(victim->handle);
            in_use_ -= victim->bytes;
            cache_.erase(victim);
            ++cache_evictions_;
        }
        in_use_ += need;  // reserved while building
        peak_ = std::max(peak_, in_use_);
        CacheEntry ce;
        ce.key = spectrum_key(j->req);
        ce.bytes = need;
        ce.refs = 1;
        ce.building = true;
        ce.last_use = ++use_clock_;
        cache_.push_back(ce);
        cf_request unit = j->req;
        unit.xi.amp = 1.0;
        builds_.push_back(Build{&cache_.back(), unit});
        ++cache_misses_;
        j->built_for = true;
        cv_build_.notify_one();
        return &cache_.back();
    }

    int builds_in_progress() const {
        int n = 0;
        for (auto& e : cache_) n += e.building ? 1 : 0;
        return n;
    }

    // The embedding thread: builds queued spectra one at a time, with the
    // lock released while the backend works.
    void build_loop() {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_build_.wait(lk, [this] { return builds_stop_ || !builds_.empty(); });
            if (builds_stop_) break;
            const Build b = builds_.front();
            builds_.pop_front();
            void* handle = nullptr;
            cf_embed_report rep{};
            lk.unlock();
            const cf_status st = be_->embed(b.req, &handle, &rep);
            lk.lock();
            CacheEntry* e = b.entry;
            e->handle = st == CF_OK ? handle : nullptr;
            e->status = st;
            e->rep_unit = rep;
            e->building = false;
            e->refs -= 1;
            if (st != CF_OK) {
                in_use_ -= e->bytes;
                e->bytes = 0;
            }
            cv_work_.notify_all();
        }
        // builds that never ran: their entries hold no embedding
        for (const Build& b : builds_) {
            b.entry->building = false;
            b.entry->refs -= 1;
            b.entry->status = CF_ERR_BUSY;
            in_use_ -= b.entry->bytes;
            b.entry->bytes = 0;
        }
        builds_.clear();
    }

    // Admits the first queued request whose spectrum is resident (and its
    // batch mates) into a free slot; starts the builds of missing spectra on
    // the way (at most kMaxBuilds at a time) and completes requests whose
    // spectrum failed.  True if the queue or a slot changed.
    static constexpr int kMaxBuilds = 4;
    static long long cells_of(const cf_request& r) {
        long long c = 2ll * r.R;
        for (int a = 0; a < r.grid.ndim; ++a) c *= r.grid.n[a];
        return c;
    }
    bool small(const Job* j) const {
        return cfg_.small_request_cells > 0 && cells_of(j->req) <= (long long)cfg_.small_request_cells;
    }

    bool admit(std::unique_lock<std::mutex>&) {
        int slot = -1;
        for (int i = 0; i < cfg_.max_inflight; ++i)
            if (slots_[i].jobs.empty()) {
                slot = i;
                break;
            }
        // the reserved slot, for small requests only
        const bool small_only = slot < 0 && (int)slots_.size() > cfg_.max_inflight &&
                                slots_[cfg_.max_inflight].jobs.empty();
        if (small_only) slot = cfg_.max_inflight;
        if (slot < 0 || queue_.empty()) return false;
        Job* head = nullptr;
        CacheEntry* e = nullptr;
        for (size_t q = 0; q < queue_.size() && q < 256 && !head; ++q) {
            Job* j = queue_[q];
            if (small_only && !small(j)) continue;
            CacheEntry* ce = find_entry(spectrum_key(j->req));
            if (!ce) {
                if (builds_in_progress() >= kMaxBuilds) continue;
                bool rejected = false;
                ce = start_build(j, &rejected);
                if (rejected) {
                    queue_.erase(queue_.begin() + (long)q);
                    complete(j, CF_ERR_NOMEM, now_s());
                    return true;
                }
                continue;  // being built, or waiting for memory to build it
            }
            if (ce->building) continue;
            if (ce->status != CF_OK) {
                queue_.erase(queue_.begin() + (long)q);
                if (!j->built_for) {
                    j->cache_hit = 1;
                    ++cache_hits_;
                }
                j->rep = scale_report(ce->rep_unit, j->req.xi.amp);
                complete(j, ce->status, now_s());
                return true;
            }
            head = j;
            e = ce;
        }
        if (!head) return false;
        e->last_use = ++use_clock_;
        // batch: the head plus queued requests of the same shape whose
        // spectrum is already resident
        std::vector<Job*> batch{head};
        int nreal = head->req.R;
        const std::string sk = shape_key(head->req);
        const size_t at = (size_t)(std::find(queue_.begin(), queue_.end(), head) - queue_.begin());
        for (size_t q = at + 1; q < queue_.size() && q < 256; ++q) {
            Job* c = queue_[q];
            if (nreal + c->req.R > cfg_.max_batch_realizations) break;
            if (shape_key(c->req) != sk) continue;
            if (small_only && !small(c)) continue;
            CacheEntry* ce = find_entry(spectrum_key(c->req));
            if (!ce || ce->building || ce->status != CF_OK) continue;
            batch.push_back(c);
            nreal += c->req.R;
        }
        auto bytes_of = [&](const std::vector<Job*>& b) {
            size_t t = be_->batch_bytes(b);
            for (Job* x : b) t += be_->result_bytes(x->req);
            return t;
        };
        size_t need = bytes_of(batch);
        while (batch.size() > 1 && in_use_ + need > cfg_.hbm_budget) {
            batch.pop_back();
            need = bytes_of(batch);
        }
        // pin the batch's embeddings so that making room cannot evict them
        std::vector<CacheEntry*> pinned;
        for (Job* b : batch) {
            CacheEntry* ce = find_entry(spectrum_key(b->req));
            ce->refs += 1;
            pinned.push_back(ce);
        }
        const bool fits = in_use_ + need <= cfg_.hbm_budget || make_room(need);
        for (CacheEntry* ce : pinned) ce->refs -= 1;
        if (!fits) {
            if (!anything_in_flight() && builds_in_progress() == 0 && in_use_ + need > cfg_.hbm_budget) {
                // cannot run even alone after everything evictable is gone
                bool others = false;
                for (auto& kv : jobs_)
                    if (kv.second->state == DONE && kv.second->result_bytes) others = true;
                if (!others) {
                    queue_.erase(std::find(queue_.begin(), queue_.end(), head));
                    complete(head, CF_ERR_NOMEM, now_s());
                    return true;
                }
            }
            return false;
        }
        // take the batch out of the queue
        for (Job* b : batch) queue_.erase(std::find(queue_.begin(), queue_.end(), b));
        const double t = now_s();
        Slot& sl = slots_[slot];
        size_t temp = be_->batch_bytes(batch);
        for (Job* b : batch) {
            CacheEntry* ce = find_entry(spectrum_key(b->req));
            ce->refs += 1;
            ce->last_use = ++use_clock_;
            if (!b->built_for) {
                b->cache_hit = 1;
                ++cache_hits_;
            }
            b->emb = ce;
            b->rep = scale_report(ce->rep_unit, b->req.xi.amp);
            b->state = RUNNING;
            b->t_start = t;
            b->result_bytes = be_->result_bytes(b->req);
        }
        cf_status st = CF_OK;
        for (Job* b : batch) {
            if (st == CF_OK) st = be_->alloc_result(slot, b);
        }
        if (st == CF_OK) st = be_->launch(slot, batch);
        if (st != CF_OK) {
            for (Job* b : batch) {
                b->emb->refs -= 1;
                if (b->dev_fields || b->dev_counts) be_->free_result(b);
                b->result_bytes = 0;
                complete(b, st, now_s());
            }
            return true;
        }
        size_t results = 0;
        for (Job* b : batch) results += b->result_bytes;
        in_use_ += temp + results;
        peak_ = std::max(peak_, in_use_);
        sl.jobs = batch;
        sl.bytes = temp;
        ++batches_;
        batched_requests_ += batch.size();
        realizations_ += (uint64_t)nreal;
        return true;
    }

    void run() {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            bool progress = retire();
            if (stopping_) {
                if (!anything_in_flight()) break;
            } else {
                while (admit(lk)) progress = true;
            }
            if (stopping_ && !anything_in_flight()) break;
            if (!progress) cv_work_.wait_for(lk, std::chrono::microseconds(anything_in_flight() ? 50 : 2000));
        }
        // queued requests end unserved
        const double t = now_s();
        for (Job* j : queue_) complete(j, CF_ERR_BUSY, t);
        queue_.clear();
    }

    cf_serve_cfg cfg_;
    Backend* be_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::thread worker_, embedder_;
    struct Build {
        CacheEntry* entry;
        cf_request req;  // at amplitude 1
    };
    std::deque<Build> builds_;
    std::condition_variable cv_build_;
    bool builds_stop_ = false;
    std::deque<Job*> queue_;
    std::map<uint64_t, Job*> jobs_;
    std::list<CacheEntry> cache_;
    std::vector<Slot> slots_;
    uint64_t next_ticket_ = 0, use_clock_ = 0;
    bool stopping_ = false, stopped_ = false;
    size_t in_use_ = 0, peak_ = 0;
    uint64_t submitted_ = 0, completed_ = 0, failed_ = 0, rejected_ = 0;
    uint64_t cache_hits_ = 0, cache_misses_ = 0, cache_evictions_ = 0;
    uint64_t batches_ = 0, batched_requests_ = 0, realizations_ = 0, done_realizations_ = 0;
    double first_submit_ = 0, last_done_ = 0;
    std::vector<double> latencies_;
};

}  // namespace cfserve
