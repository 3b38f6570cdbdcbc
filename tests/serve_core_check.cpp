// CPU check of the serving scheduler (cf_serve_core.h) with a fake backend:
// device work is simulated by completion times.  Run by test_serve_core.py;
// prints one JSON object per scenario.
#include <stdio.h>

#include <atomic>
#include <set>
#include <thread>

#include "../paper_1406_6072_gb300/csrc/cf_serve_core.h"

using namespace cfserve;

struct FakeBackend : Backend {
    double per_real = 1e-4;        // simulated seconds per realization
    std::atomic<int> embeds{0}, allocs{0}, frees{0}, emb_frees{0}, launches{0};
    std::vector<double> until;     // per slot completion time
    std::vector<int> busy;
    std::mutex m;
    std::vector<uint64_t> start_order;
    FakeBackend(int nslots) : until(nslots, 0.0), busy(nslots, 0) {}
    static long long cells(const cf_request& r) {
        long long c = 1;
        for (int a = 0; a < r.grid.ndim; ++a) c *= r.grid.n[a];
        return c;
    }
    size_t embed_bytes(const cf_request& r) override { return (size_t)cells(r) * (1 << r.grid.ndim) * 36; }
    cf_status embed(const cf_request& r, void** h, cf_embed_report* rep) override {
        embeds++;
        if (r.xi.scale > 40.0 && r.xi.scale < 60.0)  // stands for a slow build (a large 3D spectrum)
            std::this_thread::sleep_for(std::chrono::milliseconds(300));
        memset(rep, 0, sizeof *rep);
        rep->lambda_max = 1.0;
        if (r.xi.scale > 100.0) {  // stands for a non-PSD spectrum
            *h = nullptr;
            rep->n_negative = 3;
            return CF_ERR_NOT_PSD;
        }
        *h = new int(1);
        return CF_OK;
    }
    void free_embedding(void* h) override {
        emb_frees++;
        delete (int*)h;
    }
    size_t result_bytes(const cf_request& r) override {
        return (size_t)cells(r) * 2 * r.R * (4 + (r.want_counts ? 4 : 0));
    }
    size_t batch_bytes(const std::vector<Job*>& jobs) override { return 1000; }
    cf_status alloc_result(int slot, Job* j) override {
        allocs++;
        j->dev_fields = new char[1];
        return CF_OK;
    }
    void free_result(Job* j) override {
        frees++;
        delete[] (char*)j->dev_fields;
        j->dev_fields = nullptr;
    }
    cf_status launch(int slot, const std::vector<Job*>& jobs) override {
        std::lock_guard<std::mutex> lk(m);
        launches++;
        int n = 0;
        for (auto* j : jobs) {
            n += j->req.R;
            start_order.push_back(j->ticket);
        }
        until[slot] = now_s() + per_real * n;
        busy[slot] = 1;
        return CF_OK;
    }
    bool done(int slot) override { return now_s() >= until[slot]; }
    void finish(int slot) override { busy[slot] = 0; }
};

static cf_request make_req(int side, int ndim, int R, double scale) {
    cf_request r;
    memset(&r, 0, sizeof r);
    r.grid.ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        r.grid.n[a] = a < ndim ? side : 1;
        r.grid.cell[a] = 1.0;
    }
    r.xi.kind = CF_XI_GAUSSIAN;
    r.xi.amp = 1.0;
    r.xi.scale = scale;
    r.R = R;
    r.seed = 1;
    return r;
}

static cf_serve_cfg make_cfg(size_t budget, int slots, int queue, int cache, int maxb) {
    cf_serve_cfg c;
    memset(&c, 0, sizeof c);
    c.max_inflight = slots;
    c.queue_capacity = queue;
    c.cache_entries = cache;
    c.max_batch_realizations = maxb;
    c.hbm_budget = budget;
    return c;
}

int main() {
    // 1. mixed requests: all complete, batching happens, latency stats ordered
    {
        FakeBackend be(3);
        Scheduler s(make_cfg(1ull << 32, 3, 1000, 8, 64), &be);
        std::vector<uint64_t> t;
        for (int i = 0; i < 60; ++i) {
            uint64_t k;
            cf_request r = make_req(i % 3 == 0 ? 64 : 32, i % 5 == 0 ? 3 : 2, 1 + i % 7, 2.0 + (i % 4));
            r.xi.amp = 0.5 + 0.1 * (i % 5);
            s.submit(r, &k);
            t.push_back(k);
        }
        int ok = 0;
        double lat_max = 0;
        for (auto k : t) {
            cf_result res;
            if (s.wait(k, 5000000, &res) == CF_OK && res.status == CF_OK) ++ok;
            lat_max = std::max(lat_max, res.latency_ms);
            s.release(k);
        }
        cf_serve_statistics st;
        s.stats(&st);
        printf("{\"scenario\": \"mixed\", \"ok\": %d, \"completed\": %llu, \"batches\": %llu, \"batched_requests\": %llu, "
               "\"p50\": %.4f, \"p99\": %.4f, \"lat_max\": %.4f, \"cache_hits\": %llu, \"cache_misses\": %llu, "
               "\"bytes_in_use\": %zu, \"allocs\": %d, \"frees\": %d, \"embeds\": %d}\n",
               ok, (unsigned long long)st.completed, (unsigned long long)st.batches,
               (unsigned long long)st.batched_requests, st.p50_ms, st.p99_ms, lat_max,
               (unsigned long long)st.cache_hits, (unsigned long long)st.cache_misses, st.bytes_in_use,
               be.allocs.load(), be.frees.load(), be.embeds.load());
    }
    // 2. budget admits one request at a time; peak stays within it
    {
        FakeBackend be(4);
        const cf_request r = make_req(32, 2, 4, 2.0);
        const size_t one = be.embed_bytes(r) + be.result_bytes(r) + 1000;
        Scheduler s(make_cfg(one + be.result_bytes(r) / 2, 4, 100, 4, 4), &be);
        std::vector<uint64_t> t;
        for (int i = 0; i < 12; ++i) {
            uint64_t k;
            s.submit(r, &k);
            t.push_back(k);
        }
        int ok = 0;
        for (auto k : t) {
            cf_result res;
            if (s.wait(k, 5000000, &res) == CF_OK && res.status == CF_OK) ++ok;
            s.release(k);
        }
        cf_serve_statistics st;
        s.stats(&st);
        printf("{\"scenario\": \"budget\", \"ok\": %d, \"peak\": %zu, \"budget\": %zu, \"batches\": %llu}\n", ok,
               st.bytes_peak, st.budget, (unsigned long long)st.batches);
    }
    // 3. a request larger than the whole budget is rejected; others still run
    {
        FakeBackend be(2);
        Scheduler s(make_cfg(200000, 2, 100, 4, 64), &be);
        uint64_t big, small;
        s.submit(make_req(256, 2, 8, 2.0), &big);
        s.submit(make_req(8, 2, 1, 2.0), &small);
        cf_result rb, rs;
        s.wait(big, 5000000, &rb);
        s.wait(small, 5000000, &rs);
        printf("{\"scenario\": \"reject\", \"big\": %d, \"small\": %d}\n", rb.status, rs.status);
    }
    // 4. a non-PSD spectrum fails once and the failure is cached
    {
        FakeBackend be(2);
        Scheduler s(make_cfg(1ull << 30, 2, 100, 4, 64), &be);
        uint64_t a, b;
        s.submit(make_req(16, 2, 1, 500.0), &a);
        cf_result ra, rb;
        s.wait(a, 5000000, &ra);
        s.submit(make_req(16, 2, 1, 500.0), &b);
        s.wait(b, 5000000, &rb);
        printf("{\"scenario\": \"notpsd\", \"a\": %d, \"b\": %d, \"b_hit\": %d, \"neg\": %lld, \"embeds\": %d}\n",
               ra.status, rb.status, rb.cache_hit, (long long)rb.embed.n_negative, be.embeds.load());
    }
    // 5. full queue -> BUSY; 6. wait timeout; 7. release semantics
    {
        FakeBackend be(1);
        be.per_real = 0.2;
        Scheduler s(make_cfg(1ull << 30, 1, 2, 4, 1), &be);
        uint64_t a, b, c, d;
        const cf_status sa = s.submit(make_req(8, 2, 1, 2.0), &a);
        // let the worker take a off the queue
        std::this_thread::sleep_for(std::chrono::milliseconds(50));
        const cf_status sb = s.submit(make_req(8, 2, 1, 3.0), &b);
        const cf_status sc = s.submit(make_req(8, 2, 1, 4.0), &c);
        const cf_status sd = s.submit(make_req(8, 2, 1, 5.0), &d);
        cf_result r;
        const cf_status w = s.wait(a, 1000, &r);
        const cf_status rel_early = s.release(a);
        const cf_status w2 = s.wait(a, 5000000, &r);
        const cf_status rel = s.release(a);
        const cf_status rel2 = s.release(a);
        const cf_status unk = s.poll(987654, &r);
        printf("{\"scenario\": \"queue\", \"sa\": %d, \"sb\": %d, \"sc\": %d, \"sd\": %d, \"wait_short\": %d, "
               "\"release_early\": %d, \"wait_long\": %d, \"release\": %d, \"release_again\": %d, \"unknown\": %d}\n",
               sa, sb, sc, sd, w, rel_early, w2, rel, rel2, unk);
        s.stop();
        printf("{\"scenario\": \"stop\", \"allocs\": %d, \"frees\": %d, \"embeds\": %d, \"emb_frees\": %d}\n",
               be.allocs.load(), be.frees.load(), be.embeds.load(), be.emb_frees.load());
    }
    // 8. LRU: more spectra than cache entries
    {
        FakeBackend be(1);
        Scheduler s(make_cfg(1ull << 30, 1, 100, 2, 64), &be);
        for (int i = 0; i < 6; ++i) {
            uint64_t k;
            s.submit(make_req(16, 2, 1, 2.0 + (i % 3)), &k);
            cf_result r;
            s.wait(k, 5000000, &r);
            s.release(k);
        }
        cf_serve_statistics st;
        s.stats(&st);
        printf("{\"scenario\": \"lru\", \"evictions\": %llu, \"misses\": %llu, \"hits\": %llu}\n",
               (unsigned long long)st.cache_evictions, (unsigned long long)st.cache_misses,
               (unsigned long long)st.cache_hits);
    }
    // 9. FIFO: requests of one shape whose spectra are resident start in
    // submission order (the three spectra are built first)
    {
        FakeBackend be(2);
        Scheduler s(make_cfg(1ull << 30, 2, 1000, 8, 3), &be);
        for (int i = 0; i < 3; ++i) {
            uint64_t k;
            s.submit(make_req(16, 2, 1, 2.0 + i), &k);
            cf_result r;
            s.wait(k, 5000000, &r);
            s.release(k);
        }
        {
            std::lock_guard<std::mutex> lk(be.m);
            be.start_order.clear();
        }
        std::vector<uint64_t> t;
        for (int i = 0; i < 30; ++i) {
            uint64_t k;
            s.submit(make_req(16, 2, 1 + i % 2, 2.0 + (i % 3)), &k);
            t.push_back(k);
        }
        for (auto k : t) {
            cf_result r;
            s.wait(k, 5000000, &r);
            s.release(k);
        }
        // how many positions a request started after its submission position
        // (later requests may ride along in an earlier batch; none waits long)
        long max_delay = 0;
        for (size_t i = 0; i < be.start_order.size(); ++i) {
            const long submitted_pos = (long)(be.start_order[i] - t[0]);
            max_delay = std::max(max_delay, (long)i - submitted_pos);
        }
        printf("{\"scenario\": \"fifo\", \"started\": %zu, \"max_delay\": %ld}\n", be.start_order.size(), max_delay);
    }
    // 10. a slow build does not hold up requests whose spectrum is resident:
    // they are admitted and complete while it runs; then it completes too
    {
        FakeBackend be(2);
        Scheduler s(make_cfg(1ull << 30, 2, 1000, 8, 8), &be);
        uint64_t warm;
        s.submit(make_req(16, 2, 1, 2.0), &warm);
        cf_result r;
        s.wait(warm, 5000000, &r);
        s.release(warm);
        uint64_t slow;
        s.submit(make_req(32, 3, 2, 50.0), &slow);  // its spectrum takes 300 ms to build
        std::vector<uint64_t> fast;
        for (int i = 0; i < 10; ++i) {
            uint64_t k;
            s.submit(make_req(16, 2, 1 + i % 3, 2.0), &k);
            fast.push_back(k);
        }
        int fast_ok = 0;
        double fast_max = 0;
        for (auto k : fast) {
            cf_result rr;
            if (s.wait(k, 5000000, &rr) == CF_OK && rr.status == CF_OK) ++fast_ok;
            fast_max = std::max(fast_max, rr.latency_ms);
            s.release(k);
        }
        cf_result rs;
        const cf_status ws = s.wait(slow, 5000000, &rs);
        printf("{\"scenario\": \"overtake\", \"fast_ok\": %d, \"fast_max_ms\": %.3f, \"slow\": %d, "
               "\"slow_status\": %d, \"slow_ms\": %.3f, \"slow_hit\": %d}\n",
               fast_ok, fast_max, (int)ws, (int)rs.status, rs.latency_ms, rs.cache_hit);
        s.release(slow);
    }
    // 11. a slot reserved for small requests: with the only general slot busy
    // on a long batch, small requests still run (and large ones wait)
    {
        FakeBackend be(2);
        cf_serve_cfg c = make_cfg(1ull << 30, 1, 1000, 8, 64);
        c.small_request_cells = 2 * 4 * 16 * 16;  // up to 4 realizations of 16^2
        Scheduler s(c, &be);
        uint64_t warm;
        s.submit(make_req(16, 2, 1, 2.0), &warm);
        cf_result r;
        s.wait(warm, 5000000, &r);
        s.release(warm);
        be.per_real = 0.02;                          // the large batch takes 40 x 20 ms
        uint64_t big, big2;
        s.submit(make_req(16, 2, 40, 2.0), &big);    // 2 * 40 * 256 cells: not small
        std::this_thread::sleep_for(std::chrono::milliseconds(20));
        be.per_real = 1e-4;
        s.submit(make_req(16, 2, 40, 2.0), &big2);   // waits for the general slot
        std::vector<uint64_t> sm;
        for (int i = 0; i < 6; ++i) {
            uint64_t k;
            s.submit(make_req(16, 2, 1 + i % 4, 2.0), &k);
            sm.push_back(k);
        }
        double small_max = 0;
        int small_ok = 0;
        for (auto k : sm) {
            cf_result rr;
            if (s.wait(k, 5000000, &rr) == CF_OK && rr.status == CF_OK) ++small_ok;
            small_max = std::max(small_max, rr.latency_ms);
            s.release(k);
        }
        cf_result rb, rb2;
        s.wait(big, 10000000, &rb);
        s.wait(big2, 10000000, &rb2);
        printf("{\"scenario\": \"reserved\", \"small_ok\": %d, \"small_max_ms\": %.3f, \"big_ms\": %.3f, "
               "\"big2_status\": %d, \"big2_queue_ms\": %.3f}\n",
               small_ok, small_max, rb.latency_ms, (int)rb2.status, rb2.queue_ms);
        s.release(big);
        s.release(big2);
    }
    {  // a request larger than one batch is refused at submission
        FakeBackend be(1);
        Scheduler s(make_cfg(1ull << 30, 1, 10, 2, 8), &be);
        uint64_t a = 0, b = 0;
        const cf_status too_big = s.submit(make_req(16, 2, 9, 2.0), &a);
        const cf_status fits = s.submit(make_req(16, 2, 8, 2.0), &b);
        cf_result r;
        s.wait(b, 5000000, &r);
        printf("{\"scenario\": \"oversize\", \"too_big\": %d, \"fits\": %d, \"status\": %d}\n", (int)too_big,
               (int)fits, (int)r.status);
        s.release(b);
    }
    return 0;
}
