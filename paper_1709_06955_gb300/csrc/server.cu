// Serving loop: continuous batching of top-k SimRank queries over one resident graph store.
//
// Requests (queries and edge-update batches) enter one FIFO.  Worker threads, each with its own workspace
// and CUDA stream, take the next batch of queries from the head of the FIFO as soon as they are free: up to
// max_batch queries, admitted while the estimated score-buffer memory of the batches in flight stays within
// the budget.  Requests that arrive while other batches run are admitted by the next free worker, so batches
// of different workers overlap on the device.  An update batch at the head of the FIFO is applied between
// batches: the worker builds the next store version beside the current one and publishes it -- batches in
// flight keep reading the version they started with -- and every query behind it sees the new edge set.  Each
// result records the epoch it saw and its submit-to-completion latency.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>

#include "engine.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    bool is_update = false;
    probesim_query q{};
    uint64_t ticket = 0;
    Clock::time_point submitted;
    std::vector<int32_t> src, dst;  // update batch
    bool insert = true;
};

struct Done {
    probesim_result r{};
    std::vector<int32_t> ids;
    std::vector<float> vals;
};

}  // namespace

struct probesim_server {
    probesim_graph *g = nullptr;
    probesim_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> fifo;
    std::deque<Done> done;
    int64_t queued_queries = 0;
    bool stop = false;
    bool updating = false;  // an update batch has left the FIFO but is not applied yet: hold admissions
    double mem_in_flight = 0.0;
    int32_t batches_in_flight = 0;
    uint64_t next_ticket = 1;
    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, updates_applied = 0, failed = 0;
    double batch_queries = 0.0;
    std::vector<double> latencies;
    Clock::time_point first_submit{}, last_done{};
    bool any_submit = false;
    std::vector<std::thread> workers;
    std::vector<Workspace *> ws;
    std::vector<cudaStream_t> streams;
};

// Device bytes a query takes in a batch.  The regrouped deterministic engine holds about 0.25 n_r score vectors
// of n FP32 in three buffers at its widest depth.  The frontier and randomized engines hold an estimate row
// (8 + 4 bytes per node) and walk rows of the query's n_r walks (8 bytes per node slot); their level tables and
// hash sets adapt to the worker's share of the budget (passes, deferred ranges, walk ranges).
static double query_bytes(const probesim_server *s, const probesim_query &q) {
    const double nr = (double)ps::num_walks_for(s->g, q.eps), n = (double)s->g->n;
    const probesim_config &c = s->g->cfg;
    if (c.probe_mode != PROBESIM_PROBE_DETERMINISTIC || c.eps_p > 0.f) return 12.0 * n + 8.0 * c.l_max * nr;
    return 3.0 * 4.0 * n * std::max(1.0, 0.25 * nr);
}

static void worker_loop(probesim_server *s, int wid) {
    Workspace *ws = s->ws[wid];
    cudaStream_t st = s->streams[wid];
    cudaSetDevice(s->g->device);
    const int32_t kmax = s->cfg.kmax;
    std::vector<Request> batch;
    std::vector<probesim_query> qs;
    std::vector<int32_t> ids;
    std::vector<float> vals;
    for (;;) {
        batch.clear();
        Request update;
        bool have_update = false;
        double mem = 0.0;
        // a batch takes its store version before the queue lock is released, so an update batch behind it in the
        // FIFO cannot change what it reads; the update builds the next version beside it
        std::shared_ptr<StoreVersion> snap;
        uint64_t epoch = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || (!s->fifo.empty() && !s->updating); });
            if (s->stop) return;
            if (s->fifo.front().is_update) {
                update = std::move(s->fifo.front());
                s->fifo.pop_front();
                have_update = true;
                s->updating = true;
            } else {
                while (!s->fifo.empty() && !s->fifo.front().is_update && (int32_t)batch.size() < s->cfg.max_batch) {
                    const double b = query_bytes(s, s->fifo.front().q);
                    const bool fits = s->mem_in_flight + mem + b <= s->cfg.memory_budget_bytes;
                    if (!fits && !(batch.empty() && s->batches_in_flight == 0)) break;  // admit when memory frees up
                    mem += b;
                    batch.push_back(std::move(s->fifo.front()));
                    s->fifo.pop_front();
                }
                if (batch.empty()) {  // waiting for memory: let a finishing batch wake us
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                    continue;
                }
                s->queued_queries -= (int64_t)batch.size();
                s->mem_in_flight += mem;
                s->batches_in_flight += 1;
                snap = s->g->current();
                epoch = snap->epoch;
            }
        }
        if (have_update) {  // epoch boundary: queries behind it wait (admissions held), those in flight do not
            int64_t applied = 0;
            probesim_status rc = ps::apply_updates(s->g, update.src.data(), update.dst.data(), (int64_t)update.src.size(),
                                                   update.insert, &applied, st);
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc == PROBESIM_OK) s->updates_applied += 1; else s->failed += 1;
            s->updating = false;
            s->cv_work.notify_all();
            continue;
        }
        const Clock::time_point t_start = Clock::now();
        qs.resize(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) qs[i] = batch[i].q;
        const int32_t B = (int32_t)batch.size();
        ids.assign((size_t)B * kmax, -1);
        vals.assign((size_t)B * kmax, 0.f);
        const probesim_status rc = ps::topk_core(s->g, ws, snap, qs.data(), B, kmax, ids.data(), vals.data(), st);
        snap.reset();
        const Clock::time_point t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (int32_t i = 0; i < B; ++i) {
                Done d;
                d.r.ticket = batch[i].ticket;
                d.r.query_id = batch[i].q.query_id;
                d.r.node = batch[i].q.node;
                d.r.k = batch[i].q.k;
                d.r.status = (int32_t)rc;
                d.r.epoch = epoch;
                d.r.batch_size = B;
                d.r.worker = wid;
                d.r.queue_ms = std::chrono::duration<double, std::milli>(t_start - batch[i].submitted).count();
                d.r.latency_ms = std::chrono::duration<double, std::milli>(t_end - batch[i].submitted).count();
                d.ids.assign(ids.begin() + (size_t)i * kmax, ids.begin() + (size_t)(i + 1) * kmax);
                d.vals.assign(vals.begin() + (size_t)i * kmax, vals.begin() + (size_t)(i + 1) * kmax);
                s->latencies.push_back(d.r.latency_ms);
                s->done.push_back(std::move(d));
            }
            s->completed += B;
            if (rc != PROBESIM_OK) s->failed += B;
            s->batches += 1;
            s->batch_queries += B;
            s->last_done = t_end;
            s->mem_in_flight -= mem;
            s->batches_in_flight -= 1;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

extern "C" {

probesim_status probesim_server_config_default(probesim_server_config *cfg) {
    if (!cfg) return ps::fail_status(PROBESIM_E_INVALID, "cfg is null");
    // measured on R-MAT 2^20 at saturation: several workers overlap one query's host-side schedule with
    // another's kernels, while wide batches cost more in the accumulate than they save
    cfg->workers = 3;
    cfg->max_batch = 2;
    cfg->kmax = 100;
    cfg->queue_capacity = 100000;
    cfg->memory_budget_bytes = 0.0;
    return PROBESIM_OK;
}

probesim_status probesim_server_create(probesim_graph *g, const probesim_server_config *cfg, probesim_server **out) {
    if (!g || !out) return ps::fail_status(PROBESIM_E_INVALID, "null argument");
    *out = nullptr;
    probesim_server_config c;
    if (cfg) c = *cfg; else probesim_server_config_default(&c);
    if (c.workers < 1 || c.workers > 8) return ps::fail_status(PROBESIM_E_INVALID, "workers must lie in [1, 8]");
    if (c.max_batch < 1 || c.max_batch > 4096) return ps::fail_status(PROBESIM_E_INVALID, "max_batch must lie in [1, 4096]");
    if (c.kmax < 1 || c.kmax > 4096 || c.kmax > g->n - 1)
        return ps::fail_status(PROBESIM_E_INVALID, "kmax must lie in [1, min(4096, n-1)]");
    if (c.queue_capacity < 1) return ps::fail_status(PROBESIM_E_INVALID, "queue_capacity must be >= 1");
    if (!(c.memory_budget_bytes >= 0.0)) return ps::fail_status(PROBESIM_E_INVALID, "memory_budget_bytes must be >= 0");
    if (c.memory_budget_bytes == 0.0) c.memory_budget_bytes = (double)g->budget;
    probesim_server *s = new (std::nothrow) probesim_server();
    if (!s) return ps::fail_status(PROBESIM_E_NOMEM, "host allocation failed");
    s->g = g;
    s->cfg = c;
    cudaSetDevice(g->device);
    for (int i = 0; i < c.workers; ++i) {
        Workspace *ws = new (std::nothrow) Workspace();
        cudaStream_t st = nullptr;
        if (!ws || ws->pin_s.ensure(65536) != cudaSuccess ||
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete ws;
            probesim_server_destroy(s);
            return ps::fail_status(PROBESIM_E_NOMEM, "server workspace allocation failed");
        }
        ws->budget = (size_t)(c.memory_budget_bytes / c.workers);  // the workers' calls share the budget
        s->ws.push_back(ws);
        s->streams.push_back(st);
    }
    for (int i = 0; i < c.workers; ++i) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return PROBESIM_OK;
}

probesim_status probesim_server_submit(probesim_server *s, const probesim_query *q, int32_t nq, uint64_t *tickets) {
    if (!s || !q || nq < 1) return ps::fail_status(PROBESIM_E_INVALID, "null argument or nq < 1");
    probesim_status rc = ps::check_queries(s->g, q, nq, true, s->cfg.kmax);
    if (rc != PROBESIM_OK) return rc;
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queued_queries + nq > s->cfg.queue_capacity) {
            s->rejected += nq;
            return ps::fail_status(PROBESIM_E_BUSY, "server queue full");
        }
        if (!s->any_submit) {
            s->first_submit = now;
            s->any_submit = true;
        }
        for (int32_t i = 0; i < nq; ++i) {
            Request r;
            r.q = q[i];
            r.ticket = s->next_ticket++;
            r.submitted = now;
            if (tickets) tickets[i] = r.ticket;
            s->fifo.push_back(std::move(r));
        }
        s->queued_queries += nq;
        s->submitted += nq;
    }
    s->cv_work.notify_all();
    return PROBESIM_OK;
}

probesim_status probesim_server_update(probesim_server *s, const int32_t *src, const int32_t *dst, int64_t k,
                                       int32_t insert) {
    if (!s || k < 0 || (k > 0 && (!src || !dst))) return ps::fail_status(PROBESIM_E_INVALID, "bad update batch");
    const int32_t n = s->g->n;
    Request r;
    r.is_update = true;
    r.insert = insert != 0;
    r.src.assign(src, src + k);
    r.dst.assign(dst, dst + k);
    for (int64_t e = 0; e < k; ++e)
        if (r.src[e] < 0 || r.src[e] >= n || r.dst[e] < 0 || r.dst[e] >= n)
            return ps::fail_status(PROBESIM_E_RANGE, "edge id outside [0, n)");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->fifo.push_back(std::move(r));
    }
    s->cv_work.notify_all();
    return PROBESIM_OK;
}

probesim_status probesim_server_poll(probesim_server *s, int32_t max_results, int32_t kmax, probesim_result *res,
                                     int32_t *ids, float *vals, int32_t *count, int32_t wait_ms) {
    if (!s || !res || !ids || !vals || !count || max_results < 1 || kmax < 1)
        return ps::fail_status(PROBESIM_E_INVALID, "null argument or bad size");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int32_t c = 0;
    while (c < max_results && !s->done.empty()) {
        Done &d = s->done.front();
        res[c] = d.r;
        const int32_t kk = std::min(kmax, s->cfg.kmax);
        for (int32_t i = 0; i < kmax; ++i) {
            ids[(int64_t)c * kmax + i] = i < kk ? d.ids[i] : -1;
            vals[(int64_t)c * kmax + i] = i < kk ? d.vals[i] : 0.f;
        }
        s->done.pop_front();
        ++c;
    }
    *count = c;
    return PROBESIM_OK;
}

probesim_status probesim_server_get_stats(probesim_server *s, probesim_server_stats *out) {
    if (!s || !out) return ps::fail_status(PROBESIM_E_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->failed = s->failed;
    out->batches = s->batches;
    out->updates_applied = s->updates_applied;
    out->mean_batch = s->batches ? s->batch_queries / (double)s->batches : 0.0;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        auto pct = [&](double p) {
            const size_t i = std::min(l.size() - 1, (size_t)(p * (double)(l.size() - 1) + 0.5));
            std::nth_element(l.begin(), l.begin() + i, l.end());
            return l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : s->latencies) sum += x;
        out->mean_ms = sum / (double)s->latencies.size();
        const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        out->qps = span > 0 ? (double)s->completed / span : 0.0;
    }
    return PROBESIM_OK;
}

probesim_status probesim_server_destroy(probesim_server *s) {
    if (!s) return PROBESIM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread &t : s->workers)
        if (t.joinable()) t.join();
    for (size_t i = 0; i < s->ws.size(); ++i) {
        if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
        s->ws[i]->release();
        delete s->ws[i];
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    }
    delete s;
    return PROBESIM_OK;
}

}  // extern "C"
