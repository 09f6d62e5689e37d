// C ABI of libprobesim.so: the graph store, the query engine and the entry points of include/probesim.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <shared_mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine.cuh"

using namespace ps;

// ------------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

void ps::set_last_error(const char *msg) { g_last_error = msg; }

static probesim_status fail(probesim_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

probesim_status ps::fail_status(probesim_status st, const std::string &msg) { return fail(st, msg); }

#define PS_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            return fail(_e == cudaErrorMemoryAllocation ? PROBESIM_E_NOMEM : PROBESIM_E_CUDA,          \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                           \
        }                                                                                              \
    } while (0)

// an allocation of one walk range's buffers in the randomized PROBE: when it fails, the range is split
#define PS_ALLOC_RANGE(expr)                                                                           \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            cudaGetLastError();                                                                        \
            *too_big = true;                                                                           \
            return fail(PROBESIM_E_NOMEM, std::string(#expr) + ": " + cudaGetErrorString(_e));         \
        }                                                                                              \
    } while (0)

// an allocation of a batch's working buffers: when it fails on a call of several queries, the caller splits it
#define PS_ALLOC(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            cudaGetLastError();                                                                        \
            *too_big = B > 1;                                                                          \
            return fail(PROBESIM_E_NOMEM, std::string(#expr) + ": " + cudaGetErrorString(_e));         \
        }                                                                                              \
    } while (0)

#define PS_TRY(expr)                                  \
    do {                                              \
        probesim_status _s = (expr);                  \
        if (_s != PROBESIM_OK) return _s;             \
    } while (0)

static uint32_t threshold_stop(double c) { return (uint32_t)std::floor((1.0 - std::sqrt(c)) * 4294967296.0); }
static uint32_t threshold_keep(double c) {
    const double t = std::floor(std::sqrt(c) * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

static int64_t num_walks(double c, double eps, double delta, int64_t n) {
    return (int64_t)std::ceil(3.0 * c / (eps * eps) * std::log((double)n / delta));
}

int64_t ps::num_walks_for(const probesim_graph *g, double eps) { return num_walks(g->cfg.c, eps, g->cfg.delta, g->n); }

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------------------------------------
// graph store
// ------------------------------------------------------------------------------------------------

// Builds the device graph store from the caller's edge list (device arrays of the caller's ids) with the kernels
// of graph_build.cu and publishes it as the first version.  Repeated edges and loops are dropped.  Internally nodes
// are renumbered by descending out-degree (ties by the caller's id): the pull kernel gathers score rows of
// in-neighbours, which are mostly high-out-degree nodes, so their rows become contiguous and stay cached.  I(v)
// keeps the caller's source-id order (walks pick the k-th entry of that order) but holds internal ids; O(x) holds
// internal ids in ascending order; ext2int / int2ext map at the boundary.
static probesim_status build_graph(probesim_graph *g, int32_t n, const int32_t *d_src, const int32_t *d_dst, int64_t m,
                                   cudaStream_t st) {
    struct Scratch {  // the build's temporaries, freed on every return
        DevBuf ka, kb, kc, cnt, off, part, ext_off, outdeg, rka, rkb, indeg_i, outdeg_i, hist, flag;
        ~Scratch() {
            for (DevBuf *b : {&ka, &kb, &kc, &cnt, &off, &part, &ext_off, &outdeg, &rka, &rkb, &indeg_i, &outdeg_i,
                              &hist, &flag})
                b->release();
        }
    } t;
    auto bitlen = [](uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; };
    const int bs = std::max(1, bitlen((uint64_t)std::max(1, n - 1)));  // bits of a node id
    const uint32_t smask = (uint32_t)(((uint64_t)1 << bs) - 1);
    const uint64_t end_key = (uint64_t)(uint32_t)n << bs;
    const int64_t M = std::max<int64_t>(1, m);
    const int64_t big = std::max<int64_t>(M, n);
    const int64_t ntiles = radix_tiles(big);
    PS_CUDA(t.ka.ensure(8 * (size_t)(M + 1)));
    PS_CUDA(t.kb.ensure(8 * (size_t)(M + 1)));
    PS_CUDA(t.cnt.ensure(8 * (size_t)(256 * ntiles)));
    PS_CUDA(t.off.ensure(8 * (size_t)(256 * ntiles + 1)));
    PS_CUDA(t.part.ensure(8 * (size_t)scan64_partials_needed(std::max<int64_t>(256 * ntiles, big + 1))));
    PS_CUDA(t.flag.ensure(sizeof(int32_t)));
    long long *cnt = t.cnt.as<long long>(), *off = t.off.as<long long>(), *part = t.part.as<long long>();
    // 1-3: sorted unique edge keys (dst << bs | src, caller's ids)
    PS_CUDA(cudaMemsetAsync(t.flag.p, 0, sizeof(int32_t), st));
    launch_build_keys(d_src, d_dst, m, n, bs, t.ka.as<uint64_t>(), t.flag.as<int32_t>(), st);
    int32_t bad = 0;
    PS_CUDA(cudaMemcpyAsync(&bad, t.flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(PROBESIM_E_RANGE, "edge id outside [0, n)");
    uint64_t *sorted = radix_sort_u64(t.ka.as<uint64_t>(), t.kb.as<uint64_t>(), m, bs + bitlen(n), cnt, off, part, st);
    long long *pre = reinterpret_cast<long long *>(sorted == t.ka.as<uint64_t>() ? t.kb.p : t.ka.p);
    launch_build_flags(sorted, m, end_key, pre, st);
    launch_scan64(pre, m, part, pre, st);  // in place: pre[m] = the number of distinct edges
    long long mu_ll = 0;
    PS_CUDA(cudaMemcpyAsync(&mu_ll, pre + std::max<int64_t>(0, m), sizeof(long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t mu = m > 0 ? (int64_t)mu_ll : 0;
    PS_CUDA(t.kc.ensure(8 * (size_t)std::max<int64_t>(1, mu)));
    uint64_t *ukeys = t.kc.as<uint64_t>();
    launch_build_compact(sorted, m, end_key, pre, ukeys, st);
    // 4: in-list offsets and out-degrees by caller id, then the renumbering
    PS_CUDA(t.ext_off.ensure(8 * ((size_t)n + 1)));
    PS_CUDA(t.outdeg.ensure(8 * (size_t)n));
    PS_CUDA(t.rka.ensure(8 * (size_t)n));
    PS_CUDA(t.rkb.ensure(8 * (size_t)n));
    PS_CUDA(t.indeg_i.ensure(8 * (size_t)n));
    PS_CUDA(t.outdeg_i.ensure(8 * (size_t)n));
    long long *ext_off = t.ext_off.as<long long>();
    unsigned long long *outdeg = t.outdeg.as<unsigned long long>();
    PS_CUDA(cudaMemsetAsync(outdeg, 0, 8 * (size_t)n, st));
    launch_build_ext_off(ukeys, mu, n, bs, ext_off, st);
    launch_build_outdeg(ukeys, mu, smask, outdeg, st);
    launch_build_rank_keys(outdeg, n, mu, bs, t.rka.as<uint64_t>(), st);
    const uint64_t *rk =
        radix_sort_u64(t.rka.as<uint64_t>(), t.rkb.as<uint64_t>(), n, bs + bitlen((uint64_t)mu), cnt, off, part, st);
    PS_CUDA(g->ext2int.ensure(sizeof(int32_t) * n));
    PS_CUDA(g->int2ext.ensure(sizeof(int32_t) * n));
    launch_build_perm(rk, n, smask, ext_off, outdeg, g->int2ext.as<int32_t>(), g->ext2int.as<int32_t>(),
                      t.indeg_i.as<long long>(), t.outdeg_i.as<long long>(), st);
    // 5: the CSR arrays in internal ids
    auto sv = std::make_shared<StoreVersion>();
    PS_CUDA(sv->in_off.ensure(sizeof(int64_t) * ((size_t)n + 1)));
    PS_CUDA(sv->out_off.ensure(sizeof(int64_t) * ((size_t)n + 1)));
    PS_CUDA(sv->in_col.ensure(sizeof(int32_t) * std::max<int64_t>(1, mu)));
    PS_CUDA(sv->out_col.ensure(sizeof(int32_t) * std::max<int64_t>(1, mu)));
    launch_scan64(t.indeg_i.as<long long>(), n, part, sv->in_off.as<long long>(), st);
    launch_scan64(t.outdeg_i.as<long long>(), n, part, sv->out_off.as<long long>(), st);
    uint64_t *okeys = t.ka.as<uint64_t>();  // the edge-key buffers are free again (the unique keys live in kc)
    launch_build_in_col(n, g->int2ext.as<int32_t>(), ext_off, sv->in_off.as<int64_t>(), ukeys, smask,
                        g->ext2int.as<int32_t>(), bs, sv->in_col.as<int32_t>(), okeys, st);
    const uint64_t *osorted = radix_sort_u64(okeys, t.kb.as<uint64_t>(), mu, 2 * bs, cnt, off, part, st);
    launch_build_out_col(osorted, mu, smask, sv->out_col.as<int32_t>(), st);
    // w and the pull pieces (in-lists cut into at most kPiece edges, longest first)
    const int64_t cap_pieces = (int64_t)n + mu / kPiece + 1;
    PS_CUDA(sv->w.ensure(sizeof(float) * n));
    PS_CUDA(sv->piece_v.ensure(sizeof(int32_t) * cap_pieces));
    PS_CUDA(sv->piece_beg.ensure(sizeof(int64_t) * cap_pieces));
    PS_CUDA(sv->piece_len.ensure(sizeof(int32_t) * cap_pieces));
    PS_CUDA(sv->split_v.ensure(sizeof(int32_t) * (size_t)n));
    PS_CUDA(t.hist.ensure(sizeof(unsigned long long) * (2 * (kPiece + 1) + 2)));
    launch_upd_w(n, sv->in_off.as<long long>(), (float)std::sqrt(g->cfg.c), sv->w.as<float>(),
                 t.indeg_i.as<long long>(), st);
    unsigned long long *hist = t.hist.as<unsigned long long>(), *cursor = hist + (kPiece + 1),
                       *nsplit = cursor + (kPiece + 1);
    launch_upd_pieces(n, sv->in_off.as<long long>(), hist, cursor, sv->split_v.as<int32_t>(), nsplit,
                      sv->piece_v.as<int32_t>(), sv->piece_beg.as<int64_t>(), sv->piece_len.as<int32_t>(), st);
    std::vector<unsigned long long> hh(kPiece + 2);
    long long ends[2] = {0, 0};
    int32_t n_active = 0;
    PS_CUDA(cudaMemsetAsync(t.flag.p, 0, sizeof(int32_t), st));
    launch_active_rows(sv->out_off.as<int64_t>(), n, t.flag.as<int32_t>(), st);
    PS_CUDA(cudaMemcpyAsync(&n_active, t.flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned long long) * (kPiece + 1), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(hh.data() + kPiece + 1, nsplit, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&ends[0], sv->in_off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&ends[1], sv->out_off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
    g->h_ext2int.resize(n);
    PS_CUDA(cudaMemcpyAsync(g->h_ext2int.data(), g->ext2int.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaStreamSynchronize(st));
    if (ends[0] != mu || ends[1] != mu) return fail(PROBESIM_E_CUDA, "internal: the built lists disagree on m");
    int64_t npieces = 0;
    for (int len = 0; len <= kPiece; ++len) npieces += (int64_t)hh[len];
    DeviceGraph &d = sv->dg;
    d.n = n;
    d.m = mu;
    d.in_off = sv->in_off.as<int64_t>();
    d.in_col = sv->in_col.as<int32_t>();
    d.out_off = sv->out_off.as<int64_t>();
    d.out_col = sv->out_col.as<int32_t>();
    d.w = sv->w.as<float>();
    d.n_pieces = npieces;
    d.piece_v = sv->piece_v.as<int32_t>();
    d.piece_beg = sv->piece_beg.as<int64_t>();
    d.piece_len = sv->piece_len.as<int32_t>();
    d.n_split = (int32_t)hh[kPiece + 1];
    d.n_active = n_active;
    d.split_v = sv->split_v.as<int32_t>();
    d.ext2int = g->ext2int.as<int32_t>();
    d.int2ext = g->int2ext.as<int32_t>();
    g->n = n;
    g->publish(sv);
    return PROBESIM_OK;
}

// Device memory one call on workspace ws may take (a server gives each worker a share of the graph's budget).
static size_t budget_of(const probesim_graph *g, const Workspace *ws) {
    return ws->budget ? ws->budget : g->budget.load();
}

// Copies an int32 array that may live on the device to the host.
static probesim_status fetch_ids(const int32_t *p, int64_t k, std::vector<int32_t> &out) {
    out.resize(std::max<int64_t>(1, k));
    if (k == 0) return PROBESIM_OK;
    if (is_device_ptr(p)) {
        PS_CUDA(cudaMemcpy(out.data(), p, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), p, sizeof(int32_t) * k);
    }
    return PROBESIM_OK;
}

// ------------------------------------------------------------------------------------------------
// query engine
// ------------------------------------------------------------------------------------------------
struct BatchPlan {
    int32_t B = 0, W = 0;
    std::vector<int32_t> node, base, k0;
    std::vector<uint32_t> qid;
    std::vector<float> inv_nr;
};

static probesim_status plan_batch(probesim_graph *g, const probesim_query *q, int32_t B, BatchPlan &P) {
    P.B = B;
    P.node.resize(B);
    P.base.resize(B + 1);
    P.k0.resize(B);
    P.qid.resize(B);
    P.inv_nr.resize(B);
    int64_t W = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t nr = num_walks(g->cfg.c, q[b].eps, g->cfg.delta, g->n);
        const int64_t kb = std::max<int64_t>(0, q[b].walk_begin);
        const int64_t ke = q[b].walk_end <= 0 ? nr : std::min<int64_t>(q[b].walk_end, nr);
        P.node[b] = q[b].node;
        P.qid[b] = q[b].query_id;
        P.k0[b] = (int32_t)std::min(kb, ke);
        P.base[b] = (int32_t)W;
        W += std::max<int64_t>(0, ke - kb);
        P.inv_nr[b] = (float)(1.0 / (double)nr);
        if (W > (int64_t)1 << 30) return fail(PROBESIM_E_INVALID, "too many walks in one call");
    }
    P.base[B] = (int32_t)W;
    P.W = (int32_t)W;
    return PROBESIM_OK;
}

// Uploads the batch arrays; returns the device view.
static probesim_status upload_batch(Workspace *ws, const BatchPlan &P, QueryBatch &qb, cudaStream_t st) {
    const int32_t B = P.B;
    const size_t bytes = sizeof(int32_t) * (4 * (size_t)B + 1) + sizeof(float) * B + 64;
    PS_CUDA(ws->pin_q.ensure(bytes));
    PS_CUDA(ws->qbuf.ensure(bytes));
    char *h = ws->pin_q.as<char>();
    int32_t *hn = reinterpret_cast<int32_t *>(h);
    std::memcpy(hn, P.node.data(), sizeof(int32_t) * B);
    std::memcpy(hn + B, P.qid.data(), sizeof(uint32_t) * B);
    std::memcpy(hn + 2 * B, P.base.data(), sizeof(int32_t) * (B + 1));
    std::memcpy(hn + 3 * B + 1, P.k0.data(), sizeof(int32_t) * B);
    std::memcpy(hn + 4 * B + 1, P.inv_nr.data(), sizeof(float) * B);
    PS_CUDA(cudaMemcpyAsync(ws->qbuf.p, h, bytes, cudaMemcpyHostToDevice, st));
    int32_t *d = ws->qbuf.as<int32_t>();
    qb.B = B;
    qb.node = d;
    qb.qid = reinterpret_cast<const uint32_t *>(d + B);
    qb.walk_base = d + 2 * B;
    qb.walk_k0 = d + 3 * B + 1;
    qb.inv_nr = reinterpret_cast<const float *>(d + 4 * B + 1);
    return PROBESIM_OK;
}

static int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct Timer {
    Workspace *ws;
    cudaStream_t st;
    size_t used = 0;
    cudaEvent_t get() {
        if (used == ws->ev.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ws->ev.push_back(e);
        }
        return ws->ev[used++];
    }
};

// Brackets groups of launches with events when profiling is on; times are summed per phase after the
// batch's final synchronisation.
struct PhaseTimer {
    Timer *tm;
    bool on;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    int cur = -1;
    cudaEvent_t e0 = nullptr;
    void begin(int phase) {
        if (!on) return;
        cur = phase;
        e0 = tm->get();
        cudaEventRecord(e0, tm->st);
    }
    void end() {
        if (!on || cur < 0) return;
        cudaEvent_t e1 = tm->get();
        cudaEventRecord(e1, tm->st);
        marks.push_back({cur, {e0, e1}});
        cur = -1;
    }
    void collect(probesim_stats &st) {
        for (auto &m : marks) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, m.second.first, m.second.second) == cudaSuccess) st.phase_ms[m.first] += ms;
        }
    }
};

// Runs the query path for one batch into d_out ([B][n] on the device).  Returns PROBESIM_E_NOMEM with
// *too_big set when the level buffers of this batch would exceed the workspace budget.
static probesim_status run_batch(probesim_graph *g, Workspace *ws, const probesim_query *q, int32_t B, float *d_out,
                                 cudaStream_t st, bool *too_big) {
    *too_big = false;
    const DeviceGraph &dg = ws->dg;
    const int32_t n = dg.n;
    const int32_t L = g->cfg.l_max;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, B, P));
    if ((size_t)P.W * L * 4 > budget_of(g, ws) / 4 && B > 1) {
        *too_big = true;
        return PROBESIM_E_NOMEM;
    }
    QueryBatch qb;
    PS_TRY(upload_batch(ws, P, qb, st));
    int64_t launches = 0;
    Timer tm{ws, st};
    PhaseTimer ph{&tm, ws->profiling != 0};
    // 1. walks (Def. 3)
    PS_CUDA(ws->walks.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_CUDA(ws->lens.ensure(sizeof(int32_t) * std::max<int32_t>(1, P.W)));
    PS_CUDA(ws->ctr.ensure(sizeof(LaunchCounters)));
    LaunchCounters *d_ctr = ws->ctr.as<LaunchCounters>();
    PS_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(LaunchCounters), st));
    ph.begin(0);
    launch_walks(dg, qb, P.W, L, g->t_stop, g->cfg.seed, ws->walks.as<int32_t>(), ws->lens.as<int32_t>(), false, d_ctr, st);
    ph.end();
    ++launches;
    LaunchCounters *h_ctr = ws->pin_s.as<LaunchCounters>();
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t walk_nodes = (int64_t)h_ctr->walk_nodes;
    ws->stats.walks += P.W;
    ws->stats.walk_nodes += walk_nodes;
    // 2. reverse-reachability tree (Alg. 4) in a hash table at load <= 1/2
    TrieTable t;
    t.cap = next_pow2(std::max<int64_t>(1024, 2 * (walk_nodes + B) + 64));
    const size_t cap = (size_t)t.cap;
    PS_CUDA(ws->t_key.ensure(8 * cap));
    PS_CUDA(ws->t_node.ensure(4 * cap));
    PS_CUDA(ws->t_parent.ensure(4 * cap));
    PS_CUDA(ws->t_depth.ensure(4 * cap));
    PS_CUDA(ws->t_query.ensure(4 * cap));
    PS_CUDA(ws->t_weight.ensure(4 * cap));
    PS_CUDA(ws->t_height.ensure(4 * cap));
    PS_CUDA(ws->t_slot.ensure(4 * cap));
    PS_CUDA(ws->t_gamma.ensure(4 * cap));
    PS_CUDA(ws->t_G.ensure(4 * cap));
    t.key = ws->t_key.as<unsigned long long>();
    t.node = ws->t_node.as<int32_t>();
    t.parent = ws->t_parent.as<int32_t>();
    t.depth = ws->t_depth.as<int32_t>();
    t.query = ws->t_query.as<int32_t>();
    t.weight = ws->t_weight.as<int32_t>();
    t.height = ws->t_height.as<int32_t>();
    t.slot = ws->t_slot.as<int32_t>();
    t.gamma = ws->t_gamma.as<float>();
    t.G = ws->t_G.as<float>();
    ph.begin(1);
    PS_CUDA(cudaMemsetAsync(t.key, 0xFF, 8 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.weight, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.height, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.G, 0, 4 * cap, st));
    launch_trie_insert(dg, qb, P.W, L, ws->walks.as<int32_t>(), ws->lens.as<int32_t>(), t, d_ctr, st);
    ++launches;
    // 3. level schedule: nodes, dense columns (pulled) and push columns per depth
    const int32_t D1 = L + 2;
    PS_CUDA(ws->counts.ensure(sizeof(int32_t) * 5 * D1));
    int32_t *d_ncount = ws->counts.as<int32_t>(), *d_scount = d_ncount + D1, *d_hcount = d_ncount + 2 * D1,
            *d_ncur = d_ncount + 3 * D1;
    PS_CUDA(cudaMemsetAsync(d_ncount, 0, sizeof(int32_t) * 4 * D1, st));
    launch_sched_count(t, d_ncount, d_scount, d_hcount, st);
    ph.end();
    ++launches;
    int32_t *h_cnt = reinterpret_cast<int32_t *>(ws->pin_s.as<char>() + 256);
    PS_CUDA(cudaMemcpyAsync(h_cnt, d_ncount, sizeof(int32_t) * 3 * D1, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (h_ctr->overflow) return fail(PROBESIM_E_CUDA, "internal: walk tree table overflow");
    std::vector<int32_t> ncount(h_cnt, h_cnt + D1), scount(h_cnt + D1, h_cnt + 2 * D1),
        hcount(h_cnt + 2 * D1, h_cnt + 3 * D1);
    int32_t Dmax = 0;
    for (int32_t d = 0; d < D1; ++d)
        if (ncount[d] > 0) Dmax = d;
    std::vector<int32_t> node_off(D1 + 1, 0), dw(D1, 0);
    for (int32_t d = 0; d < D1; ++d) node_off[d + 1] = node_off[d] + ncount[d];
    const int32_t total_nodes = node_off[D1];
    ws->stats.tree_nodes += total_nodes;
    for (int32_t d = 0; d < D1; ++d) ws->stats.vectors += scount[d] + hcount[d];
    PS_CUDA(ws->offs.ensure(sizeof(int32_t) * (D1 + 1)));
    int32_t *d_node_off = ws->offs.as<int32_t>();
    int32_t *h_offs = h_cnt + 3 * D1;
    std::memcpy(h_offs, node_off.data(), sizeof(int32_t) * (D1 + 1));
    PS_CUDA(cudaMemcpyAsync(d_node_off, h_offs, sizeof(int32_t) * (D1 + 1), cudaMemcpyHostToDevice, st));
    PS_CUDA(ws->node_list.ensure(sizeof(int32_t) * std::max(1, total_nodes)));
    ph.begin(1);
    launch_node_lists(t, d_node_off, d_ncur, ws->node_list.as<int32_t>(), st);
    // columns.  Every dense node's "heir" (its dense child with the deepest chain below it) takes over its
    // column one depth down, so along a chain of heirs the MD column of the child already is the D column of
    // the parent and nothing is copied.  Push columns (height 2) sit in a block after the dense columns.
    int32_t ncol_nodes = 0;
    for (int32_t d = 0; d < D1; ++d) ncol_nodes += scount[d] + hcount[d];
    PS_CUDA(ws->col_export.ensure(sizeof(int32_t) * (5 * (size_t)std::max(1, ncol_nodes) + 1)));
    int32_t *d_exp = ws->col_export.as<int32_t>(), *d_expn = d_exp + 5 * (size_t)std::max(1, ncol_nodes);
    PS_CUDA(cudaMemsetAsync(d_expn, 0, sizeof(int32_t), st));
    launch_sched_export(t, d_exp, d_expn, st);
    ph.end();
    launches += 2;
    PS_CUDA(ws->pin_q.ensure(sizeof(int32_t) * (5 * (size_t)std::max(1, ncol_nodes) + 64)));
    int32_t *h_exp = ws->pin_q.as<int32_t>();
    PS_CUDA(cudaMemcpyAsync(h_exp, d_exp, sizeof(int32_t) * 5 * (size_t)ncol_nodes, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const auto host0 = std::chrono::steady_clock::now();  // the host-side schedule starts (the device waits)
    // export rows: 0 entry, 1 depth, 2 parent entry, 3 dense, 4 query
    std::vector<std::vector<int32_t>> dense_at(D1), push_at(D1);
    for (int32_t i = 0; i < ncol_nodes; ++i) (h_exp[5 * i + 3] ? dense_at : push_at)[h_exp[5 * i + 1]].push_back(i);
    // the export row of every node's parent (-1: none).  Tree entries are slots of the table, so a flat array
    // indexes them unless the table is much larger than the exported set
    std::vector<int32_t> prow(ncol_nodes, -1);
    if (t.cap <= 32 * (int64_t)ncol_nodes + 65536) {
        std::vector<int32_t> row_of((size_t)t.cap, -1);
        for (int32_t i = 0; i < ncol_nodes; ++i) row_of[h_exp[5 * i]] = i;
        for (int32_t i = 0; i < ncol_nodes; ++i) {
            const int32_t pe = h_exp[5 * i + 2];
            if (pe >= 0) prow[i] = row_of[pe];
        }
    } else {
        std::unordered_map<int32_t, int32_t> row_of;
        row_of.reserve(2 * (size_t)ncol_nodes + 1);
        for (int32_t i = 0; i < ncol_nodes; ++i) row_of[h_exp[5 * i]] = i;
        for (int32_t i = 0; i < ncol_nodes; ++i) {
            const auto it = row_of.find(h_exp[5 * i + 2]);
            if (it != row_of.end()) prow[i] = it->second;
        }
    }
    // heights are not exported; the heir is the dense child with the deepest dense descendant chain, found
    // bottom-up, ties to the smaller entry
    std::vector<int32_t> chain(ncol_nodes, 0), heir(ncol_nodes, -1), col(ncol_nodes, -1);
    for (int32_t d = Dmax; d >= 1; --d)
        for (int32_t i : dense_at[d]) {
            const int32_t pr = prow[i];
            if (pr < 0) continue;
            const int32_t h = heir[pr];
            if (h < 0 || chain[i] > chain[h] || (chain[i] == chain[h] && h_exp[5 * i] < h_exp[5 * h])) heir[pr] = i;
            chain[pr] = std::max(chain[pr], chain[i] + 1);
        }
    // a dense node without a dense heir takes its first push child (smallest entry) as "push heir": that
    // child's pushed column is then the node's D column, in place, and the accumulate has nothing to copy
    std::vector<int32_t> pheir(ncol_nodes, -1);
    for (int32_t d = 1; d <= Dmax; ++d)
        for (int32_t i : push_at[d]) {
            const int32_t pr = prow[i];
            if (pr < 0 || heir[pr] >= 0) continue;
            if (pheir[pr] < 0 || h_exp[5 * i] < h_exp[5 * pheir[pr]]) pheir[pr] = i;
        }
    std::vector<char> is_pheir(ncol_nodes, 0);
    for (int32_t i = 0; i < ncol_nodes; ++i)
        if (pheir[i] >= 0) is_pheir[pheir[i]] = 1;
    // a chain is a maximal path of heirs (ending, possibly, in a push heir); all its nodes share one column.
    // Chains are coloured deepest bottom
    // first, each taking the smallest column whose chains all start more than one depth below its bottom
    // (every chain coloured before it ends at least as deep, so that is "free over its depth range and the
    // depth below"); the columns in use at a depth then stay close to the number of dense nodes there.
    std::vector<char> is_heir(ncol_nodes, 0);
    for (int32_t i = 0; i < ncol_nodes; ++i)
        if (heir[i] >= 0) is_heir[heir[i]] = 1;
    struct Chain {
        int32_t head, top, bottom;
    };
    std::vector<Chain> chains;
    for (int32_t d = 0; d <= Dmax; ++d)
        for (int32_t i : dense_at[d]) {
            if (is_heir[i]) continue;
            int32_t x = i, bot = d;
            while (heir[x] >= 0) x = heir[x], ++bot;
            if (pheir[x] >= 0) ++bot;
            chains.push_back({i, d, bot});
        }
    std::sort(chains.begin(), chains.end(), [&](const Chain &x, const Chain &y) {
        if (x.bottom != y.bottom) return x.bottom > y.bottom;
        if (x.top != y.top) return x.top < y.top;
        return h_exp[5 * x.head] < h_exp[5 * y.head];
    });
    // per column: the smallest top depth of the chains holding it, kept in a max segment tree over the
    // columns (columns not opened yet hold INT32_MAX) so the first column above a depth is found in log time
    int32_t seg_leaves = 1;
    while (seg_leaves < std::max<int32_t>(1, (int32_t)chains.size())) seg_leaves <<= 1;
    std::vector<int32_t> top_min(2 * (size_t)seg_leaves, INT32_MAX);
    for (const Chain &ch : chains) {
        // a column whose chain ends at depth d stays unused at depth d+1 too: there the accumulate sets it to
        // the chain bottom's D, while other groups may still read what a chain starting at d+1 left in it.
        // The chain takes the first column all of whose chains start below ch.bottom + 1.
        int32_t i = 1;
        while (i < seg_leaves) i = top_min[2 * i] > ch.bottom + 1 ? 2 * i : 2 * i + 1;
        const int32_t c = i - seg_leaves;
        top_min[i] = std::min(top_min[i], ch.top);
        for (i >>= 1; i >= 1; i >>= 1) top_min[i] = std::max(top_min[2 * i], top_min[2 * i + 1]);
        int32_t last = ch.head;
        for (int32_t x = ch.head; x >= 0; x = heir[x]) col[x] = c, last = x;
        if (pheir[last] >= 0) col[pheir[last]] = c;
    }
    std::vector<int32_t> width(D1, 0), rho(B, -1);
    for (int32_t d = 0; d <= Dmax; ++d) {
        int32_t w = 0;
        for (int32_t i : dense_at[d]) w = std::max(w, col[i] + 1);
        width[d] = w;
        if (d == 0)
            for (int32_t i : dense_at[0]) rho[h_exp[5 * i + 4]] = col[i];
    }
    // pull tiles per depth: full 32-column tiles (or 16-column halves, if the tuner prefers them) and one
    // narrower tail tile of 1..16 columns; dw = the columns the pull covers
    std::vector<int32_t> nfull(D1, 0), tail(D1, 0);
    for (int32_t d = 0; d <= Dmax; ++d) {
        int32_t full = width[d] / 32, rem = width[d] - 32 * full;
        if (rem > 16) ++full, rem = 0;
        nfull[d] = full;
        tail[d] = rem > 0 ? pull_tile_for(rem, 16) : 0;
        dw[d] = 32 * full + tail[d];
    }
    // push nodes of a depth that keep a column of their own (the others inherited their parent's)
    std::vector<int32_t> hinh(D1, 0);
    for (int32_t d = 0; d <= Dmax; ++d) {
        std::vector<int32_t> &pa = push_at[d];
        const size_t before = pa.size();
        pa.erase(std::remove_if(pa.begin(), pa.end(), [&](int32_t x) { return is_pheir[x] != 0; }), pa.end());
        hinh[d] = (int32_t)(before - pa.size());
    }
    // MD of depth d is read in place as D of depth d-1, so its matrix holds the columns of both depths:
    // max(dw[d-1], dw[d]) dense columns (inherited push columns among them), then the push block at h0[d]
    std::vector<int32_t> h0v(D1, 0), rpv(D1, 0);
    std::vector<ColLayout> lay(D1);
    int64_t max_floats = 4 * (int64_t)n;
    for (int32_t d = 0; d <= Dmax; ++d) {
        const int32_t dense_w = std::max(dw[d], d >= 1 ? dw[d - 1] : 0);
        h0v[d] = round_up(std::max(dense_w, 1), 4);
        rpv[d] = round_up(h0v[d] + (int32_t)push_at[d].size(), 4);
        lay[d] = make_layout(n, rpv[d]);
        max_floats = std::max<int64_t>(max_floats, lay[d].size());
        ws->stats.max_columns = std::max<int64_t>(ws->stats.max_columns, rpv[d]);
    }
    // push columns of a depth: grouped by parent (in parent column order), so a parent's push children are
    // adjacent for the accumulate
    for (int32_t d = 0; d <= Dmax; ++d) {
        std::vector<int32_t> &pa = push_at[d];
        auto pcol = [&](int32_t x) { return d >= 1 && prow[x] >= 0 ? col[prow[x]] : -1; };
        std::sort(pa.begin(), pa.end(), [&](int32_t x, int32_t y) {
            const int32_t px = pcol(x), py = pcol(y);
            return px != py ? px < py : h_exp[5 * x] < h_exp[5 * y];
        });
        for (size_t r = 0; r < pa.size(); ++r) col[pa[r]] = h0v[d] + (int32_t)r;
    }
    const size_t level_bytes2 = 2 * (size_t)max_floats * sizeof(float);
    if (level_bytes2 > budget_of(g, ws)) {
        *too_big = B > 1;
        return fail(PROBESIM_E_NOMEM, "score vectors of one query exceed the workspace budget");
    }
    // accumulate groups per depth d (dense parents at d): dst = parent column (| set flag when it has no heir
    // of either kind), srcs = columns (at d+1) of its children other than the heir
    std::vector<std::vector<int32_t>> kids(ncol_nodes);
    for (int32_t i = 0; i < ncol_nodes; ++i) {
        const int32_t pr = prow[i];
        if (pr >= 0 && heir[pr] != i && pheir[pr] != i) kids[pr].push_back(col[i]);
    }
    // Each group is cut into parts of at most four sources, stored as a destination (bit 30: set, for a node
    // without heir) and an int4 of sources (-1 = none).  The first part of every group runs in the
    // accumulate's first phase, the others add in a second phase (so one node with many children does not
    // hold up a block).  Records of depth d: first parts [p1_at[d], p1_at[d+1]), later parts likewise.
    std::vector<int32_t> pairs, p1dst, p1src, p2dst, p2src, p1_at(D1 + 1, 0), p2_at(D1 + 1, 0);
    pairs.reserve(2 * (size_t)ncol_nodes);
    for (int32_t i = 0; i < ncol_nodes; ++i) {
        pairs.push_back(h_exp[5 * i]);
        pairs.push_back(col[i]);
    }
    auto put_part = [](std::vector<int32_t> &dst, std::vector<int32_t> &src, int32_t dcol, const std::vector<int32_t> &k,
                       size_t from) {
        dst.push_back(dcol);
        for (size_t j = 0; j < 4; ++j) src.push_back(from + j < k.size() ? k[from + j] : -1);
    };
    for (int32_t d = 0; d < D1; ++d) {
        p1_at[d] = (int32_t)p1dst.size();
        p2_at[d] = (int32_t)p2dst.size();
        if (d > Dmax) continue;
        // groups in destination order, sources ascending
        std::sort(dense_at[d].begin(), dense_at[d].end(), [&](int32_t x, int32_t y) { return col[x] < col[y]; });
        for (int32_t i : dense_at[d]) {
            std::sort(kids[i].begin(), kids[i].end());
            const bool own = heir[i] < 0 && pheir[i] < 0;  // no heir of any kind: the column is set
            if (kids[i].empty() && !own) continue;            // its column already is its heir's MD
            put_part(p1dst, p1src, col[i] | (own ? (1 << 30) : 0), kids[i], 0);
            for (size_t f = 4; f < kids[i].size(); f += 4) put_part(p2dst, p2src, col[i], kids[i], f);
        }
    }
    p1_at[D1] = (int32_t)p1dst.size();
    p2_at[D1] = (int32_t)p2dst.size();
    // zero masks of the pull at each depth: an inherited push column inside the pulled tiles is written as 0
    // there (the push fills it afterwards); one 32-bit word per 32 columns, words of depth d at zoff[d]
    std::vector<int32_t> zmask, zoff(D1 + 1, 0), zany(D1, 0);
    for (int32_t d = 0; d < D1; ++d) {
        zoff[d] = (int32_t)zmask.size();
        zmask.resize(zmask.size() + (size_t)(dw[d] + 31) / 32, 0);
    }
    zoff[D1] = (int32_t)zmask.size();
    for (int32_t i = 0; i < ncol_nodes; ++i) {
        if (!is_pheir[i]) continue;
        const int32_t d = h_exp[5 * i + 1], c = col[i];
        if (c < dw[d]) {
            zmask[zoff[d] + c / 32] |= (int32_t)(1u << (c % 32));
            zany[d] = 1;
        }
    }
    // upload: slot pairs, super-root columns, part destinations, zero masks, part sources (int4, 16-byte aligned)
    const size_t sched_ints =
        pairs.size() + B + p1dst.size() + p2dst.size() + zmask.size() + p1src.size() + p2src.size() + 8;
    PS_CUDA(ws->sched.ensure(sizeof(int32_t) * std::max<size_t>(1, sched_ints)));
    PS_CUDA(ws->pin_q.ensure(sizeof(int32_t) * std::max<size_t>(1, sched_ints)));
    int32_t *h_sched = ws->pin_q.as<int32_t>();
    size_t o = 0;
    auto put = [&](const std::vector<int32_t> &v) {
        const size_t at = o;
        if (!v.empty()) std::memcpy(h_sched + o, v.data(), sizeof(int32_t) * v.size());
        o += v.size();
        return at;
    };
    const size_t o_pairs = put(pairs), o_rho = put(rho), o_p1dst = put(p1dst), o_p2dst = put(p2dst),
                 o_zmask = put(zmask);
    o = (o + 3) / 4 * 4;
    const size_t o_p1src = put(p1src), o_p2src = put(p2src);
    int32_t *d_sched = ws->sched.as<int32_t>();
    PS_CUDA(cudaMemcpyAsync(d_sched, h_sched, sizeof(int32_t) * o, cudaMemcpyHostToDevice, st));
    ws->stats.phase_ms[9] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host0).count();
    launch_set_slots(t, d_sched + o_pairs, (int32_t)(pairs.size() / 2), st);
    ++launches;
    const int32_t *d_rho = d_sched + o_rho;
    // 4. level loop, deepest depth first.  Two score buffers: A receives this depth's MD; B holds the depth
    // below, which becomes this depth's D in place (accumulate + gamma scatter) before the pull reads it.
    PS_CUDA(ws->md_a.ensure((size_t)max_floats * sizeof(float)));
    PS_CUDA(ws->md_b.ensure((size_t)max_floats * sizeof(float)));
    float *A = ws->md_a.as<float>(), *Bm = ws->md_b.as<float>();
    const int32_t *node_list = ws->node_list.as<int32_t>();
    // the full tiles' launch: 32-column tiles, their 16-column halves, 32-column tiles two per pass, or 32-column
    // tiles gathered by the TMA
    const int32_t wide = g->tune_wide == 16 || g->tune_wide == kPullPairs || g->tune_wide == kPullTma ? g->tune_wide : 32;
    const int32_t tw = wide == 16 ? 16 : 32;
    int32_t *d_pull_err = nullptr;
    if (wide == kPullTma) {
        PS_CUDA(ws->pull_err.ensure(sizeof(int32_t)));
        d_pull_err = ws->pull_err.as<int32_t>();
        PS_CUDA(cudaMemsetAsync(d_pull_err, 0, sizeof(int32_t), st));
    }
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks;
    // Without profiling, the push block and the tail tile of a depth run on a second stream beside the
    // accumulate and the full-tile pull: they write other columns of A than the full tiles do.  With
    // profiling everything stays on the caller's stream, so the phase times do not overlap.
    const bool overlap = !ws->profiling;
    auto zmask_at = [&](int32_t d) -> const uint32_t * {
        return zany[d] ? reinterpret_cast<const uint32_t *>(d_sched + o_zmask + zoff[d]) : nullptr;
    };
    if (overlap) PS_CUDA(ws->ensure_side());
    cudaStream_t ss = overlap ? ws->side : st;
    for (int32_t d = Dmax; d >= 0; --d) {
        const int32_t S = scount[d], H = hcount[d];
        const ColLayout La = lay[d], Lb = d + 1 <= Dmax ? lay[d + 1] : make_layout(n, 4);
        const bool side_work = H > 0 || (S > 0 && tail[d] > 0);
        if (overlap && side_work) {  // side work of this depth starts after everything before it
            PS_CUDA(cudaEventRecord(ws->ev_start, st));
            PS_CUDA(cudaStreamWaitEvent(ss, ws->ev_start, 0));
        }
        if (H > 0) {  // height-2 columns: zero, then push from the grandchildren's gamma
            // zeroed: the push block, and the inherited columns outside the pulled tiles (the pull writes 0 into
            // those inside them); inherited columns are pushed after the pull, below
            const int32_t z0 = hinh[d] > 0 ? dw[d] : h0v[d];
            ph.begin(6);
            launch_zero_cols(n, A, La, z0, rpv[d] - z0, ss);
            launch_push_h2(dg, node_list + node_off[d + 2], ncount[d + 2], t, A, La, h0v[d], false, ss);
            ph.end();
            launches += 2;
        }
        if (S > 0) {
            ph.begin(2);  // D of this depth's dense nodes, in place in B (the MD of depth d+1)
            const int32_t np1 = p1_at[d + 1] - p1_at[d], np2 = p2_at[d + 1] - p2_at[d];
            if (np1 > 0)
                launch_accumulate(dg.n_active, Bm, Lb, d_sched + o_p1dst + p1_at[d],
                                  reinterpret_cast<const int4 *>(d_sched + o_p1src) + p1_at[d], np1,
                                  d_sched + o_p2dst + p2_at[d],
                                  reinterpret_cast<const int4 *>(d_sched + o_p2src) + p2_at[d], np2, st);
            ph.end();
            ++launches;
            if (d + 2 <= Dmax) {
                ph.begin(3);
                launch_scatter_gamma(node_list + node_off[d + 2], ncount[d + 2], t, Bm, Lb, st);
                ph.end();
                ++launches;
            }
            ph.begin(4);
            launch_zero_spare_row(Bm, Lb, dw[d], st);  // the pull's padding gathers read it
            if (dg.n_split > 0) {
                launch_zero_split_rows(dg, A, La, dw[d], st);
                ++launches;
            }
            ph.end();
            ++launches;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (ws->profiling) {
                e0 = tm.get();
                e1 = tm.get();
                PS_CUDA(cudaEventRecord(e0, st));
            }
            if (tail[d] > 0) {  // the tail tile lies inside one group (or row) of each layout
                if (overlap) {
                    PS_CUDA(cudaEventRecord(ws->ev_ready, st));
                    PS_CUDA(cudaStreamWaitEvent(ss, ws->ev_ready, 0));
                }
                const int32_t c = 32 * nfull[d];
                launch_pull(dg, Bm + Lb.base(c), Lb.rpitch(c), 0, 1 << 30, A + La.base(c), La.rpitch(c), 0, 1 << 30, 1,
                            tail[d], g->tune_bps[tail[d]], zmask_at(d) ? zmask_at(d) + nfull[d] : nullptr, ss);
                ++launches;
            }
            if (nfull[d] > 0 && wide == kPullTma) {  // 32-column tiles, rows gathered by the TMA
                PS_CUDA(launch_pull_tma(dg, Bm, Lb.rpitch(0), Lb.K > 0 ? kGroup : Lb.R, Lb.tile_stride(), Lb.tile_sub(32),
                                        A, La.rpitch(0), La.tile_stride(), La.tile_sub(32), nfull[d],
                                        g->tune_bps[kPullTma], zmask_at(d), d_pull_err, st));
                ++launches;
            } else if (nfull[d] > 0) {  // 32-column tiles (or their 16-column halves, or pairs of them)
                const int32_t nt = nfull[d] * (32 / tw);
                launch_pull(dg, Bm, Lb.rpitch(0), Lb.tile_stride(), Lb.tile_sub(tw), A, La.rpitch(0), La.tile_stride(),
                            La.tile_sub(tw), nt, wide, g->tune_bps[wide], zmask_at(d), st);
                ++launches;
            }
            if (ws->profiling) {
                PS_CUDA(cudaEventRecord(e1, st));
                marks.push_back({e0, e1});
            }
            ws->stats.probe_launches += 1;
            ws->stats.edge_gathers += dg.m * (int64_t)S;
            ws->stats.probe_bytes += 4.0 * dg.m + 16.0 * dg.n_pieces + 4.0 * n + 8.0 * (double)n * S;
        }
        if (overlap && side_work) {  // the gamma of this depth (and every later step) waits for the side work
            PS_CUDA(cudaEventRecord(ws->ev_side, ss));
            PS_CUDA(cudaStreamWaitEvent(st, ws->ev_side, 0));
        }
        if (hinh[d] > 0) {  // push nodes in inherited columns: after the pull has written those columns as 0
            ph.begin(6);
            launch_push_h2(dg, node_list + node_off[d + 2], ncount[d + 2], t, A, La, h0v[d], true, st);
            ph.end();
            ++launches;
        }
        if (d >= 1) {
            ph.begin(7);
            launch_gamma(dg, node_list + node_off[d], ncount[d], t, qb.inv_nr, (S + H) > 0 ? A : nullptr, La, st);
            ph.end();
            ++launches;
        }
        std::swap(A, Bm);
        ws->stats.levels += 1;
    }
    float *MD0 = Bm;  // after the last swap, the super-roots' MD
    // 5. estimates: s(u, v) = MD(super-root)[v], s(u, u) = 1
    ph.begin(8);
    launch_finalize(n, B, qb.node, d_rho, scount[0] > 0 ? MD0 : nullptr, lay[0], dg.ext2int, g->cfg.shift, d_out, st);
    ph.end();
    ++launches;
    PS_CUDA(cudaGetLastError());
    int32_t pull_err = 0;
    if (d_pull_err) PS_CUDA(cudaMemcpyAsync(&pull_err, d_pull_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (pull_err) return fail(PROBESIM_E_TIMEOUT, "a TMA row gather of the pull did not complete in time");
    ph.collect(ws->stats);
    for (auto &mk : marks) {
        float ms = 0.f;
        PS_CUDA(cudaEventElapsedTime(&ms, mk.first, mk.second));
        ws->stats.probe_ms += ms;
        ws->stats.phase_ms[5] += ms;
    }
    ws->stats.kernel_launches += launches;
    return PROBESIM_OK;
}

// Walks of a planned batch (Def. 3): uploads the queries, launches the walk kernel and reads back the walk
// node count and the longest walk.
static probesim_status batch_walks(probesim_graph *g, Workspace *ws, const BatchPlan &P, QueryBatch &qb,
                                   int64_t *walk_nodes, int32_t *max_len, int64_t &launches, cudaStream_t st) {
    const int32_t L = g->cfg.l_max;
    PS_TRY(upload_batch(ws, P, qb, st));
    PS_CUDA(ws->walks.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_CUDA(ws->lens.ensure(sizeof(int32_t) * std::max<int32_t>(1, P.W)));
    PS_CUDA(ws->ctr.ensure(sizeof(LaunchCounters)));
    LaunchCounters *d_ctr = ws->ctr.as<LaunchCounters>();
    PS_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(LaunchCounters), st));
    launch_walks(ws->dg, qb, P.W, L, g->t_stop, g->cfg.seed, ws->walks.as<int32_t>(), ws->lens.as<int32_t>(), false,
                 d_ctr, st);
    ++launches;
    LaunchCounters *h_ctr = ws->pin_s.as<LaunchCounters>();
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    *walk_nodes = (int64_t)h_ctr->walk_nodes;
    *max_len = h_ctr->max_len;
    ws->stats.walks += P.W;
    ws->stats.walk_nodes += *walk_nodes;
    return PROBESIM_OK;
}

// Randomized PROBE (Alg. 3) instances of the walks w0 .. w1-1, one per (walk, prefix length i >= 2) -- or, with
// walk_slot and t_sw, only those whose prefix's tree slot is flagged -- run level by level over hash-set
// frontiers.  Adds the member counts of the final levels into counts ([B][n], internal ids).  An allocation that
// fails sets *too_big (here: the walk range is too large) and returns PROBESIM_E_NOMEM.
static probesim_status rand_range(probesim_graph *g, Workspace *ws, const QueryBatch &qb, int32_t B, int32_t w0,
                                  int32_t w1, int32_t max_len, const int32_t *walk_slot, const uint8_t *t_sw,
                                  int32_t *counts, int64_t &launches, cudaStream_t st, bool *too_big) {
    *too_big = false;
    const int32_t W = w1 - w0;
    const DeviceGraph &dg = ws->dg;
    const int32_t L = g->cfg.l_max;
    PS_ALLOC_RANGE(ws->r_cnt.ensure(sizeof(long long) * std::max(1, W)));
    PS_ALLOC_RANGE(ws->r_off.ensure(sizeof(long long) * (W + 1)));
    PS_ALLOC_RANGE(ws->r_part.ensure(sizeof(long long) * scan64_partials_needed(W)));
    launch_inst_count(ws->lens.as<int32_t>(), w0, W, ws->r_cnt.as<long long>(), walk_slot, t_sw, L, st);
    launch_scan64(ws->r_cnt.as<long long>(), W, ws->r_part.as<long long>(), ws->r_off.as<long long>(), st);
    launches += 4;
    long long *h_ll = reinterpret_cast<long long *>(ws->pin_s.as<char>() + 32768);
    PS_CUDA(cudaMemcpyAsync(h_ll, ws->r_off.as<long long>() + W, sizeof(long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t NI = h_ll[0];
    if (NI >= ((int64_t)1 << 31)) return fail(PROBESIM_E_INVALID, "too many probe instances in one call");
    if (NI == 0) return PROBESIM_OK;
    PS_ALLOC_RANGE(ws->r_iwalk.ensure(sizeof(int32_t) * NI));
    PS_ALLOC_RANGE(ws->r_ilen.ensure(sizeof(int32_t) * NI));
    PS_ALLOC_RANGE(ws->r_iq.ensure(sizeof(int32_t) * NI));
    PS_ALLOC_RANGE(ws->r_ik.ensure(sizeof(uint32_t) * NI));
    PS_ALLOC_RANGE(ws->r_ctr.ensure(sizeof(unsigned long long) * 4));
    unsigned long long *d_fc = ws->r_ctr.as<unsigned long long>();
    int32_t *d_over = reinterpret_cast<int32_t *>(d_fc + 2);
    int cur = 0;
    int64_t cap = next_pow2(std::max<int64_t>(1024, 2 * NI));
    PS_ALLOC_RANGE(ws->r_keys[cur].ensure(8 * (size_t)cap));
    PS_ALLOC_RANGE(ws->r_fi[cur].ensure(4 * (size_t)NI));
    PS_ALLOC_RANGE(ws->r_fn[cur].ensure(4 * (size_t)NI));
    PS_CUDA(cudaMemsetAsync(ws->r_keys[cur].p, 0xFF, 8 * (size_t)cap, st));
    PS_CUDA(cudaMemsetAsync(d_fc, 0, sizeof(unsigned long long) * 4, st));
    launch_inst_init(qb, dg, ws->lens.as<int32_t>(), w0, W, L, ws->walks.as<int32_t>(), ws->r_off.as<long long>(),
                     ws->r_iwalk.as<int32_t>(), ws->r_ilen.as<int32_t>(), ws->r_iq.as<int32_t>(), ws->r_ik.as<uint32_t>(),
                     ws->r_fi[cur].as<int32_t>(), ws->r_fn[cur].as<int32_t>(), d_fc, ws->r_keys[cur].as<unsigned long long>(),
                     cap, d_over, walk_slot, t_sw, st);
    ++launches;
    PS_CUDA(cudaMemcpyAsync(h_ll, d_fc, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (reinterpret_cast<int32_t *>(h_ll + 2)[0]) return fail(PROBESIM_E_CUDA, "internal: frontier set overflow");
    int64_t F = (int64_t)((unsigned long long *)h_ll)[0];
    int64_t cur_cap = cap;
    for (int32_t j = 0; j + 2 <= max_len && F > 0; ++j) {
        // out-degree prefix sums of the frontier
        PS_ALLOC_RANGE(ws->r_deg.ensure(sizeof(long long) * F));
        PS_ALLOC_RANGE(ws->r_pref.ensure(sizeof(long long) * (F + 1)));
        PS_ALLOC_RANGE(ws->r_part.ensure(sizeof(long long) * scan64_partials_needed(F)));
        launch_frontier_degree(ws->r_fi[cur].as<int32_t>(), ws->r_fn[cur].as<int32_t>(), F, ws->r_ilen.as<int32_t>(), j,
                               dg.out_off, ws->r_deg.as<long long>(), st);
        launch_scan64(ws->r_deg.as<long long>(), F, ws->r_part.as<long long>(), ws->r_pref.as<long long>(), st);
        launches += 4;
        PS_CUDA(cudaMemcpyAsync(h_ll, ws->r_pref.as<long long>() + F, sizeof(long long), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        const int64_t E = h_ll[0];
        if (E <= 0) break;
        const int nx = cur ^ 1;
        const int64_t ncap = next_pow2(std::max<int64_t>(1024, 2 * E));
        if ((size_t)(8 * ncap + 8 * E) > budget_of(g, ws) / 4 && w1 - w0 > 1) {  // a smaller walk range fits the budget
            *too_big = true;
            return fail(PROBESIM_E_NOMEM, "randomized PROBE level exceeds a quarter of the memory budget");
        }
        PS_ALLOC_RANGE(ws->r_keys[nx].ensure(8 * (size_t)ncap));
        PS_ALLOC_RANGE(ws->r_fi[nx].ensure(4 * (size_t)E));
        PS_ALLOC_RANGE(ws->r_fn[nx].ensure(4 * (size_t)E));
        PS_CUDA(cudaMemsetAsync(ws->r_keys[nx].p, 0xFF, 8 * (size_t)ncap, st));
        PS_CUDA(cudaMemsetAsync(d_fc, 0, sizeof(unsigned long long), st));
        RandLevel Lv;
        Lv.fr_inst = ws->r_fi[cur].as<int32_t>();
        Lv.fr_node = ws->r_fn[cur].as<int32_t>();
        Lv.F = F;
        Lv.prefix = ws->r_pref.as<long long>();
        Lv.E = E;
        Lv.cur_keys = ws->r_keys[cur].as<unsigned long long>();
        Lv.cur_cap = cur_cap;
        Lv.next_keys = ws->r_keys[nx].as<unsigned long long>();
        Lv.next_cap = ncap;
        Lv.next_inst = ws->r_fi[nx].as<int32_t>();
        Lv.next_node = ws->r_fn[nx].as<int32_t>();
        Lv.next_count = d_fc;
        Lv.counts = counts;
        Lv.overflow = d_over;
        Lv.j = j;
        launch_rand_level(dg, ws->walks.as<int32_t>(), L, ws->r_iwalk.as<int32_t>(), ws->r_ilen.as<int32_t>(),
                          ws->r_iq.as<int32_t>(), ws->r_ik.as<uint32_t>(), qb.qid, g->cfg.seed, g->t_keep, Lv, st);
        ++launches;
        ws->stats.edge_gathers += E;
        PS_CUDA(cudaMemcpyAsync(h_ll, d_fc, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        if (reinterpret_cast<int32_t *>(h_ll + 2)[0]) return fail(PROBESIM_E_CUDA, "internal: frontier set overflow");
        F = (int64_t)((unsigned long long *)h_ll)[0];
        cur = nx;
        cur_cap = ncap;
        ws->stats.levels += 1;
    }
    return PROBESIM_OK;
}

// All instances of the call (see rand_range), into ws->r_counts.  When the whole walk range does not fit, the
// walks are taken in halves, quarters, ..., each counted into a side buffer added once the range completes, so
// the integer member counts come out the same whatever the split.
static probesim_status rand_instances(probesim_graph *g, Workspace *ws, const QueryBatch &qb, int32_t B, int32_t W,
                                      int32_t max_len, const int32_t *walk_slot, const uint8_t *t_sw, int64_t &launches,
                                      cudaStream_t st, bool *too_big) {
    const size_t cn = (size_t)B * g->n;
    PS_ALLOC(ws->r_counts.ensure(sizeof(int32_t) * cn));
    PS_CUDA(cudaMemsetAsync(ws->r_counts.p, 0, sizeof(int32_t) * cn, st));
    bool oom = false;
    probesim_status s = rand_range(g, ws, qb, B, 0, W, max_len, walk_slot, t_sw, ws->r_counts.as<int32_t>(), launches,
                                   st, &oom);
    if (s == PROBESIM_OK || !oom || W <= 1) {
        if (oom) *too_big = B > 1;
        return s;
    }
    DevBuf *big[] = {&ws->r_keys[0], &ws->r_keys[1], &ws->r_fi[0], &ws->r_fi[1], &ws->r_fn[0], &ws->r_fn[1],
                     &ws->r_deg, &ws->r_pref};
    for (DevBuf *b : big) b->release();
    PS_CUDA(cudaMemsetAsync(ws->r_counts.p, 0, sizeof(int32_t) * cn, st));
    PS_ALLOC(ws->r_counts2.ensure(sizeof(int32_t) * cn));
    int32_t span = (W + 1) / 2;
    for (int32_t w0 = 0; w0 < W;) {
        const int32_t w1 = std::min(W, w0 + span);
        PS_CUDA(cudaMemsetAsync(ws->r_counts2.p, 0, sizeof(int32_t) * cn, st));
        s = rand_range(g, ws, qb, B, w0, w1, max_len, walk_slot, t_sw, ws->r_counts2.as<int32_t>(), launches, st, &oom);
        if (s == PROBESIM_OK) {
            launch_add_i32(ws->r_counts.as<int32_t>(), ws->r_counts2.as<int32_t>(), (int64_t)cn, st);
            ++launches;
            w0 = w1;
        } else if (oom && span > 1) {
            span = (span + 1) / 2;
            for (DevBuf *b : big) b->release();
        } else {
            if (oom) *too_big = B > 1;
            return s;
        }
    }
    g_last_error.clear();  // the allocation failures that cut the walk range are not errors
    return PROBESIM_OK;
}

// Randomized PROBE (Alg. 3) for every probe of Alg. 1: one instance per (walk, prefix length); the estimate is
// the member count of the final levels divided by n_r.
static probesim_status run_batch_rand(probesim_graph *g, Workspace *ws, const probesim_query *q, int32_t B,
                                      float *d_out, cudaStream_t st, bool *too_big) {
    *too_big = false;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, B, P));
    QueryBatch qb;
    int64_t launches = 0, walk_nodes = 0;
    int32_t max_len = 0;
    PS_TRY(batch_walks(g, ws, P, qb, &walk_nodes, &max_len, launches, st));
    PS_TRY(rand_instances(g, ws, qb, B, P.W, max_len, nullptr, nullptr, launches, st, too_big));
    launch_rand_finalize(g->n, B, qb.node, ws->r_counts.as<int32_t>(), qb.inv_nr, ws->dg.ext2int, g->cfg.shift, d_out,
                         st);
    ++launches;
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaStreamSynchronize(st));
    ws->stats.kernel_launches += launches;
    return PROBESIM_OK;
}

// Frontier engine (frontier.cu): every prefix of the batch's walk trees probed on its own with Pruning Rule 2,
// and, in PROBESIM_PROBE_SWITCH mode, the switch of Sec. 4.4 handing large probes to Alg. 3.
static probesim_status run_batch_frontier(probesim_graph *g, Workspace *ws, const probesim_query *q, int32_t B,
                                          float *d_out, cudaStream_t st, bool *too_big) {
    *too_big = false;
    const DeviceGraph &dg = ws->dg;
    const int32_t n = dg.n, L = g->cfg.l_max;
    const bool sw_mode = g->cfg.probe_mode == PROBESIM_PROBE_SWITCH;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, B, P));
    int64_t max_w = 1;
    for (int32_t b = 0; b < B; ++b) {
        if (num_walks(g->cfg.c, q[b].eps, g->cfg.delta, n) > kFrontierMaxWalks)
            return fail(PROBESIM_E_INVALID, "eps too small: Pruning Rule 2 and the switch take at most 2^18 walks per query");
        max_w = std::max<int64_t>(max_w, P.base[b + 1] - P.base[b]);
    }
    if ((size_t)P.W * L * 8 > budget_of(g, ws) / 4 && B > 1) {
        *too_big = true;
        return PROBESIM_E_NOMEM;
    }
    QueryBatch qb;
    int64_t launches = 0, walk_nodes = 0;
    int32_t max_len = 0;
    PS_TRY(batch_walks(g, ws, P, qb, &walk_nodes, &max_len, launches, st));
    // reverse-reachability tree (Alg. 4) with the slot of every walk prefix
    TrieTable t;
    t.cap = next_pow2(std::max<int64_t>(1024, 2 * (walk_nodes + B) + 64));
    const size_t cap = (size_t)t.cap;
    PS_ALLOC(ws->t_key.ensure(8 * cap));
    PS_ALLOC(ws->t_node.ensure(4 * cap));
    PS_ALLOC(ws->t_parent.ensure(4 * cap));
    PS_ALLOC(ws->t_depth.ensure(4 * cap));
    PS_ALLOC(ws->t_query.ensure(4 * cap));
    PS_ALLOC(ws->t_weight.ensure(4 * cap));
    PS_ALLOC(ws->t_height.ensure(4 * cap));
    PS_ALLOC(ws->f_wslot.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_ALLOC(ws->f_tsw.ensure(cap));
    t.key = ws->t_key.as<unsigned long long>();
    t.node = ws->t_node.as<int32_t>();
    t.parent = ws->t_parent.as<int32_t>();
    t.depth = ws->t_depth.as<int32_t>();
    t.query = ws->t_query.as<int32_t>();
    t.weight = ws->t_weight.as<int32_t>();
    t.height = ws->t_height.as<int32_t>();
    t.walk_slot = ws->f_wslot.as<int32_t>();
    uint8_t *t_sw = ws->f_tsw.as<uint8_t>();
    PS_CUDA(cudaMemsetAsync(t.key, 0xFF, 8 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.weight, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.height, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t_sw, 0, cap, st));
    LaunchCounters *d_ctr = ws->ctr.as<LaunchCounters>();
    launch_trie_insert(dg, qb, P.W, L, ws->walks.as<int32_t>(), ws->lens.as<int32_t>(), t, d_ctr, st);
    // the probes: tree nodes of depth >= 2
    PS_ALLOC(ws->f_slot.ensure(sizeof(int32_t) * std::max<int64_t>(1, walk_nodes)));
    PS_ALLOC(ws->f_misc.ensure(64));
    int32_t *d_np = ws->f_misc.as<int32_t>();
    unsigned long long *d_fctr = reinterpret_cast<unsigned long long *>(ws->f_misc.as<char>() + 8);
    PS_CUDA(cudaMemsetAsync(d_np, 0, 64, st));
    launch_fr_list(t, ws->f_slot.as<int32_t>(), d_np, st);
    launches += 2;
    LaunchCounters *h_ctr = ws->pin_s.as<LaunchCounters>();
    long long *h_ll = reinterpret_cast<long long *>(ws->pin_s.as<char>() + 32768);
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(h_ll, d_np, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (h_ctr->overflow) return fail(PROBESIM_E_CUDA, "internal: walk tree table overflow");
    const int32_t NP = reinterpret_cast<int32_t *>(h_ll)[0];
    ws->stats.probes += NP;
    ws->stats.tree_nodes += NP;
    // per-probe state, the two frontier lists, the estimate sums
    FrontierProbes PR;
    PR.P = NP;
    PS_ALLOC(ws->f_anc.ensure(sizeof(int32_t) * std::max(1, NP)));
    PS_ALLOC(ws->f_deg.ensure(sizeof(unsigned long long) * std::max(1, NP)));
    PS_ALLOC(ws->f_state.ensure(sizeof(int32_t) * std::max(1, NP)));
    PS_ALLOC(ws->f_rsize.ensure(sizeof(long long) * (NP + 1)));
    PS_ALLOC(ws->f_roff.ensure(sizeof(long long) * (NP + 1)));
    PS_ALLOC(ws->f_dsize.ensure(sizeof(long long) * (NP + 1)));
    PS_ALLOC(ws->f_doff.ensure(sizeof(long long) * (NP + 1)));
    PR.slot = ws->f_slot.as<int32_t>();
    PR.anc = ws->f_anc.as<int32_t>();
    PR.deg = ws->f_deg.as<unsigned long long>();
    PR.state = ws->f_state.as<int32_t>();
    PR.rsize = ws->f_rsize.as<long long>();
    PR.roff = ws->f_roff.as<long long>();
    PR.dsize = ws->f_dsize.as<long long>();
    PR.doff = ws->f_doff.as<long long>();
    const size_t accn = (size_t)B * n;
    PS_ALLOC(ws->f_acc.ensure(sizeof(unsigned long long) * accn));
    PS_CUDA(cudaMemsetAsync(ws->f_acc.p, 0, sizeof(unsigned long long) * accn, st));
    // host tables: thr[w] = floor(c0 * w * n) in FP64 (the switch compares the integer out-degree sum with it),
    // pw[k] = sqrt(c)^k rounded to FP32 (Rule 2's factor)
    const size_t nthr = sw_mode ? (size_t)max_w + 1 : 0;
    const size_t tab_bytes = 256 * sizeof(float) + nthr * sizeof(long long);
    PS_ALLOC(ws->f_tab.ensure(tab_bytes));
    PS_ALLOC(ws->pin_q.ensure(tab_bytes));
    {
        char *h = ws->pin_q.as<char>();
        float *pw = reinterpret_cast<float *>(h);
        const double sc = std::sqrt(g->cfg.c);
        for (int k = 0; k < 256; ++k) pw[k] = (float)std::pow(sc, (double)k);
        long long *thr = reinterpret_cast<long long *>(h + 256 * sizeof(float));
        for (size_t w = 0; w < nthr; ++w) {
            const double x = std::floor((double)g->cfg.c0 * (double)w * (double)n);
            thr[w] = x >= 9.0e18 ? (long long)9000000000000000000ll : (long long)x;
        }
        PS_CUDA(cudaMemcpyAsync(ws->f_tab.p, h, tab_bytes, cudaMemcpyHostToDevice, st));
    }
    const float *d_pw = ws->f_tab.as<float>();
    const long long *d_thr = sw_mode ? reinterpret_cast<const long long *>(ws->f_tab.as<char>() + 256 * sizeof(float)) : nullptr;
    // The deterministic rounds work on tasks: a probe range [p0, p1) at level j with its frontier entries.  A
    // level whose next frontier might not fit the list budget processes the passes that fit and defers the other
    // probes, with their level-j entries, to a stack; they resume once the processed range has run out.  Every
    // probe's last-level pushes land in the estimate exactly once, whatever the split.
    const long long pass_slots =
        std::max<long long>((long long)n, (long long)(budget_of(g, ws) / 4 / sizeof(FrontierSlot)));
    const long long list_cap = std::max<long long>((long long)n, (long long)(budget_of(g, ws) / 8 / 12));
    auto list_of = [&](int k) {
        FrontierList F;
        F.p = ws->f_lp[k].as<int32_t>();
        F.x = ws->f_lx[k].as<int32_t>();
        F.val = ws->f_lv[k].as<float>();
        return F;
    };
    auto grow_list = [&](int k, long long need, long long keep, cudaStream_t s) -> cudaError_t {
        cudaError_t e = ws->f_lp[k].grow(sizeof(int32_t) * need, sizeof(int32_t) * keep, s);
        if (e == cudaSuccess) e = ws->f_lx[k].grow(sizeof(int32_t) * need, sizeof(int32_t) * keep, s);
        if (e == cudaSuccess) e = ws->f_lv[k].grow(sizeof(float) * need, sizeof(float) * keep, s);
        return e;
    };
    struct Task {
        int32_t p0, p1, j;
        long long at, count;  // entries on the deferral stack
    };
    std::vector<Task> stack;
    long long stack_top = 0;
    int cur = 0;
    int64_t nF = NP;
    int32_t p0 = 0, p1 = NP, j = 0;
    PS_ALLOC(grow_list(cur, std::max<int64_t>(1, nF), 0, st));
    launch_fr_init(t, PR, list_of(cur), st);
    ++launches;
    for (;;) {
        if (nF == 0) {  // the range ran out: resume the last deferred one
            if (stack.empty()) break;
            const Task tk = stack.back();
            stack.pop_back();
            PS_ALLOC(grow_list(cur, std::max<long long>(1, tk.count), 0, st));
            const FrontierList F = list_of(cur);
            PS_CUDA(cudaMemcpyAsync(F.p, ws->f_sp.as<int32_t>() + tk.at, sizeof(int32_t) * tk.count, cudaMemcpyDeviceToDevice, st));
            PS_CUDA(cudaMemcpyAsync(F.x, ws->f_sx.as<int32_t>() + tk.at, sizeof(int32_t) * tk.count, cudaMemcpyDeviceToDevice, st));
            PS_CUDA(cudaMemcpyAsync(F.val, ws->f_sv.as<float>() + tk.at, sizeof(float) * tk.count, cudaMemcpyDeviceToDevice, st));
            stack_top = tk.at;
            p0 = tk.p0, p1 = tk.p1, j = tk.j, nF = tk.count;
            ws->stats.deferred += 1;
        }
        const FrontierList F = list_of(cur);
        const int32_t np_ = p1 - p0;
        PS_ALLOC(ws->f_wp.ensure(sizeof(long long) * (nF + 1)));
        PS_ALLOC(ws->r_part.ensure(sizeof(long long) * scan64_partials_needed(std::max<int64_t>(nF, np_))));
        long long *wp = ws->f_wp.as<long long>();
        launch_fr_prune(F, nF, t, PR, dg.out_off, d_pw, g->cfg.eps_p, j, wp, st);
        launch_fr_regions(t, PR, p0, p1, j, n, d_thr, t_sw, st);
        launch_fr_work(F, nF, PR, wp, st);
        launch_scan64(wp, nF, ws->r_part.as<long long>(), wp, st);  // in place: wp[f] = first work item of entry f
        launch_scan64(PR.rsize + p0, np_, ws->r_part.as<long long>(), PR.roff + p0, st);
        launch_scan64(PR.dsize + p0, np_, ws->r_part.as<long long>(), PR.doff + p0, st);
        launches += 12;
        PS_CUDA(cudaMemcpyAsync(h_ll, wp + nF, sizeof(long long), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(h_ll + 1, PR.roff + p1, sizeof(long long), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(h_ll + 2, PR.doff + p1, sizeof(long long), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        const long long E = h_ll[0], T = h_ll[1], Dtot = h_ll[2];
        ws->stats.edge_gathers += E;
        ws->stats.levels += 1;
        if (E == 0) {  // nothing left to push: every probe of the range ended, switched or was pruned
            nF = 0;
            continue;
        }
        const int nx = cur ^ 1;
        // passes: probe ranges whose regions fit pass_slots (roff and doff are relative to p0)
        std::vector<int32_t> cuts{p0};
        if (T > pass_slots) {
            std::vector<long long> roff(np_ + 1);
            PS_CUDA(cudaMemcpyAsync(roff.data(), PR.roff + p0, sizeof(long long) * (np_ + 1), cudaMemcpyDeviceToHost, st));
            PS_CUDA(cudaStreamSynchronize(st));
            int32_t a = 0;
            while (a < np_) {
                int32_t b = (int32_t)(std::upper_bound(roff.begin() + a + 1, roff.end(), roff[a] + pass_slots) -
                                      roff.begin()) - 1;
                if (b <= a) b = a + 1;
                cuts.push_back(p0 + b);
                a = b;
            }
        } else {
            cuts.push_back(p1);
        }
        const int32_t npass = (int32_t)cuts.size() - 1;
        // per cut: first entry, work prefix, region offset, next-entry bound offset
        std::vector<long long> cb(4 * (size_t)(npass + 1));
        if (npass == 1) {
            cb = {0, 0, 0, 0, nF, E, T, Dtot};
        } else {
            PS_ALLOC(ws->f_cuts.ensure(sizeof(int32_t) * cuts.size() + 32 * cuts.size() + 16));
            int32_t *d_cuts = ws->f_cuts.as<int32_t>();
            long long *d_cb = reinterpret_cast<long long *>(ws->f_cuts.as<char>() + ((sizeof(int32_t) * cuts.size() + 15) / 16 * 16));
            PS_CUDA(cudaMemcpyAsync(d_cuts, cuts.data(), sizeof(int32_t) * cuts.size(), cudaMemcpyHostToDevice, st));
            launch_fr_bounds(F.p, nF, wp, PR.roff, PR.doff, d_cuts, (int32_t)cuts.size(), d_cb, st);
            ++launches;
            PS_CUDA(cudaMemcpyAsync(cb.data(), d_cb, sizeof(long long) * cb.size(), cudaMemcpyDeviceToHost, st));
            PS_CUDA(cudaStreamSynchronize(st));
        }
        ws->stats.table_passes += npass;
        ws->stats.max_table_slots = std::max<int64_t>(ws->stats.max_table_slots, T);
        const long long tslots = std::max<long long>(1, std::min<long long>(T, pass_slots + n));
        {
            const void *k0 = ws->f_keys.p;
            PS_ALLOC(ws->f_keys.ensure(sizeof(FrontierSlot) * tslots));
            if (ws->f_keys.p != k0 || !ws->f_table_clean) {  // new memory, or a failed call left slots behind
                PS_CUDA(cudaMemsetAsync(ws->f_keys.p, 0, ws->f_keys.cap, st));
                ws->f_table_clean = true;
            }
        }
        PS_ALLOC(ws->f_bcnt.ensure(sizeof(long long) * (fr_compact_blocks(tslots) + 1)));
        PS_ALLOC(ws->f_bpre.ensure(sizeof(long long) * (fr_compact_blocks(tslots) + 1)));
        PS_ALLOC(ws->r_part.ensure(sizeof(long long) * scan64_partials_needed(std::max<int64_t>(
                                       std::max<int64_t>(nF, np_), fr_compact_blocks(tslots)))));
        long long out_n = 0;
        int32_t pk = p1;  // probes [p0, pk) advance to level j + 1
        for (int32_t c = 0; c < npass; ++c) {
            const long long f_lo = cb[4 * c], e_lo = cb[4 * c + 1], r0 = cb[4 * c + 2], d0 = cb[4 * c + 3];
            const long long f_hi = cb[4 * (c + 1)], e_hi = cb[4 * (c + 1) + 1], r1 = cb[4 * (c + 1) + 2],
                            d1 = cb[4 * (c + 1) + 3];
            if (out_n > 0 && out_n + (d1 - d0) > list_cap) {  // defer probes [cuts[c], p1) at level j
                const long long cnt = nF - f_lo;
                PS_ALLOC(ws->f_sp.grow(sizeof(int32_t) * (stack_top + cnt), sizeof(int32_t) * stack_top, st));
                PS_ALLOC(ws->f_sx.grow(sizeof(int32_t) * (stack_top + cnt), sizeof(int32_t) * stack_top, st));
                PS_ALLOC(ws->f_sv.grow(sizeof(float) * (stack_top + cnt), sizeof(float) * stack_top, st));
                PS_CUDA(cudaMemcpyAsync(ws->f_sp.as<int32_t>() + stack_top, F.p + f_lo, sizeof(int32_t) * cnt, cudaMemcpyDeviceToDevice, st));
                PS_CUDA(cudaMemcpyAsync(ws->f_sx.as<int32_t>() + stack_top, F.x + f_lo, sizeof(int32_t) * cnt, cudaMemcpyDeviceToDevice, st));
                PS_CUDA(cudaMemcpyAsync(ws->f_sv.as<float>() + stack_top, F.val + f_lo, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st));
                stack.push_back({cuts[c], p1, j, stack_top, cnt});
                stack_top += cnt;
                pk = cuts[c];
                break;
            }
            const long long Tc = r1 - r0;
            FrontierExpand a;
            a.wp = wp;
            a.f_lo = f_lo;
            a.f_hi = f_hi;
            a.e_lo = e_lo;
            a.e_hi = e_hi;
            a.j = j;
            a.tab = ws->f_keys.as<FrontierSlot>();
            a.rbase = r0;
            a.acc = ws->f_acc.as<unsigned long long>();
            a.n = n;
            if (Tc > 0) ws->f_table_clean = false;  // until this pass's compaction has emptied its slots
            launch_fr_expand(dg, t, PR, F, a, st);
            ++launches;
            if (Tc > 0) {  // count the pass's occupied slots, grow the next list to hold them, write them
                const int64_t nb = fr_compact_blocks(Tc);
                launch_fr_count(a.tab, Tc, ws->f_bcnt.as<long long>(), st);
                launch_scan64(ws->f_bcnt.as<long long>(), nb, ws->r_part.as<long long>(), ws->f_bpre.as<long long>(), st);
                PS_CUDA(cudaMemcpyAsync(h_ll, ws->f_bpre.as<long long>() + nb, sizeof(long long), cudaMemcpyDeviceToHost, st));
                PS_CUDA(cudaStreamSynchronize(st));
                const long long need = std::max<long long>(1, out_n + h_ll[0]);
                PS_ALLOC(grow_list(nx, need, out_n, st));
                launch_fr_write(a.tab, Tc, PR.roff, cuts[c], cuts[c + 1], r0, ws->f_bpre.as<long long>(),
                                list_of(nx), out_n, need, st);
                launches += 5;
                out_n += h_ll[0];
                ws->f_table_clean = true;
            }
        }
        launch_fr_advance(t, PR, p0, pk, st);
        ++launches;
        p1 = pk;
        nF = out_n;
        cur = nx;
        ++j;
    }
    launch_fr_count_switched(PR, d_fctr, st);
    PS_CUDA(cudaMemcpyAsync(h_ll, d_fctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t switched = h_ll[0];
    ws->stats.switched += switched;
    // Sec. 4.4: Alg. 3 for every walk through a switched tree node
    const int32_t *counts = nullptr;
    if (switched > 0) {
        // the deterministic rounds' tables and lists are done with: their memory goes to Alg. 3's hash sets
        for (DevBuf *b : {&ws->f_keys, &ws->f_lp[0], &ws->f_lp[1], &ws->f_lx[0], &ws->f_lx[1],
                          &ws->f_lv[0], &ws->f_lv[1], &ws->f_wp, &ws->f_sp, &ws->f_sx, &ws->f_sv})
            b->release();
        PS_TRY(rand_instances(g, ws, qb, B, P.W, max_len, t.walk_slot, t_sw, launches, st, too_big));
        counts = ws->r_counts.as<int32_t>();
    }
    launch_fr_finalize(n, B, qb.node, ws->f_acc.as<unsigned long long>(), counts, qb.inv_nr, dg.ext2int, g->cfg.shift,
                       d_out, st);
    ++launches;
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaStreamSynchronize(st));
    ws->stats.kernel_launches += launches;
    return PROBESIM_OK;
}

// Runs all nq queries, splitting batches that do not fit the workspace budget.
static probesim_status run_queries(probesim_graph *g, Workspace *ws, const probesim_query *q, int32_t nq, float *d_out,
                                   cudaStream_t st) {
    int32_t done = 0;
    int32_t chunk = nq;
    while (done < nq) {
        const int32_t B = std::min(chunk, nq - done);
        bool too_big = false;
        float *out = d_out + (int64_t)done * g->n;
        probesim_status s;
        if (g->cfg.probe_mode == PROBESIM_PROBE_RANDOMIZED)
            s = run_batch_rand(g, ws, q + done, B, out, st, &too_big);
        else if (g->cfg.probe_mode == PROBESIM_PROBE_SWITCH || g->cfg.eps_p > 0.f)
            s = run_batch_frontier(g, ws, q + done, B, out, st, &too_big);
        else
            s = run_batch(g, ws, q + done, B, out, st, &too_big);
        if (s == PROBESIM_OK) {
            done += B;
            continue;
        }
        if (too_big && B > 1) {
            chunk = std::max(1, B / 2);
            continue;
        }
        return s;
    }
    if (chunk < nq) g_last_error.clear();  // the budget messages of batches that were split are not errors
    return PROBESIM_OK;
}

probesim_status ps::check_queries(const probesim_graph *g, const probesim_query *q, int32_t nq, bool topk,
                                     int32_t kmax) {
    if (!q || nq <= 0) return fail(PROBESIM_E_INVALID, "queries: null pointer or nq <= 0");
    if (nq > 65535) return fail(PROBESIM_E_INVALID, "at most 65535 queries per call");
    for (int32_t i = 0; i < nq; ++i) {
        if (q[i].node < 0 || q[i].node >= g->n) return fail(PROBESIM_E_RANGE, "query node outside [0, n)");
        if (!(q[i].eps > 0.0 && q[i].eps < 1.0)) return fail(PROBESIM_E_INVALID, "query eps must lie in (0, 1)");
        if (topk && (q[i].k < 1 || q[i].k > kmax)) return fail(PROBESIM_E_INVALID, "query k must lie in [1, kmax]");
    }
    return PROBESIM_OK;
}

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

const char *probesim_last_error(void) { return g_last_error.c_str(); }

probesim_status probesim_config_default(probesim_config *cfg) {
    if (!cfg) return fail(PROBESIM_E_INVALID, "cfg is null");
    cfg->c = 0.6;
    cfg->delta = 0.01;
    cfg->l_max = 64;
    cfg->eps_p = 0.f;
    cfg->c0 = 1.f;
    cfg->probe_mode = PROBESIM_PROBE_DETERMINISTIC;
    cfg->seed = 3;
    cfg->shift = 0.f;
    return PROBESIM_OK;
}

probesim_status probesim_split_error(double eps_a, double c, int32_t shift, probesim_error_split *out) {
    if (!out) return fail(PROBESIM_E_INVALID, "out is null");
    if (!(eps_a > 0.0 && eps_a < 1.0)) return fail(PROBESIM_E_INVALID, "eps_a must lie in (0, 1)");
    if (!(c > 0.0 && c < 1.0)) return fail(PROBESIM_E_INVALID, "c must lie in (0, 1)");
    const double sc = std::sqrt(c);
    const double eps = eps_a / 2.0, rest = eps_a / 2.0;
    // Rule 1: error in [0, sqrt(c)^l_max] per walk, centred by the shift
    const double eps_t = shift ? rest : rest / 2.0;
    int32_t l_max = (int32_t)std::ceil(std::log(eps_t) / std::log(sc));
    l_max = std::max(1, std::min(255, l_max));
    // Rule 2: (1 + eps) * E[l (l - 1) / 2] * eps_p = rest / 2
    const double per_walk = sc / ((1.0 - sc) * (1.0 - sc));
    double ep = rest / 2.0 / ((1.0 + eps) * per_walk);
    float epf = (float)ep;
    if ((double)epf > ep) epf = std::nextafter(epf, 0.f);
    out->eps = eps;
    out->eps_t = eps_t;
    out->l_max = l_max;
    out->eps_p = epf;
    out->shift = shift ? (float)(eps_t / 2.0) : 0.f;
    const double r1 = std::pow(sc, (double)l_max) * (shift ? 0.5 : 1.0);
    out->bound = eps + (1.0 + eps) * per_walk * (double)epf + r1;
    out->bound_paper = eps + (1.0 + eps) / (1.0 - sc) * (double)epf + r1;
    return PROBESIM_OK;
}

probesim_status probesim_graph_create(int32_t n, const int32_t *src, const int32_t *dst, int64_t m,
                                      const probesim_config *cfg, void *stream, probesim_graph **out) {
    g_last_error.clear();
    if (!out) return fail(PROBESIM_E_INVALID, "out is null");
    *out = nullptr;
    if (n < 1) return fail(PROBESIM_E_INVALID, "n must be >= 1");
    if (m < 0 || m >= ((int64_t)1 << 31)) return fail(PROBESIM_E_INVALID, "m must lie in [0, 2^31)");
    if (m > 0 && (!src || !dst)) return fail(PROBESIM_E_INVALID, "src/dst is null");
    probesim_config c;
    if (cfg) c = *cfg; else probesim_config_default(&c);
    if (!(c.c > 0.0 && c.c < 1.0)) return fail(PROBESIM_E_INVALID, "c must lie in (0, 1)");
    if (!(c.delta > 0.0 && c.delta < 1.0)) return fail(PROBESIM_E_INVALID, "delta must lie in (0, 1)");
    if (c.l_max < 1 || c.l_max > 255) return fail(PROBESIM_E_INVALID, "l_max must lie in [1, 255]");
    if (!(c.eps_p >= 0.f) || !(c.c0 >= 0.f) || !(c.shift >= 0.f))
        return fail(PROBESIM_E_INVALID, "eps_p, c0 and shift must be >= 0");
    if (c.probe_mode < 0 || c.probe_mode > 2) return fail(PROBESIM_E_INVALID, "unknown probe_mode");
    probesim_graph *g = new (std::nothrow) probesim_graph();
    if (!g) return fail(PROBESIM_E_NOMEM, "host allocation failed");
    g->cfg = c;
    g->t_stop = threshold_stop(c.c);
    g->t_keep = threshold_keep(c.c);
    cudaGetDevice(&g->device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    g->budget0 = (size_t)(0.6 * (double)tot);
    g->budget = g->budget0;
    if (g->ws0.pin_s.ensure(65536) != cudaSuccess) {
        delete g;
        return fail(PROBESIM_E_NOMEM, "pinned host allocation failed");
    }
    probesim_status s;
    {   // the edge list on the device (copied there when the caller's arrays are on the host), then the build
        const bool on_dev = m == 0 || (is_device_ptr(src) && is_device_ptr(dst));
        DevBuf staged;
        const int32_t *d_src = src, *d_dst = dst;
        s = PROBESIM_OK;
        if (!on_dev) {
            cudaError_t e = staged.ensure(2 * sizeof(int32_t) * (size_t)m);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(staged.p, src, sizeof(int32_t) * m, cudaMemcpyDefault, (cudaStream_t)stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(staged.as<int32_t>() + m, dst, sizeof(int32_t) * m, cudaMemcpyDefault,
                                    (cudaStream_t)stream);
            if (e != cudaSuccess)
                s = fail(e == cudaErrorMemoryAllocation ? PROBESIM_E_NOMEM : PROBESIM_E_CUDA,
                         std::string("staging the edge list: ") + cudaGetErrorString(e));
            d_src = staged.as<int32_t>();
            d_dst = staged.as<int32_t>() + m;
        }
        if (s == PROBESIM_OK) s = build_graph(g, n, d_src, d_dst, m, (cudaStream_t)stream);
        cudaStreamSynchronize((cudaStream_t)stream);
        staged.release();
    }
    if (s != PROBESIM_OK) {
        probesim_graph_destroy(g);
        return s;
    }
    {   // update batches allocate store versions from the device's stream-ordered pool: let it keep about three
        // versions' worth of memory between updates instead of returning it to the driver at every synchronisation
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) {
            const std::shared_ptr<StoreVersion> v = g->current();
            uint64_t keep = 0;
            for (DevBuf *b : {&v->in_off, &v->in_col, &v->out_off, &v->out_col, &v->w, &v->piece_v, &v->piece_beg,
                              &v->piece_len, &v->split_v})
                keep += b->cap;
            keep *= 3;
            uint64_t cur = 0;
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur);
            if (cur < keep) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    *out = g;
    return PROBESIM_OK;
}

probesim_status probesim_pair_mc(probesim_graph *g, const int32_t *u, const int32_t *v, const uint32_t *key_u,
                                 const uint32_t *key_v, int32_t npairs, int64_t r, int64_t *meets, float *est,
                                 void *stream) {
    if (!g || !u || !v || !key_u || !key_v || !meets) return fail(PROBESIM_E_INVALID, "null argument");
    if (npairs < 1 || npairs > 65535) return fail(PROBESIM_E_INVALID, "npairs must lie in [1, 65535]");
    if (r < 1 || r >= ((int64_t)1 << 32)) return fail(PROBESIM_E_INVALID, "r must lie in [1, 2^32)");
    for (int32_t i = 0; i < npairs; ++i)
        if (u[i] < 0 || u[i] >= g->n || v[i] < 0 || v[i] >= g->n) return fail(PROBESIM_E_RANGE, "node outside [0, n)");
    std::lock_guard<std::mutex> lk(g->mu);
    const std::shared_ptr<StoreVersion> snap = g->current();
    g_last_error.clear();
    Workspace *ws = &g->ws0;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = 4 * (size_t)npairs;
    PS_CUDA(ws->pm_in.ensure(sizeof(int32_t) * words));
    PS_CUDA(ws->pm_meets.ensure(sizeof(unsigned long long) * npairs));
    PS_CUDA(ws->pin_q.ensure(std::max(sizeof(int32_t) * words, sizeof(unsigned long long) * npairs)));
    int32_t *h = ws->pin_q.as<int32_t>();
    std::memcpy(h, u, sizeof(int32_t) * npairs);
    std::memcpy(h + npairs, v, sizeof(int32_t) * npairs);
    std::memcpy(h + 2 * npairs, key_u, sizeof(uint32_t) * npairs);
    std::memcpy(h + 3 * npairs, key_v, sizeof(uint32_t) * npairs);
    int32_t *d = ws->pm_in.as<int32_t>();
    PS_CUDA(cudaMemcpyAsync(d, h, sizeof(int32_t) * words, cudaMemcpyHostToDevice, st));
    unsigned long long *dm = ws->pm_meets.as<unsigned long long>();
    PS_CUDA(cudaMemsetAsync(dm, 0, sizeof(unsigned long long) * npairs, st));
    launch_pair_mc(snap->dg, d, d + npairs, reinterpret_cast<const uint32_t *>(d + 2 * npairs),
                   reinterpret_cast<const uint32_t *>(d + 3 * npairs), npairs, r, g->cfg.l_max, g->cfg.seed, g->t_stop,
                   dm, st);
    PS_CUDA(cudaGetLastError());
    std::vector<unsigned long long> hm(npairs);
    PS_CUDA(cudaMemcpyAsync(hm.data(), dm, sizeof(unsigned long long) * npairs, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> m64(hm.begin(), hm.end());
    std::vector<float> e(npairs);
    for (int32_t i = 0; i < npairs; ++i) e[i] = u[i] == v[i] ? 1.f : (float)((double)hm[i] / (double)r);
    if (is_device_ptr(meets)) PS_CUDA(cudaMemcpy(meets, m64.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice));
    else std::memcpy(meets, m64.data(), sizeof(int64_t) * npairs);
    if (est) {
        if (is_device_ptr(est)) PS_CUDA(cudaMemcpy(est, e.data(), sizeof(float) * npairs, cudaMemcpyHostToDevice));
        else std::memcpy(est, e.data(), sizeof(float) * npairs);
    }
    return PROBESIM_OK;
}

probesim_status probesim_set_memory_budget(probesim_graph *g, double bytes) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (!(bytes >= 0.0)) return fail(PROBESIM_E_INVALID, "bytes must be >= 0");
    std::lock_guard<std::mutex> lk(g->mu);
    g->budget = bytes > 0.0 ? (size_t)bytes : g->budget0;
    return PROBESIM_OK;
}

probesim_status probesim_graph_destroy(probesim_graph *g) {
    if (!g) return PROBESIM_OK;
    g->store.reset();
    DevBuf *bufs[] = {&g->ext2int, &g->int2ext, &g->u_batch, &g->u_valid,
                      &g->u_vpre, &g->u_delta, &g->u_deg, &g->u_part, &g->u_hist};
    for (DevBuf *b : bufs) b->release();
    g->ws0.release();
    delete g;
    return PROBESIM_OK;
}

probesim_status probesim_graph_info(const probesim_graph *g, int32_t *n, int64_t *m, uint64_t *epoch) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    const std::shared_ptr<StoreVersion> v = const_cast<probesim_graph *>(g)->current();
    if (n) *n = g->n;
    if (m) *m = v->dg.m;
    if (epoch) *epoch = v->epoch;
    return PROBESIM_OK;
}

}  // extern "C"

probesim_status ps::apply_updates(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k, bool insert,
                                  int64_t *applied, cudaStream_t st) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (k < 0 || (k > 0 && (!src || !dst))) return fail(PROBESIM_E_INVALID, "bad update batch");
    std::lock_guard<std::mutex> lk(g->update_mu);
    g_last_error.clear();
    std::vector<int32_t> hs, hd;
    PS_TRY(fetch_ids(src, k, hs));
    PS_TRY(fetch_ids(dst, k, hd));
    const int32_t n = g->n;
    const std::shared_ptr<StoreVersion> old = g->current();  // read only; queries may be reading it too
    for (int64_t e = 0; e < k; ++e)
        if (hs[e] < 0 || hs[e] >= n || hd[e] < 0 || hd[e] >= n) return fail(PROBESIM_E_RANGE, "edge id outside [0, n)");
    // the batch without loops and repeats, in the two row orders
    std::vector<uint64_t> in_keys, out_keys;
    in_keys.reserve(k);
    for (int64_t e = 0; e < k; ++e) {
        if (hs[e] == hd[e]) continue;
        in_keys.push_back(((uint64_t)(uint32_t)g->h_ext2int[hd[e]] << 32) | (uint32_t)hs[e]);  // (dst int, src ext)
    }
    std::sort(in_keys.begin(), in_keys.end());
    in_keys.erase(std::unique(in_keys.begin(), in_keys.end()), in_keys.end());
    const int64_t K = (int64_t)in_keys.size();
    if (K == 0) {  // nothing changes but the epoch: the next version shares the current one's arrays
        auto nv = std::make_shared<StoreVersion>();
        nv->base = old;
        nv->dg = old->dg;
        nv->epoch = old->epoch + 1;
        g->publish(nv);
        if (applied) *applied = 0;
        return PROBESIM_OK;
    }
    out_keys.resize(K);
    std::vector<int32_t> hb(5 * K);
    int32_t *in_dst = hb.data(), *in_src = in_dst + K, *in_src_ext = in_src + K, *out_src = in_src_ext + K,
            *out_dst = out_src + K;
    for (int64_t e = 0; e < K; ++e) {
        const int32_t d_int = (int32_t)(in_keys[e] >> 32), s_ext = (int32_t)(in_keys[e] & 0xffffffffu);
        const int32_t s_int = g->h_ext2int[s_ext];
        in_dst[e] = d_int;
        in_src[e] = s_int;
        in_src_ext[e] = s_ext;
        out_keys[e] = ((uint64_t)(uint32_t)s_int << 32) | (uint32_t)d_int;
    }
    std::sort(out_keys.begin(), out_keys.end());
    for (int64_t e = 0; e < K; ++e) {
        out_src[e] = (int32_t)(out_keys[e] >> 32);
        out_dst[e] = (int32_t)(out_keys[e] & 0xffffffffu);
    }
    const DeviceGraph &dg = old->dg;
    auto nv = std::make_shared<StoreVersion>();  // the next version, built beside the current one
    PS_CUDA(g->u_batch.ensure(sizeof(int32_t) * 5 * K));
    PS_CUDA(g->u_valid.ensure(sizeof(long long) * 2 * K));
    PS_CUDA(g->u_vpre.ensure(sizeof(long long) * 2 * (K + 1)));
    PS_CUDA(g->u_delta.ensure(sizeof(long long) * 2 * (size_t)n));
    PS_CUDA(g->u_deg.ensure(sizeof(long long) * 2 * ((size_t)n + 1)));
    PS_CUDA(g->u_part.ensure(sizeof(long long) * scan64_partials_needed(std::max<int64_t>(K, n))));
    PS_CUDA(g->u_hist.ensure(sizeof(unsigned long long) * (2 * (kPiece + 1) + 2)));
    PS_CUDA(cudaMemcpyAsync(g->u_batch.p, hb.data(), sizeof(int32_t) * 5 * K, cudaMemcpyHostToDevice, st));
    int32_t *db = g->u_batch.as<int32_t>();
    UpdateBatchArgs a;
    a.k = K;
    a.in_dst = db; a.in_src = db + K; a.in_src_ext = db + 2 * K; a.out_src = db + 3 * K; a.out_dst = db + 4 * K;
    a.in_valid = g->u_valid.as<long long>();
    a.out_valid = a.in_valid + K;
    long long *in_vpre = g->u_vpre.as<long long>(), *out_vpre = in_vpre + (K + 1);
    a.in_vpre = in_vpre;
    a.out_vpre = out_vpre;
    a.insert = insert;
    long long *in_delta = g->u_delta.as<long long>(), *out_delta = in_delta + n;
    PS_CUDA(cudaMemsetAsync(in_delta, 0, sizeof(long long) * 2 * (size_t)n, st));
    launch_upd_mark(dg, a, in_delta, out_delta, st);
    launch_scan64(a.in_valid, K, g->u_part.as<long long>(), in_vpre, st);
    launch_scan64(a.out_valid, K, g->u_part.as<long long>(), out_vpre, st);
    // new offsets
    long long *deg = g->u_deg.as<long long>(), *deg_out = deg + (n + 1);
    DevBuf &n_in_off = nv->in_off, &n_out_off = nv->out_off, &n_in_col = nv->in_col, &n_out_col = nv->out_col;
    PS_CUDA(n_in_off.alloc_pooled(sizeof(int64_t) * ((size_t)n + 1), st));
    PS_CUDA(n_out_off.alloc_pooled(sizeof(int64_t) * ((size_t)n + 1), st));
    launch_upd_degrees(n, dg.in_off, in_delta, deg, st);
    launch_scan64(deg, n, g->u_part.as<long long>(), n_in_off.as<long long>(), st);
    launch_upd_degrees(n, dg.out_off, out_delta, deg_out, st);
    launch_scan64(deg_out, n, g->u_part.as<long long>(), n_out_off.as<long long>(), st);
    long long hm[3] = {0, 0, 0};
    PS_CUDA(cudaMemcpyAsync(&hm[0], n_in_off.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&hm[1], n_out_off.as<long long>() + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&hm[2], in_vpre + K, sizeof(long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t m2 = hm[0];
    if (m2 != hm[1]) return fail(PROBESIM_E_CUDA, "internal: in- and out-lists disagree after the update");
    if (m2 >= ((int64_t)1 << 31)) return fail(PROBESIM_E_INVALID, "edge count would reach 2^31");
    PS_CUDA(n_in_col.alloc_pooled(sizeof(int32_t) * std::max<int64_t>(1, m2), st));
    PS_CUDA(n_out_col.alloc_pooled(sizeof(int32_t) * std::max<int64_t>(1, m2), st));
    launch_upd_rows(dg, a, true, n_in_off.as<long long>(), n_in_col.as<int32_t>(), st);
    launch_upd_rows(dg, a, false, n_out_off.as<long long>(), n_out_col.as<int32_t>(), st);
    // w and pieces of the new in-lists
    const int64_t cap_pieces = (int64_t)n + m2 / kPiece + 1;
    DevBuf &n_pv = nv->piece_v, &n_pb = nv->piece_beg, &n_pl = nv->piece_len, &n_split = nv->split_v;
    PS_CUDA(n_pv.alloc_pooled(sizeof(int32_t) * cap_pieces, st));
    PS_CUDA(n_pb.alloc_pooled(sizeof(int64_t) * cap_pieces, st));
    PS_CUDA(n_pl.alloc_pooled(sizeof(int32_t) * cap_pieces, st));
    PS_CUDA(n_split.alloc_pooled(sizeof(int32_t) * (size_t)n, st));
    PS_CUDA(nv->w.alloc_pooled(sizeof(float) * (size_t)n, st));
    launch_upd_w(n, n_in_off.as<long long>(), (float)std::sqrt(g->cfg.c), nv->w.as<float>(), deg, st);
    unsigned long long *hist = g->u_hist.as<unsigned long long>(), *cursor = hist + (kPiece + 1),
                       *nsplit = cursor + (kPiece + 1);
    launch_upd_pieces(n, n_in_off.as<long long>(), hist, cursor, n_split.as<int32_t>(), nsplit, n_pv.as<int32_t>(),
                      n_pb.as<int64_t>(), n_pl.as<int32_t>(), st);
    // the rows with out-edges after the batch (the last slot of the histogram buffer is free)
    int32_t *d_active = reinterpret_cast<int32_t *>(nsplit + 1);
    PS_CUDA(cudaMemsetAsync(d_active, 0, sizeof(int32_t), st));
    launch_active_rows(n_out_off.as<int64_t>(), n, d_active, st);
    std::vector<unsigned long long> hh(kPiece + 2);
    int32_t n_active = 0;
    PS_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned long long) * (kPiece + 1), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(hh.data() + kPiece + 1, nsplit, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&n_active, d_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaStreamSynchronize(st));
    int64_t npieces = 0;
    for (int len = 0; len <= kPiece; ++len) npieces += (int64_t)hh[len];
    // publish the new version: queries that start from now on read it, those in flight keep the old one
    DeviceGraph &ng = nv->dg;
    ng = dg;
    ng.m = m2;
    ng.in_off = nv->in_off.as<int64_t>();
    ng.out_off = nv->out_off.as<int64_t>();
    ng.in_col = nv->in_col.as<int32_t>();
    ng.out_col = nv->out_col.as<int32_t>();
    ng.w = nv->w.as<float>();
    ng.n_pieces = npieces;
    ng.piece_v = nv->piece_v.as<int32_t>();
    ng.piece_beg = nv->piece_beg.as<int64_t>();
    ng.piece_len = nv->piece_len.as<int32_t>();
    ng.n_split = (int32_t)hh[kPiece + 1];
    ng.split_v = nv->split_v.as<int32_t>();
    ng.n_active = n_active;
    nv->epoch = old->epoch + 1;
    g->publish(nv);
    if (applied) *applied = hm[2];
    return PROBESIM_OK;
}

extern "C" {

probesim_status probesim_insert_edges(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k,
                                      int64_t *applied, void *stream) {
    return apply_updates(g, src, dst, k, true, applied, (cudaStream_t)stream);
}

probesim_status probesim_delete_edges(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k,
                                      int64_t *applied, void *stream) {
    return apply_updates(g, src, dst, k, false, applied, (cudaStream_t)stream);
}

probesim_status probesim_num_walks(const probesim_graph *g, double eps, int64_t *n_r) {
    if (!g || !n_r) return fail(PROBESIM_E_INVALID, "null argument");
    if (!(eps > 0.0 && eps < 1.0)) return fail(PROBESIM_E_INVALID, "eps must lie in (0, 1)");
    *n_r = num_walks(g->cfg.c, eps, g->cfg.delta, g->n);
    return PROBESIM_OK;
}

probesim_status probesim_sample_walks(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t *nodes,
                                      int32_t *lens, int64_t capacity, void *stream) {
    if (!g || !nodes || !lens) return fail(PROBESIM_E_INVALID, "null argument");
    PS_TRY(check_queries(g, q, nq, false, 0));
    std::lock_guard<std::mutex> lk(g->mu);
    const std::shared_ptr<StoreVersion> snap = g->current();
    g_last_error.clear();
    Workspace *ws = &g->ws0;
    cudaStream_t st = (cudaStream_t)stream;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, nq, P));
    if (P.W > capacity) return fail(PROBESIM_E_INVALID, "walk buffer too small");
    QueryBatch qb;
    PS_TRY(upload_batch(ws, P, qb, st));
    const int32_t L = g->cfg.l_max;
    const bool dev_nodes = is_device_ptr(nodes), dev_lens = is_device_ptr(lens);
    PS_CUDA(ws->walks.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_CUDA(ws->lens.ensure(sizeof(int32_t) * std::max<int32_t>(1, P.W)));
    PS_CUDA(ws->ctr.ensure(sizeof(LaunchCounters)));
    PS_CUDA(cudaMemsetAsync(ws->ctr.p, 0, sizeof(LaunchCounters), st));
    int32_t *wd = dev_nodes ? nodes : ws->walks.as<int32_t>();
    int32_t *ld = dev_lens ? lens : ws->lens.as<int32_t>();
    launch_walks(snap->dg, qb, P.W, L, g->t_stop, g->cfg.seed, wd, ld, true, ws->ctr.as<LaunchCounters>(), st);
    ps::launch_map_ids(wd, (int64_t)P.W * L, snap->dg.int2ext, st);
    PS_CUDA(cudaGetLastError());
    if (!dev_nodes)
        PS_CUDA(cudaMemcpyAsync(nodes, wd, sizeof(int32_t) * (size_t)P.W * L, cudaMemcpyDeviceToHost, st));
    if (!dev_lens) PS_CUDA(cudaMemcpyAsync(lens, ld, sizeof(int32_t) * (size_t)P.W, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    return PROBESIM_OK;
}

}  // extern "C"

// Single-source estimates of nq queries into `scores` (host or device) using workspace ws.  The caller holds
// the store lock (shared) and owns ws.
probesim_status ps::single_source_core(probesim_graph *g, Workspace *ws, const std::shared_ptr<StoreVersion> &snap,
                                          const probesim_query *q, int32_t nq, float *scores, cudaStream_t st) {
    ws->stats = probesim_stats{};
    ws->snap = snap;
    ws->dg = snap->dg;
    struct Release {
        Workspace *w;
        ~Release() { w->snap.reset(); }
    } release{ws};
    const bool dev = is_device_ptr(scores);
    float *d_out = scores;
    const size_t out_bytes = sizeof(float) * (size_t)nq * g->n;
    if (!dev) {
        PS_CUDA(ws->out_stage.ensure(out_bytes));
        d_out = ws->out_stage.as<float>();
    }
    PS_TRY(run_queries(g, ws, q, nq, d_out, st));
    if (!dev) {
        PS_CUDA(cudaMemcpyAsync(scores, d_out, out_bytes, cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
    }
    return PROBESIM_OK;
}

// Top-k of nq queries (ids/vals host or device, [nq][kmax]) using workspace ws; same locking as above.
probesim_status ps::topk_core(probesim_graph *g, Workspace *ws, const std::shared_ptr<StoreVersion> &snap,
                                 const probesim_query *q, int32_t nq, int32_t kmax, int32_t *ids, float *vals,
                                 cudaStream_t st) {
    ws->stats = probesim_stats{};
    ws->snap = snap;
    ws->dg = snap->dg;
    struct Release {
        Workspace *w;
        ~Release() { w->snap.reset(); }
    } release{ws};
    const int32_t n = g->n;
    // scores of a chunk of queries, then the selection
    const int32_t chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)(budget_of(g, ws) / 8) / ((int64_t)n * 4)));
    PS_CUDA(ws->out_stage.ensure(sizeof(float) * (size_t)chunk * n));
    const int nblk = topk_blocks_per_query(n);
    PS_CUDA(ws->tk_hist.ensure(sizeof(unsigned) * 256 * chunk));
    PS_CUDA(ws->tk_state.ensure(sizeof(unsigned) * 4 * chunk));
    PS_CUDA(ws->tk_tie.ensure(sizeof(unsigned) * (size_t)nblk * chunk));
    PS_CUDA(ws->tk_cid.ensure(sizeof(int32_t) * (size_t)kmax * chunk));
    PS_CUDA(ws->tk_cval.ensure(sizeof(float) * (size_t)kmax * chunk));
    PS_CUDA(ws->tk_qk.ensure(sizeof(int32_t) * 2 * chunk));
    const bool dev_ids = is_device_ptr(ids), dev_vals = is_device_ptr(vals);
    if (!dev_ids) PS_CUDA(ws->tk_ids.ensure(sizeof(int32_t) * (size_t)kmax * chunk));
    if (!dev_vals) PS_CUDA(ws->tk_vals.ensure(sizeof(float) * (size_t)kmax * chunk));
    std::vector<int32_t> hq(2 * chunk);
    for (int32_t done = 0; done < nq; done += chunk) {
        const int32_t B = std::min(chunk, nq - done);
        PS_TRY(run_queries(g, ws, q + done, B, ws->out_stage.as<float>(), st));
        for (int32_t b = 0; b < B; ++b) {
            hq[b] = q[done + b].node;
            hq[chunk + b] = q[done + b].k;
        }
        int32_t *d_qn = ws->tk_qk.as<int32_t>(), *d_qk = d_qn + chunk;
        PS_CUDA(cudaMemcpyAsync(d_qn, hq.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaMemcpyAsync(d_qk, hq.data() + chunk, sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
        TopkScratch sc;
        sc.hist = ws->tk_hist.as<unsigned>();
        sc.state = ws->tk_state.as<unsigned>();
        sc.tiecnt = ws->tk_tie.as<unsigned>();
        sc.cand_id = ws->tk_cid.as<int32_t>();
        sc.cand_val = ws->tk_cval.as<float>();
        int32_t *oi = dev_ids ? ids + (int64_t)done * kmax : ws->tk_ids.as<int32_t>();
        float *ov = dev_vals ? vals + (int64_t)done * kmax : ws->tk_vals.as<float>();
        launch_topk(n, B, ws->out_stage.as<float>(), d_qn, d_qk, kmax, sc, oi, ov, st, &ws->stats.kernel_launches);
        PS_CUDA(cudaGetLastError());
        if (!dev_ids)
            PS_CUDA(cudaMemcpyAsync(ids + (int64_t)done * kmax, oi, sizeof(int32_t) * (size_t)B * kmax,
                                    cudaMemcpyDeviceToHost, st));
        if (!dev_vals)
            PS_CUDA(cudaMemcpyAsync(vals + (int64_t)done * kmax, ov, sizeof(float) * (size_t)B * kmax,
                                    cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
    }
    return PROBESIM_OK;
}

extern "C" {

probesim_status probesim_single_source(probesim_graph *g, const probesim_query *q, int32_t nq, float *scores,
                                       void *stream) {
    if (!g || !scores) return fail(PROBESIM_E_INVALID, "null argument");
    PS_TRY(check_queries(g, q, nq, false, 0));
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    return single_source_core(g, &g->ws0, g->current(), q, nq, scores, (cudaStream_t)stream);
}

probesim_status probesim_topk(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t kmax, int32_t *ids,
                              float *vals, void *stream) {
    if (!g || !ids || !vals) return fail(PROBESIM_E_INVALID, "null argument");
    if (kmax < 1 || kmax > 4096 || kmax > g->n - 1) return fail(PROBESIM_E_INVALID, "kmax must lie in [1, min(4096, n-1)]");
    PS_TRY(check_queries(g, q, nq, true, kmax));
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    return topk_core(g, &g->ws0, g->current(), q, nq, kmax, ids, vals, (cudaStream_t)stream);
}

// Times the pull on this graph's in-lists for every tile width in {1, 2, 4, 8, 16, 32} and blocks-per-SM in
// {2, 4, 8, 16} over a random score matrix, keeps the fastest shape per width, and picks the full tiles' launch
// (16-column halves, 32-column tiles, or 32-column tiles two per pass) by time per column.  The choice is stored in the graph and used by every later query.
probesim_status probesim_autotune(probesim_graph *g, void *stream) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    std::lock_guard<std::mutex> lk(g->mu);
    const std::shared_ptr<StoreVersion> snap = g->current();
    g_last_error.clear();
    cudaStream_t st = (cudaStream_t)stream;
    const DeviceGraph &dg = snap->dg;
    const int32_t n = dg.n, P = 64;
    Workspace *ws = &g->ws0;
    PS_CUDA(ws->md_a.ensure((size_t)(n + 1) * P * sizeof(float)));  // a spare row after the n rows
    PS_CUDA(ws->md_b.ensure((size_t)(n + 1) * P * sizeof(float)));
    PS_CUDA(cudaMemsetAsync(ws->md_a.p, 0x3c, (size_t)(n + 1) * P * sizeof(float), st));  // any finite values
    const int32_t tiles[] = {1, 2, 4, 8, 16}, bpss[] = {2, 4, 8, 16};
    Timer tm{ws, st};
    // times one configuration: three runs after a warm-up run, in ms
    auto time_pull = [&](auto &&launch) -> float {
        float total = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEvent_t e0 = tm.get(), e1 = tm.get();
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) total += ms;
        }
        return total;
    };
    float *Da = ws->md_a.as<float>(), *Mb = ws->md_b.as<float>();
    // tail tiles: one narrow tile over a compact [n][T] block
    for (int32_t T : tiles) {
        float best = 1e30f;
        for (int32_t bps : bpss) {
            const float ms = time_pull([&] { launch_pull(dg, Da, T, 0, 1, Mb, T, 0, 1, 1, T, bps, nullptr, st); });
            if (ms < best) best = ms, g->tune_bps[T] = bps;
        }
    }
    // wide tiles: two 32-column tiles of a node-major [n][64] matrix, as 32-column tiles, 16-column halves, or one
    // pass over both
    double per_col[kPullTma + 1] = {0};
    int32_t wide_bps[kPullTma + 1] = {0};
    for (int32_t T : {16, 32, kPullPairs}) {
        float best = 1e30f;
        for (int32_t bps : bpss) {
            const int32_t nt = T == 16 ? 4 : 2;
            const float ms =
                time_pull([&] { launch_pull(dg, Da, P, 0, 1 << 30, Mb, P, 0, 1 << 30, nt, T, bps, nullptr, st); });
            if (ms < best) best = ms, wide_bps[T] = bps;
        }
        per_col[T] = best / 3.0 / 64.0;
    }
    if (pull_tma_available()) {  // the TMA gathers (one block of 192 KB shared memory per SM)
        PS_CUDA(ws->pull_err.ensure(sizeof(int32_t)));
        PS_CUDA(cudaMemsetAsync(ws->pull_err.p, 0, sizeof(int32_t), st));
        cudaError_t le = cudaSuccess;
        const float best = time_pull([&] {
            le = launch_pull_tma(dg, Da, P, P, 0, 1 << 30, Mb, P, 0, 1 << 30, 2, 1, nullptr, ws->pull_err.as<int32_t>(),
                                 st);
        });
        PS_CUDA(le);
        wide_bps[kPullTma] = 1;
        int32_t herr = 0;
        PS_CUDA(cudaMemcpyAsync(&herr, ws->pull_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        if (herr) return fail(PROBESIM_E_TIMEOUT, "a TMA row gather of the pull did not complete in time");
        per_col[kPullTma] = best / 3.0 / 64.0;
    }
    PS_CUDA(cudaGetLastError());
    int32_t pick = 32;
    for (int32_t T : {16, kPullPairs, kPullTma})
        if (per_col[T] > 0 && per_col[T] < per_col[pick]) pick = T;
    g->tune_bps[32] = wide_bps[32];
    g->tune_bps[pick] = wide_bps[pick];
    g->tune_wide = pick;
    g->tuned = 1;
    PS_CUDA(cudaGetLastError());
    return PROBESIM_OK;
}

probesim_status probesim_set_tuning(probesim_graph *g, int32_t wide_tile, const int32_t *blocks_per_sm) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (wide_tile != 16 && wide_tile != 32 && wide_tile != kPullPairs && wide_tile != kPullTma)
        return fail(PROBESIM_E_INVALID, "wide_tile must be 16, 32, 64 or 96");
    if (wide_tile == kPullTma && !pull_tma_available())
        return fail(PROBESIM_E_UNSUPPORTED, "no tensor-map encoder in this driver");
    if (blocks_per_sm)
        for (int i = 0; i < 8; ++i)
            if (blocks_per_sm[i] < 1 || blocks_per_sm[i] > 32)
                return fail(PROBESIM_E_INVALID, "blocks_per_sm must lie in [1, 32]");
    std::lock_guard<std::mutex> lk(g->mu);
    g->tune_wide = wide_tile;
    if (blocks_per_sm) {
        for (int i = 0; i < 6; ++i) g->tune_bps[1 << i] = blocks_per_sm[i];
        g->tune_bps[kPullPairs] = blocks_per_sm[6];
        g->tune_bps[kPullTma] = blocks_per_sm[7];
    }
    return PROBESIM_OK;
}

probesim_status probesim_get_tuning(const probesim_graph *g, int32_t *wide_tile, int32_t *blocks_per_sm) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (wide_tile) *wide_tile = g->tune_wide;
    if (blocks_per_sm)
        for (int i = 0; i < 6; ++i) blocks_per_sm[i] = g->tune_bps[1 << i] ? g->tune_bps[1 << i] : 8;
    return PROBESIM_OK;
}

probesim_status probesim_set_profiling(probesim_graph *g, int32_t on) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    std::lock_guard<std::mutex> lk(g->mu);
    g->ws0.profiling = on ? 1 : 0;
    return PROBESIM_OK;
}

probesim_status probesim_get_stats(const probesim_graph *g, probesim_stats *out) {
    if (!g || !out) return fail(PROBESIM_E_INVALID, "null argument");
    *out = g->ws0.stats;
    return PROBESIM_OK;
}

}  // extern "C"
