// C ABI of libprobesim.so: the graph store, the query engine and the entry points of include/probesim.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

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

#define PS_CUDA(expr)                                                                                  \
    do {                                                                                               \
        cudaError_t _e = (expr);                                                                       \
        if (_e != cudaSuccess) {                                                                       \
            return fail(_e == cudaErrorMemoryAllocation ? PROBESIM_E_NOMEM : PROBESIM_E_CUDA,          \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                           \
        }                                                                                              \
    } while (0)

#define PS_TRY(expr)                                  \
    do {                                              \
        probesim_status _s = (expr);                  \
        if (_s != PROBESIM_OK) return _s;             \
    } while (0)

// ------------------------------------------------------------------------------------------------
// device buffers that grow on demand and are freed with the graph
// ------------------------------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t nb = std::max<size_t>(256, bytes + bytes / 8);
        cudaError_t e = cudaMalloc(&p, nb);
        if (e == cudaSuccess) cap = nb; else cudaGetLastError();
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

struct PinnedBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t nb = std::max<size_t>(256, bytes + bytes / 8);
        cudaError_t e = cudaMallocHost(&p, nb);
        if (e == cudaSuccess) cap = nb; else cudaGetLastError();
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

struct probesim_graph {
    std::mutex mu;
    probesim_config cfg{};
    uint32_t t_stop = 0;
    int device = 0;
    DeviceGraph dg;
    // device arrays of the graph store
    DevBuf in_off, in_col, out_off, out_col, w, piece_v, piece_beg, piece_len, split_v;
    // host copy of the edge set as sorted keys (dst << 32 | src), used to apply update batches
    std::vector<uint64_t> keys;
    uint64_t epoch = 0;
    // query workspace
    DevBuf qbuf, walks, lens, ctr;
    DevBuf t_key, t_node, t_parent, t_depth, t_query, t_weight, t_height, t_slot, t_gamma, t_G;
    DevBuf counts, offs, node_list, slot_entry, nchild, child_off, child_list, ccur, rho_slot;
    DevBuf md_a, md_b, dmat, out_stage;
    DevBuf tk_hist, tk_state, tk_tie, tk_cid, tk_cval, tk_ids, tk_vals, tk_qk;
    PinnedBuf pin_q;  // query arrays of one batch
    PinnedBuf pin_s;  // counters and schedule offsets (fixed size, allocated at creation)
    // profiling
    int profiling = 0;
    std::vector<cudaEvent_t> ev;
    probesim_stats stats{};
    size_t budget = 0;
};

static uint32_t threshold_stop(double c) { return (uint32_t)std::floor((1.0 - std::sqrt(c)) * 4294967296.0); }

static int64_t num_walks(double c, double eps, double delta, int64_t n) {
    return (int64_t)std::ceil(3.0 * c / (eps * eps) * std::log((double)n / delta));
}

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

// Builds in-CSR (rows by destination, sources ascending), out-CSR (rows by source, destinations
// ascending), w[v] = sqrt(c)/|I(v)| and the pull pieces from the sorted unique keys, and uploads them.
static probesim_status upload_graph(probesim_graph *g, int32_t n, cudaStream_t st) {
    const std::vector<uint64_t> &K = g->keys;
    const int64_t m = (int64_t)K.size();
    std::vector<int64_t> in_off(n + 1, 0), out_off(n + 1, 0);
    std::vector<int32_t> in_col(std::max<int64_t>(1, m)), out_col(std::max<int64_t>(1, m));
    for (int64_t e = 0; e < m; ++e) {
        in_off[(K[e] >> 32) + 1]++;
        out_off[(K[e] & 0xffffffffu) + 1]++;
        in_col[e] = (int32_t)(K[e] & 0xffffffffu);
    }
    for (int32_t v = 0; v < n; ++v) {
        in_off[v + 1] += in_off[v];
        out_off[v + 1] += out_off[v];
    }
    {
        std::vector<int64_t> cur(out_off.begin(), out_off.end() - 1);
        for (int64_t e = 0; e < m; ++e) {  // keys ascend by destination: each out-row fills in ascending order
            const int32_t src = (int32_t)(K[e] & 0xffffffffu);
            out_col[cur[src]++] = (int32_t)(K[e] >> 32);
        }
    }
    const float sc = (float)std::sqrt(g->cfg.c);
    std::vector<float> w(n);
    for (int32_t v = 0; v < n; ++v) {
        const int64_t d = in_off[v + 1] - in_off[v];
        w[v] = d > 0 ? sc / (float)d : 0.f;
    }
    // pieces: in-lists cut into at most kPiece edges; ordered by length, longest first (counting sort)
    std::vector<int32_t> split;
    std::vector<int64_t> per_len(kPiece + 2, 0);
    for (int32_t v = 0; v < n; ++v) {
        const int64_t d = in_off[v + 1] - in_off[v];
        if (d > kPiece) {
            split.push_back(v);
            per_len[kPiece] += d / kPiece;
            if (d % kPiece) per_len[d % kPiece] += 1;
        } else {
            per_len[d] += 1;
        }
    }
    std::vector<int64_t> start(kPiece + 2, 0);  // longest first: bucket kPiece, kPiece-1, ..., 0
    for (int len = kPiece, acc = 0; len >= 0; --len) { start[len] = acc; acc += (int)per_len[len]; }
    int64_t npieces = 0;
    for (int len = 0; len <= kPiece; ++len) npieces += per_len[len];
    std::vector<int32_t> pv(std::max<int64_t>(1, npieces)), pl(std::max<int64_t>(1, npieces));
    std::vector<int64_t> pb(std::max<int64_t>(1, npieces));
    {
        std::vector<int64_t> cur(start);
        auto put = [&](int32_t v, int64_t beg, int64_t len, bool sp) {
            const int64_t i = cur[len]++;
            pv[i] = v;
            pb[i] = beg;
            pl[i] = (int32_t)len | (sp ? (int32_t)0x80000000 : 0);
        };
        for (int32_t v = 0; v < n; ++v) {
            const int64_t beg = in_off[v], d = in_off[v + 1] - beg;
            if (d <= kPiece) { put(v, beg, d, false); continue; }
            const int64_t full = d / kPiece, rest = d % kPiece;
            for (int64_t c = 0; c < full; ++c) put(v, beg + c * kPiece, kPiece, true);
            if (rest) put(v, beg + full * kPiece, rest, true);
        }
    }
    pv.resize(npieces);
    pb.resize(npieces);
    pl.resize(npieces);
    PS_CUDA(g->in_off.ensure(sizeof(int64_t) * (n + 1)));
    PS_CUDA(g->out_off.ensure(sizeof(int64_t) * (n + 1)));
    PS_CUDA(g->in_col.ensure(sizeof(int32_t) * std::max<int64_t>(1, m)));
    PS_CUDA(g->out_col.ensure(sizeof(int32_t) * std::max<int64_t>(1, m)));
    PS_CUDA(g->w.ensure(sizeof(float) * n));
    PS_CUDA(g->piece_v.ensure(sizeof(int32_t) * std::max<size_t>(1, pv.size())));
    PS_CUDA(g->piece_beg.ensure(sizeof(int64_t) * std::max<size_t>(1, pb.size())));
    PS_CUDA(g->piece_len.ensure(sizeof(int32_t) * std::max<size_t>(1, pl.size())));
    PS_CUDA(g->split_v.ensure(sizeof(int32_t) * std::max<size_t>(1, split.size())));
    PS_CUDA(cudaMemcpyAsync(g->in_off.p, in_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(g->out_off.p, out_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (m > 0) {
        PS_CUDA(cudaMemcpyAsync(g->in_col.p, in_col.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaMemcpyAsync(g->out_col.p, out_col.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    }
    PS_CUDA(cudaMemcpyAsync(g->w.p, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(g->piece_v.p, pv.data(), sizeof(int32_t) * pv.size(), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(g->piece_beg.p, pb.data(), sizeof(int64_t) * pb.size(), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(g->piece_len.p, pl.data(), sizeof(int32_t) * pl.size(), cudaMemcpyHostToDevice, st));
    if (!split.empty())
        PS_CUDA(cudaMemcpyAsync(g->split_v.p, split.data(), sizeof(int32_t) * split.size(), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaStreamSynchronize(st));
    DeviceGraph &d = g->dg;
    d.n = n;
    d.m = m;
    d.in_off = g->in_off.as<int64_t>();
    d.in_col = g->in_col.as<int32_t>();
    d.out_off = g->out_off.as<int64_t>();
    d.out_col = g->out_col.as<int32_t>();
    d.w = g->w.as<float>();
    d.n_pieces = (int64_t)pv.size();
    d.piece_v = g->piece_v.as<int32_t>();
    d.piece_beg = g->piece_beg.as<int64_t>();
    d.piece_len = g->piece_len.as<int32_t>();
    d.n_split = (int32_t)split.size();
    d.split_v = g->split_v.as<int32_t>();
    return PROBESIM_OK;
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
        const int64_t nr = num_walks(g->cfg.c, q[b].eps, g->cfg.delta, g->dg.n);
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
static probesim_status upload_batch(probesim_graph *g, const BatchPlan &P, QueryBatch &qb, cudaStream_t st) {
    const int32_t B = P.B;
    const size_t bytes = sizeof(int32_t) * (4 * (size_t)B + 1) + sizeof(float) * B + 64;
    PS_CUDA(g->pin_q.ensure(bytes));
    PS_CUDA(g->qbuf.ensure(bytes));
    char *h = g->pin_q.as<char>();
    int32_t *hn = reinterpret_cast<int32_t *>(h);
    std::memcpy(hn, P.node.data(), sizeof(int32_t) * B);
    std::memcpy(hn + B, P.qid.data(), sizeof(uint32_t) * B);
    std::memcpy(hn + 2 * B, P.base.data(), sizeof(int32_t) * (B + 1));
    std::memcpy(hn + 3 * B + 1, P.k0.data(), sizeof(int32_t) * B);
    std::memcpy(hn + 4 * B + 1, P.inv_nr.data(), sizeof(float) * B);
    PS_CUDA(cudaMemcpyAsync(g->qbuf.p, h, bytes, cudaMemcpyHostToDevice, st));
    int32_t *d = g->qbuf.as<int32_t>();
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
    probesim_graph *g;
    cudaStream_t st;
    size_t used = 0;
    cudaEvent_t get() {
        if (used == g->ev.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            g->ev.push_back(e);
        }
        return g->ev[used++];
    }
};

// Runs the query path for one batch into d_out ([B][n] on the device).  Returns PROBESIM_E_NOMEM with
// *too_big set when the level buffers of this batch would exceed the workspace budget.
static probesim_status run_batch(probesim_graph *g, const probesim_query *q, int32_t B, float *d_out, cudaStream_t st,
                                 bool *too_big) {
    *too_big = false;
    const DeviceGraph &dg = g->dg;
    const int32_t n = dg.n;
    const int32_t L = g->cfg.l_max;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, B, P));
    if ((size_t)P.W * L * 4 > g->budget / 4 && B > 1) {
        *too_big = true;
        return PROBESIM_E_NOMEM;
    }
    QueryBatch qb;
    PS_TRY(upload_batch(g, P, qb, st));
    int64_t launches = 0;
    // 1. walks (Def. 3)
    PS_CUDA(g->walks.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_CUDA(g->lens.ensure(sizeof(int32_t) * std::max<int32_t>(1, P.W)));
    PS_CUDA(g->ctr.ensure(sizeof(LaunchCounters)));
    LaunchCounters *d_ctr = g->ctr.as<LaunchCounters>();
    PS_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(LaunchCounters), st));
    launch_walks(dg, qb, P.W, L, g->t_stop, g->cfg.seed, g->walks.as<int32_t>(), g->lens.as<int32_t>(), false, d_ctr, st);
    ++launches;
    LaunchCounters *h_ctr = g->pin_s.as<LaunchCounters>();
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const int64_t walk_nodes = (int64_t)h_ctr->walk_nodes;
    g->stats.walks += P.W;
    g->stats.walk_nodes += walk_nodes;
    // 2. reverse-reachability tree (Alg. 4) in a hash table at load <= 1/2
    TrieTable t;
    t.cap = next_pow2(std::max<int64_t>(1024, 2 * (walk_nodes + B) + 64));
    const size_t cap = (size_t)t.cap;
    PS_CUDA(g->t_key.ensure(8 * cap));
    PS_CUDA(g->t_node.ensure(4 * cap));
    PS_CUDA(g->t_parent.ensure(4 * cap));
    PS_CUDA(g->t_depth.ensure(4 * cap));
    PS_CUDA(g->t_query.ensure(4 * cap));
    PS_CUDA(g->t_weight.ensure(4 * cap));
    PS_CUDA(g->t_height.ensure(4 * cap));
    PS_CUDA(g->t_slot.ensure(4 * cap));
    PS_CUDA(g->t_gamma.ensure(4 * cap));
    PS_CUDA(g->t_G.ensure(4 * cap));
    t.key = g->t_key.as<unsigned long long>();
    t.node = g->t_node.as<int32_t>();
    t.parent = g->t_parent.as<int32_t>();
    t.depth = g->t_depth.as<int32_t>();
    t.query = g->t_query.as<int32_t>();
    t.weight = g->t_weight.as<int32_t>();
    t.height = g->t_height.as<int32_t>();
    t.slot = g->t_slot.as<int32_t>();
    t.gamma = g->t_gamma.as<float>();
    t.G = g->t_G.as<float>();
    PS_CUDA(cudaMemsetAsync(t.key, 0xFF, 8 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.weight, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.height, 0, 4 * cap, st));
    PS_CUDA(cudaMemsetAsync(t.G, 0, 4 * cap, st));
    launch_trie_insert(dg, qb, P.W, L, g->walks.as<int32_t>(), g->lens.as<int32_t>(), t, d_ctr, st);
    ++launches;
    // 3. level schedule: nodes and vector slots per depth
    const int32_t D1 = L + 2;
    PS_CUDA(g->counts.ensure(sizeof(int32_t) * 4 * D1));
    int32_t *d_ncount = g->counts.as<int32_t>(), *d_scount = d_ncount + D1, *d_ncur = d_ncount + 2 * D1;
    PS_CUDA(cudaMemsetAsync(d_ncount, 0, sizeof(int32_t) * 3 * D1, st));
    launch_sched_count(t, d_ncount, d_scount, st);
    ++launches;
    int32_t *h_cnt = reinterpret_cast<int32_t *>(g->pin_s.as<char>() + 256);
    PS_CUDA(cudaMemcpyAsync(h_cnt, d_ncount, sizeof(int32_t) * 2 * D1, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(LaunchCounters), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    if (h_ctr->overflow) return fail(PROBESIM_E_CUDA, "internal: walk tree table overflow");
    std::vector<int32_t> ncount(h_cnt, h_cnt + D1), scount(h_cnt + D1, h_cnt + 2 * D1);
    int32_t Dmax = 0;
    for (int32_t d = 0; d < D1; ++d)
        if (ncount[d] > 0) Dmax = d;
    std::vector<int32_t> node_off(D1 + 1, 0), slot_off(D1 + 1, 0), pitch(D1, 0), tile(D1, 1);
    int64_t maxpitch = 1;
    for (int32_t d = 0; d < D1; ++d) {
        node_off[d + 1] = node_off[d] + ncount[d];
        slot_off[d + 1] = slot_off[d] + scount[d];
        if (scount[d] > 0) {
            tile[d] = pull_tile_for(scount[d]);
            pitch[d] = round_up(scount[d], tile[d]);
            maxpitch = std::max<int64_t>(maxpitch, pitch[d]);
        }
    }
    const int32_t total_nodes = node_off[D1], S_total = slot_off[D1];
    g->stats.tree_nodes += total_nodes;
    g->stats.vectors += S_total;
    const size_t level_bytes = 3 * (size_t)n * (size_t)maxpitch * sizeof(float);
    if (level_bytes > g->budget) {
        *too_big = B > 1;
        return fail(PROBESIM_E_NOMEM, "score vectors of one query exceed the workspace budget");
    }
    PS_CUDA(g->offs.ensure(sizeof(int32_t) * 2 * (D1 + 1)));
    int32_t *d_node_off = g->offs.as<int32_t>(), *d_slot_off = d_node_off + D1 + 1;
    int32_t *h_offs = h_cnt + 2 * D1;
    std::memcpy(h_offs, node_off.data(), sizeof(int32_t) * (D1 + 1));
    std::memcpy(h_offs + D1 + 1, slot_off.data(), sizeof(int32_t) * (D1 + 1));
    PS_CUDA(cudaMemcpyAsync(d_node_off, h_offs, sizeof(int32_t) * 2 * (D1 + 1), cudaMemcpyHostToDevice, st));
    PS_CUDA(g->node_list.ensure(sizeof(int32_t) * std::max(1, total_nodes)));
    PS_CUDA(g->slot_entry.ensure(sizeof(int32_t) * std::max(1, S_total)));
    PS_CUDA(g->nchild.ensure(sizeof(int32_t) * std::max(1, S_total)));
    PS_CUDA(g->child_off.ensure(sizeof(int32_t) * (S_total + 1)));
    PS_CUDA(g->child_list.ensure(sizeof(int32_t) * std::max(1, S_total)));
    PS_CUDA(g->ccur.ensure(sizeof(int32_t) * std::max(1, S_total)));
    PS_CUDA(g->rho_slot.ensure(sizeof(int32_t) * B));
    PS_CUDA(cudaMemsetAsync(g->nchild.p, 0, sizeof(int32_t) * std::max(1, S_total), st));
    PS_CUDA(cudaMemsetAsync(g->ccur.p, 0, sizeof(int32_t) * std::max(1, S_total), st));
    PS_CUDA(cudaMemsetAsync(g->rho_slot.p, 0xFF, sizeof(int32_t) * B, st));
    launch_sched_lists(t, d_node_off, d_slot_off, d_ncur, g->node_list.as<int32_t>(), g->slot_entry.as<int32_t>(),
                       g->nchild.as<int32_t>(), g->rho_slot.as<int32_t>(), st);
    launch_scan_exclusive(g->nchild.as<int32_t>(), g->child_off.as<int32_t>(), S_total, st);
    launch_sched_children(t, g->slot_entry.as<int32_t>(), S_total, d_slot_off, g->child_off.as<int32_t>(),
                          g->ccur.as<int32_t>(), g->child_list.as<int32_t>(), st);
    launches += 3;
    // 4. level loop, deepest depth first
    const size_t vec_bytes = (size_t)n * (size_t)maxpitch * sizeof(float);
    PS_CUDA(g->md_a.ensure(vec_bytes));
    PS_CUDA(g->md_b.ensure(vec_bytes));
    PS_CUDA(g->dmat.ensure(vec_bytes));
    float *prev = g->md_a.as<float>(), *cur = g->md_b.as<float>(), *Dm = g->dmat.as<float>();
    const int32_t *node_list = g->node_list.as<int32_t>();
    Timer tm{g, st};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks;
    for (int32_t d = Dmax; d >= 0; --d) {
        const int32_t S = scount[d], pd = pitch[d];
        if (S > 0) {
            if (d + 1 <= Dmax && scount[d + 1] > 0) {
                launch_dbuild(n, prev, pitch[d + 1], Dm, pd, S, g->child_off.as<int32_t>() + slot_off[d],
                              g->child_list.as<int32_t>(), st);
                ++launches;
            } else {
                PS_CUDA(cudaMemsetAsync(Dm, 0, (size_t)n * pd * sizeof(float), st));
            }
            if (d + 2 <= Dmax) {
                launch_scatter_gamma(node_list + node_off[d + 2], ncount[d + 2], t, Dm, pd, st);
                ++launches;
            }
            if (dg.n_split > 0) {
                launch_zero_split_rows(dg, cur, pd, st);
                ++launches;
            }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (g->profiling) {
                e0 = tm.get();
                e1 = tm.get();
                PS_CUDA(cudaEventRecord(e0, st));
            }
            launch_pull(dg, Dm, cur, pd, tile[d], st);
            ++launches;
            if (g->profiling) {
                PS_CUDA(cudaEventRecord(e1, st));
                marks.push_back({e0, e1});
            }
            g->stats.probe_launches += 1;
            g->stats.edge_gathers += dg.m * (int64_t)S;
            g->stats.probe_bytes += 4.0 * dg.m + 16.0 * dg.n_pieces + 4.0 * n + 8.0 * (double)n * S;
        }
        if (d >= 1) {
            launch_gamma(dg, node_list + node_off[d], ncount[d], t, qb.inv_nr, S > 0 ? cur : nullptr, pd, st);
            ++launches;
        }
        std::swap(prev, cur);
        g->stats.levels += 1;
    }
    // 5. estimates: s(u, v) = MD(super-root)[v], s(u, u) = 1
    launch_finalize(n, B, qb.node, g->rho_slot.as<int32_t>(), scount[0] > 0 ? prev : nullptr, std::max(1, pitch[0]),
                    d_out, st);
    ++launches;
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaStreamSynchronize(st));
    for (auto &mk : marks) {
        float ms = 0.f;
        PS_CUDA(cudaEventElapsedTime(&ms, mk.first, mk.second));
        g->stats.probe_ms += ms;
    }
    g->stats.kernel_launches += launches;
    return PROBESIM_OK;
}

// Runs all nq queries, splitting batches that do not fit the workspace budget.
static probesim_status run_queries(probesim_graph *g, const probesim_query *q, int32_t nq, float *d_out,
                                   cudaStream_t st) {
    int32_t done = 0;
    int32_t chunk = nq;
    while (done < nq) {
        const int32_t B = std::min(chunk, nq - done);
        bool too_big = false;
        probesim_status s = run_batch(g, q + done, B, d_out + (int64_t)done * g->dg.n, st, &too_big);
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
    return PROBESIM_OK;
}

static probesim_status check_queries(const probesim_graph *g, const probesim_query *q, int32_t nq, bool topk,
                                     int32_t kmax) {
    if (!q || nq <= 0) return fail(PROBESIM_E_INVALID, "queries: null pointer or nq <= 0");
    if (nq > 65535) return fail(PROBESIM_E_INVALID, "at most 65535 queries per call");
    for (int32_t i = 0; i < nq; ++i) {
        if (q[i].node < 0 || q[i].node >= g->dg.n) return fail(PROBESIM_E_RANGE, "query node outside [0, n)");
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
    if (!(c.eps_p >= 0.f) || !(c.c0 >= 0.f)) return fail(PROBESIM_E_INVALID, "eps_p and c0 must be >= 0");
    if (c.probe_mode < 0 || c.probe_mode > 2) return fail(PROBESIM_E_INVALID, "unknown probe_mode");
    if (c.probe_mode != PROBESIM_PROBE_DETERMINISTIC || c.eps_p != 0.f)
        return fail(PROBESIM_E_UNSUPPORTED, "this build runs the deterministic PROBE without Pruning Rule 2");
    std::vector<int32_t> hs, hd;
    PS_TRY(fetch_ids(src, m, hs));
    PS_TRY(fetch_ids(dst, m, hd));
    for (int64_t e = 0; e < m; ++e)
        if (hs[e] < 0 || hs[e] >= n || hd[e] < 0 || hd[e] >= n) return fail(PROBESIM_E_RANGE, "edge id outside [0, n)");
    probesim_graph *g = new (std::nothrow) probesim_graph();
    if (!g) return fail(PROBESIM_E_NOMEM, "host allocation failed");
    g->cfg = c;
    g->t_stop = threshold_stop(c.c);
    cudaGetDevice(&g->device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    g->budget = (size_t)(0.6 * (double)tot);
    if (g->pin_s.ensure(65536) != cudaSuccess) {
        delete g;
        return fail(PROBESIM_E_NOMEM, "pinned host allocation failed");
    }
    g->keys.reserve(m);
    for (int64_t e = 0; e < m; ++e)
        if (hs[e] != hd[e]) g->keys.push_back(((uint64_t)(uint32_t)hd[e] << 32) | (uint32_t)hs[e]);
    std::sort(g->keys.begin(), g->keys.end());
    g->keys.erase(std::unique(g->keys.begin(), g->keys.end()), g->keys.end());
    probesim_status s = upload_graph(g, n, (cudaStream_t)stream);
    if (s != PROBESIM_OK) {
        probesim_graph_destroy(g);
        return s;
    }
    *out = g;
    return PROBESIM_OK;
}

probesim_status probesim_graph_destroy(probesim_graph *g) {
    if (!g) return PROBESIM_OK;
    DevBuf *bufs[] = {&g->in_off, &g->in_col, &g->out_off, &g->out_col, &g->w, &g->piece_v, &g->piece_beg,
                      &g->piece_len, &g->split_v, &g->qbuf, &g->walks, &g->lens, &g->ctr, &g->t_key, &g->t_node,
                      &g->t_parent, &g->t_depth, &g->t_query, &g->t_weight, &g->t_height, &g->t_slot, &g->t_gamma,
                      &g->t_G, &g->counts, &g->offs, &g->node_list, &g->slot_entry, &g->nchild, &g->child_off,
                      &g->child_list, &g->ccur, &g->rho_slot, &g->md_a, &g->md_b, &g->dmat, &g->out_stage,
                      &g->tk_hist, &g->tk_state, &g->tk_tie, &g->tk_cid, &g->tk_cval, &g->tk_ids, &g->tk_vals,
                      &g->tk_qk};
    for (DevBuf *b : bufs) b->release();
    g->pin_q.release();
    g->pin_s.release();
    for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
    delete g;
    return PROBESIM_OK;
}

probesim_status probesim_graph_info(const probesim_graph *g, int32_t *n, int64_t *m, uint64_t *epoch) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (n) *n = g->dg.n;
    if (m) *m = g->dg.m;
    if (epoch) *epoch = g->epoch;
    return PROBESIM_OK;
}

static probesim_status apply_updates(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k, bool insert,
                                     int64_t *applied, cudaStream_t st) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    if (k < 0 || (k > 0 && (!src || !dst))) return fail(PROBESIM_E_INVALID, "bad update batch");
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    std::vector<int32_t> hs, hd;
    PS_TRY(fetch_ids(src, k, hs));
    PS_TRY(fetch_ids(dst, k, hd));
    const int32_t n = g->dg.n;
    for (int64_t e = 0; e < k; ++e)
        if (hs[e] < 0 || hs[e] >= n || hd[e] < 0 || hd[e] >= n) return fail(PROBESIM_E_RANGE, "edge id outside [0, n)");
    std::vector<uint64_t> batch;
    batch.reserve(k);
    for (int64_t e = 0; e < k; ++e)
        if (hs[e] != hd[e]) batch.push_back(((uint64_t)(uint32_t)hd[e] << 32) | (uint32_t)hs[e]);
    std::sort(batch.begin(), batch.end());
    batch.erase(std::unique(batch.begin(), batch.end()), batch.end());
    std::vector<uint64_t> next;
    int64_t changed = 0;
    if (insert) {
        std::vector<uint64_t> fresh;
        std::set_difference(batch.begin(), batch.end(), g->keys.begin(), g->keys.end(), std::back_inserter(fresh));
        changed = (int64_t)fresh.size();
        next.reserve(g->keys.size() + fresh.size());
        std::merge(g->keys.begin(), g->keys.end(), fresh.begin(), fresh.end(), std::back_inserter(next));
    } else {
        next.reserve(g->keys.size());
        std::set_difference(g->keys.begin(), g->keys.end(), batch.begin(), batch.end(), std::back_inserter(next));
        changed = (int64_t)(g->keys.size() - next.size());
    }
    if ((int64_t)next.size() >= ((int64_t)1 << 31)) return fail(PROBESIM_E_INVALID, "edge count would reach 2^31");
    if (changed > 0) {
        g->keys.swap(next);
        PS_TRY(upload_graph(g, n, st));
    }
    g->epoch += 1;
    if (applied) *applied = changed;
    return PROBESIM_OK;
}

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
    *n_r = num_walks(g->cfg.c, eps, g->cfg.delta, g->dg.n);
    return PROBESIM_OK;
}

probesim_status probesim_sample_walks(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t *nodes,
                                      int32_t *lens, int64_t capacity, void *stream) {
    if (!g || !nodes || !lens) return fail(PROBESIM_E_INVALID, "null argument");
    PS_TRY(check_queries(g, q, nq, false, 0));
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    cudaStream_t st = (cudaStream_t)stream;
    BatchPlan P;
    PS_TRY(plan_batch(g, q, nq, P));
    if (P.W > capacity) return fail(PROBESIM_E_INVALID, "walk buffer too small");
    QueryBatch qb;
    PS_TRY(upload_batch(g, P, qb, st));
    const int32_t L = g->cfg.l_max;
    const bool dev_nodes = is_device_ptr(nodes), dev_lens = is_device_ptr(lens);
    PS_CUDA(g->walks.ensure(sizeof(int32_t) * std::max<int64_t>(1, (int64_t)P.W * L)));
    PS_CUDA(g->lens.ensure(sizeof(int32_t) * std::max<int32_t>(1, P.W)));
    PS_CUDA(g->ctr.ensure(sizeof(LaunchCounters)));
    PS_CUDA(cudaMemsetAsync(g->ctr.p, 0, sizeof(LaunchCounters), st));
    int32_t *wd = dev_nodes ? nodes : g->walks.as<int32_t>();
    int32_t *ld = dev_lens ? lens : g->lens.as<int32_t>();
    launch_walks(g->dg, qb, P.W, L, g->t_stop, g->cfg.seed, wd, ld, true, g->ctr.as<LaunchCounters>(), st);
    PS_CUDA(cudaGetLastError());
    if (!dev_nodes)
        PS_CUDA(cudaMemcpyAsync(nodes, wd, sizeof(int32_t) * (size_t)P.W * L, cudaMemcpyDeviceToHost, st));
    if (!dev_lens) PS_CUDA(cudaMemcpyAsync(lens, ld, sizeof(int32_t) * (size_t)P.W, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    return PROBESIM_OK;
}

probesim_status probesim_single_source(probesim_graph *g, const probesim_query *q, int32_t nq, float *scores,
                                       void *stream) {
    if (!g || !scores) return fail(PROBESIM_E_INVALID, "null argument");
    PS_TRY(check_queries(g, q, nq, false, 0));
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    g->stats = probesim_stats{};
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_ptr(scores);
    float *d_out = scores;
    const size_t out_bytes = sizeof(float) * (size_t)nq * g->dg.n;
    if (!dev) {
        PS_CUDA(g->out_stage.ensure(out_bytes));
        d_out = g->out_stage.as<float>();
    }
    PS_TRY(run_queries(g, q, nq, d_out, st));
    if (!dev) {
        PS_CUDA(cudaMemcpyAsync(scores, d_out, out_bytes, cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
    }
    return PROBESIM_OK;
}

probesim_status probesim_topk(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t kmax, int32_t *ids,
                              float *vals, void *stream) {
    if (!g || !ids || !vals) return fail(PROBESIM_E_INVALID, "null argument");
    if (kmax < 1 || kmax > 4096 || kmax > g->dg.n - 1) return fail(PROBESIM_E_INVALID, "kmax must lie in [1, min(4096, n-1)]");
    PS_TRY(check_queries(g, q, nq, true, kmax));
    std::lock_guard<std::mutex> lk(g->mu);
    g_last_error.clear();
    g->stats = probesim_stats{};
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = g->dg.n;
    // scores of a chunk of queries, then the selection
    const int32_t chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)(g->budget / 8) / ((int64_t)n * 4)));
    PS_CUDA(g->out_stage.ensure(sizeof(float) * (size_t)chunk * n));
    const int nblk = topk_blocks_per_query(n);
    PS_CUDA(g->tk_hist.ensure(sizeof(unsigned) * 256 * chunk));
    PS_CUDA(g->tk_state.ensure(sizeof(unsigned) * 4 * chunk));
    PS_CUDA(g->tk_tie.ensure(sizeof(unsigned) * (size_t)nblk * chunk));
    PS_CUDA(g->tk_cid.ensure(sizeof(int32_t) * (size_t)kmax * chunk));
    PS_CUDA(g->tk_cval.ensure(sizeof(float) * (size_t)kmax * chunk));
    PS_CUDA(g->tk_qk.ensure(sizeof(int32_t) * 2 * chunk));
    const bool dev_ids = is_device_ptr(ids), dev_vals = is_device_ptr(vals);
    if (!dev_ids) PS_CUDA(g->tk_ids.ensure(sizeof(int32_t) * (size_t)kmax * chunk));
    if (!dev_vals) PS_CUDA(g->tk_vals.ensure(sizeof(float) * (size_t)kmax * chunk));
    std::vector<int32_t> hq(2 * chunk);
    for (int32_t done = 0; done < nq; done += chunk) {
        const int32_t B = std::min(chunk, nq - done);
        PS_TRY(run_queries(g, q + done, B, g->out_stage.as<float>(), st));
        for (int32_t b = 0; b < B; ++b) {
            hq[b] = q[done + b].node;
            hq[chunk + b] = q[done + b].k;
        }
        int32_t *d_qn = g->tk_qk.as<int32_t>(), *d_qk = d_qn + chunk;
        PS_CUDA(cudaMemcpyAsync(d_qn, hq.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaMemcpyAsync(d_qk, hq.data() + chunk, sizeof(int32_t) * B, cudaMemcpyHostToDevice, st));
        TopkScratch sc;
        sc.hist = g->tk_hist.as<unsigned>();
        sc.state = g->tk_state.as<unsigned>();
        sc.tiecnt = g->tk_tie.as<unsigned>();
        sc.cand_id = g->tk_cid.as<int32_t>();
        sc.cand_val = g->tk_cval.as<float>();
        int32_t *oi = dev_ids ? ids + (int64_t)done * kmax : g->tk_ids.as<int32_t>();
        float *ov = dev_vals ? vals + (int64_t)done * kmax : g->tk_vals.as<float>();
        launch_topk(n, B, g->out_stage.as<float>(), d_qn, d_qk, kmax, sc, oi, ov, st, &g->stats.kernel_launches);
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

probesim_status probesim_set_profiling(probesim_graph *g, int32_t on) {
    if (!g) return fail(PROBESIM_E_INVALID, "graph is null");
    std::lock_guard<std::mutex> lk(g->mu);
    g->profiling = on ? 1 : 0;
    return PROBESIM_OK;
}

probesim_status probesim_get_stats(const probesim_graph *g, probesim_stats *out) {
    if (!g || !out) return fail(PROBESIM_E_INVALID, "null argument");
    *out = g->stats;
    return PROBESIM_OK;
}

}  // extern "C"
