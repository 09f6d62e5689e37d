// Host-side engine types shared by the C ABI (probesim.cu) and the serving loop (server.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <vector>

#include "internal.cuh"

// ------------------------------------------------------------------------------------------------
// device buffers that grow on demand and are freed with the graph
// ------------------------------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    bool pooled = false;  // from the stream-ordered pool (cudaMallocAsync): freed with cudaFreeAsync
    // allocates exactly `bytes` from the device's stream-ordered pool on stream s (no device-wide synchronisation,
    // unlike cudaMalloc / cudaFree); for buffers that are written once, such as a new version of the graph store
    cudaError_t alloc_pooled(size_t bytes, cudaStream_t s) {
        release();
        cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(256, bytes), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return e;
        }
        cap = std::max<size_t>(256, bytes);
        pooled = true;
        return cudaSuccess;
    }
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
    // grows to at least `bytes`, keeping the first `keep` bytes (copied on stream s)
    cudaError_t grow(size_t bytes, size_t keep, cudaStream_t s) {
        if (bytes <= cap && p) return cudaSuccess;
        void *q = nullptr;
        const size_t nb = std::max<size_t>(256, bytes + bytes / 4);
        cudaError_t e = cudaMalloc(&q, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        if (p && keep > 0) e = cudaMemcpyAsync(q, p, std::min(keep, cap), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && p) e = cudaStreamSynchronize(s);
        if (p) cudaFree(p);
        p = q;
        cap = nb;
        return e;
    }
    // A pooled buffer returns to the pool on the calling thread's default stream, without waiting: its readers
    // have synchronised their own streams before they let go of it.
    void release() {
        if (p) {
            if (pooled) cudaFreeAsync(p, cudaStreamPerThread);
            else cudaFree(p);
        }
        p = nullptr;
        cap = 0;
        pooled = false;
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

// One version of the graph store.  A query holds the version it started with; an update batch builds the next
// version beside it and publishes it, so queries never wait for updates nor updates for queries, and a version's
// device memory is freed when its last reader lets go.
struct StoreVersion {
    DevBuf in_off, in_col, out_off, out_col, w, piece_v, piece_beg, piece_len, split_v;
    std::shared_ptr<StoreVersion> base;  // set when this version reuses base's arrays (an update that changed nothing)
    ps::DeviceGraph dg;
    uint64_t epoch = 0;
    ~StoreVersion() {
        for (DevBuf *b : {&in_off, &in_col, &out_off, &out_col, &w, &piece_v, &piece_beg, &piece_len, &split_v})
            b->release();
    }
};

// Per-call device and pinned buffers; a graph owns one for direct calls, a server one per worker.
struct Workspace {
    DevBuf qbuf, walks, lens, ctr;
    DevBuf t_key, t_node, t_parent, t_depth, t_query, t_weight, t_height, t_slot, t_gamma, t_G;
    DevBuf counts, offs, node_list, col_export, sched;  // level schedule: exported column nodes, uploaded plan
    DevBuf md_a, md_b, out_stage;                       // the two score buffers; host-output staging
    DevBuf r_cnt, r_off, r_part, r_iwalk, r_ilen, r_iq, r_ik, r_fi[2], r_fn[2], r_keys[2], r_deg, r_pref, r_counts,
        r_counts2, r_ctr;
    DevBuf tk_hist, tk_state, tk_tie, tk_cid, tk_cval, tk_ids, tk_vals, tk_qk;
    // frontier engine: walk-prefix slots, switched flags, probes, frontier lists, next-level table, estimates
    DevBuf f_wslot, f_tsw, f_slot, f_misc, f_anc, f_deg, f_state, f_rsize, f_roff, f_dsize, f_doff, f_acc, f_tab, f_wp,
        f_lp[2], f_lx[2], f_lv[2], f_sp, f_sx, f_sv, f_cuts, f_keys, f_bcnt, f_bpre;
    DevBuf pm_in, pm_meets;  // pairwise Monte Carlo: pairs and keys, meet counts
    DevBuf pull_err;         // set by the TMA pull when a stage's wait gives up
    bool f_table_clean = false;  // f_keys (the level table) holds only empty slots (every pass's compaction empties
                                 // its slots)
    PinnedBuf pin_q;  // query arrays of one batch
    PinnedBuf pin_s;  // counters and schedule offsets (fixed size, allocated at creation)
    int profiling = 0;
    size_t budget = 0;  // device memory one call on this workspace may take; 0 = the graph's budget
    std::shared_ptr<StoreVersion> snap;  // the store version of the call in progress
    ps::DeviceGraph dg;                  // its device view
    std::vector<cudaEvent_t> ev;
    probesim_stats stats{};
    // a second stream for work of a depth that runs beside the pull (the push block, the tail tile), and the
    // events that order it against the caller's stream; created on first use
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ev_ready = nullptr, ev_side = nullptr;
    cudaError_t ensure_side() {
        if (side) return cudaSuccess;
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_side, cudaEventDisableTiming);
        return e;
    }
    void release() {
        DevBuf *bufs[] = {&qbuf, &walks, &lens, &ctr, &t_key, &t_node, &t_parent, &t_depth, &t_query, &t_weight,
                          &t_height, &t_slot, &t_gamma, &t_G, &counts, &offs, &node_list, &col_export,
                          &sched, &md_a, &md_b, &out_stage, &r_cnt, &r_off,
                          &r_part, &r_iwalk, &r_ilen, &r_iq, &r_ik, &r_fi[0], &r_fi[1], &r_fn[0], &r_fn[1],
                          &r_keys[0], &r_keys[1], &r_deg, &r_pref, &r_counts, &r_counts2, &r_ctr, &tk_hist, &tk_state, &tk_tie,
                          &tk_cid, &tk_cval, &tk_ids, &tk_vals, &tk_qk, &f_wslot, &f_tsw, &f_slot, &f_misc, &f_anc,
                          &f_deg, &f_state, &f_rsize, &f_roff, &f_dsize, &f_doff, &f_acc, &f_tab, &f_wp, &f_lp[0],
                          &f_lp[1], &f_lx[0], &f_lx[1], &f_lv[0], &f_lv[1], &f_sp, &f_sx, &f_sv, &f_cuts, &f_keys,
                          &f_bcnt, &f_bpre, &pm_in, &pm_meets, &pull_err};
        for (DevBuf *b : bufs) b->release();
        f_table_clean = false;
        pin_q.release();
        pin_s.release();
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        for (cudaEvent_t *e : {&ev_start, &ev_ready, &ev_side})
            if (*e) cudaEventDestroy(*e), *e = nullptr;
        if (side) cudaStreamDestroy(side), side = nullptr;
    }
};

struct probesim_graph {
    std::mutex mu;              // serialises direct calls (they share ws0)
    std::mutex update_mu;       // serialises update batches
    std::mutex store_ptr_mu;    // guards the pointer to the current store version
    std::shared_ptr<StoreVersion> store;
    probesim_config cfg{};
    uint32_t t_stop = 0;
    uint32_t t_keep = 0;
    int device = 0;
    int32_t n = 0;              // node count (fixed; updates change edges only)
    DevBuf ext2int, int2ext;    // the id maps, shared by every store version
    std::shared_ptr<StoreVersion> current() {
        std::lock_guard<std::mutex> lk(store_ptr_mu);
        return store;
    }
    void publish(std::shared_ptr<StoreVersion> v) {
        std::lock_guard<std::mutex> lk(store_ptr_mu);
        store.swap(v);  // the old version is released outside the lock, by whichever reader holds it last
    }
    std::vector<int32_t> h_ext2int;  // host copy of the id map (update batches are sorted by internal ids)
    // update scratch
    DevBuf u_batch, u_valid, u_vpre, u_delta, u_deg, u_part, u_hist;
    uint64_t epoch = 0;
    Workspace ws0;
    std::atomic<size_t> budget{0};  // device memory one call's working buffers may take (set while calls run)
    size_t budget0 = 0;  // the default: 60% of device memory at creation
    // pull launch shape chosen by probesim_autotune (defaults until then)
    int32_t tune_wide = 32;       // full tiles: 16, 32, kPullPairs (32-column tiles two per pass) or kPullTma
    int32_t tune_bps[128] = {0};  // blocks per SM per tile width, kPullPairs / kPullTma for those (0 = default)
    int32_t tuned = 0;
};


namespace ps {
// Status helpers (probesim.cu): set the calling thread's message and return the status.
probesim_status fail_status(probesim_status st, const std::string &msg);
// Checks a query array against the graph (ids, eps, k <= kmax when topk).
probesim_status check_queries(const probesim_graph *g, const probesim_query *q, int32_t nq, bool topk, int32_t kmax);
// Estimates and top-k of nq queries with workspace ws on stream st, over store version snap.  The caller owns ws.
probesim_status single_source_core(probesim_graph *g, Workspace *ws, const std::shared_ptr<StoreVersion> &snap,
                                   const probesim_query *q, int32_t nq, float *scores, cudaStream_t st);
probesim_status topk_core(probesim_graph *g, Workspace *ws, const std::shared_ptr<StoreVersion> &snap,
                          const probesim_query *q, int32_t nq, int32_t kmax, int32_t *ids, float *vals, cudaStream_t st);
// Applies one update batch: builds the next store version from the current one and publishes it (serialised with
// other update batches, never waiting for queries).
probesim_status apply_updates(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k, bool insert,
                              int64_t *applied, cudaStream_t st);
int64_t num_walks_for(const probesim_graph *g, double eps);
}  // namespace ps
