// sqrt(c)-walks (Def. 3, Pruning Rule 1), the reverse-reachability tree of Alg. 4 as a hash table, and
// the level schedule derived from it.
#include "internal.cuh"

namespace ps {

// Which query of the launch walk `wid` belongs to (walk_base is sorted, B is small).
__device__ __forceinline__ int32_t query_of(const int32_t *walk_base, int32_t B, int32_t wid) {
    int32_t lo = 0, hi = B;  // walk_base[lo] <= wid < walk_base[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (walk_base[mid] <= wid) lo = mid; else hi = mid;
    }
    return lo;
}

// One thread per walk, in internal node ids.  At node v: stop when the draw x0 is below t_stop (probability 1 - sqrt(c)),
// stop when |I(v)| = 0, stop when the walk already holds l_max nodes; otherwise move to entry
// floor(x1 * |I(v)| / 2^32) of I(v).
__global__ void __launch_bounds__(256) k_walks(const int64_t *__restrict__ in_off, const int32_t *__restrict__ in_col,
                                               const int32_t *__restrict__ ext2int, QueryBatch q, int32_t W, int32_t l_max, uint32_t t_stop,
                                               uint32_t seed, int32_t *__restrict__ walks,
                                               int32_t *__restrict__ lens, bool pad, LaunchCounters *ctr) {
    const int32_t wid = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t len = 0;
    if (wid < W) {
        const int32_t b = query_of(q.walk_base, q.B, wid);
        const uint32_t k = (uint32_t)(q.walk_k0[b] + (wid - q.walk_base[b]));
        const uint32_t key1 = q.qid[b];
        int32_t v = ext2int[q.node[b]];
        int32_t *row = walks + (int64_t)wid * l_max;
        row[len++] = v;
        for (uint32_t s = 0;; ++s) {
            if (len >= l_max) break;
            const U32x4 r = philox4x32_10(k, s, 0u, 0u, seed, key1);
            if (r.x < t_stop) break;
            const int64_t beg = in_off[v];
            const uint32_t d = (uint32_t)(in_off[v + 1] - beg);
            if (d == 0) break;
            v = in_col[beg + __umulhi(r.y, d)];
            row[len++] = v;
        }
        if (pad)
            for (int32_t t = len; t < l_max; ++t) row[t] = -1;
        lens[wid] = len;
    }
    // block-level reduction of the length sum and maximum
    __shared__ unsigned long long s_sum[8];
    __shared__ int32_t s_max[8];
    unsigned long long sum = (unsigned long long)len;
    int32_t mx = len;
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s_sum[warp] = sum; s_max[warp] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bs = 0;
        int32_t bm = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { bs += s_sum[i]; bm = max(bm, s_max[i]); }
        atomicAdd(&ctr->walk_nodes, bs);
        atomicMax(&ctr->max_len, bm);
    }
}

void launch_walks(const DeviceGraph &g, const QueryBatch &q, int32_t W, int32_t l_max, uint32_t t_stop,
                  uint32_t seed, int32_t *walks, int32_t *lens, bool pad, LaunchCounters *ctr, cudaStream_t s) {
    if (W <= 0) return;
    k_walks<<<(W + 255) / 256, 256, 0, s>>>(g.in_off, g.in_col, g.ext2int, q, W, l_max, t_stop, seed, walks, lens, pad, ctr);
}

// splitmix64 finalizer as the table hash
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Returns the slot holding `key`, inserting it if absent; -1 when the table is full (every probe is
// bounded by the capacity, so the loop always ends).
__device__ __forceinline__ int64_t table_insert(unsigned long long *keys, int64_t cap, unsigned long long key) {
    int64_t h = (int64_t)(mix64(key) & (unsigned long long)(cap - 1));
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long cur = keys[h];
        if (cur == key) return h;
        if (cur == kEmptyKey) {
            cur = atomicCAS(&keys[h], kEmptyKey, key);
            if (cur == kEmptyKey || cur == key) return h;
        }
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

// One thread per walk: inserts the super-root, then the prefixes (u_1), (u_1,u_2), ... (Alg. 4 lines
// 5-11).  A node's weight counts the walks through it; its height is the longest walk suffix below it.
__global__ void __launch_bounds__(256) k_trie_insert(QueryBatch q, int32_t W, int32_t l_max,
                                                     const int32_t *__restrict__ walks,
                                                     const int32_t *__restrict__ lens, TrieTable t,
                                                     LaunchCounters *ctr) {
    const int32_t wid = blockIdx.x * blockDim.x + threadIdx.x;
    if (wid >= W) return;
    const int32_t b = query_of(q.walk_base, q.B, wid);
    const int32_t len = lens[wid];
    const int32_t *row = walks + (int64_t)wid * l_max;
    int64_t p = table_insert(t.key, t.cap, ((unsigned long long)kRhoTag << 32) | (uint32_t)b);
    if (p < 0) { atomicExch(&ctr->overflow, 1); return; }
    t.node[p] = -1;
    t.parent[p] = -1;
    t.depth[p] = 0;
    t.query[p] = b;
    atomicMax(&t.height[p], len);
    for (int32_t i = 1; i <= len; ++i) {
        const int32_t u = row[i - 1];
        const int64_t s = table_insert(t.key, t.cap, ((unsigned long long)(uint32_t)p << 32) | (uint32_t)u);
        if (s < 0) { atomicExch(&ctr->overflow, 1); return; }
        if (t.walk_slot) t.walk_slot[(int64_t)wid * l_max + i - 1] = (int32_t)s;
        t.node[s] = u;
        t.parent[s] = (int32_t)p;
        t.depth[s] = i;
        t.query[s] = b;
        atomicAdd(&t.weight[s], 1);
        atomicMax(&t.height[s], len - i);
        p = s;
    }
}

void launch_trie_insert(const DeviceGraph &g, const QueryBatch &q, int32_t W, int32_t l_max, const int32_t *walks,
                        const int32_t *lens, TrieTable t, LaunchCounters *ctr, cudaStream_t s) {
    (void)g;
    if (W <= 0) return;
    k_trie_insert<<<(W + 255) / 256, 256, 0, s>>>(q, W, l_max, walks, lens, t, ctr);
}

// Counts tree nodes and vector columns per depth.  A node owns a score-vector column when its subtree has
// height >= 2: only then is the sum of its children's contributions more than a sparse set of nodes.
// Height >= 3 nodes (and a super-root of height 2) get "dense" columns filled by the pull; height-2 nodes
// get "push" columns filled from their grandchildren's few gamma terms.  Dense columns take local indices
// 0.., push columns are encoded -2 - local until the host knows the dense width of the depth.
__global__ void k_sched_count(TrieTable t, int32_t *ncount, int32_t *scount, int32_t *hcount) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= t.cap) return;
    if (t.key[e] == kEmptyKey) return;
    const int32_t d = t.depth[e], h = t.height[e];
    atomicAdd(&ncount[d], 1);
    if (h >= 3 || (d == 0 && h >= 2)) t.slot[e] = atomicAdd(&scount[d], 1);
    else if (h == 2) t.slot[e] = -2 - atomicAdd(&hcount[d], 1);
    else t.slot[e] = -1;
}

void launch_sched_count(TrieTable t, int32_t *ncount, int32_t *scount, int32_t *hcount, cudaStream_t s) {
    k_sched_count<<<(unsigned)((t.cap + 255) / 256), 256, 0, s>>>(t, ncount, scount, hcount);
}

// Exports every node that owns a column (dense or push): entry, depth, parent entry, dense flag, query.
__global__ void k_sched_export(TrieTable t, int32_t *out, int32_t *count) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= t.cap) return;
    if (t.key[e] == kEmptyKey) return;
    const int32_t sl = t.slot[e];
    if (sl == -1) return;
    const int32_t i = atomicAdd(count, 1);
    out[5 * i + 0] = (int32_t)e;
    out[5 * i + 1] = t.depth[e];
    out[5 * i + 2] = t.parent[e];
    out[5 * i + 3] = sl >= 0 ? 1 : 0;
    out[5 * i + 4] = t.query[e];
}

void launch_sched_export(TrieTable t, int32_t *out, int32_t *count, cudaStream_t s) {
    k_sched_export<<<(unsigned)((t.cap + 255) / 256), 256, 0, s>>>(t, out, count);
}

// Node lists per depth (every tree node).
__global__ void k_node_lists(TrieTable t, const int32_t *__restrict__ node_off, int32_t *ncur, int32_t *node_list) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= t.cap) return;
    if (t.key[e] == kEmptyKey) return;
    const int32_t d = t.depth[e];
    node_list[node_off[d] + atomicAdd(&ncur[d], 1)] = (int32_t)e;
}

void launch_node_lists(TrieTable t, const int32_t *node_off, int32_t *ncur, int32_t *node_list, cudaStream_t s) {
    k_node_lists<<<(unsigned)((t.cap + 255) / 256), 256, 0, s>>>(t, node_off, ncur, node_list);
}

// slot[pairs[2i]] = pairs[2i+1]
__global__ void k_set_slots(TrieTable t, const int32_t *__restrict__ pairs, int32_t count) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) t.slot[pairs[2 * i]] = pairs[2 * i + 1];
}

void launch_set_slots(TrieTable t, const int32_t *pairs, int32_t count, cudaStream_t s) {
    if (count > 0) k_set_slots<<<(count + 255) / 256, 256, 0, s>>>(t, pairs, count);
}

}  // namespace ps
