// Randomized PROBE (Alg. 3) for every probe instance of a launch: instance (walk k, prefix length i) runs
// levels j = 0..i-2 over a frontier H_j of nodes (all with score 1).  At level j each candidate x != u_{i-j-1}
// samples one in-edge (v, x) of I(x) and joins H_{j+1} with probability sqrt(c) when v is in H_j
// (Alg. 3 lines 8-11); the draws use Philox counter (k, 2^24 | i << 8 | j, x, 0) with x the caller's node id,
// so the outcome of a candidate does not depend on how often or in which order it is evaluated.
//
// Candidates: Alg. 3 takes U = union of O(y), y in H_j, or V when that union is large (lines 4-7).  A node
// outside the union has no in-neighbour in H_j and can never be selected, so both choices give the same
// H_{j+1}; the kernels always evaluate the union, one work item per (frontier entry, out-edge), with the
// frontier's out-degree prefix sums balancing the work.  Repeated candidates evaluate the same draw and the
// next level's hash set keeps one copy.  The members of H_{i-1} are counted per query node; the estimate is
// count / n_r (Alg. 1 with randomized PROBE), exact in integers.
#include "internal.cuh"

namespace ps {

// ------------------------------------------------------------------------------------------------
// exclusive scan of int64 values (three passes: block sums, scan of the block sums, block scans)
// ------------------------------------------------------------------------------------------------
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *s_warp, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_warp[lane] = t;  // inclusive per warp
    }
    __syncthreads();
    const long long base = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_partials(const long long *__restrict__ in, int64_t count,
                                                              long long *__restrict__ partial) {
    __shared__ long long s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long local = 0;
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = base + (int64_t)r * kScanBlock + threadIdx.x;
        if (i < count) local += in[i];
    }
    long long total;
    block_exclusive_scan(local, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// one block scans the block sums in place (any count, in chunks of kScanBlock)
__global__ void __launch_bounds__(kScanBlock) k_scan_partials_scan(long long *partial, int64_t nblocks) {
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nblocks; c0 += kScanBlock) {
        const int64_t i = c0 + threadIdx.x;
        const long long v = i < nblocks ? partial[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, s_warp, &total);
        if (i < nblocks) partial[i] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_final(const long long *__restrict__ in, int64_t count,
                                                           const long long *__restrict__ partial,
                                                           long long *__restrict__ out) {
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (threadIdx.x == 0) s_carry = partial[blockIdx.x];
    __syncthreads();
    for (int r = 0; r < kScanItems; ++r) {
        const int64_t i = base + (int64_t)r * kScanBlock + threadIdx.x;
        const long long v = i < count ? in[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, s_warp, &total);
        if (i < count) out[i] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += total;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = s_carry;
}

int64_t scan64_partials_needed(int64_t count) { return (count + kScanTile - 1) / kScanTile + 1; }

// out[0..count] = exclusive prefix sums of in[0..count), out[count] = total.  partial holds
// scan64_partials_needed(count) entries.
void launch_scan64(const long long *in, int64_t count, long long *partial, long long *out, cudaStream_t s) {
    if (count <= 0) {
        cudaMemsetAsync(out, 0, sizeof(long long), s);
        return;
    }
    const int64_t nb = (count + kScanTile - 1) / kScanTile;
    k_scan_partials<<<(unsigned)nb, kScanBlock, 0, s>>>(in, count, partial);
    k_scan_partials_scan<<<1, kScanBlock, 0, s>>>(partial, nb);
    k_scan_final<<<(unsigned)nb, kScanBlock, 0, s>>>(in, count, partial, out);
}

// ------------------------------------------------------------------------------------------------
// probe instances
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t walk_query(const int32_t *walk_base, int32_t B, int32_t wid) {
    int32_t lo = 0, hi = B;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (walk_base[mid] <= wid) lo = mid; else hi = mid;
    }
    return lo;
}

// A slot in an append list for each lane that calls it: the lanes executing the call together (__activemask) take
// consecutive slots with one atomic on the shared counter, instead of one atomic each on the same address.
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
}

// instance (w, i) runs unless a filter is given and the tree slot of its prefix is not flagged
__device__ __forceinline__ bool inst_on(const int32_t *walk_slot, const uint8_t *t_sw, int32_t l_max, int32_t w, int32_t i) {
    return !walk_slot || t_sw[walk_slot[(int64_t)w * l_max + i - 1]];
}

// per walk w0 + i of a walk range: number of probes (len - 1, or the flagged ones)
__global__ void k_inst_count(const int32_t *__restrict__ lens, int32_t w0, int32_t nw, long long *cnt,
                             const int32_t *__restrict__ walk_slot, const uint8_t *__restrict__ t_sw, int32_t l_max) {
    const int32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 >= nw) return;
    const int32_t w = w0 + i0;
    long long c = 0;
    for (int32_t i = 2; i <= lens[w]; ++i) c += inst_on(walk_slot, t_sw, l_max, w, i);
    cnt[i0] = c;
}

__global__ void k_add_i32(int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// instance (walk w, prefix length i) for i = 2..len; its level-0 frontier {u_i} goes into the table and list
__device__ __forceinline__ unsigned long long rmix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// inserts key; returns 1 if it was absent, 0 if present, -1 if the table is full
__device__ __forceinline__ int set_insert(unsigned long long *keys, int64_t cap, unsigned long long key) {
    int64_t h = (int64_t)(rmix(key) & (unsigned long long)(cap - 1));
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long cur = keys[h];
        if (cur == key) return 0;
        if (cur == kEmptyKey) {
            cur = atomicCAS(&keys[h], kEmptyKey, key);
            if (cur == kEmptyKey) return 1;
            if (cur == key) return 0;
        }
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

__device__ __forceinline__ bool set_contains(const unsigned long long *keys, int64_t cap, unsigned long long key) {
    int64_t h = (int64_t)(rmix(key) & (unsigned long long)(cap - 1));
    for (int64_t probe = 0; probe < cap; ++probe) {
        const unsigned long long cur = keys[h];
        if (cur == key) return true;
        if (cur == kEmptyKey) return false;
        h = (h + 1) & (cap - 1);
    }
    return false;
}

__global__ void k_inst_init(QueryBatch q, const int64_t *__restrict__ out_off, const int32_t *__restrict__ lens,
                            int32_t w0, int32_t nw, int32_t l_max, const int32_t *__restrict__ walks,
                            const long long *__restrict__ inst_off, int32_t *inst_walk, int32_t *inst_len,
                            int32_t *inst_q, uint32_t *inst_k, int32_t *fr_inst, int32_t *fr_node,
                            unsigned long long *fr_count, unsigned long long *keys, int64_t cap, int32_t *overflow,
                            const int32_t *__restrict__ walk_slot, const uint8_t *__restrict__ t_sw) {
    const int32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 >= nw) return;
    const int32_t w = w0 + i0;
    const int32_t len = lens[w];
    int64_t id = inst_off[i0];
    const int32_t b = walk_query(q.walk_base, q.B, w);
    const uint32_t k = (uint32_t)(q.walk_k0[b] + (w - q.walk_base[b]));
    for (int32_t i = 2; i <= len; ++i) {
        if (!inst_on(walk_slot, t_sw, l_max, w, i)) continue;
        inst_walk[id] = w;
        inst_len[id] = i;
        inst_q[id] = b;
        inst_k[id] = k;
        const int32_t u = walks[(int64_t)w * l_max + i - 1];  // H_0 = {u_i}
        if (set_insert(keys, cap, ((unsigned long long)id << 32) | (uint32_t)u) < 0) atomicExch(overflow, 1);
        if (out_off[u + 1] > out_off[u]) {
            const unsigned long long pos = warp_append(fr_count);
            fr_inst[pos] = (int32_t)id;
            fr_node[pos] = u;
        }
        ++id;
    }
}

// out-degree of every frontier entry whose instance still has a level to run
__global__ void k_frontier_degree(const int32_t *__restrict__ fr_inst, const int32_t *__restrict__ fr_node, int64_t F,
                                  const int32_t *__restrict__ inst_len, int32_t j, const int64_t *__restrict__ out_off,
                                  long long *deg) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int32_t y = fr_node[f];
    deg[f] = (inst_len[fr_inst[f]] - 2 >= j) ? (long long)(out_off[y + 1] - out_off[y]) : 0;
}

constexpr int kLevelThreads = 256;
constexpr int kLevelItems = 2048;  // work items per block pass

// One pass per block over kLevelItems consecutive work items; the block's slice of the prefix sums is
// staged in shared memory so each item finds its frontier entry with a short search.
__global__ void __launch_bounds__(kLevelThreads) k_rand_level(DeviceGraph g, const int32_t *__restrict__ walks,
                                                              int32_t l_max, const int32_t *__restrict__ inst_walk,
                                                              const int32_t *__restrict__ inst_len,
                                                              const int32_t *__restrict__ inst_q,
                                                              const uint32_t *__restrict__ inst_k,
                                                              const uint32_t *__restrict__ qkey, uint32_t seed,
                                                              uint32_t t_keep, RandLevel L) {
    __shared__ long long s_pref[kLevelItems + 1];
    __shared__ int64_t s_f0, s_nf;
    const int64_t nblk = (L.E + kLevelItems - 1) / kLevelItems;
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int64_t t0 = blk * kLevelItems, t1 = min(L.E, t0 + kLevelItems);
        if (threadIdx.x == 0) {
            int64_t lo = 0, hi = L.F;  // entry of item t0
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (L.prefix[mid] <= t0) lo = mid; else hi = mid;
            }
            int64_t lo2 = lo, hi2 = L.F;  // entry of item t1 - 1
            while (hi2 - lo2 > 1) {
                const int64_t mid = (lo2 + hi2) >> 1;
                if (L.prefix[mid] <= t1 - 1) lo2 = mid; else hi2 = mid;
            }
            s_f0 = lo;
            s_nf = lo2 - lo + 1;
        }
        __syncthreads();
        const int64_t f0 = s_f0, nf = s_nf;
        const bool staged = nf <= kLevelItems;
        if (staged)
            for (int64_t a = threadIdx.x; a <= nf; a += blockDim.x) s_pref[a] = L.prefix[f0 + a];
        __syncthreads();
        for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            int64_t f;
            if (staged) {
                int64_t lo = 0, hi = nf;
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (s_pref[mid] <= t) lo = mid; else hi = mid;
                }
                f = f0 + lo;
            } else {
                int64_t lo = f0, hi = L.F;
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (L.prefix[mid] <= t) lo = mid; else hi = mid;
                }
                f = lo;
            }
            const int32_t inst = L.fr_inst[f];
            const int32_t y = L.fr_node[f];
            const int32_t x = g.out_col[g.out_off[y] + (t - L.prefix[f])];
            const int32_t wid = inst_walk[inst];
            const int32_t i = inst_len[inst];
            if (x == walks[(int64_t)wid * l_max + (i - L.j - 2)]) continue;  // x = u_{i-j-1}
            const int32_t b = inst_q[inst];
            const U32x4 r = philox4x32_10(inst_k[inst], (1u << 24) | ((uint32_t)i << 8) | (uint32_t)L.j,
                                          (uint32_t)g.int2ext[x], 0u, seed, qkey[b]);
            if (r.y >= t_keep) continue;  // kept with probability sqrt(c)
            const int64_t beg = g.in_off[x];
            const uint32_t d = (uint32_t)(g.in_off[x + 1] - beg);
            const int32_t v = g.in_col[beg + __umulhi(r.x, d)];  // the sampled in-edge (v, x)
            if (!set_contains(L.cur_keys, L.cur_cap, ((unsigned long long)inst << 32) | (uint32_t)v)) continue;
            const int ins = set_insert(L.next_keys, L.next_cap, ((unsigned long long)inst << 32) | (uint32_t)x);
            if (ins < 0) { atomicExch(L.overflow, 1); continue; }
            if (ins == 0) continue;
            if (i - 2 == L.j) {
                atomicAdd(L.counts + (int64_t)b * g.n + x, 1);  // member of H_{i-1}: the probe's result
            } else if (g.out_off[x + 1] > g.out_off[x]) {    // only nodes with out-edges can expand
                const unsigned long long pos = warp_append(L.next_count);
                L.next_inst[pos] = inst;
                L.next_node[pos] = x;
            }
        }
        __syncthreads();
    }
}

__global__ void k_rand_finalize(int32_t n, int32_t B, const int32_t *__restrict__ qnode,
                                const int32_t *__restrict__ counts, const float *__restrict__ inv_nr,
                                const int32_t *__restrict__ ext2int, float shift, float *__restrict__ out) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t b = blockIdx.y;
    if (v >= n) return;
    float s = (float)counts[(int64_t)b * n + ext2int[v]] * inv_nr[b] + shift;
    if ((int32_t)v == qnode[b]) s = 1.f;
    out[(int64_t)b * n + v] = s;
}

void launch_inst_count(const int32_t *lens, int32_t w0, int32_t nw, long long *cnt, const int32_t *walk_slot,
                       const uint8_t *t_sw, int32_t l_max, cudaStream_t s) {
    if (nw > 0) k_inst_count<<<(nw + 255) / 256, 256, 0, s>>>(lens, w0, nw, cnt, walk_slot, t_sw, l_max);
}
void launch_inst_init(const QueryBatch &q, const DeviceGraph &g, const int32_t *lens, int32_t w0, int32_t nw,
                      int32_t l_max, const int32_t *walks, const long long *inst_off, int32_t *inst_walk,
                      int32_t *inst_len, int32_t *inst_q, uint32_t *inst_k, int32_t *fr_inst, int32_t *fr_node,
                      unsigned long long *fr_count, unsigned long long *keys, int64_t cap, int32_t *overflow,
                      const int32_t *walk_slot, const uint8_t *t_sw, cudaStream_t s) {
    if (nw > 0)
        k_inst_init<<<(nw + 255) / 256, 256, 0, s>>>(q, g.out_off, lens, w0, nw, l_max, walks, inst_off, inst_walk,
                                                     inst_len, inst_q, inst_k, fr_inst, fr_node, fr_count, keys, cap,
                                                     overflow, walk_slot, t_sw);
}
void launch_add_i32(int32_t *a, const int32_t *b, int64_t count, cudaStream_t s) {
    if (count > 0) k_add_i32<<<grid_for(count, 256, 8), 256, 0, s>>>(a, b, count);
}
void launch_frontier_degree(const int32_t *fr_inst, const int32_t *fr_node, int64_t F, const int32_t *inst_len, int32_t j,
                            const int64_t *out_off, long long *deg, cudaStream_t s) {
    if (F > 0)
        k_frontier_degree<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(fr_inst, fr_node, F, inst_len, j, out_off, deg);
}
void launch_rand_level(const DeviceGraph &g, const int32_t *walks, int32_t l_max, const int32_t *inst_walk,
                       const int32_t *inst_len, const int32_t *inst_q, const uint32_t *inst_k, const uint32_t *qkey,
                       uint32_t seed, uint32_t t_keep, const RandLevel &L, cudaStream_t s) {
    if (L.E <= 0) return;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (L.E + kLevelItems - 1) / kLevelItems;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_rand_level<<<(unsigned)blocks, kLevelThreads, 0, s>>>(g, walks, l_max, inst_walk, inst_len, inst_q, inst_k, qkey,
                                                            seed, t_keep, L);
}
void launch_rand_finalize(int32_t n, int32_t B, const int32_t *qnode, const int32_t *counts, const float *inv_nr,
                          const int32_t *ext2int, float shift, float *out, cudaStream_t s) {
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)B);
    k_rand_finalize<<<grid, 256, 0, s>>>(n, B, qnode, counts, inv_nr, ext2int, shift, out);
}

}  // namespace ps
