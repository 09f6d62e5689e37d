// Frontier PROBE engine: every walk prefix of a call's reverse-reachability trees probed on its own, as Alg. 4
// runs Alg. 2, with Pruning Rule 2 (Sec. 4.1) and the best-of-both switch of Sec. 4.4.
//
// A probe is a tree node r_q (q >= 2) of weight w, the prefix (u_1..u_q); it runs levels j = 0..q-2 of
// Alg. 2.  All probes of a call advance one level per round, and the frontier H_j of every probe is one
// list of entries (probe, node, score), grouped by probe in probe order.  A round:
//   prune    Rule 2: drop x when Score(x) * sqrt(c)^(q-j-1) <= eps_p; sum the out-degrees of the rest
//   switch   Sec. 4.4: a probe whose sum exceeds c0 * w * n leaves the deterministic rounds; Alg. 3 then
//            runs on its whole partial walk once per walk through the tree node (rand_probe.cu)
//   expand   every kept entry x pushes sqrt(c)/|I(v)| * Score(x) to each v in O(x), v != u_{q-j-1}, into
//            the probe's region of the next level's table -- open addressing over a power of two, or a
//            dense slab of n slots when the probe's out-degree sum is a sizeable fraction of n -- or, at
//            the probe's last level (j = q-2), straight into its query's estimate with weight w; a slot holds
//            its node and its sum in one 16-byte pair, so the sum's atomic finds the sector the key lookup loaded
//   compact  the regions' occupied slots, in slot order, become H_{j+1}, still grouped by probe; the compaction
//            empties the slots it reads, so the table needs no clearing between passes
// Work items are (entry, out-edge) pairs balanced by prefix sums over the entries' out-degrees, so a hub's
// out-list is spread over many threads and consecutive threads read consecutive out-edges.
//
// Scores are FP32 products accumulated in 2^-44 fixed point (int64 atomics).  The sums are exact whatever
// order the atomics land in, so the frontier sets, the pruning and switch decisions and the estimates are
// the same alone and in any batch, and a run repeats bit for bit.  Every score is at most 1 and every
// query's estimate sum at most n_r, so values stay below 2^62 for n_r <= 2^18 (checked by the host).
#include <algorithm>

#include "internal.cuh"

namespace ps {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 2048;      // work items per block pass of the expansion
constexpr int kCompactTile = 4096; // table slots per block of the compaction

__device__ __forceinline__ float fx_to_f(long long v) { return __ll2float_rn(v) * __int_as_float((127 - kFixShift) << 23); }
__device__ __forceinline__ long long f_to_fx(float x) { return __float2ll_rn(x * __int_as_float((127 + kFixShift) << 23)); }

__device__ __forceinline__ uint32_t node_hash(int32_t v) {
    return (uint32_t)(((unsigned long long)(uint32_t)v * 0x9E3779B97F4A7C15ull) >> 32);
}

// largest index i in [lo, hi) with pre[i] <= t (pre nondecreasing, pre[lo] <= t)
__device__ __forceinline__ int64_t search_le(const long long *pre, int64_t lo, int64_t hi, long long t) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// tree slots of depth >= 2: the probes
__global__ void k_fr_list(TrieTable t, int32_t *slot, int32_t *count) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= t.cap || t.key[e] == kEmptyKey || t.depth[e] < 2) return;
    slot[atomicAdd(count, 1)] = (int32_t)e;
}

// H_0 = {(u_q, 1)} for every probe; the first excluded node is u_{q-1}, the parent's
__global__ void k_fr_init(TrieTable t, FrontierProbes P, FrontierList F) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.P) return;
    const int32_t s = P.slot[p];
    F.p[p] = p;
    F.x[p] = t.node[s];
    F.val[p] = 1.f;
    P.anc[p] = t.parent[s];
    P.deg[p] = 0;
    P.state[p] = 0;
}

// Rule 2 and the out-degree sums: work[f] = |O(x)| for kept entries, else 0.  Entries are grouped by probe, so
// a warp sums each run of one probe's entries (a segmented shuffle scan) and the run's last lane adds it:
// one atomic per run instead of one per entry on a counter that a large probe's millions of entries share.
__global__ void k_fr_prune(FrontierList F, int64_t nF, TrieTable t, FrontierProbes P, const int64_t *__restrict__ out_off,
                           const float *__restrict__ pw, float eps_p, int32_t j, long long *__restrict__ work) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = f < nF;
    const int32_t p = valid ? F.p[f] : -1;
    unsigned long long x = 0;
    if (valid) {
        const int32_t v = F.x[f];
        bool keep = true;
        if (eps_p > 0.f) {
            const int32_t q = t.depth[P.slot[p]];
            keep = F.val[f] * pw[q - j - 1] > eps_p;
        }
        x = keep ? (unsigned long long)(out_off[v + 1] - out_off[v]) : 0ull;
        work[f] = (long long)x;
    }
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        const int32_t q = __shfl_up_sync(0xffffffffu, p, o);
        if (lane >= o && q == p) x += y;
    }
    const int32_t pn = __shfl_down_sync(0xffffffffu, p, 1);
    if (valid && (lane == 31 || pn != p) && x > 0) atomicAdd(&P.deg[p], x);
}

// Per probe of [p0, p1): the switch decision (Sec. 4.4), the size of its region of the next level's table and a
// bound on its next level's entries.  thr[w] = floor(c0 * w * n) (host FP64); the probe switches when its
// out-degree sum exceeds thr[w].  The decision is idempotent, so a probe range that resumes a level decides the
// same again.
__global__ void k_fr_regions(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1, int32_t j, int32_t n,
                             const long long *__restrict__ thr, uint8_t *t_sw) {
    const int32_t p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const unsigned long long d = P.deg[p];
    P.deg[p] = 0;
    long long r = 0, D = 0;
    if (d > 0) {
        const int32_t s = P.slot[p];
        if (thr && (long long)d > thr[t.weight[s]]) {
            P.state[p] |= kProbeSwitched;
            t_sw[s] = 1;
        } else if (j < t.depth[s] - 2) {
            D = (long long)d < (long long)n ? (long long)d : (long long)n;
            if (4 * D >= (long long)n) {  // dense slab: slot v holds node v
                P.state[p] |= kProbeDense;
                r = n;
            } else {
                P.state[p] &= ~kProbeDense;
                r = 2;
                while (r < 2 * D) r <<= 1;
            }
        }
    }
    P.rsize[p] = r;
    P.dsize[p] = D;
}

__global__ void k_fr_count_switched(FrontierProbes P, unsigned long long *count) {
    const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool sw = p < P.P && (P.state[p] & kProbeSwitched);
    const unsigned m = __ballot_sync(0xffffffffu, sw);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

// entries of switched probes do no deterministic work
__global__ void k_fr_work(FrontierList F, int64_t nF, FrontierProbes P, long long *__restrict__ work) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f < nF && (P.state[F.p[f]] & kProbeSwitched)) work[f] = 0;
}

// One pass per block over kItems consecutive work items (entry f, out-edge e).  The block's slice of the
// work prefix sums is staged in shared memory when it is short, so an item finds its entry with a short search.
__global__ void __launch_bounds__(kThreads) k_fr_expand(DeviceGraph g, TrieTable t, FrontierProbes P, FrontierList F,
                                                        FrontierExpand a) {
    __shared__ long long s_pref[kItems + 1];
    __shared__ int64_t s_f0, s_nf;
    const long long E = a.e_hi - a.e_lo;
    const int64_t nblk = (E + kItems - 1) / kItems;
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long t0 = a.e_lo + blk * kItems, t1 = min(a.e_hi, t0 + kItems);
        if (threadIdx.x == 0) {
            const int64_t lo = search_le(a.wp, a.f_lo, a.f_hi, t0);
            const int64_t hi = search_le(a.wp, lo, a.f_hi, t1 - 1);
            s_f0 = lo;
            s_nf = hi - lo + 1;
        }
        __syncthreads();
        const int64_t f0 = s_f0, nf = s_nf;
        const bool staged = nf <= kItems;
        if (staged)
            for (int64_t i = threadIdx.x; i <= nf; i += blockDim.x) s_pref[i] = a.wp[f0 + i];
        __syncthreads();
        for (long long it = t0 + threadIdx.x; it < t1; it += blockDim.x) {
            int64_t f;
            if (staged) {
                int64_t lo = 0, hi = nf;
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (s_pref[mid] <= it) lo = mid; else hi = mid;
                }
                f = f0 + lo;
            } else {
                f = search_le(a.wp, f0, a.f_hi, it);
            }
            const int32_t p = F.p[f], x = F.x[f];
            const long long e = it - a.wp[f];
            const int32_t v = g.out_col[g.out_off[x] + e];
            const int32_t s = P.slot[p];
            if (v == t.node[P.anc[p]]) continue;  // level j excludes u_{q-j-1}
            const long long c = f_to_fx(g.w[v] * F.val[f]);
            if (a.j == t.depth[s] - 2) {  // last level: weight * Score into the query's estimate
                atomicAdd(a.acc + (int64_t)t.query[s] * a.n + v, (unsigned long long)(c * (long long)t.weight[s]));
                continue;
            }
            const long long off = P.roff[p] - a.rbase, R = P.roff[p + 1] - P.roff[p];
            const int32_t key = v + 1;
            if (P.state[p] & kProbeDense) {
                FrontierSlot &slot = a.tab[off + v];
                slot.key = key;
                atomicAdd(&slot.val, (unsigned long long)c);
            } else {
                long long h = node_hash(v) & (R - 1);
                for (long long probe = 0; probe < R; ++probe) {
                    FrontierSlot &slot = a.tab[off + h];
                    int32_t cur = slot.key;
                    if (cur == 0) {
                        cur = atomicCAS(&slot.key, 0, key);
                        if (cur == 0) cur = key;
                    }
                    if (cur == key) {
                        atomicAdd(&slot.val, (unsigned long long)c);
                        break;
                    }
                    h = (h + 1) & (R - 1);
                }
            }
        }
        __syncthreads();
    }
}

// occupied slots per block of kCompactTile table slots
__global__ void __launch_bounds__(kThreads) k_fr_count(const FrontierSlot *__restrict__ tab, long long T,
                                                       long long *__restrict__ bcount) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kCompactTile;
    int c = 0;
    for (int i = threadIdx.x; i < kCompactTile; i += blockDim.x) {
        const long long k = base + i;
        if (k < T && tab[k].key != 0) ++c;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) bcount[blockIdx.x] = s_cnt;
}

// writes the occupied slots of each block, in slot order, at out_base + bpre[block], and empties them again, so
// the table is clean for the next pass without a memset
__global__ void __launch_bounds__(kThreads) k_fr_write(FrontierSlot *__restrict__ tab, long long T,
                                                       const long long *__restrict__ roff, int32_t p0, int32_t p1,
                                                       long long rbase, const long long *__restrict__ bpre,
                                                       FrontierList out, long long out_base, long long out_cap) {
    __shared__ int s_warp[kThreads / 32];
    __shared__ long long s_run;
    __shared__ int32_t s_plo, s_phi;
    const long long base = (long long)blockIdx.x * kCompactTile;
    if (threadIdx.x == 0) {
        s_run = out_base + bpre[blockIdx.x];
        // the probes whose regions hold this block's first and last slots: the per-slot search stays between them
        const long long last = min(T, base + kCompactTile) - 1;
        int32_t lo = p0, hi = p1;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (roff[mid] - rbase <= base) lo = mid; else hi = mid;
        }
        s_plo = lo;
        hi = p1;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (roff[mid] - rbase <= last) lo = mid; else hi = mid;
        }
        s_phi = lo + 1;
    }
    __syncthreads();
    const int32_t plo = s_plo, phi = s_phi;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < kCompactTile; r += kThreads) {
        const long long k = base + r + threadIdx.x;
        const bool occ = k < T && tab[k].key != 0;
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) before += s_warp[w];
            total += s_warp[w];
        }
        const long long pos = s_run + before + __popc(m & ((1u << lane) - 1));
        if (occ && pos < out_cap) {  // the host sees a total above out_cap and fails the call
            // the probe whose region holds slot k: largest p in [plo, phi) with roff[p] - rbase <= k
            int32_t lo = plo, hi = phi;
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (roff[mid] - rbase <= k) lo = mid; else hi = mid;
            }
            out.p[pos] = lo;
            out.x[pos] = tab[k].key - 1;
            out.val[pos] = fx_to_f((long long)tab[k].val);
        }
        if (occ) *reinterpret_cast<ulonglong2 *>(tab + k) = make_ulonglong2(0ull, 0ull);
        __syncthreads();
        if (threadIdx.x == 0) s_run += total;
        __syncthreads();
    }
}

// the next level excludes the next ancestor up (probes [p0, p1))
__global__ void k_fr_advance(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1) {
    const int32_t p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int32_t a = P.anc[p];
    if (a >= 0) P.anc[p] = t.parent[a];
}

// for each given probe: its first entry in the probe-sorted frontier, the work prefix there, and the region and
// entry-bound offsets at the probe
__global__ void k_fr_bounds(const int32_t *__restrict__ fp, int64_t nF, const long long *__restrict__ wp,
                            const long long *__restrict__ roff, const long long *__restrict__ doff,
                            const int32_t *__restrict__ probes, int32_t count, long long *__restrict__ out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int32_t p = probes[i];
    int64_t lo = 0, hi = nF;  // lower bound of p
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (fp[mid] < p) lo = mid + 1; else hi = mid;
    }
    out[4 * i] = lo;
    out[4 * i + 1] = wp[lo];
    out[4 * i + 2] = roff[p];
    out[4 * i + 3] = doff[p];
}

// s(u, v) = (fixed-point deterministic sum + randomized member count) / n_r + shift, s(u, u) = 1
__global__ void k_fr_finalize(int32_t n, const int32_t *__restrict__ qnode, const unsigned long long *__restrict__ acc,
                              const int32_t *__restrict__ counts, const float *__restrict__ inv_nr,
                              const int32_t *__restrict__ ext2int, float shift, float *__restrict__ out) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t b = blockIdx.y;
    if (v >= n) return;
    const int64_t i = (int64_t)b * n + ext2int[v];
    long long tot = (long long)acc[i];
    if (counts) tot += (long long)counts[i] << kFixShift;
    float s = fx_to_f(tot) * inv_nr[b] + shift;
    if ((int32_t)v == qnode[b]) s = 1.f;
    out[(int64_t)b * n + v] = s;
}

inline unsigned blocks_for(int64_t count, int threads = kThreads) {
    return (unsigned)std::max<int64_t>(1, (count + threads - 1) / threads);
}

}  // namespace

void launch_fr_list(TrieTable t, int32_t *slot, int32_t *count, cudaStream_t s) {
    k_fr_list<<<blocks_for(t.cap), kThreads, 0, s>>>(t, slot, count);
}
void launch_fr_init(TrieTable t, FrontierProbes P, FrontierList F, cudaStream_t s) {
    if (P.P > 0) k_fr_init<<<blocks_for(P.P), kThreads, 0, s>>>(t, P, F);
}
void launch_fr_prune(FrontierList F, int64_t nF, TrieTable t, FrontierProbes P, const int64_t *out_off, const float *pw,
                     float eps_p, int32_t j, long long *work, cudaStream_t s) {
    if (nF > 0) k_fr_prune<<<blocks_for(nF), kThreads, 0, s>>>(F, nF, t, P, out_off, pw, eps_p, j, work);
}
void launch_fr_regions(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1, int32_t j, int32_t n, const long long *thr,
                       uint8_t *t_sw, cudaStream_t s) {
    if (p1 > p0) k_fr_regions<<<blocks_for(p1 - p0), kThreads, 0, s>>>(t, P, p0, p1, j, n, thr, t_sw);
}
void launch_fr_count_switched(FrontierProbes P, unsigned long long *count, cudaStream_t s) {
    cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (P.P > 0) k_fr_count_switched<<<blocks_for(P.P), kThreads, 0, s>>>(P, count);
}
void launch_fr_work(FrontierList F, int64_t nF, FrontierProbes P, long long *work, cudaStream_t s) {
    if (nF > 0) k_fr_work<<<blocks_for(nF), kThreads, 0, s>>>(F, nF, P, work);
}
void launch_fr_expand(const DeviceGraph &g, TrieTable t, FrontierProbes P, FrontierList F, const FrontierExpand &a,
                      cudaStream_t s) {
    const long long E = a.e_hi - a.e_lo;
    if (E <= 0) return;
    const int blocks = grid_for((E + kItems - 1) / kItems, 1, 8);
    k_fr_expand<<<blocks, kThreads, 0, s>>>(g, t, P, F, a);
}
int64_t fr_compact_blocks(long long T) { return (T + kCompactTile - 1) / kCompactTile; }
void launch_fr_count(const FrontierSlot *tab, long long T, long long *bcount, cudaStream_t s) {
    if (T > 0) k_fr_count<<<(unsigned)fr_compact_blocks(T), kThreads, 0, s>>>(tab, T, bcount);
}
void launch_fr_write(FrontierSlot *tab, long long T, const long long *roff, int32_t p0,
                     int32_t p1, long long rbase, const long long *bpre, FrontierList out, long long out_base,
                     long long out_cap, cudaStream_t s) {
    if (T > 0)
        k_fr_write<<<(unsigned)fr_compact_blocks(T), kThreads, 0, s>>>(tab, T, roff, p0, p1, rbase, bpre, out,
                                                                       out_base, out_cap);
}
void launch_fr_advance(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1, cudaStream_t s) {
    if (p1 > p0) k_fr_advance<<<blocks_for(p1 - p0), kThreads, 0, s>>>(t, P, p0, p1);
}
void launch_fr_bounds(const int32_t *fp, int64_t nF, const long long *wp, const long long *roff, const long long *doff,
                      const int32_t *probes, int32_t count, long long *out, cudaStream_t s) {
    if (count > 0) k_fr_bounds<<<blocks_for(count), kThreads, 0, s>>>(fp, nF, wp, roff, doff, probes, count, out);
}
void launch_fr_finalize(int32_t n, int32_t B, const int32_t *qnode, const unsigned long long *acc, const int32_t *counts,
                        const float *inv_nr, const int32_t *ext2int, float shift, float *out, cudaStream_t s) {
    dim3 grid(blocks_for(n), (unsigned)B);
    k_fr_finalize<<<grid, kThreads, 0, s>>>(n, qnode, acc, counts, inv_nr, ext2int, shift, out);
}

}  // namespace ps
