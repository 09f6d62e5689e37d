// Device-side initial build of the graph store from an edge list (the directed graph of Sec. 2.1: in-lists I(v)
// for the sqrt(c)-walks and PROBE's weights, out-lists O(x) for the probes' pushes).  A graph of 10^9 edges is
// sorted and laid out on the GPU in about a second, where a host sort takes minutes.
//
//   1. a key per edge, (destination << bs) | source in the caller's ids; a loop gets the key n << bs, which sorts
//      after every edge; an id outside [0, n) raises a flag the host reads
//   2. an LSD radix sort of the keys (below)
//   3. repeats and loops dropped: a flag per key, its prefix sums, a compaction
//   4. the caller-id in-list offsets (run boundaries of the sorted keys) and out-degrees; the renumbering by
//      descending out-degree, ties by caller id, as a radix sort of n keys ((m - outdeg) << bs | id)
//   5. the in-lists per internal row in the caller's source order (each row's run of sorted keys mapped through
//      ext2int), and the out-lists from a radix sort of (source << bs | destination) in internal ids
// w and the pull pieces then come from the kernels the update path uses.
//
// Radix sort: 8-bit digits, least significant first, tiles of 4096 keys.  Per digit pass, one kernel counts
// each tile's digits into a digit-major table, whose exclusive prefix sums are every (digit, tile)'s first output
// index; a second kernel ranks each key among the tile's earlier keys of its digit (warps take 32 keys a round in
// index order and rank them with __match_any_sync against per-warp running counts, so the sort is stable),
// stages the tile in shared memory in digit order and writes each digit's run contiguously.
#include <algorithm>

#include "internal.cuh"

namespace ps {

constexpr int kRadix = 256;
constexpr int kRadixThreads = 256;  // one thread per digit in the per-tile digit scans
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixKPT = 16;       // keys per thread
constexpr int kRadixTile = kRadixThreads * kRadixKPT;
constexpr int kWarpKeys = 32 * kRadixKPT;
static_assert(kRadixThreads == kRadix, "the digit scans use one thread per digit");

int64_t radix_tiles(int64_t count) { return (count + kRadixTile - 1) / kRadixTile; }

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint64_t *__restrict__ keys, int64_t count,
                                                              int shift, long long *__restrict__ counts,
                                                              int64_t ntiles) {
    __shared__ unsigned int h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t base = blockIdx.x * (int64_t)kRadixTile;
#pragma unroll 4
    for (int r = 0; r < kRadixKPT; ++r) {
        const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        const uint32_t d = i < count ? (uint32_t)(keys[i] >> shift) & (kRadix - 1) : kRadix;
        // lanes with the same digit add once (skewed digits would otherwise serialise on one counter)
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < kRadix && (peers >> lane) == 1u) atomicAdd(&h[d], (unsigned)__popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive prefix sum of one value per thread over a block of kRadixThreads threads
__device__ __forceinline__ uint32_t radix_block_exclusive(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    return before + x - v;
}

__global__ void __launch_bounds__(kRadixThreads, 3) k_radix_scatter(const uint64_t *__restrict__ in,
                                                                 uint64_t *__restrict__ out, int64_t count, int shift,
                                                                 const long long *__restrict__ offsets,
                                                                 int64_t ntiles) {
    __shared__ uint32_t wcnt[kRadixWarps][kRadix];  // per warp: keys of each digit so far, then its first rank
    __shared__ uint32_t dstart[kRadix];             // first tile-local position of each digit
    __shared__ long long goff[kRadix];              // output index of the digit's first key, minus dstart
    __shared__ uint32_t s_warp[kRadixWarps];
    __shared__ uint64_t stage[kRadixTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * kRadix; i += kRadixThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = blockIdx.x * (int64_t)kRadixTile;
    const int64_t base = tile0 + (int64_t)warp * kWarpKeys;
    uint64_t key[kRadixKPT];
    uint32_t rank[kRadixKPT];
#pragma unroll
    for (int r = 0; r < kRadixKPT; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < count;
        key[r] = ok ? in[i] : 0ull;
        const uint32_t d = ok ? (uint32_t)(key[r] >> shift) & (kRadix - 1) : kRadix;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = ok ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (ok && (peers >> lane) == 1u) wcnt[warp][d] = before + __popc(peers);  // the peers' highest lane
        __syncwarp();
        rank[r] = before + __popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t s = 0;
        for (int w = 0; w < kRadixWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = s;
            s += c;
        }
        const uint32_t st = radix_block_exclusive(s, s_warp);
        dstart[d] = st;
        goff[d] = offsets[(int64_t)d * ntiles + blockIdx.x] - (long long)st;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixKPT; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < count) {
            const uint32_t d = (uint32_t)(key[r] >> shift) & (kRadix - 1);
            stage[dstart[d] + wcnt[warp][d] + rank[r]] = key[r];
        }
    }
    __syncthreads();
    const int64_t left = count - tile0;
    const int valid = left < kRadixTile ? (int)left : kRadixTile;
    for (int j = threadIdx.x; j < valid; j += kRadixThreads) {
        const uint64_t k = stage[j];
        out[goff[(k >> shift) & (kRadix - 1)] + j] = k;
    }
}

uint64_t *radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t count, int bits, long long *counts,
                         long long *offsets, long long *partial, cudaStream_t s) {
    if (count <= 1) return keys;
    const int64_t nt = radix_tiles(count);
    uint64_t *a = keys, *b = tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nt, kRadixThreads, 0, s>>>(a, count, shift, counts, nt);
        launch_scan64(counts, (int64_t)kRadix * nt, partial, offsets, s);
        k_radix_scatter<<<(unsigned)nt, kRadixThreads, 0, s>>>(a, b, count, shift, offsets, nt);
        std::swap(a, b);
    }
    return a;
}

// ------------------------------------------------------------------------------------------------
// build steps
// ------------------------------------------------------------------------------------------------
static unsigned build_blocks(int64_t work, int threads) {
    return (unsigned)std::min<int64_t>((work + threads - 1) / threads, (int64_t)152 * 32);
}

__global__ void k_build_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m, int32_t n,
                             int bs, uint64_t *__restrict__ keys, int32_t *bad) {
    const uint64_t loop_key = (uint64_t)(uint32_t)n << bs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = src[i], d = dst[i];
        if ((uint32_t)s >= (uint32_t)n || (uint32_t)d >= (uint32_t)n) {
            atomicOr(bad, 1);
            keys[i] = loop_key;
            continue;
        }
        keys[i] = s == d ? loop_key : (((uint64_t)(uint32_t)d << bs) | (uint32_t)s);
    }
}

// flag[i] = 1 for the first copy of each edge key (keys sorted; loop keys and those after them dropped)
__global__ void k_build_flags(const uint64_t *__restrict__ keys, int64_t m, uint64_t end_key, long long *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        flag[i] = (k < end_key && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

__global__ void k_build_compact(const uint64_t *__restrict__ keys, int64_t m, uint64_t end_key,
                                const long long *__restrict__ pre, uint64_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (k < end_key && (i == 0 || keys[i - 1] != k)) out[pre[i]] = k;
    }
}

// ext_off[v] = first index of destination v's run in the sorted unique keys, v = 0..n (each v written once: by the
// key that starts the first run at or after v, or by index mu for the rows after the last run).  One pass over the
// keys; the thread at a run boundary also fills the nodes without in-edges just before it, so a long stretch of
// such nodes is written by one thread (on power-law inputs the stretches are short).
__global__ void k_build_ext_off(const uint64_t *__restrict__ ukeys, int64_t mu, int32_t n, int bs,
                                long long *__restrict__ ext_off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= mu; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = i == 0 ? -1 : (int64_t)(ukeys[i - 1] >> bs);
        const int64_t cur = i == mu ? (int64_t)n : (int64_t)(ukeys[i] >> bs);
        for (int64_t v = prev + 1; v <= cur; ++v) ext_off[v] = i;
    }
}

__global__ void k_build_outdeg(const uint64_t *__restrict__ ukeys, int64_t mu, uint32_t smask,
                               unsigned long long *outdeg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mu; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&outdeg[ukeys[i] & smask], 1ull);
}

__global__ void k_build_rank_keys(const unsigned long long *__restrict__ outdeg, int32_t n, int64_t mu, int bs,
                                  uint64_t *__restrict__ rk) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        rk[v] = ((uint64_t)(mu - (int64_t)outdeg[v]) << bs) | (uint64_t)v;
}

// the renumbering, and each internal row's in- and out-degree
__global__ void k_build_perm(const uint64_t *__restrict__ rk, int32_t n, uint32_t smask,
                             const long long *__restrict__ ext_off, const unsigned long long *__restrict__ outdeg,
                             int32_t *__restrict__ int2ext, int32_t *__restrict__ ext2int, long long *__restrict__ indeg_i,
                             long long *__restrict__ outdeg_i) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(rk[i] & smask);
        int2ext[i] = v;
        ext2int[v] = (int32_t)i;
        indeg_i[i] = ext_off[v + 1] - ext_off[v];
        outdeg_i[i] = (long long)outdeg[v];
    }
}

// one warp per internal row i: its in-list in the caller's source order, in internal ids, and the (source, i) key
// of each of its edges for the out-list sort
__global__ void __launch_bounds__(256) k_build_in_col(int32_t n, const int32_t *__restrict__ int2ext,
                                                      const long long *__restrict__ ext_off,
                                                      const int64_t *__restrict__ in_off,
                                                      const uint64_t *__restrict__ ukeys, uint32_t smask,
                                                      const int32_t *__restrict__ ext2int, int bs,
                                                      int32_t *__restrict__ in_col, uint64_t *__restrict__ okeys) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const int32_t v = int2ext[i];
        const long long e0 = ext_off[v], d = ext_off[v + 1] - e0;
        const int64_t b = in_off[i];
        for (long long j = lane; j < d; j += 32) {
            const int32_t x = ext2int[ukeys[e0 + j] & smask];
            in_col[b + j] = x;
            okeys[b + j] = ((uint64_t)(uint32_t)x << bs) | (uint64_t)i;
        }
    }
}

__global__ void k_build_out_col(const uint64_t *__restrict__ okeys, int64_t mu, uint32_t smask,
                                int32_t *__restrict__ out_col) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mu; e += (int64_t)gridDim.x * blockDim.x)
        out_col[e] = (int32_t)(okeys[e] & smask);
}

__global__ void k_active_rows(const int64_t *__restrict__ out_off, int32_t n, int32_t *res) {
    int32_t best = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (out_off[v + 1] > out_off[v]) best = (int32_t)v + 1;
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(res, best);
}

void launch_active_rows(const int64_t *out_off, int32_t n, int32_t *res, cudaStream_t s) {
    k_active_rows<<<build_blocks(n, 256), 256, 0, s>>>(out_off, n, res);
}

void launch_build_keys(const int32_t *src, const int32_t *dst, int64_t m, int32_t n, int bs, uint64_t *keys,
                       int32_t *bad, cudaStream_t s) {
    if (m > 0) k_build_keys<<<build_blocks(m, 256), 256, 0, s>>>(src, dst, m, n, bs, keys, bad);
}
void launch_build_flags(const uint64_t *keys, int64_t m, uint64_t end_key, long long *flag, cudaStream_t s) {
    if (m > 0) k_build_flags<<<build_blocks(m, 256), 256, 0, s>>>(keys, m, end_key, flag);
}
void launch_build_compact(const uint64_t *keys, int64_t m, uint64_t end_key, const long long *pre, uint64_t *out,
                          cudaStream_t s) {
    if (m > 0) k_build_compact<<<build_blocks(m, 256), 256, 0, s>>>(keys, m, end_key, pre, out);
}
void launch_build_ext_off(const uint64_t *ukeys, int64_t mu, int32_t n, int bs, long long *ext_off, cudaStream_t s) {
    k_build_ext_off<<<build_blocks(mu + 1, 256), 256, 0, s>>>(ukeys, mu, n, bs, ext_off);
}
void launch_build_outdeg(const uint64_t *ukeys, int64_t mu, uint32_t smask, unsigned long long *outdeg,
                         cudaStream_t s) {
    if (mu > 0) k_build_outdeg<<<build_blocks(mu, 256), 256, 0, s>>>(ukeys, mu, smask, outdeg);
}
void launch_build_rank_keys(const unsigned long long *outdeg, int32_t n, int64_t mu, int bs, uint64_t *rk,
                            cudaStream_t s) {
    k_build_rank_keys<<<build_blocks(n, 256), 256, 0, s>>>(outdeg, n, mu, bs, rk);
}
void launch_build_perm(const uint64_t *rk, int32_t n, uint32_t smask, const long long *ext_off,
                       const unsigned long long *outdeg, int32_t *int2ext, int32_t *ext2int, long long *indeg_i,
                       long long *outdeg_i, cudaStream_t s) {
    k_build_perm<<<build_blocks(n, 256), 256, 0, s>>>(rk, n, smask, ext_off, outdeg, int2ext, ext2int, indeg_i,
                                                       outdeg_i);
}
void launch_build_in_col(int32_t n, const int32_t *int2ext, const long long *ext_off, const int64_t *in_off,
                         const uint64_t *ukeys, uint32_t smask, const int32_t *ext2int, int bs, int32_t *in_col,
                         uint64_t *okeys, cudaStream_t s) {
    k_build_in_col<<<build_blocks((int64_t)n * 32, 256), 256, 0, s>>>(n, int2ext, ext_off, in_off, ukeys, smask,
                                                                       ext2int, bs, in_col, okeys);
}
void launch_build_out_col(const uint64_t *okeys, int64_t mu, uint32_t smask, int32_t *out_col, cudaStream_t s) {
    if (mu > 0) k_build_out_col<<<build_blocks(mu, 256), 256, 0, s>>>(okeys, mu, smask, out_col);
}

}  // namespace ps
