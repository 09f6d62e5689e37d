// Top-k (Def. 2): the k nodes v != u with the largest estimates, ordered by (estimate descending,
// id ascending).  Radix select over order-preserving 32-bit keys of the FP32 scores, four 8-bit
// passes, many blocks per query; then the entries above the threshold plus the smallest-id ties at the
// threshold are collected and sorted in one block per query.
#include "internal.cuh"

namespace ps {

constexpr int kTopkThreads = 256;

__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fval(uint32_t k) {
    const uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

int topk_blocks_per_query(int32_t n) {
    int64_t b = ((int64_t)n + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

// state[b*4 + 0] = prefix, [1] = k remaining, [2] = count above threshold (cursor), [3] = unused
__global__ void k_topk_init(int32_t B, const int32_t *__restrict__ qk, unsigned int *state, unsigned int *hist) {
    const int32_t b = blockIdx.x;
    if (threadIdx.x == 0) {
        state[b * 4 + 0] = 0u;
        state[b * 4 + 1] = (unsigned int)qk[b];
        state[b * 4 + 2] = 0u;
        state[b * 4 + 3] = 0u;
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[b * 256 + i] = 0u;
}

__global__ void __launch_bounds__(kTopkThreads) k_topk_hist(int32_t n, const float *__restrict__ scores,
                                                            const int32_t *__restrict__ qnode,
                                                            const unsigned int *__restrict__ state, unsigned int *hist,
                                                            int shift) {
    __shared__ unsigned int s_h[256];
    const int32_t b = blockIdx.y;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_h[i] = 0u;
    __syncthreads();
    const uint32_t prefix = state[b * 4 + 0];
    const uint32_t hi_mask = shift >= 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    const int64_t per = ((int64_t)n + gridDim.x - 1) / gridDim.x;
    const int64_t beg = blockIdx.x * per, end = min((int64_t)n, beg + per);
    const float *row = scores + (int64_t)b * n;
    const int32_t u = qnode[b];
    for (int64_t v = beg + threadIdx.x; v < end; v += blockDim.x) {
        if ((int32_t)v == u) continue;
        const uint32_t k = fkey(row[v]);
        if ((k & hi_mask) == prefix) atomicAdd(&s_h[(k >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (s_h[i]) atomicAdd(&hist[b * 256 + i], s_h[i]);
}

__global__ void k_topk_select(unsigned int *state, unsigned int *hist, int shift) {
    const int32_t b = blockIdx.x;
    if (threadIdx.x == 0) {
        uint32_t krem = state[b * 4 + 1];
        uint32_t cum = 0;
        int d = 255;
        for (; d > 0; --d) {
            const uint32_t h = hist[b * 256 + d];
            if (cum + h >= krem) break;
            cum += h;
        }
        state[b * 4 + 0] |= ((uint32_t)d << shift);
        state[b * 4 + 1] = krem - cum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[b * 256 + i] = 0u;
}

// Entries strictly above the threshold go to the candidate list; ties are counted per block.
__global__ void __launch_bounds__(kTopkThreads) k_topk_collect(int32_t n, const float *__restrict__ scores,
                                                               const int32_t *__restrict__ qnode, unsigned int *state,
                                                               unsigned int *tiecnt, int32_t kmax, int32_t *cand_id,
                                                               float *cand_val) {
    __shared__ unsigned int s_ties;
    const int32_t b = blockIdx.y;
    if (threadIdx.x == 0) s_ties = 0u;
    __syncthreads();
    const uint32_t thr = state[b * 4 + 0];
    const int64_t per = ((int64_t)n + gridDim.x - 1) / gridDim.x;
    const int64_t beg = blockIdx.x * per, end = min((int64_t)n, beg + per);
    const float *row = scores + (int64_t)b * n;
    const int32_t u = qnode[b];
    unsigned int ties = 0;
    for (int64_t v = beg + threadIdx.x; v < end; v += blockDim.x) {
        if ((int32_t)v == u) continue;
        const uint32_t k = fkey(row[v]);
        if (k > thr) {
            const unsigned int pos = atomicAdd(&state[b * 4 + 2], 1u);
            if (pos < (unsigned)kmax) {
                cand_id[(int64_t)b * kmax + pos] = (int32_t)v;
                cand_val[(int64_t)b * kmax + pos] = row[v];
            }
        } else if (k == thr) {
            ++ties;
        }
    }
    if (ties) atomicAdd(&s_ties, ties);
    __syncthreads();
    if (threadIdx.x == 0) tiecnt[(int64_t)b * gridDim.x + blockIdx.x] = s_ties;
}

// Exclusive scan of the per-block tie counts of each query (at most 1024 blocks).
__global__ void __launch_bounds__(1024) k_topk_tiebase(unsigned int *tiecnt, int nblk) {
    __shared__ unsigned int s[1024];
    const int32_t b = blockIdx.x;
    const int t = threadIdx.x;
    const unsigned int mine = t < nblk ? tiecnt[(int64_t)b * nblk + t] : 0u;
    s[t] = mine;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned int v = t >= off ? s[t - off] : 0u;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    if (t < nblk) tiecnt[(int64_t)b * nblk + t] = s[t] - mine;
}

// The k_remaining ties with the smallest ids, in id order across blocks.
__global__ void __launch_bounds__(kTopkThreads) k_topk_ties(int32_t n, const float *__restrict__ scores,
                                                            const int32_t *__restrict__ qnode,
                                                            const unsigned int *__restrict__ state,
                                                            const unsigned int *__restrict__ tiebase, int32_t kmax,
                                                            int32_t *cand_id, float *cand_val) {
    __shared__ unsigned int s_warp[kTopkThreads / 32];
    __shared__ unsigned int s_base;
    const int32_t b = blockIdx.y;
    const uint32_t thr = state[b * 4 + 0];
    const uint32_t krem = state[b * 4 + 1];
    const uint32_t above = state[b * 4 + 2];
    const int64_t per = ((int64_t)n + gridDim.x - 1) / gridDim.x;
    const int64_t beg = blockIdx.x * per, end = min((int64_t)n, beg + per);
    const float *row = scores + (int64_t)b * n;
    const int32_t u = qnode[b];
    if (threadIdx.x == 0) s_base = tiebase[(int64_t)b * gridDim.x + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = beg; c0 < end; c0 += blockDim.x) {
        const int64_t v = c0 + threadIdx.x;
        const bool tie = v < end && (int32_t)v != u && fkey(row[v]) == thr;
        const unsigned int bal = __ballot_sync(0xffffffffu, tie);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        unsigned int wbase = 0, total = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            if (i < warp) wbase += s_warp[i];
            total += s_warp[i];
        }
        const unsigned int rank = s_base + wbase + __popc(bal & ((1u << lane) - 1u));
        if (tie && rank < krem && above + rank < (unsigned)kmax) {
            cand_id[(int64_t)b * kmax + above + rank] = (int32_t)v;
            cand_val[(int64_t)b * kmax + above + rank] = row[v];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
    }
}

// Bitonic sort of each query's k candidates by (value desc, id asc); outputs padded with -1 / 0.
__global__ void __launch_bounds__(1024) k_topk_sort(const int32_t *__restrict__ qk, int32_t kmax,
                                                    const int32_t *__restrict__ cand_id,
                                                    const float *__restrict__ cand_val, int32_t *ids, float *vals) {
    extern __shared__ unsigned char s_raw[];
    const int32_t b = blockIdx.x;
    const int32_t k = qk[b];
    int P = 1;
    while (P < k) P <<= 1;
    float *sv = reinterpret_cast<float *>(s_raw);
    int32_t *si = reinterpret_cast<int32_t *>(sv + P);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < k) {
            sv[i] = cand_val[(int64_t)b * kmax + i];
            si[i] = cand_id[(int64_t)b * kmax + i];
        } else {
            sv[i] = -__int_as_float(0x7f800000);  // -inf sorts last
            si[i] = 0x7fffffff;
        }
    }
    __syncthreads();
    // "a before b" when a.val > b.val, or equal values and a.id < b.id
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool i_first = sv[i] > sv[j] || (sv[i] == sv[j] && si[i] < si[j]);
                    if (up != i_first) {
                        const float tv = sv[i]; sv[i] = sv[j]; sv[j] = tv;
                        const int32_t ti = si[i]; si[i] = si[j]; si[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < kmax; i += blockDim.x) {
        ids[(int64_t)b * kmax + i] = i < k ? si[i] : -1;
        vals[(int64_t)b * kmax + i] = i < k ? sv[i] : 0.f;
    }
}

// Loads the module that holds the top-k kernels (under lazy loading a module loads, and may allocate device
// memory, on its first use; querying a kernel's attributes is such a use).
cudaError_t topk_preload() {
    const void *fns[] = {(const void *)k_topk_init, (const void *)k_topk_hist, (const void *)k_topk_select,
                         (const void *)k_topk_collect, (const void *)k_topk_tiebase, (const void *)k_topk_ties,
                         (const void *)k_topk_sort};
    for (const void *f : fns) {
        cudaFuncAttributes a;
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void launch_topk(int32_t n, int32_t B, const float *scores, const int32_t *qnode, const int32_t *qk, int32_t kmax,
                 TopkScratch sc, int32_t *ids, float *vals, cudaStream_t s, int64_t *launches) {
    const int nblk = topk_blocks_per_query(n);
    k_topk_init<<<B, 256, 0, s>>>(B, qk, sc.state, sc.hist);
    dim3 grid(nblk, B);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        k_topk_hist<<<grid, kTopkThreads, 0, s>>>(n, scores, qnode, sc.state, sc.hist, shift);
        k_topk_select<<<B, 256, 0, s>>>(sc.state, sc.hist, shift);
    }
    k_topk_collect<<<grid, kTopkThreads, 0, s>>>(n, scores, qnode, sc.state, sc.tiecnt, kmax, sc.cand_id, sc.cand_val);
    k_topk_tiebase<<<B, 1024, 0, s>>>(sc.tiecnt, nblk);
    k_topk_ties<<<grid, kTopkThreads, 0, s>>>(n, scores, qnode, sc.state, sc.tiecnt, kmax, sc.cand_id, sc.cand_val);
    int P = 1;
    while (P < kmax) P <<= 1;
    k_topk_sort<<<B, 1024, (size_t)P * 8, s>>>(qk, kmax, sc.cand_id, sc.cand_val, ids, vals);
    if (launches) *launches += 13;
}

}  // namespace ps
