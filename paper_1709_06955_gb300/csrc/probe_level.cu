// PROBE level loop over the reverse-reachability tree (Alg. 2 / Alg. 4), regrouped.
//
// Alg. 4 probes every tree node r_q (the prefix (u_1..u_q)) with q-1 levels of Alg. 2 and adds
// w_q/n_r * PROBE(u_1..u_q).  Writing one level of Alg. 2 as a linear map, Score_{j+1} = X_a M Score_j
// with (M y)[v] = sqrt(c)/|I(v)| * sum_{x in I(v)} y[x] and X_a zeroing entry a = u_{q-j-1}, the sum over
// all tree nodes factors along the tree (Horner's rule): for a tree node t with graph node a,
//     C(t)  = sum over children s of Y(s),        Y(s) = w_s/n_r e_{a_s} + X_{a_s} M C(s),
// and the estimate is M C(root) (entry u then set to 1).  Because X_a only removes entry a,
//     X_a M C = M C - beta e_a,   beta = (M C)[a] = sqrt(c)/|I(a)| * sum_{x in I(a)} C[x],
// so with gamma_s = w_s/n_r - beta_s the children of one tree node share one application of M:
//     C(t) = M D(t) + sum_s gamma_s e_{a_s},  D(t) = sum over children s of C(s).
// A tree node whose subtree has height >= 2 owns a score vector MD(t) = M D(t) (a column); lower nodes
// only contribute their sparse gamma terms.  For height >= 3 the column is "dense" and computed by the
// pull; for height 2, D(t) is just the gamma terms of t's grandchildren (all leaves), so the column is
// "pushed": MD(t) = sum_g gamma_g * sum_{x in O(a_g)} sqrt(c)/|I(x)| e_x.  The level loop runs from the
// deepest depth to the virtual super-root (depth 0, whose only child is the root u):
//   dbuild   D(t)[x]  = sum of the children's MD columns                (segmented row sums, dense t)
//   scatter  D(t)[a_g] += gamma_g for every grandchild g of t            (sparse terms, dense t)
//   pull     MD(t)[v] = sqrt(c)/|I(v)| * sum_{x in I(v)} D(t)[x]         (the dominant kernel, dense t)
//   push     MD(t)[x] += sqrt(c)/|I(x)| * gamma_g, x in O(a_g)           (height-2 t)
//   gamma    gamma_t  = w_t/n_r - sqrt(c)/|I(a_t)| * (sum_{x in I(a_t)} MD(t)[x] + G_t),  G_parent += gamma_t
// The result is exactly Alg. 4's (up to FP32 rounding); the work is one pull per slot instead of
// q-1 pushes per tree node.  Score vectors of one depth are stored node-major, [n][pitch] FP32.
#include <algorithm>

#include "internal.cuh"

namespace ps {

// ------------------------------------------------------------------------------------------------
// dbuild: one warp per row x; D[x][p] = sum_{c in children(p)} MDp[x][c], zero for padding columns.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dbuild(int32_t n, const float *__restrict__ MDp, int32_t pp,
                                                float *__restrict__ D, int32_t pd, int32_t S,
                                                const int32_t *__restrict__ child_off,
                                                const int32_t *__restrict__ child_list) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < n; x += nwarps) {
        const float *src = MDp + x * pp;
        float *dst = D + x * pd;
        for (int32_t p = lane; p < pd; p += 32) {
            float acc = 0.f;
            if (p < S) {
                const int32_t cb = __ldg(child_off + p), ce = __ldg(child_off + p + 1);
                for (int32_t c = cb; c < ce; ++c) acc += __ldg(src + __ldg(child_list + c));
            }
            dst[p] = acc;
        }
    }
}

static int grid_for(int64_t work, int threads, int per_sm) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

// dbuild through shared memory: a block copies R consecutive rows of MDp (one contiguous range of about 32 KB,
// whatever the width) into shared memory and forms the R output rows of D (one contiguous range) from it,
// one output element per thread and step; the depth's child lists sit in shared memory.  Both global
// transfers are fully coalesced.
constexpr int kDbThreads = 256;

__global__ void __launch_bounds__(kDbThreads) k_dbuild_smem(int32_t n, const float *__restrict__ MDp, int32_t pp,
                                                            float *__restrict__ D, int32_t pd, int32_t S,
                                                            const int32_t *__restrict__ child_off,
                                                            const int32_t *__restrict__ child_list, int32_t R) {
    extern __shared__ float sm[];
    float *rows = sm;
    int32_t *s_off = reinterpret_cast<int32_t *>(sm + (size_t)R * pp);
    int32_t *s_list = s_off + (S + 1);
    const int32_t base = child_off[0], nk = child_off[S] - base;
    for (int32_t i = threadIdx.x; i <= S; i += blockDim.x) s_off[i] = child_off[i] - base;
    for (int32_t i = threadIdx.x; i < nk; i += blockDim.x) s_list[i] = child_list[base + i];
    __syncthreads();
    for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < n; r0 += (int64_t)gridDim.x * R) {
        const int32_t nr = (int32_t)min((int64_t)R, (int64_t)n - r0);
        const int32_t cnt = nr * pp;
        const float *src = MDp + r0 * pp;
        if ((pp & 3) == 0) {
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            float4 *d4 = reinterpret_cast<float4 *>(rows);
            for (int32_t i = threadIdx.x; i < cnt / 4; i += blockDim.x) d4[i] = __ldcs(s4 + i);
        } else {
            for (int32_t i = threadIdx.x; i < cnt; i += blockDim.x) rows[i] = __ldcs(src + i);
        }
        __syncthreads();
        float *dst = D + r0 * pd;
        const int32_t ocnt = nr * pd;
        for (int32_t o = threadIdx.x; o < ocnt; o += blockDim.x) {
            const int32_t r = o / pd, p = o - r * pd;
            float acc = 0.f;
            if (p < S) {
                const float *row = rows + r * pp;
                const int32_t ce = s_off[p + 1];
                for (int32_t c = s_off[p]; c < ce; ++c) acc += row[s_list[c]];
            }
            __stcs(dst + o, acc);
        }
        __syncthreads();
    }
}

void launch_dbuild(int32_t n, const float *MDp, int32_t pp, float *D, int32_t pd, int32_t S, const int32_t *child_off,
                   const int32_t *child_list, cudaStream_t s) {
    // rows per block step: about 32 KB of MDp rows at any width; the child lists need (S + 1 + children) ints,
    // children <= pp
    const int32_t R = (int32_t)std::max<int64_t>(1, std::min<int64_t>(4096, 8192 / std::max(1, pp)));
    const int64_t smem = 4 * (int64_t)R * pp + 4 * ((int64_t)S + 1 + pp);
    if (smem <= 160 * 1024 && (int64_t)R * std::max(pp, pd) < ((int64_t)1 << 30)) {
        cudaFuncSetAttribute(k_dbuild_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        const int blocks = grid_for((int64_t)(n + R - 1) / R * kDbThreads, kDbThreads, 4);
        k_dbuild_smem<<<blocks, kDbThreads, (size_t)smem, s>>>(n, MDp, pp, D, pd, S, child_off, child_list, R);
        return;
    }
    const int blocks = grid_for((int64_t)n * 32, 256, 8);
    k_dbuild<<<blocks, 256, 0, s>>>(n, MDp, pp, D, pd, S, child_off, child_list);
}

// zero the listed columns of every row: one warp per row
__global__ void __launch_bounds__(256) k_zero_listed(int32_t n, float *D, int32_t pitch, const int32_t *__restrict__ cols,
                                                     int32_t count) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        float *row = D + v * pitch;
        for (int32_t c = lane; c < count; c += 32) row[__ldg(cols + c)] = 0.f;
    }
}

void launch_zero_listed(int32_t n, float *D, int32_t pitch, const int32_t *cols, int32_t count, cudaStream_t s) {
    if (count <= 0) return;
    const int blocks = grid_for((int64_t)n * 32, 256, 8);
    k_zero_listed<<<blocks, 256, 0, s>>>(n, D, pitch, cols, count);
}

// zero columns [c0, c0 + width) of every row: one warp per row
__global__ void __launch_bounds__(256) k_zero_cols(int32_t n, float *MD, int32_t pitch, int32_t c0, int32_t width) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        float *row = MD + v * pitch + c0;
        for (int32_t c = lane; c < width; c += 32) row[c] = 0.f;
    }
}

void launch_zero_cols(int32_t n, float *MD, int32_t pitch, int32_t c0, int32_t width, cudaStream_t s) {
    if (width <= 0) return;
    const int blocks = grid_for((int64_t)n * 32, 256, 8);
    k_zero_cols<<<blocks, 256, 0, s>>>(n, MD, pitch, c0, width);
}

// ------------------------------------------------------------------------------------------------
// scatter: for every tree node g at depth t+2 whose grandparent has a dense column (< dw),
// D[a_g][slot(grandparent(g))] += gamma_g.
// ------------------------------------------------------------------------------------------------
__global__ void k_scatter_gamma(const int32_t *__restrict__ nodes, int32_t cnt, TrieTable t, float *D, int32_t pd,
                                int32_t dw) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int32_t e = nodes[i];
    const int32_t sl = t.slot[t.parent[t.parent[e]]];
    if (sl < 0 || sl >= dw) return;
    atomicAdd(D + (int64_t)t.node[e] * pd + sl, t.gamma[e]);
}

void launch_scatter_gamma(const int32_t *nodes, int32_t cnt, TrieTable t, float *D, int32_t pd, int32_t dw,
                          cudaStream_t s) {
    if (cnt <= 0) return;
    k_scatter_gamma<<<(cnt + 255) / 256, 256, 0, s>>>(nodes, cnt, t, D, pd, dw);
}

// ------------------------------------------------------------------------------------------------
// push: one warp per tree node g at depth t+2 whose grandparent p has a push column (>= dw):
// MD[x][slot(p)] += sqrt(c)/|I(x)| * gamma_g for every x in O(a_g).
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_push_h2(const int64_t *__restrict__ out_off, const int32_t *__restrict__ out_col,
                                                 const float *__restrict__ w, const int32_t *__restrict__ nodes,
                                                 int32_t cnt, TrieTable t, float *MD, int32_t pitch, int32_t h0) {
    const int lane = threadIdx.x & 31;
    const int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= cnt) return;
    const int32_t e = nodes[i];
    const int32_t p = t.parent[t.parent[e]];  // the height-2 node
    const int32_t sl = t.slot[p];
    if (sl < h0) return;
    const int32_t a = t.node[e];
    const float g = t.gamma[e];
    const int64_t beg = out_off[a], end = out_off[a + 1];
    for (int64_t k = beg + lane; k < end; k += 32) {
        const int32_t x = __ldg(out_col + k);
        atomicAdd(MD + (int64_t)x * pitch + sl, __ldg(w + x) * g);
    }
}

void launch_push_h2(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, float *MD, int32_t pitch,
                    int32_t h0, cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t threads = (int64_t)cnt * 32;
    k_push_h2<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(g.out_off, g.out_col, g.w, nodes, cnt, t, MD, pitch, h0);
}

// ------------------------------------------------------------------------------------------------
// accumulate: D of the dense nodes of a depth, in place in the previous level's MD buffer.  A dense node's
// column already holds its heir's MD (the heir inherits the column); each group g adds (or, for a node
// without heir, sets) the sum of its other children's columns: B[v][dst_g] (+)= sum of B[v][src], src in
// srcs[off_g .. off_g+1).  One warp per row: every group's sum is formed before any column is written, so a
// column that is both a source and a later destination is read first.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_accumulate(int32_t n, float *B, int32_t pitch, const int32_t *__restrict__ gdst,
                                                    const int32_t *__restrict__ goff, const int32_t *__restrict__ srcs,
                                                    int32_t ngroups) {
    extern __shared__ float acc_sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *mine = acc_sm + (size_t)wib * ngroups;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        float *row = B + v * pitch;
        for (int32_t gi = lane; gi < ngroups; gi += 32) {
            float sum = 0.f;
            const int32_t e = __ldg(goff + gi + 1);
            for (int32_t k = __ldg(goff + gi); k < e; ++k) sum += row[__ldg(srcs + k)];
            mine[gi] = sum;
        }
        __syncwarp();
        for (int32_t gi = lane; gi < ngroups; gi += 32) {
            const int32_t d = __ldg(gdst + gi);
            const int32_t c = d & 0x3fffffff;
            row[c] = (d & (1 << 30)) ? mine[gi] : row[c] + mine[gi];  // bit 30: set (no heir)
        }
        __syncwarp();
    }
}

void launch_accumulate(int32_t n, float *B, int32_t pitch, const int32_t *gdst, const int32_t *goff, const int32_t *srcs,
                       int32_t ngroups, cudaStream_t s) {
    if (ngroups <= 0) return;
    int warps = 8;
    while (warps > 1 && (size_t)warps * ngroups * 4 > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * ngroups * 4;
    cudaFuncSetAttribute(k_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    const int threads = warps * 32;
    const int blocks = grid_for((int64_t)n * 32, threads, 2048 / threads);
    k_accumulate<<<blocks, threads, smem, s>>>(n, B, pitch, gdst, goff, srcs, ngroups);
}

// ------------------------------------------------------------------------------------------------
// Rows of vertices whose in-list is cut into several pieces receive atomic adds: zero them first.
// ------------------------------------------------------------------------------------------------
__global__ void k_zero_rows(const int32_t *__restrict__ rows, int32_t cnt, float *MD, int32_t pitch, int32_t width) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)cnt * width;
    if (i >= total) return;
    const int64_t r = i / width, c = i - r * width;
    MD[(int64_t)rows[r] * pitch + c] = 0.f;
}

void launch_zero_split_rows(const DeviceGraph &g, float *MD, int32_t pitch, int32_t width, cudaStream_t s) {
    const int64_t total = (int64_t)g.n_split * width;
    if (total <= 0) return;
    k_zero_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g.split_v, g.n_split, MD, pitch, width);
}

// ------------------------------------------------------------------------------------------------
// pull: MD[v][tile] = w[v] * sum_{x in I(v)} D[x][tile] over one tile of T columns (grid.y = tile).
// A group of L = T/4 lanes (1 lane for T <= 2) owns one piece of an in-list and gathers VEC = min(T,4)
// floats per lane per in-neighbour row; pieces are ordered longest first so the groups of a warp run
// similar trip counts.  Column indices are loaded eight at a time and broadcast within the group, so
// eight row gathers are in flight per lane.
// ------------------------------------------------------------------------------------------------
template <int VEC>
struct VecT;
template <>
struct VecT<1> {
    using type = float;
    __device__ static float load(const float *p) { return __ldg(p); }
};
template <>
struct VecT<2> {
    using type = float2;
    __device__ static float2 load(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
};
template <>
struct VecT<4> {
    using type = float4;
    __device__ static float4 load(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
};

__device__ __forceinline__ void vadd(float &a, float b) { a += b; }
__device__ __forceinline__ void vadd(float2 &a, float2 b) { a.x += b.x; a.y += b.y; }
__device__ __forceinline__ void vadd(float4 &a, float4 b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
__device__ __forceinline__ float vscale(float a, float s) { return a * s; }
__device__ __forceinline__ float2 vscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float4 vscale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
template <class V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float vzero<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vatomic(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void vatomic(float *p, float2 v) { atomicAdd(reinterpret_cast<float2 *>(p), v); }
__device__ __forceinline__ void vatomic(float *p, float4 v) { atomicAdd(reinterpret_cast<float4 *>(p), v); }
__device__ __forceinline__ void vstore(float *p, float v) { *p = v; }
__device__ __forceinline__ void vstore(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void vstore(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

template <int T>
__global__ void __launch_bounds__(256, (T == 32 || T <= 2) ? 4 : 3) k_pull(const int32_t *__restrict__ piece_v, const int64_t *__restrict__ piece_beg,
                                              const int32_t *__restrict__ piece_len, int64_t n_pieces,
                                              const int32_t *__restrict__ in_col, const float *__restrict__ w,
                                              const float *__restrict__ D, int32_t dpitch, float *__restrict__ MD,
                                              int32_t pitch) {
    constexpr int VEC = T >= 4 ? 4 : T;
    constexpr int L = T / VEC;         // lanes per group
    constexpr int CH = 8;              // in-neighbours per chunk
    constexpr int PER = CH / L;        // column indices loaded per lane per chunk
    using V = typename VecT<VEC>::type;
    const int lane = threadIdx.x & 31;
    const int lig = lane % L;
    const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane - lig));
    const int32_t col0 = blockIdx.y * T + lig * VEC;
    const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / L;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / L;
    // Software pipeline over this group's pieces p, p + ngroups, ...: the metadata of the piece after next and
    // the column indices of the next chunk (or of the next piece's first chunk) are loaded while the current
    // chunk's row gathers are in flight, so a short piece costs about one gather round trip.
    auto load_meta = [&](int64_t q, int32_t &v, int64_t &beg, int32_t &info) {
        if (q < n_pieces) {
            v = __ldg(piece_v + q);
            beg = __ldg(piece_beg + q);
            info = __ldg(piece_len + q);
        } else {
            v = 0, beg = 0, info = 0;
        }
    };
    auto load_idx = [&](int64_t beg, int32_t len, int32_t e0, int32_t(&mine)[PER]) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int32_t e = e0 + lig + L * r;
            mine[r] = e < len ? __ldg(in_col + beg + e) : -1;
        }
    };
    int64_t p = gid;
    int32_t v, info, v1, info1;
    int64_t beg, beg1;
    load_meta(p, v, beg, info);
    load_meta(p + ngroups, v1, beg1, info1);
    int32_t mine[PER];
    load_idx(beg, info & 0x7fffffff, 0, mine);
    for (; p < n_pieces; p += ngroups) {
        int32_t v2, info2;
        int64_t beg2;
        load_meta(p + 2 * ngroups, v2, beg2, info2);
        const float wv = __ldg(w + v);
        const int32_t len = info & 0x7fffffff;
        V acc = vzero<V>();
        for (int32_t e0 = 0;;) {
            V val[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int32_t x = L == 1 ? mine[j] : __shfl_sync(gmask, mine[j / L], j % L, L);
                val[j] = x >= 0 ? VecT<VEC>::load(D + (int64_t)x * dpitch + col0) : vzero<V>();
            }
            e0 += CH;
            const bool more = e0 < len;
            if (more) load_idx(beg, len, e0, mine);
            else load_idx(beg1, info1 & 0x7fffffff, 0, mine);
#pragma unroll
            for (int j = 0; j < CH; ++j) vadd(acc, val[j]);
            if (!more) break;
        }
        const V res = vscale(acc, wv);
        float *dst = MD + (int64_t)v * pitch + col0;
        if (info < 0) vatomic(dst, res); else vstore(dst, res);
        v = v1, beg = beg1, info = info1;
        v1 = v2, beg1 = beg2, info1 = info2;
    }
}

int32_t pull_tile_for(int32_t S, int32_t wide) {
    if (S <= 1) return 1;
    if (S <= 2) return 2;
    if (S <= 4) return 4;
    if (S <= 8) return 8;
    if (S <= 16 || wide <= 16) return 16;
    return 32;
}

void launch_pull(const DeviceGraph &g, const float *D, int32_t dpitch, float *MD, int32_t pitch, int32_t width,
                 int32_t tile, int32_t blocks_per_sm, cudaStream_t s) {
    const int32_t ntiles = width / tile;
    const int L = tile >= 4 ? tile / 4 : 1;
    const int64_t threads_needed = g.n_pieces * L;
    const int blocks = grid_for(threads_needed, 256, blocks_per_sm > 0 ? blocks_per_sm : 8);
    dim3 grid(blocks, ntiles);
    switch (tile) {
        case 1: k_pull<1><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
        case 2: k_pull<2><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
        case 4: k_pull<4><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
        case 8: k_pull<8><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
        case 16: k_pull<16><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
        default: k_pull<32><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, pitch); break;
    }
}

// ------------------------------------------------------------------------------------------------
// gamma: one warp per tree node t at the current depth.
//   beta_t  = sqrt(c)/|I(a_t)| * (sum_{x in I(a_t)} MD(t)[x] + G_t)   (the score PROBE would give a_t)
//   gamma_t = w_t / n_r - beta_t;  G_parent += gamma_t
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gamma(const int64_t *__restrict__ in_off, const int32_t *__restrict__ in_col,
                                               const float *__restrict__ w, const int32_t *__restrict__ nodes,
                                               int32_t cnt, TrieTable t, const float *__restrict__ inv_nr,
                                               const float *__restrict__ MD, int32_t pc) {
    const int lane = threadIdx.x & 31;
    const int32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= cnt) return;
    const int32_t e = nodes[i];
    const int32_t a = t.node[e];
    const int32_t sl = t.slot[e];
    float sum = 0.f;
    if (sl >= 0 && MD != nullptr) {
        const int64_t beg = in_off[a], end = in_off[a + 1];
        for (int64_t k = beg + lane; k < end; k += 32) sum += __ldg(MD + (int64_t)__ldg(in_col + k) * pc + sl);
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        const float beta = __ldg(w + a) * (sum + t.G[e]);
        const float g = (float)t.weight[e] * inv_nr[t.query[e]] - beta;
        t.gamma[e] = g;
        const int32_t p = t.parent[e];
        if (p >= 0) atomicAdd(&t.G[p], g);
    }
}

void launch_gamma(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, const float *inv_nr,
                  const float *MD, int32_t pc, cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t threads = (int64_t)cnt * 32;
    k_gamma<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(g.in_off, g.in_col, g.w, nodes, cnt, t, inv_nr, MD, pc);
}

// ------------------------------------------------------------------------------------------------
// finalize: out[q][v] = MD0[ext2int[v]][rho_slot(q)] for the caller's node id v, out[q][u_q] = 1 (s(u,u) = 1).
// ------------------------------------------------------------------------------------------------
__global__ void k_finalize(int32_t n, int32_t B, const int32_t *__restrict__ qnode, const int32_t *__restrict__ rho_slot,
                           const float *__restrict__ MD0, int32_t p0, const int32_t *__restrict__ ext2int,
                           float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t q = blockIdx.y;
    if (i >= n) return;
    const int32_t sl = rho_slot[q];
    float v = sl >= 0 ? MD0[(int64_t)ext2int[i] * p0 + sl] : 0.f;
    if ((int32_t)i == qnode[q]) v = 1.f;
    out[(int64_t)q * n + i] = v;
}

void launch_finalize(int32_t n, int32_t B, const int32_t *qnode, const int32_t *rho_slot, const float *MD0,
                     int32_t p0, const int32_t *ext2int, float *out, cudaStream_t s) {
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)B);
    k_finalize<<<grid, 256, 0, s>>>(n, B, qnode, rho_slot, MD0, p0, ext2int, out);
}

__global__ void k_map_ids(int32_t *ids, int64_t count, const int32_t *__restrict__ map) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count && ids[i] >= 0) ids[i] = map[ids[i]];
}

void launch_map_ids(int32_t *ids, int64_t count, const int32_t *map, cudaStream_t s) {
    if (count <= 0) return;
    k_map_ids<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ids, count, map);
}

}  // namespace ps
