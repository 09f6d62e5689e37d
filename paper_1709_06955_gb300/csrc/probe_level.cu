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
//   accumulate D(t)[x] = sum of the children's MD columns, in place      (dense t; an heir's column is reused)
//   scatter  D(t)[a_g] += gamma_g for every grandchild g of t            (sparse terms, dense t)
//   pull     MD(t)[v] = sqrt(c)/|I(v)| * sum_{x in I(v)} D(t)[x]         (the dominant kernel, dense t)
//   push     MD(t)[x] += sqrt(c)/|I(x)| * gamma_g, x in O(a_g)           (height-2 t)
//   gamma    gamma_t  = w_t/n_r - sqrt(c)/|I(a_t)| * (sum_{x in I(a_t)} MD(t)[x] + G_t),  G_parent += gamma_t
// The result is exactly Alg. 4's (up to FP32 rounding); the work is one pull per slot instead of
// q-1 pushes per tree node.  The score vectors of one depth form an [n] x pitch FP32 matrix in the ColLayout
// of internal.cuh: node-major up to 256 columns, else groups of 256 columns, each an [n][256] block.
#include <algorithm>

#include "internal.cuh"

namespace ps {

// zero columns [c0, c0 + w4 * 4) of every row (c0 a multiple of 4), one float4 per thread; consecutive
// threads take consecutive float4s of a row
__global__ void k_zero_cols(int32_t n, float *MD, ColLayout L, int32_t c0, int32_t w4) {
    const int64_t total = (int64_t)n * w4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / w4;
        const int32_t c = c0 + 4 * (int32_t)(i - v * w4);
        *reinterpret_cast<float4 *>(MD + L.at(v, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// zero columns [c0, c1) of every row, c1 - c0 < 4 (the head of a range that does not start on a float4)
__global__ void k_zero_cols_head(int32_t n, float *MD, ColLayout L, int32_t c0, int32_t c1) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    for (int32_t c = c0; c < c1; ++c) MD[L.at(v, c)] = 0.f;
}

// zeroes columns [c0, c0 + width) rounded up to a multiple of 4 (inside the pitch)
void launch_zero_cols(int32_t n, float *MD, ColLayout L, int32_t c0, int32_t width, cudaStream_t s) {
    if (width <= 0) return;
    const int32_t end = (c0 + width + 3) / 4 * 4, a0 = (c0 + 3) / 4 * 4;
    if (a0 > c0) k_zero_cols_head<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, MD, L, c0, std::min(a0, end));
    if (end > a0) {
        const int32_t w4 = (end - a0) / 4;
        const int blocks = grid_for((int64_t)n * w4, 256, 8);
        k_zero_cols<<<blocks, 256, 0, s>>>(n, MD, L, a0, w4);
    }
}

// a tree node with a push column: subtree height 2, below the super-root
__device__ __forceinline__ bool is_push_node(const TrieTable &t, int32_t e) { return t.height[e] == 2 && t.depth[e] != 0; }

// ------------------------------------------------------------------------------------------------
// scatter: for every tree node g at depth t+2 whose grandparent is dense,
// D[a_g][slot(grandparent(g))] += gamma_g.
// ------------------------------------------------------------------------------------------------
__global__ void k_scatter_gamma(const int32_t *__restrict__ nodes, int32_t cnt, TrieTable t, float *D, ColLayout L) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int32_t e = nodes[i];
    const int32_t gp = t.parent[t.parent[e]];
    const int32_t sl = t.slot[gp];
    if (sl < 0 || is_push_node(t, gp)) return;
    atomicAdd(D + L.at(t.node[e], sl), t.gamma[e]);
}

void launch_scatter_gamma(const int32_t *nodes, int32_t cnt, TrieTable t, float *D, ColLayout L, cudaStream_t s) {
    if (cnt <= 0) return;
    k_scatter_gamma<<<(cnt + 255) / 256, 256, 0, s>>>(nodes, cnt, t, D, L);
}

// ------------------------------------------------------------------------------------------------
// push: for every tree node g at depth t+2 whose grandparent p is a push node:
// MD[x][slot(p)] += sqrt(c)/|I(x)| * gamma_g for every x in O(a_g).  A push node's column is either in the
// push block of its depth (slot >= h0) or the column it inherited from its parent (slot < h0); one launch
// serves one of the two kinds.  One block per node g: an out-list can hold tens of thousands of edges
// (hubs), so the block's threads split it and a hub does not hold up the launch.
// ------------------------------------------------------------------------------------------------
constexpr int kListThreads = 128;

__global__ void __launch_bounds__(kListThreads) k_push_h2(const int64_t *__restrict__ out_off,
                                                          const int32_t *__restrict__ out_col,
                                                          const float *__restrict__ w, const int32_t *__restrict__ nodes,
                                                          TrieTable t, float *MD, ColLayout L, int32_t h0,
                                                          int32_t inherited) {
    const int32_t e = nodes[blockIdx.x];
    const int32_t p = t.parent[t.parent[e]];  // the height-2 node
    const int32_t sl = t.slot[p];
    if (sl < 0 || !is_push_node(t, p) || (sl < h0) != (inherited != 0)) return;
    const int32_t a = t.node[e];
    const float g = t.gamma[e];
    const int64_t beg = out_off[a], end = out_off[a + 1];
    float *col = MD + L.base(sl);
    const int32_t rp = L.rpitch(sl);
    for (int64_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
        const int32_t x = __ldg(out_col + k);
        atomicAdd(col + (int64_t)x * rp, __ldg(w + x) * g);
    }
}

void launch_push_h2(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, float *MD, ColLayout L,
                    int32_t h0, bool inherited, cudaStream_t s) {
    if (cnt <= 0) return;
    k_push_h2<<<(unsigned)cnt, kListThreads, 0, s>>>(g.out_off, g.out_col, g.w, nodes, t, MD, L, h0, inherited ? 1 : 0);
}

// ------------------------------------------------------------------------------------------------
// accumulate: D of the dense nodes of a depth, in place in the previous level's MD buffer.  A dense node's
// column already holds its heir's MD (the heir inherits the column); each group g adds (or, for a node
// without heir, sets) the sum of its other children's columns: B[v][dst_g] (+)= sum of B[v][src], src in
// srcs[off_g .. off_g+1).  No destination is a source of any group (the column assignment guarantees it), so
// the groups are independent.  Groups are cut into parts of at most four sources.  One warp per row, lanes
// over the parts; the later parts of groups with more than four sources add atomically after the row's first
// parts are done.  Heirs and push heirs leave few parts per depth, so the kernel touches a few sectors of
// each row in place (measured faster than streaming whole rows through shared memory at every batch width).
// Only rows below n_active are accumulated: a row of a node without out-edges is never read once accumulated (the
// pull and the gamma gather in-neighbours' rows), and the renumbering puts those nodes last.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float acc_part_sum(const float *B, const ColLayout &L, int64_t v, int4 sc) {
    float sum = 0.f;
    if (sc.x >= 0) sum += B[L.at(v, sc.x)];
    if (sc.y >= 0) sum += B[L.at(v, sc.y)];
    if (sc.z >= 0) sum += B[L.at(v, sc.z)];
    if (sc.w >= 0) sum += B[L.at(v, sc.w)];
    return sum;
}

__global__ void __launch_bounds__(256) k_accumulate(int32_t n, float *B, ColLayout L, const int32_t *__restrict__ p1dst,
                                                    const int4 *__restrict__ p1src, int32_t np1,
                                                    const int32_t *__restrict__ p2dst, const int4 *__restrict__ p2src,
                                                    int32_t np2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        for (int32_t pi = lane; pi < np1; pi += 32) {
            const float sum = acc_part_sum(B, L, v, __ldg(p1src + pi));
            const int32_t d = __ldg(p1dst + pi);
            float *dst = B + L.at(v, d & 0x3fffffff);
            *dst = (d & (1 << 30)) ? sum : *dst + sum;  // bit 30: no heir, the column is set
        }
        if (np2 > 0) {
            __syncwarp();
            for (int32_t pi = lane; pi < np2; pi += 32)
                atomicAdd(B + L.at(v, __ldg(p2dst + pi)), acc_part_sum(B, L, v, __ldg(p2src + pi)));
            __syncwarp();
        }
    }
}

void launch_accumulate(int32_t n, float *B, ColLayout L, const int32_t *p1dst, const int4 *p1src, int32_t np1,
                       const int32_t *p2dst, const int4 *p2src, int32_t np2, cudaStream_t s) {
    if (np1 <= 0) return;
    k_accumulate<<<grid_for((int64_t)n * 32, 256, 8), 256, 0, s>>>(n, B, L, p1dst, p1src, np1, p2dst, p2src, np2);
}

// ------------------------------------------------------------------------------------------------
// Rows of vertices whose in-list is cut into several pieces receive atomic adds: zero them first.
// ------------------------------------------------------------------------------------------------
__global__ void k_zero_rows(const int32_t *__restrict__ rows, int32_t cnt, float *MD, ColLayout L, int32_t width) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)cnt * width;
    if (i >= total) return;
    const int64_t r = i / width;
    const int32_t c = (int32_t)(i - r * width);
    MD[L.at(rows[r], c)] = 0.f;
}

__global__ void k_zero_spare_row(float *MD, ColLayout L, int32_t width) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < width) MD[L.at(L.n, c)] = 0.f;
}

void launch_zero_spare_row(float *MD, ColLayout L, int32_t width, cudaStream_t s) {
    if (width <= 0) return;
    k_zero_spare_row<<<(width + 255) / 256, 256, 0, s>>>(MD, L, width);
}

void launch_zero_split_rows(const DeviceGraph &g, float *MD, ColLayout L, int32_t width, cudaStream_t s) {
    const int64_t total = (int64_t)g.n_split * width;
    if (total <= 0) return;
    k_zero_rows<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g.split_v, g.n_split, MD, L, width);
}

// ------------------------------------------------------------------------------------------------
// gamma, for every tree node t at the current depth:
//   beta_t  = sqrt(c)/|I(a_t)| * (sum_{x in I(a_t)} MD(t)[x] + G_t)   (the score PROBE would give a_t)
//   gamma_t = w_t / n_r - beta_t;  G_parent += gamma_t
// ------------------------------------------------------------------------------------------------
// One block per tree node (the in-list of a hub is long); four independent gathers per thread in flight.
__global__ void __launch_bounds__(kListThreads) k_gamma(const int64_t *__restrict__ in_off,
                                                        const int32_t *__restrict__ in_col,
                                                        const float *__restrict__ w, const int32_t *__restrict__ nodes,
                                                        TrieTable t, const float *__restrict__ inv_nr,
                                                        const float *__restrict__ MD, ColLayout Lc) {
    __shared__ float part[kListThreads / 32];
    const int32_t e = nodes[blockIdx.x];
    const int32_t a = t.node[e];
    const int32_t sl = t.slot[e];
    float sum = 0.f;
    if (sl >= 0 && MD != nullptr) {
        const int64_t beg = in_off[a], end = in_off[a + 1];
        const float *col = MD + Lc.base(sl);
        const int32_t rp = Lc.rpitch(sl);
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int64_t k = beg + threadIdx.x;
        for (; k + 3 * kListThreads < end; k += 4 * kListThreads) {
            const int32_t x0 = __ldg(in_col + k), x1 = __ldg(in_col + k + kListThreads);
            const int32_t x2 = __ldg(in_col + k + 2 * kListThreads), x3 = __ldg(in_col + k + 3 * kListThreads);
            sum += __ldg(col + (int64_t)x0 * rp);
            s1 += __ldg(col + (int64_t)x1 * rp);
            s2 += __ldg(col + (int64_t)x2 * rp);
            s3 += __ldg(col + (int64_t)x3 * rp);
        }
        for (; k < end; k += kListThreads) sum += __ldg(col + (int64_t)__ldg(in_col + k) * rp);
        sum += s1 + s2 + s3;
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int i = 0; i < kListThreads / 32; ++i) tot += part[i];
        const float beta = __ldg(w + a) * (tot + t.G[e]);
        const float g = (float)t.weight[e] * inv_nr[t.query[e]] - beta;
        t.gamma[e] = g;
        const int32_t p = t.parent[e];
        if (p >= 0) atomicAdd(&t.G[p], g);
    }
}

void launch_gamma(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, const float *inv_nr,
                  const float *MD, ColLayout L, cudaStream_t s) {
    if (cnt <= 0) return;
    k_gamma<<<(unsigned)cnt, kListThreads, 0, s>>>(g.in_off, g.in_col, g.w, nodes, t, inv_nr, MD, L);
}

// ------------------------------------------------------------------------------------------------
// finalize: out[q][v] = MD0[ext2int[v]][rho_slot(q)] + shift for the caller's node id v, out[q][u_q] = 1 (s(u,u) = 1).
// ------------------------------------------------------------------------------------------------
__global__ void k_finalize(int32_t n, int32_t B, const int32_t *__restrict__ qnode, const int32_t *__restrict__ rho_slot,
                           const float *__restrict__ MD0, ColLayout L, const int32_t *__restrict__ ext2int,
                           float shift, float *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t q = blockIdx.y;
    if (i >= n) return;
    const int32_t sl = rho_slot[q];
    float v = (sl >= 0 ? MD0[L.at(ext2int[i], sl)] : 0.f) + shift;
    if ((int32_t)i == qnode[q]) v = 1.f;
    out[(int64_t)q * n + i] = v;
}

void launch_finalize(int32_t n, int32_t B, const int32_t *qnode, const int32_t *rho_slot, const float *MD0,
                     ColLayout L, const int32_t *ext2int, float shift, float *out, cudaStream_t s) {
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)B);
    k_finalize<<<grid, 256, 0, s>>>(n, B, qnode, rho_slot, MD0, L, ext2int, shift, out);
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
