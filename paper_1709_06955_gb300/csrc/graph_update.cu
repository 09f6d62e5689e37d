// Device-side update of the graph store: one batch of edge insertions or deletions merged into the CSR
// arrays without rebuilding them on the host.
//
// The host sorts the (deduplicated, loop-free) batch twice: by (destination, source in the caller's id order)
// for the in-lists, whose order is the caller's source-id order (walks pick the k-th entry of it), and by
// (source, destination in internal id order) for the out-lists.  The device then
//   1. marks the batch entries that change the graph (an insert of an absent edge, a delete of a present one)
//      by binary search in the current rows, and counts the change of every row's degree;
//   2. forms the new offsets (prefix sums of the new degrees);
//   3. writes every row in parallel: an old entry that survives moves to its old index plus the number of
//      inserted entries ordered before it, minus the number of deleted entries ordered before it; an inserted
//      entry goes to the number of old entries ordered before it plus its rank among the inserts;
//   4. recomputes w[v] = sqrt(c)/|I(v)| and the pull pieces (a counting sort by piece length).
#include <algorithm>

#include "internal.cuh"

namespace ps {

struct UpdateBatch {
    int64_t k = 0;
    // in-order: sorted by (dst internal, src external)
    const int32_t *in_dst = nullptr, *in_src = nullptr, *in_src_ext = nullptr;
    // out-order: sorted by (src internal, dst internal)
    const int32_t *out_src = nullptr, *out_dst = nullptr;
    long long *in_valid = nullptr, *out_valid = nullptr;  // 1 if the entry changes the graph
    const long long *in_vpre = nullptr, *out_vpre = nullptr;  // exclusive prefix sums of the flags (k + 1)
    bool insert = true;
};

// first index in [lo, hi) of row entries whose key is >= x, keys read through `key`
template <class Key>
__device__ __forceinline__ int64_t lower_bound_row(int64_t lo, int64_t hi, uint32_t x, Key key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key(mid) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// 1. validity of each batch entry (in-order and out-order copies get the same decision) and degree deltas
__global__ void k_upd_mark(DeviceGraph g, UpdateBatch b, long long *in_delta, long long *out_delta) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= b.k) return;
    {
        const int32_t v = b.in_dst[e];
        const uint32_t xe = (uint32_t)b.in_src_ext[e];
        const int64_t beg = g.in_off[v], end = g.in_off[v + 1];
        const int64_t pos = lower_bound_row(beg, end, xe, [&](int64_t i) { return (uint32_t)g.int2ext[g.in_col[i]]; });
        const bool exists = pos < end && (uint32_t)g.int2ext[g.in_col[pos]] == xe;
        const bool valid = b.insert ? !exists : exists;
        b.in_valid[e] = valid ? 1 : 0;
        if (valid) atomicAdd(reinterpret_cast<unsigned long long *>(&in_delta[v]), b.insert ? 1ull : ~0ull);  // +-1
    }
    {
        const int32_t x = b.out_src[e];
        const uint32_t v = (uint32_t)b.out_dst[e];
        const int64_t beg = g.out_off[x], end = g.out_off[x + 1];
        const int64_t pos = lower_bound_row(beg, end, v, [&](int64_t i) { return (uint32_t)g.out_col[i]; });
        const bool exists = pos < end && (uint32_t)g.out_col[pos] == v;
        const bool valid = b.insert ? !exists : exists;
        b.out_valid[e] = valid ? 1 : 0;
        if (valid) atomicAdd(reinterpret_cast<unsigned long long *>(&out_delta[x]), b.insert ? 1ull : ~0ull);
    }
}

// new degree per row
__global__ void k_upd_degrees(int32_t n, const int64_t *__restrict__ off, const long long *__restrict__ delta,
                              long long *deg) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < n) deg[v] = (off[v + 1] - off[v]) + delta[v];
}

// rows touched by the batch: [first, last) range of a row's entries in the sorted batch
__device__ __forceinline__ void batch_range(const int32_t *rows, int64_t k, int32_t v, int64_t *first, int64_t *last) {
    int64_t lo = 0, hi = k;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rows[mid] < v) lo = mid + 1; else hi = mid;
    }
    *first = lo;
    hi = k;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rows[mid] <= v) lo = mid + 1; else hi = mid;
    }
    *last = lo;
}

// 3. one warp per row.  Keys compare in the row's order: the caller's source id for in-lists, the internal
// destination id for out-lists.  Valid batch entries before a key are counted with a binary search in the
// row's batch range and the prefix sums of the validity flags.
template <bool IN>
__global__ void __launch_bounds__(256) k_upd_rows(DeviceGraph g, UpdateBatch b, const long long *__restrict__ new_off,
                                                  int32_t *__restrict__ new_col) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *rows = IN ? b.in_dst : b.out_src;
    const long long *valid = IN ? b.in_valid : b.out_valid;
    const long long *vpre = IN ? b.in_vpre : b.out_vpre;
    const int64_t *off = IN ? g.in_off : g.out_off;
    const int32_t *col = IN ? g.in_col : g.out_col;
    for (int64_t v = warp; v < g.n; v += nwarps) {
        const int64_t beg = off[v], end = off[v + 1], nb = new_off[v];
        int64_t f, l;
        batch_range(rows, b.k, (int32_t)v, &f, &l);
        if (f == l) {  // untouched row: copy
            for (int64_t i = beg + lane; i < end; i += 32) new_col[nb + (i - beg)] = col[i];
            continue;
        }
        auto bkey = [&](int64_t i) -> uint32_t { return IN ? (uint32_t)b.in_src_ext[i] : (uint32_t)b.out_dst[i]; };
        auto okey = [&](int64_t i) -> uint32_t { return IN ? (uint32_t)g.int2ext[col[i]] : (uint32_t)col[i]; };
        for (int64_t i = beg + lane; i < end; i += 32) {  // surviving old entries
            const uint32_t x = okey(i);
            const int64_t j = lower_bound_row(f, l, x, bkey);  // first batch entry with key >= x
            const long long less = vpre[j] - vpre[f];
            if (!b.insert && j < l && bkey(j) == x && valid[j]) continue;  // deleted
            new_col[nb + (i - beg) + (b.insert ? less : -less)] = col[i];
        }
        if (b.insert) {
            for (int64_t j = f + lane; j < l; j += 32) {  // inserted entries
                if (!valid[j]) continue;
                const int64_t before = lower_bound_row(beg, end, bkey(j), okey) - beg;
                new_col[nb + before + (vpre[j] - vpre[f])] = IN ? b.in_src[j] : b.out_dst[j];
            }
        }
    }
}

// 4. w and the pull pieces
__global__ void k_upd_w(int32_t n, const long long *__restrict__ new_off, float sqrt_c, float *w, long long *npieces) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const long long d = new_off[v + 1] - new_off[v];
    w[v] = d > 0 ? sqrt_c / (float)d : 0.f;
    npieces[v] = d <= kPiece ? 1 : (d + kPiece - 1) / kPiece;
}

// counts pieces per length (0..kPiece) and lists the split rows
__global__ void k_upd_piece_hist(int32_t n, const long long *__restrict__ new_off, unsigned long long *hist,
                                 int32_t *split_v, unsigned long long *n_split) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const long long d = new_off[v + 1] - new_off[v];
    if (d <= kPiece) {
        atomicAdd(&hist[d], 1ull);
    } else {
        atomicAdd(&hist[kPiece], (unsigned long long)(d / kPiece));
        if (d % kPiece) atomicAdd(&hist[d % kPiece], 1ull);
        split_v[atomicAdd(n_split, 1ull)] = (int32_t)v;
    }
}

// bucket starts, longest first: start[len] = sum of hist[l] for l > len
__global__ void k_upd_piece_starts(unsigned long long *hist, unsigned long long *cursor) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long acc = 0;
    for (int len = kPiece; len >= 0; --len) {
        cursor[len] = acc;
        acc += hist[len];
    }
}

__global__ void k_upd_piece_fill(int32_t n, const long long *__restrict__ new_off, unsigned long long *cursor,
                                 int32_t *pv, int64_t *pb, int32_t *pl) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const long long beg = new_off[v], d = new_off[v + 1] - beg;
    if (d <= kPiece) {
        const unsigned long long i = atomicAdd(&cursor[d], 1ull);
        pv[i] = (int32_t)v;
        pb[i] = beg;
        pl[i] = (int32_t)d;
        return;
    }
    const long long full = d / kPiece, rest = d % kPiece;
    for (long long c = 0; c < full; ++c) {
        const unsigned long long i = atomicAdd(&cursor[kPiece], 1ull);
        pv[i] = (int32_t)v;
        pb[i] = beg + c * kPiece;
        pl[i] = kPiece | (int32_t)0x80000000;
    }
    if (rest) {
        const unsigned long long i = atomicAdd(&cursor[rest], 1ull);
        pv[i] = (int32_t)v;
        pb[i] = beg + full * kPiece;
        pl[i] = (int32_t)rest | (int32_t)0x80000000;
    }
}

__global__ void k_i64_copy(const long long *__restrict__ a, int64_t *b, int64_t count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) b[i] = a[i];
}

static unsigned blocks_for(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

void launch_upd_mark(const DeviceGraph &g, const UpdateBatchArgs &a, long long *in_delta, long long *out_delta,
                     cudaStream_t s) {
    if (a.k <= 0) return;
    UpdateBatch b;
    b.k = a.k; b.in_dst = a.in_dst; b.in_src = a.in_src; b.in_src_ext = a.in_src_ext; b.out_src = a.out_src;
    b.out_dst = a.out_dst; b.in_valid = a.in_valid; b.out_valid = a.out_valid; b.insert = a.insert;
    b.in_vpre = a.in_vpre; b.out_vpre = a.out_vpre;
    k_upd_mark<<<blocks_for(a.k, 256), 256, 0, s>>>(g, b, in_delta, out_delta);
}

void launch_upd_degrees(int32_t n, const int64_t *off, const long long *delta, long long *deg, cudaStream_t s) {
    k_upd_degrees<<<blocks_for(n, 256), 256, 0, s>>>(n, off, delta, deg);
}

void launch_upd_rows(const DeviceGraph &g, const UpdateBatchArgs &a, bool in_lists, const long long *new_off,
                     int32_t *new_col, cudaStream_t s) {
    UpdateBatch b;
    b.k = a.k; b.in_dst = a.in_dst; b.in_src = a.in_src; b.in_src_ext = a.in_src_ext; b.out_src = a.out_src;
    b.out_dst = a.out_dst; b.in_valid = a.in_valid; b.out_valid = a.out_valid; b.insert = a.insert;
    b.in_vpre = a.in_vpre; b.out_vpre = a.out_vpre;
    const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for((int64_t)g.n * 32, 256), 152 * 16);
    if (in_lists) k_upd_rows<true><<<blocks, 256, 0, s>>>(g, b, new_off, new_col);
    else k_upd_rows<false><<<blocks, 256, 0, s>>>(g, b, new_off, new_col);
}

void launch_upd_w(int32_t n, const long long *new_off, float sqrt_c, float *w, long long *npieces, cudaStream_t s) {
    k_upd_w<<<blocks_for(n, 256), 256, 0, s>>>(n, new_off, sqrt_c, w, npieces);
}

void launch_upd_pieces(int32_t n, const long long *new_off, unsigned long long *hist, unsigned long long *cursor,
                       int32_t *split_v, unsigned long long *n_split, int32_t *pv, int64_t *pb, int32_t *pl,
                       cudaStream_t s) {
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (kPiece + 1), s);
    cudaMemsetAsync(n_split, 0, sizeof(unsigned long long), s);
    k_upd_piece_hist<<<blocks_for(n, 256), 256, 0, s>>>(n, new_off, hist, split_v, n_split);
    k_upd_piece_starts<<<1, 32, 0, s>>>(hist, cursor);
    k_upd_piece_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, new_off, cursor, pv, pb, pl);
}

void launch_i64_copy(const long long *a, int64_t *b, int64_t count, cudaStream_t s) {
    if (count > 0) k_i64_copy<<<blocks_for(count, 256), 256, 0, s>>>(a, b, count);
}

}  // namespace ps
