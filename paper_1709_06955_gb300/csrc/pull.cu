// The PROBE level pull, the dominant kernel of the deterministic path (one level of Alg. 2 for every dense
// column of a depth at once): MD[v][c] = sqrt(c)/|I(v)| * sum_{x in I(v)} D[x][c], an SpMM of the in-CSR with
// the depth's dense columns, gathered 32 columns (one tile) at a time.  Kept in a file of its own so that the
// committed ncu counters of this kernel are tied to exactly this source (bench.py checks its hash).
#include "internal.cuh"

namespace ps {

// ------------------------------------------------------------------------------------------------
// pull: MD[v][tile] = w[v] * sum_{x in I(v)} D[x][tile] over one tile of T columns (grid.y = tile), or over two
// 32-column tiles per pass.
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

// packed FP32x2 adds (one instruction for two lanes of a vector; each element rounds as a scalar add would)
__device__ __forceinline__ void vadd(float &a, float b) { a += b; }
__device__ __forceinline__ void vadd(float2 &a, float2 b) { a = __fadd2_rn(a, b); }
__device__ __forceinline__ void vadd(float4 &a, float4 b) {
    const float2 lo = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 hi = __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w));
    a = make_float4(lo.x, lo.y, hi.x, hi.y);
}
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
// MD is next read a depth later by the accumulate's streaming pass: store it evict-first, so the L2 keeps the
// gathered D tile and the in-lists
__device__ __forceinline__ void vstore(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void vstore(float *p, float2 v) { __stcs(reinterpret_cast<float2 *>(p), v); }
__device__ __forceinline__ void vstore(float *p, float4 v) { __stcs(reinterpret_cast<float4 *>(p), v); }

// element k of a vector becomes 0 where bit k of b is set
__device__ __forceinline__ float vmask(float a, uint32_t b) { return (b & 1u) ? 0.f : a; }
__device__ __forceinline__ float2 vmask(float2 a, uint32_t b) {
    return make_float2((b & 1u) ? 0.f : a.x, (b & 2u) ? 0.f : a.y);
}
__device__ __forceinline__ float4 vmask(float4 a, uint32_t b) {
    return make_float4((b & 1u) ? 0.f : a.x, (b & 2u) ? 0.f : a.y, (b & 4u) ? 0.f : a.z, (b & 8u) ? 0.f : a.w);
}

// NCH row gathers of one chunk for each of the NT tiles of the pass: in-neighbour j's index sits in lane j % L of
// the group, slot j / L; past the end of the piece the index is n, the zero spare row
template <int NCH, int L, int PER, int NT, class V, int VEC>
__device__ __forceinline__ void pull_gather(const int32_t (&mine)[PER], unsigned gmask, const float *__restrict__ D,
                                            int32_t dpitch, const int64_t (&dcol0)[NT], bool has1,
                                            V (&val)[NT][NCH]) {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
        const int32_t x = L == 1 ? mine[j] : __shfl_sync(gmask, mine[j / L], j % L, L);
        const float *row = D + (int64_t)x * dpitch;
        val[0][j] = VecT<VEC>::load(row + dcol0[0]);
        if (NT > 1) val[NT - 1][j] = has1 ? VecT<VEC>::load(row + dcol0[NT - 1]) : vzero<V>();
    }
}

// T = tile width; NT = tiles per pass (2: the 32-column tiles 2y and 2y + 1 in one pass, so every in-list and piece
// record is read once for both, with half the in-neighbours per chunk to keep the same gathers in flight)
template <int T, int NT>
__global__ void __launch_bounds__(256, (NT == 1 && (T == 32 || T <= 2)) ? 4 : 3) k_pull(const int32_t *__restrict__ piece_v, const int64_t *__restrict__ piece_beg,
                                              const int32_t *__restrict__ piece_len, int64_t n_pieces,
                                              const int32_t *__restrict__ in_col, const float *__restrict__ w,
                                              const float *__restrict__ D, int32_t dpitch, float *__restrict__ MD,
                                              int32_t pitch, int64_t dts, int32_t dsub, int64_t mts, int32_t msub,
                                              int32_t zrow, const uint32_t *__restrict__ zmask, int32_t ntiles) {
    static_assert(NT == 1 || NT == 2, "one or two tiles per pass");
    constexpr int VEC = T >= 4 ? 4 : T;
    constexpr int L = T / VEC;                  // lanes per group
    constexpr int CH = 8 / NT;                  // in-neighbours per chunk
    constexpr int PER = CH >= L ? CH / L : 1;   // column indices loaded per lane per chunk
    using V = typename VecT<VEC>::type;
    const int lane = threadIdx.x & 31;
    const int lig = lane % L;
    const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane - lig));
    int64_t dcol0[NT], mcol0[NT];
    uint32_t zbits[NT];  // this lane's columns that are written as 0 (columns a push node inherited: the push
                         // fills them later)
    const bool has1 = NT > 1 && (int32_t)blockIdx.y * NT + 1 < ntiles;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int32_t tile = (int32_t)blockIdx.y * NT + t;
        dcol0[t] = (int64_t)(tile / dsub) * dts + (tile % dsub) * T + lig * VEC;
        mcol0[t] = (int64_t)(tile / msub) * mts + (tile % msub) * T + lig * VEC;
        zbits[t] = 0;
        if (zmask != nullptr && (t == 0 || has1)) {
            const int32_t c = tile * T + lig * VEC;
            zbits[t] = (__ldg(zmask + (c >> 5)) >> (c & 31)) & ((1u << VEC) - 1u);
        }
    }
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
            mine[r] = ((CH >= L || lig < CH) && e < len) ? __ldg(in_col + beg + e) : zrow;
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
        V acc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[t] = vzero<V>();
        if (len == 0) {  // an empty in-list (about half the rows of a power-law graph): the row is zero
            load_idx(beg1, info1 & 0x7fffffff, 0, mine);
        } else {
            for (int32_t e0 = 0;;) {
                V val[NT][CH];
                pull_gather<CH, L, PER, NT, V, VEC>(mine, gmask, D, dpitch, dcol0, has1, val);
                e0 += CH;
                const bool more = e0 < len;
                if (more) load_idx(beg, len, e0, mine);
                else load_idx(beg1, info1 & 0x7fffffff, 0, mine);
#pragma unroll
                for (int j = 0; j < CH; ++j)
#pragma unroll
                    for (int t = 0; t < NT; ++t) vadd(acc[t], val[t][j]);
                if (!more) break;
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t > 0 && !has1) break;
            const V res = vmask(vscale(acc[t], wv), zbits[t]);
            float *dst = MD + (int64_t)v * pitch + mcol0[t];
            if (info < 0) vatomic(dst, res); else vstore(dst, res);
        }
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

void launch_pull(const DeviceGraph &g, const float *D, int32_t dpitch, int64_t dts, int32_t dsub, float *MD,
                 int32_t pitch, int64_t mts, int32_t msub, int32_t ntiles, int32_t tile, int32_t blocks_per_sm,
                 const uint32_t *zmask, cudaStream_t s) {
    if (ntiles <= 0) return;
    const int T = tile == kPullPairs ? 32 : tile;
    const int NT = tile == kPullPairs ? 2 : 1;
    const int L = T >= 4 ? T / 4 : 1;
    const int64_t threads_needed = g.n_pieces * L;
    const int blocks = grid_for(threads_needed, 256, blocks_per_sm > 0 ? blocks_per_sm : 8);
    dim3 grid(blocks, (ntiles + NT - 1) / NT);
#define PS_PULL(T, NT)                                                                                              \
    k_pull<T, NT><<<grid, 256, 0, s>>>(g.piece_v, g.piece_beg, g.piece_len, g.n_pieces, g.in_col, g.w, D, dpitch, MD, \
                                       pitch, dts, dsub, mts, msub, g.n, zmask, ntiles)
    switch (tile) {
        case 1: PS_PULL(1, 1); break;
        case 2: PS_PULL(2, 1); break;
        case 4: PS_PULL(4, 1); break;
        case 8: PS_PULL(8, 1); break;
        case 16: PS_PULL(16, 1); break;
        case kPullPairs: PS_PULL(32, 2); break;
        default: PS_PULL(32, 1); break;
    }
#undef PS_PULL
}

}  // namespace ps
