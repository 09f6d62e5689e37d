// The PROBE level pull over full 32-column tiles with the Tensor Memory Accelerator: MD[v][c] = sqrt(c)/|I(v)| *
// sum_{x in I(v)} D[x][c] (one level of Alg. 2 for every dense column of a depth), the in-neighbours' row segments
// fetched four rows per instruction by cp.async.bulk.tensor .tile::gather4 into shared memory.  One pass covers
// every full tile of one 256-column group of D (or all full tiles of a narrower matrix): a gathered row segment
// is up to 1 KB, so one copy moves up to 4 KB and each in-list is read once per group, not once per tile.
//
// Each warp runs its own ring of kStages stages of kRows rows: it walks its pieces (in-lists cut into at most 128
// edges, longest first) in order, keeps up to kStages stages of gathers in flight ahead of the stage it sums, and
// sums a stage from shared memory once its mbarrier has seen the stage's bytes.  A row of W columns is summed by
// LR = W/8 lanes (rounded up to a power of two) of 8 columns each, so the warp covers 32/LR rows at a time; at the
// end of a piece the row classes are added across lanes.  Every wait on a stage gives up after kMaxPolls polls (or
// as soon as another warp has failed), sets *err and leaves the kernel once the warp's other copies in flight have
// landed (again with a limit); the host turns the flag into an error.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace ps {

namespace {

constexpr int kWarps = 8;                      // warps per block (one block per SM)
constexpr int kStages = 3;                     // ring stages per warp
constexpr int kRows = 8;                       // rows per stage: two gather4 copies
constexpr int kMaxW = 256;                     // columns of one gathered row segment at most
constexpr int kStageBytes = kRows * kMaxW * 4;
constexpr int kSmemBytes = kWarps * kStages * kStageBytes;
constexpr uint32_t kMaxPolls = 1u << 20;       // polls of a stage before the warp gives up (each poll waits a while)

struct TmaMaps {
    CUtensorMap m[kTmaMaxGroups];
    int32_t width[kTmaMaxGroups];  // columns the pass over the group covers (its full tiles), a multiple of 32
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// waits for the phase with the given parity to complete; false after kMaxPolls polls, or sooner once another
// warp has raised *err (checked every 1024 polls, so a wait that succeeds at once never reads it)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const int32_t *err) {
    for (uint32_t i = 0; i < kMaxPolls; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *reinterpret_cast<const volatile int32_t *>(err) != 0) return false;
    }
    return false;
}

__global__ void __launch_bounds__(kWarps * 32, 1) k_pull_tma(const __grid_constant__ TmaMaps maps,
                                                             const int32_t *__restrict__ piece_v,
                                                             const int64_t *__restrict__ piece_beg,
                                                             const int32_t *__restrict__ piece_len, int64_t n_pieces,
                                                             const int32_t *__restrict__ in_col,
                                                             const float *__restrict__ w, float *__restrict__ MD,
                                                             int32_t pitch, int64_t mts, int32_t msub, int32_t col0,
                                                             int32_t zrow, const uint32_t *__restrict__ zmask,
                                                             int32_t *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kWarps][kStages];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const CUtensorMap *map = &maps.m[blockIdx.y];
    const int32_t W = maps.width[blockIdx.y];             // columns of this pass, a multiple of 32
    const int32_t gcol = col0 + (int32_t)blockIdx.y * kMaxW;  // this pass's first column among the launch's
    const int32_t LR = W <= 32 ? 4 : W <= 64 ? 8 : W <= 128 ? 16 : 32;  // lanes per row, 8 columns each
    const int32_t RC = 32 / LR;                            // rows a warp covers at a time
    const int32_t lc = (lane % LR) * 8;                    // this lane's first column in the row segment
    const int32_t lr = lane / LR;                          // this lane's row class
    const bool active = lc < W;
    const int32_t c = gcol + lc;                           // its first column among the launch's columns
    const int32_t t = c >> 5;                              // the full tile holding it
    const int64_t mcol = (int64_t)(t / msub) * mts + (t % msub) * 32 + (c & 31);
    uint32_t zbits = 0;
    if (zmask != nullptr && active) zbits = (__ldg(zmask + (c >> 5)) >> (c & 31)) & 0xffu;
    const int32_t row_bytes = W * 4;
    unsigned char *ring = smem + (size_t)warp * kStages * kStageBytes;
    const uint32_t ring_s = smem_addr(ring);
    uint32_t bar_s[kStages];
#pragma unroll
    for (int st = 0; st < kStages; ++st) bar_s[st] = smem_addr(&bars[warp][st]);
    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < kStages; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s[st]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    // producer: the next stage to issue (piece ip, stage is); consumer: the stage to sum (piece cp, stage cs)
    int64_t ip = blockIdx.x * (int64_t)kWarps + warp, cp = ip;
    int32_t is = 0, cs = 0;
    uint32_t issued = 0, consumed = 0;
    auto len_of = [&](int64_t q) -> int32_t { return q < n_pieces ? (__ldg(piece_len + q) & 0x7fffffff) : 0; };
    int32_t ilen = len_of(ip);
    while (ip < n_pieces && ilen == 0) ip += nwarps, ilen = len_of(ip);
    int64_t ibeg = ip < n_pieces ? __ldg(piece_beg + ip) : 0;
    // issues one stage of piece ip into the ring slot `issued % kStages`: lanes 0 and 4 each copy four rows
    auto issue = [&]() {
        const int32_t r0 = is * kRows;
        const int32_t nrow = min(kRows, ilen - r0);
        const int32_t ng4 = (nrow + 3) >> 2;
        const int32_t idx = lane < nrow ? __ldg(in_col + ibeg + r0 + lane) : zrow;
        const int q = lane >> 2;
        const int32_t c0 = __shfl_sync(0xffffffffu, idx, (4 * q) & 31), c1 = __shfl_sync(0xffffffffu, idx, (4 * q + 1) & 31),
                      c2 = __shfl_sync(0xffffffffu, idx, (4 * q + 2) & 31), c3 = __shfl_sync(0xffffffffu, idx, (4 * q + 3) & 31);
        const int slot = issued % kStages;
        if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s[slot]),
                         "r"(ng4 * 4 * row_bytes)
                         : "memory");
        __syncwarp();
        if ((lane & 3) == 0 && q < ng4) {
            const uint32_t dst = ring_s + slot * kStageBytes + q * 4 * row_bytes;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the slot's earlier reads come first
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
                "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
                "l"(map), "r"(0), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar_s[slot])
                : "memory");
        }
        ++issued;
        if ((++is) * kRows >= ilen) {
            is = 0;
            do {
                ip += nwarps;
                ilen = len_of(ip);
            } while (ip < n_pieces && ilen == 0);
            ibeg = ip < n_pieces ? __ldg(piece_beg + ip) : 0;
        }
    };
    while (issued - consumed < (uint32_t)kStages && ip < n_pieces) issue();
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.f;
    bool failed = false;
    for (; cp < n_pieces;) {
        const int32_t info = __ldg(piece_len + cp);
        const int32_t clen = info & 0x7fffffff;
        const int32_t v = __ldg(piece_v + cp);
        if (clen == 0) {  // an empty in-list: the row is zero
            if (lr == 0 && active) {
                float4 *dst = reinterpret_cast<float4 *>(MD + (int64_t)v * pitch + mcol);
                dst[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                dst[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cp += nwarps;
            continue;
        }
        const int slot = consumed % kStages;
        // every lane waits (each reads the stage); the warp gives up together if any lane ran out of polls
        if (!__all_sync(0xffffffffu, mbar_wait(bar_s[slot], (consumed / kStages) & 1u, err))) {
            failed = true;
            break;
        }
        const int32_t nrow = min(kRows, clen - cs * kRows);
        const unsigned char *stg = ring + slot * kStageBytes + lc * 4;
        for (int32_t r = lr; r < nrow; r += RC) {
            if (!active) break;
            const float4 x0 = *reinterpret_cast<const float4 *>(stg + r * row_bytes);
            const float4 x1 = *reinterpret_cast<const float4 *>(stg + r * row_bytes + 16);
            a[0] += x0.x, a[1] += x0.y, a[2] += x0.z, a[3] += x0.w;
            a[4] += x1.x, a[5] += x1.y, a[6] += x1.z, a[7] += x1.w;
        }
        __syncwarp();
        ++consumed;
        if ((++cs) * kRows >= clen) {  // the piece is summed: add the row classes, scale, write
            for (int o = LR; o < 32; o <<= 1)
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
            if (lr == 0 && active) {
                const float wv = __ldg(w + v);
                float r[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) r[k] = ((zbits >> k) & 1u) ? 0.f : a[k] * wv;
                float4 *dst = reinterpret_cast<float4 *>(MD + (int64_t)v * pitch + mcol);
                const float4 r0 = make_float4(r[0], r[1], r[2], r[3]), r1 = make_float4(r[4], r[5], r[6], r[7]);
                if (info < 0) {
                    atomicAdd(dst, r0);
                    atomicAdd(dst + 1, r1);
                } else {
                    __stcs(dst, r0);
                    __stcs(dst + 1, r1);
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = 0.f;
            cs = 0;
            cp += nwarps;
        }
        while (issued - consumed < (uint32_t)kStages && ip < n_pieces) issue();
    }
    if (failed) {
        if (lane == 0) atomicExch(err, 1);
        for (uint32_t c2 = consumed + 1; c2 < issued; ++c2)  // the warp's later copies in flight land first
            for (uint32_t i = 0; i < kMaxPolls && !mbar_try(bar_s[c2 % kStages], (c2 / kStages) & 1u); ++i) {
            }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool pull_tma_available() { return encode_fn() != nullptr; }

cudaError_t launch_pull_tma(const DeviceGraph &g, const float *D, int32_t dpitch, int32_t dcols, int64_t dts,
                            int32_t dsub, float *MD, int32_t pitch, int64_t mts, int32_t msub, int32_t ntiles,
                            int32_t blocks_per_sm, const uint32_t *zmask, int32_t *err, cudaStream_t s) {
    (void)blocks_per_sm;  // one block of kSmemBytes per SM
    if (ntiles <= 0) return cudaSuccess;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    static std::once_flag attr;
    std::call_once(attr, [] { cudaFuncSetAttribute(k_pull_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes); });
    const int blocks = grid_for(g.n_pieces * 32, kWarps * 32, 1);
    // passes of at most 256 columns: one per group of a grouped D, or the node-major row's full tiles
    const bool grouped = dsub < (1 << 29);
    const int32_t tiles_per_pass = kMaxW / 32;
    const int32_t npass = (ntiles + tiles_per_pass - 1) / tiles_per_pass;
    if (!grouped && npass > 1) return cudaErrorInvalidValue;  // a node-major D holds at most 256 columns
    for (int32_t p0 = 0; p0 < npass; p0 += kTmaMaxGroups) {
        const int32_t np = std::min(kTmaMaxGroups, npass - p0);
        TmaMaps maps;
        for (int32_t k = 0; k < np; ++k) {
            const int32_t pi = p0 + k;
            const int32_t W = 32 * std::min(tiles_per_pass, ntiles - pi * tiles_per_pass);
            maps.width[k] = W;
            const cuuint64_t dims[2] = {(cuuint64_t)dcols, (cuuint64_t)g.n + 1};
            const cuuint64_t strides[1] = {(cuuint64_t)dpitch * sizeof(float)};
            const cuuint32_t box[2] = {(cuuint32_t)W, 1};
            const cuuint32_t estr[2] = {1, 1};
            void *base = const_cast<float *>(D + (grouped ? (int64_t)pi * dts : 0));
            if (enc(&maps.m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
        }
        dim3 grid(blocks, np);
        k_pull_tma<<<grid, kWarps * 32, kSmemBytes, s>>>(maps, g.piece_v, g.piece_beg, g.piece_len, g.n_pieces,
                                                         g.in_col, g.w, MD, pitch, mts, msub, p0 * kMaxW, g.n, zmask,
                                                         err);
    }
    return cudaGetLastError();
}

}  // namespace ps
