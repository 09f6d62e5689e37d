// Pairwise Monte Carlo SimRank (Sec. 2.2, Eq. 3): s(u, v) is the probability that a sqrt(c)-walk from u and one
// from v meet, i.e. have the same i-th node for some i.  For r walk pairs the estimate is (pairs that meet) / r;
// with r >= ln(1/delta) / (2 eps^2) it is within eps of s(u, v) with probability 1 - delta (Chernoff).  It serves
// as the single-pair "expert" that gauges pooled top-k candidates on graphs too large for the Power Method.
//
// One thread per walk pair t: the two walks advance in lockstep, their i-th nodes compared at every position
// both reach.  Walk t from u draws Philox counter (t, s, 0, 0) under key (seed, key_u) at step s -- the draws
// of query key_u's walk t in the single-source path -- and likewise from v under (seed, key_v).
#include <algorithm>

#include "internal.cuh"

namespace ps {

namespace {

constexpr int kThreads = 256;

// one step of a sqrt(c)-walk at node x (internal id): false when it stops there
__device__ __forceinline__ bool walk_step(const int64_t *__restrict__ in_off, const int32_t *__restrict__ in_col,
                                          int32_t &x, uint32_t t, uint32_t s, uint32_t seed, uint32_t key,
                                          uint32_t t_stop) {
    const U32x4 r = philox4x32_10(t, s, 0u, 0u, seed, key);
    if (r.x < t_stop) return false;
    const int64_t beg = in_off[x];
    const uint32_t d = (uint32_t)(in_off[x + 1] - beg);
    if (d == 0) return false;
    x = in_col[beg + __umulhi(r.y, d)];
    return true;
}

// grid.y = pair; meets[pair] += walk pairs t in [0, r) that meet
__global__ void __launch_bounds__(kThreads) k_pair_mc(const int64_t *__restrict__ in_off, const int32_t *__restrict__ in_col,
                                                      const int32_t *__restrict__ ext2int, const int32_t *__restrict__ pu,
                                                      const int32_t *__restrict__ pv, const uint32_t *__restrict__ ku,
                                                      const uint32_t *__restrict__ kv, int64_t r, int32_t l_max,
                                                      uint32_t seed, uint32_t t_stop,
                                                      unsigned long long *__restrict__ meets) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int32_t pair = blockIdx.y;
    const int32_t u0 = ext2int[pu[pair]], v0 = ext2int[pv[pair]];
    const uint32_t keyu = ku[pair], keyv = kv[pair];
    unsigned local = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < r; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = u0, b = v0;
        bool meet = a == b;
        // positions 1, 2, ... exist while both walks continue; a walk holds at most l_max nodes
        for (uint32_t s = 0; !meet && (int32_t)s + 1 < l_max; ++s) {
            const bool ga = walk_step(in_off, in_col, a, (uint32_t)t, s, seed, keyu, t_stop);
            const bool gb = walk_step(in_off, in_col, b, (uint32_t)t, s, seed, keyv, t_stop);
            if (!ga || !gb) break;
            meet = a == b;
        }
        local += meet;
    }
    for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&s_cnt, local);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(meets + pair, (unsigned long long)s_cnt);
}

}  // namespace

void launch_pair_mc(const DeviceGraph &g, const int32_t *pu, const int32_t *pv, const uint32_t *ku, const uint32_t *kv,
                    int32_t npairs, int64_t r, int32_t l_max, uint32_t seed, uint32_t t_stop, unsigned long long *meets,
                    cudaStream_t s) {
    if (npairs <= 0 || r <= 0) return;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t bx = (r + kThreads - 1) / kThreads;  // blocks per pair: about 8 per SM over all pairs
    bx = std::min<int64_t>(bx, std::max<int64_t>(1, (int64_t)sms * 8 / npairs));
    dim3 grid((unsigned)bx, (unsigned)npairs);
    k_pair_mc<<<grid, kThreads, 0, s>>>(g.in_off, g.in_col, g.ext2int, pu, pv, ku, kv, r, l_max, seed, t_stop, meets);
}

}  // namespace ps
