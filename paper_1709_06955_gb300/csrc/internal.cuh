// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/probesim.h"

namespace ps {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
// SC'11): ten rounds of two 32x32->64-bit multiplies over a 4-word counter, the key advanced by a
// Weyl sequence between rounds.  Walk k, step s of a query keyed (seed, query_id) uses counter
// (k, s, 0, 0); a randomized PROBE draw of walk k on prefix length i, level j, candidate x uses
// counter (k, 2^24 | i << 8 | j, x, 0).
// ---------------------------------------------------------------------------------------------
struct U32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U32x4{c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------------------------
// Device graph store: in-adjacency I(v) sorted by source id (walks pick the k-th entry), out-
// adjacency O(x) sorted by destination id, w[v] = sqrt(c)/|I(v)| (0 when |I(v)| = 0), and the work
// decomposition of the pull kernel: every in-list cut into pieces of at most kPiece edges, ordered
// by length (longest first).  A piece of a vertex cut into several pieces is added atomically.
// ---------------------------------------------------------------------------------------------
constexpr int kPiece = 128;

struct DeviceGraph {
    int32_t n = 0;
    int64_t m = 0;
    int64_t *in_off = nullptr;
    int32_t *in_col = nullptr;
    int64_t *out_off = nullptr;
    int32_t *out_col = nullptr;
    float *w = nullptr;
    int64_t n_pieces = 0;
    int32_t *piece_v = nullptr;
    int64_t *piece_beg = nullptr;
    int32_t *piece_len = nullptr;  // length | (split ? 1 << 31 : 0)
    int32_t n_split = 0;           // vertices cut into more than one piece
    int32_t *split_v = nullptr;
    int32_t n_active = 0;          // every node with out-edges has an internal id below n_active (all of them
                                   // come first at creation; update batches may leave gaps)
    int32_t *ext2int = nullptr;    // caller's node id -> internal id (descending out-degree order)
    int32_t *int2ext = nullptr;    // internal id -> caller's node id
};

// The queries of one launch.
struct QueryBatch {
    int32_t B = 0;
    const int32_t *node = nullptr;     // u per query (caller's id; the kernels map it)
    const uint32_t *qid = nullptr;     // Philox key word 1 per query
    const int32_t *walk_base = nullptr;  // [B+1] prefix sums of walk counts
    const int32_t *walk_k0 = nullptr;  // index of the first walk per query
    const float *inv_nr = nullptr;     // 1/n_r per query (FP32)
};

// Reverse-reachability tree of Alg. 4 for all queries of a launch, stored as an open-addressing hash
// table keyed by (parent slot, graph node); the slot index is the tree-node id.  Every query also has a
// virtual super-root at depth 0 whose only child is the root u at depth 1.
struct TrieTable {
    int64_t cap = 0;           // power of two
    unsigned long long *key = nullptr;
    int32_t *node = nullptr;   // graph node (-1 for a super-root)
    int32_t *parent = nullptr; // parent slot (-1 for a super-root)
    int32_t *depth = nullptr;  // 0 super-root, 1 root, i for the prefix (u_1..u_i)
    int32_t *query = nullptr;  // query index in the launch
    int32_t *weight = nullptr; // walks sharing the prefix
    int32_t *height = nullptr; // longest path below the node
    int32_t *slot = nullptr;   // column of the node's score vector at its depth, -1 if it has none: dense
                               // nodes and push heirs (a push node that took its parent's column) below h0,
                               // the other push nodes in the push block from h0 on
    float *gamma = nullptr;    // normalised weight minus the excluded score (see probe_level.cu)
    float *G = nullptr;        // sum of the children's gamma
    int32_t *walk_slot = nullptr;  // optional [W][l_max]: slot of the prefix of length i of walk w at [w][i-1]
};

constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t kRhoTag = 0xFFFFFFFEu;

// Device-side counters of one launch (read back with one small copy).
struct LaunchCounters {
    unsigned long long walk_nodes;
    int32_t max_len;
    int32_t overflow;  // hash table full
};

// Column layout of the score matrix of one depth ([n] rows x pitch columns, FP32).  Up to kGroup columns
// it is plain node-major, [n][pitch].  Wider matrices are cut into groups of kGroup columns, each group one
// [n][kGroup] block (1 KB rows), stored group after group with a stride of gs floats (n * kGroup plus a
// few cache lines, so equal rows of different groups do not map to the same memory partition).  A pull
// tile of 32 columns then gathers 128 B per row from inside one block of n KB whatever the total width,
// while the kernels that touch many columns of one row (accumulate, gamma) still find them in one row.
// Every layout has one spare row, row n: the pull pads the last chunk of an in-list with index n, and that
// row is zeroed before each pull reads the matrix (launch_zero_spare_row).
constexpr int32_t kGroup = 256;
constexpr int64_t kGroupSkew = kGroup + 5 * 32;  // floats: the spare row, then five 128-byte lines

struct ColLayout {
    int64_t n = 0;
    int32_t K = 0;   // number of groups; 0 for a node-major matrix
    int32_t R = 0;   // row pitch of a node-major matrix
    int64_t gs = 0;  // group stride in floats
    __host__ __device__ int64_t base(int32_t c) const {  // offset of (row 0, column c)
        return K > 0 ? (int64_t)(c / kGroup) * gs + (c % kGroup) : (int64_t)c;
    }
    __host__ __device__ int32_t rpitch(int32_t) const { return K > 0 ? kGroup : R; }  // row pitch at column c
    __host__ __device__ int64_t at(int64_t v, int32_t c) const {
        return K > 0 ? (int64_t)(c / kGroup) * gs + v * kGroup + (c % kGroup) : v * R + c;
    }
    __host__ __device__ int64_t size() const { return K > 0 ? (int64_t)K * gs : (int64_t)R * (n + 1); }
    // a pull over consecutive tiles of T columns starting at column 0: tile j starts (j / sub) * ts + (j % sub)
    // * T floats after column 0
    int64_t tile_stride() const { return K > 0 ? gs : 0; }
    int32_t tile_sub(int32_t T) const { return K > 0 ? kGroup / T : (1 << 30); }
};
// the layout of a matrix with at least `cols` columns (cols a multiple of 4)
inline ColLayout make_layout(int32_t n, int32_t cols) {
    ColLayout L;
    L.n = n;
    if (cols <= kGroup) {
        L.R = cols;
    } else {
        L.K = (cols + kGroup - 1) / kGroup;
        L.gs = (int64_t)n * kGroup + kGroupSkew;
    }
    return L;
}

// grid size for `work` threads in blocks of `threads`, capped at per_sm blocks per SM of the current device
inline int grid_for(int64_t work, int threads, int per_sm) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

// ---------------------------------------------------------------------------------------------
// Launchers (each launches one kernel on `s`).
// ---------------------------------------------------------------------------------------------
void launch_walks(const DeviceGraph &g, const QueryBatch &q, int32_t W, int32_t l_max, uint32_t t_stop,
                  uint32_t seed, int32_t *walks, int32_t *lens, bool pad, LaunchCounters *ctr, cudaStream_t s);
void launch_trie_insert(const DeviceGraph &g, const QueryBatch &q, int32_t W, int32_t l_max, const int32_t *walks,
                        const int32_t *lens, TrieTable t, LaunchCounters *ctr, cudaStream_t s);
void launch_sched_count(TrieTable t, int32_t *ncount, int32_t *scount, int32_t *hcount, cudaStream_t s);
void launch_sched_export(TrieTable t, int32_t *out, int32_t *count, cudaStream_t s);
void launch_node_lists(TrieTable t, const int32_t *node_off, int32_t *ncur, int32_t *node_list, cudaStream_t s);
void launch_set_slots(TrieTable t, const int32_t *pairs, int32_t count, cudaStream_t s);
void launch_scatter_gamma(const int32_t *nodes, int32_t cnt, TrieTable t, float *D, ColLayout L, cudaStream_t s);
// inherited = false: push nodes whose column is in the push block (slot >= h0); true: those whose column
// was inherited from the parent (slot < h0)
void launch_push_h2(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, float *MD, ColLayout L,
                    int32_t h0, bool inherited, cudaStream_t s);
// Parts of at most four sources: p1 (the first part of every group: bit 30 of the destination = set, else add)
// then p2 (later parts: add).  Sources are -1 where absent.
void launch_accumulate(int32_t n, float *B, ColLayout L, const int32_t *p1dst, const int4 *p1src, int32_t np1,
                       const int32_t *p2dst, const int4 *p2src, int32_t np2, cudaStream_t s);
// zeroes columns [c0, c0 + width) rounded up to a multiple of 4 (c0 a multiple of 4, inside the pitch)
void launch_zero_cols(int32_t n, float *MD, ColLayout L, int32_t c0, int32_t width, cudaStream_t s);
void launch_zero_split_rows(const DeviceGraph &g, float *MD, ColLayout L, int32_t width, cudaStream_t s);
// zeroes columns [0, width) of the spare row n
void launch_zero_spare_row(float *MD, ColLayout L, int32_t width, cudaStream_t s);
// pull MD[v][c] = w[v] * sum_{x in I(v)} D[x][c] over ntiles tiles of `tile` columns.  D and MD point at the
// first tile's column in row 0; their rows are dpitch / pitch floats apart; tile j of D starts (j / dsub) * dts +
// (j % dsub) * tile floats after the first, and likewise for MD with mts / msub (ColLayout::tile_stride/sub).
// Row n of D (the spare row) must be zero over the pulled columns.
// zmask (may be null): bit i of word k set = column 32k + i of the launch's columns is written as 0.
// tile = kPullPairs: 32-column tiles (ntiles of them, strides as for tile 32) taken two per pass.
constexpr int32_t kPullPairs = 64;
void launch_pull(const DeviceGraph &g, const float *D, int32_t dpitch, int64_t dts, int32_t dsub, float *MD,
                 int32_t pitch, int64_t mts, int32_t msub, int32_t ntiles, int32_t tile, int32_t blocks_per_sm,
                 const uint32_t *zmask, cudaStream_t s);
// The pull over ntiles full 32-column tiles with TMA row gathers (pull_tma.cu); D's tiles as for launch_pull, plus
// dcols = the columns of one row of D's layout (its pitch, or a group's width).  *err is set when a stage's wait
// gives up.  Not available (cudaErrorNotSupported) when the driver gives no tensor-map encoder.
constexpr int32_t kTmaMaxGroups = 8;   // groups of D one launch addresses (one tensor map each)
constexpr int32_t kPullTma = 96;       // the tuner's name for this launch shape
bool pull_tma_available();
cudaError_t launch_pull_tma(const DeviceGraph &g, const float *D, int32_t dpitch, int32_t dcols, int64_t dts,
                            int32_t dsub, float *MD, int32_t pitch, int64_t mts, int32_t msub, int32_t ntiles,
                            int32_t blocks_per_sm, const uint32_t *zmask, int32_t *err, cudaStream_t s);
void launch_gamma(const DeviceGraph &g, const int32_t *nodes, int32_t cnt, TrieTable t, const float *inv_nr,
                  const float *MD, ColLayout L, cudaStream_t s);
// out[q][v] = estimate + shift for v != u, out[q][u] = 1
void launch_finalize(int32_t n, int32_t B, const int32_t *qnode, const int32_t *rho_slot, const float *MD0,
                     ColLayout L, const int32_t *ext2int, float shift, float *out, cudaStream_t s);
// ids[i] = map[ids[i]] for ids[i] >= 0
void launch_map_ids(int32_t *ids, int64_t count, const int32_t *map, cudaStream_t s);

// top-k: scores [B][n] on the device; ids/vals [B][kmax]
struct TopkScratch {
    unsigned int *hist = nullptr;     // [B][256]
    unsigned int *state = nullptr;    // [B][4]: prefix, k_remaining, gt count cursor, tie base
    unsigned int *tiecnt = nullptr;   // [B][blocks]
    int32_t *cand_id = nullptr;       // [B][kmax]
    float *cand_val = nullptr;        // [B][kmax]
};
int topk_blocks_per_query(int32_t n);
void launch_topk(int32_t n, int32_t B, const float *scores, const int32_t *qnode, const int32_t *qk, int32_t kmax,
                 TopkScratch sc, int32_t *ids, float *vals, cudaStream_t s, int64_t *launches);
cudaError_t topk_preload();

// frontier PROBE engine (frontier.cu): each walk prefix probed on its own, with Pruning Rule 2 and the switch
constexpr int kFixShift = 44;  // scores and estimates accumulate as int64 multiples of 2^-44
constexpr int32_t kProbeSwitched = 1, kProbeDense = 2;
constexpr int64_t kFrontierMaxWalks = (int64_t)1 << 18;  // per query: keeps every fixed-point sum below 2^62
struct FrontierProbes {
    int32_t P = 0;
    int32_t *slot = nullptr;              // tree slot of the probed prefix
    int32_t *anc = nullptr;               // tree slot of the node the current level excludes
    unsigned long long *deg = nullptr;    // out-degree sum of the current level's kept entries
    int32_t *state = nullptr;             // kProbeSwitched | kProbeDense
    long long *rsize = nullptr;           // region slots in the next level's table
    long long *roff = nullptr;            // [P+1] region offsets (exclusive prefix sums of rsize over a probe range)
    long long *dsize = nullptr;           // bound on the next level's entries: min(out-degree sum, n)
    long long *doff = nullptr;            // [P+1] its exclusive prefix sums over a probe range
};
struct FrontierList {  // entries of the frontiers, grouped by probe in probe order
    int32_t *p = nullptr;
    int32_t *x = nullptr;
    float *val = nullptr;                 // score (the fixed-point sum of its level, rounded to FP32)
};
// One slot of a level's table: node + 1 (0 = empty) and the node's score sum (2^-44 units), in 16 bytes of one
// sector, so the sum's atomic lands in the sector that the key's lookup has just brought into the L2.
struct alignas(16) FrontierSlot {
    int32_t key;
    int32_t pad;
    unsigned long long val;
};
struct FrontierExpand {
    const long long *wp = nullptr;        // [nF+1] prefix sums of the entries' work (out-degrees)
    int64_t f_lo = 0, f_hi = 0;           // entries of this pass
    long long e_lo = 0, e_hi = 0;         // work items of this pass
    int32_t j = 0;                        // level
    FrontierSlot *tab = nullptr;          // next level's table (all slots empty between passes)
    long long rbase = 0;                  // table offset of this pass's first region
    unsigned long long *acc = nullptr;    // [B][n] estimates (2^-44 units, internal ids)
    int32_t n = 0;
};
void launch_fr_list(TrieTable t, int32_t *slot, int32_t *count, cudaStream_t s);
void launch_fr_init(TrieTable t, FrontierProbes P, FrontierList F, cudaStream_t s);
void launch_fr_prune(FrontierList F, int64_t nF, TrieTable t, FrontierProbes P, const int64_t *out_off, const float *pw,
                     float eps_p, int32_t j, long long *work, cudaStream_t s);
void launch_fr_regions(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1, int32_t j, int32_t n, const long long *thr,
                       uint8_t *t_sw, cudaStream_t s);
void launch_fr_count_switched(FrontierProbes P, unsigned long long *count, cudaStream_t s);
void launch_fr_work(FrontierList F, int64_t nF, FrontierProbes P, long long *work, cudaStream_t s);
void launch_fr_expand(const DeviceGraph &g, TrieTable t, FrontierProbes P, FrontierList F, const FrontierExpand &a,
                      cudaStream_t s);
int64_t fr_compact_blocks(long long T);
void launch_fr_count(const FrontierSlot *tab, long long T, long long *bcount, cudaStream_t s);
void launch_fr_write(FrontierSlot *tab, long long T, const long long *roff, int32_t p0,
                     int32_t p1, long long rbase, const long long *bpre, FrontierList out, long long out_base,
                     long long out_cap, cudaStream_t s);
void launch_fr_advance(TrieTable t, FrontierProbes P, int32_t p0, int32_t p1, cudaStream_t s);
// per cut probe c: first entry, work prefix there, region offset and entry-bound offset
void launch_fr_bounds(const int32_t *fp, int64_t nF, const long long *wp, const long long *roff, const long long *doff,
                      const int32_t *probes, int32_t count, long long *out, cudaStream_t s);
void launch_fr_finalize(int32_t n, int32_t B, const int32_t *qnode, const unsigned long long *acc, const int32_t *counts,
                        const float *inv_nr, const int32_t *ext2int, float shift, float *out, cudaStream_t s);

// randomized PROBE (rand_probe.cu)
struct RandLevel {
    const int32_t *fr_inst = nullptr, *fr_node = nullptr;  // frontier H_j (entries with out-edges)
    int64_t F = 0;
    const long long *prefix = nullptr;  // [F+1] out-degree prefix sums
    int64_t E = 0;                      // work items (frontier out-edges)
    const unsigned long long *cur_keys = nullptr;  // set of (instance, node) in H_j
    int64_t cur_cap = 0;
    unsigned long long *next_keys = nullptr;       // set of (instance, node) in H_{j+1}
    int64_t next_cap = 0;
    int32_t *next_inst = nullptr, *next_node = nullptr;  // H_{j+1} entries with out-edges
    unsigned long long *next_count = nullptr;
    int32_t *counts = nullptr;          // [B][n] members of H_{i-1} per query (internal ids)
    int32_t *overflow = nullptr;
    int32_t j = 0;
};
int64_t scan64_partials_needed(int64_t count);
void launch_scan64(const long long *in, int64_t count, long long *partial, long long *out, cudaStream_t s);
// Instances (walk w, prefix length i), i = 2..len, of the walks w0 .. w0+nw-1; with walk_slot and t_sw given, only
// those whose prefix's tree slot is flagged in t_sw (the probes the switch of Sec. 4.4 handed to Alg. 3).
void launch_inst_count(const int32_t *lens, int32_t w0, int32_t nw, long long *cnt, const int32_t *walk_slot,
                       const uint8_t *t_sw, int32_t l_max, cudaStream_t s);
void launch_inst_init(const QueryBatch &q, const DeviceGraph &g, const int32_t *lens, int32_t w0, int32_t nw,
                      int32_t l_max, const int32_t *walks, const long long *inst_off, int32_t *inst_walk,
                      int32_t *inst_len, int32_t *inst_q, uint32_t *inst_k, int32_t *fr_inst, int32_t *fr_node,
                      unsigned long long *fr_count, unsigned long long *keys, int64_t cap, int32_t *overflow,
                      const int32_t *walk_slot, const uint8_t *t_sw, cudaStream_t s);
void launch_add_i32(int32_t *a, const int32_t *b, int64_t count, cudaStream_t s);  // a += b
void launch_frontier_degree(const int32_t *fr_inst, const int32_t *fr_node, int64_t F, const int32_t *inst_len, int32_t j,
                            const int64_t *out_off, long long *deg, cudaStream_t s);
void launch_rand_level(const DeviceGraph &g, const int32_t *walks, int32_t l_max, const int32_t *inst_walk,
                       const int32_t *inst_len, const int32_t *inst_q, const uint32_t *inst_k, const uint32_t *qkey,
                       uint32_t seed, uint32_t t_keep, const RandLevel &L, cudaStream_t s);
void launch_rand_finalize(int32_t n, int32_t B, const int32_t *qnode, const int32_t *counts, const float *inv_nr,
                          const int32_t *ext2int, float shift, float *out, cudaStream_t s);

// pairwise Monte Carlo (pair_mc.cu): meets[i] += walk pairs t in [0, r) from (pu[i], pv[i]) that meet (caller's ids)
void launch_pair_mc(const DeviceGraph &g, const int32_t *pu, const int32_t *pv, const uint32_t *ku, const uint32_t *kv,
                    int32_t npairs, int64_t r, int32_t l_max, uint32_t seed, uint32_t t_stop, unsigned long long *meets,
                    cudaStream_t s);

// device-side graph updates (graph_update.cu)
struct UpdateBatchArgs {
    int64_t k = 0;
    const int32_t *in_dst = nullptr, *in_src = nullptr, *in_src_ext = nullptr;  // sorted by (dst, src ext)
    const int32_t *out_src = nullptr, *out_dst = nullptr;                         // sorted by (src, dst)
    long long *in_valid = nullptr, *out_valid = nullptr;
    const long long *in_vpre = nullptr, *out_vpre = nullptr;
    bool insert = true;
};
void launch_upd_mark(const DeviceGraph &g, const UpdateBatchArgs &a, long long *in_delta, long long *out_delta,
                     cudaStream_t s);
void launch_upd_degrees(int32_t n, const int64_t *off, const long long *delta, long long *deg, cudaStream_t s);
void launch_upd_rows(const DeviceGraph &g, const UpdateBatchArgs &a, bool in_lists, const long long *new_off,
                     int32_t *new_col, cudaStream_t s);
void launch_upd_w(int32_t n, const long long *new_off, float sqrt_c, float *w, long long *npieces, cudaStream_t s);
void launch_upd_pieces(int32_t n, const long long *new_off, unsigned long long *hist, unsigned long long *cursor,
                       int32_t *split_v, unsigned long long *n_split, int32_t *pv, int64_t *pb, int32_t *pl,
                       cudaStream_t s);
void launch_i64_copy(const long long *a, int64_t *b, int64_t count, cudaStream_t s);

// device-side initial build of the graph store (graph_build.cu)
int64_t radix_tiles(int64_t count);
// Stable LSD radix sort of count keys by their low `bits` bits (8 per pass); tmp holds count keys, counts
// 256 * radix_tiles(count) entries, offsets one more, partial scan64_partials_needed(that).  Returns the buffer
// (keys or tmp) that holds the sorted keys.
uint64_t *radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t count, int bits, long long *counts,
                         long long *offsets, long long *partial, cudaStream_t s);
void launch_build_keys(const int32_t *src, const int32_t *dst, int64_t m, int32_t n, int bs, uint64_t *keys,
                       int32_t *bad, cudaStream_t s);
void launch_build_flags(const uint64_t *keys, int64_t m, uint64_t end_key, long long *flag, cudaStream_t s);
void launch_build_compact(const uint64_t *keys, int64_t m, uint64_t end_key, const long long *pre, uint64_t *out,
                          cudaStream_t s);
void launch_build_ext_off(const uint64_t *ukeys, int64_t mu, int32_t n, int bs, long long *ext_off, cudaStream_t s);
void launch_build_outdeg(const uint64_t *ukeys, int64_t mu, uint32_t smask, unsigned long long *outdeg,
                         cudaStream_t s);
void launch_build_rank_keys(const unsigned long long *outdeg, int32_t n, int64_t mu, int bs, uint64_t *rk,
                            cudaStream_t s);
void launch_build_perm(const uint64_t *rk, int32_t n, uint32_t smask, const long long *ext_off,
                       const unsigned long long *outdeg, int32_t *int2ext, int32_t *ext2int, long long *indeg_i,
                       long long *outdeg_i, cudaStream_t s);
void launch_build_in_col(int32_t n, const int32_t *int2ext, const long long *ext_off, const int64_t *in_off,
                         const uint64_t *ukeys, uint32_t smask, const int32_t *ext2int, int bs, int32_t *in_col,
                         uint64_t *okeys, cudaStream_t s);
void launch_build_out_col(const uint64_t *okeys, int64_t mu, uint32_t smask, int32_t *out_col, cudaStream_t s);
// *res = 1 + the largest v with out-edges (0 if none); *res must be 0 before the launch
void launch_active_rows(const int64_t *out_off, int32_t n, int32_t *res, cudaStream_t s);

// sets the message probesim_last_error() returns on the calling thread
void set_last_error(const char *msg);

// pull tile width for a vector count (wide = the widest tile allowed, 16 or 32)
int32_t pull_tile_for(int32_t S, int32_t wide = 32);
inline int32_t round_up(int32_t x, int32_t a) { return (x + a - 1) / a * a; }

}  // namespace ps
