/*
 * probesim.h -- C ABI of the GB300-native ProbeSim library (libprobesim.so).
 *
 * ProbeSim (Liu et al., "ProbeSim: Scalable Single-Source and Top-k SimRank Computations on Dynamic
 * Graphs", PVLDB 11(1), 2017) answers approximate single-source SimRank queries (Def. 1) and top-k
 * SimRank queries (Def. 2) on a directed simple graph without any index: n_r sqrt(c)-walks from the
 * query node (Alg. 1), a PROBE from every walk prefix (Alg. 2, or Alg. 3 randomized), shared walk
 * prefixes (Alg. 4) and the pruning rules of Sec. 4.1.
 *
 * Conventions shared by every entry point:
 *  - Every function returns a probesim_status; no exception or signal crosses the ABI.  On failure
 *    probesim_last_error() returns a message for the calling thread.
 *  - Node ids are int32 in [0, n).  An id outside that range makes the call fail with
 *    PROBESIM_E_RANGE before anything is applied.
 *  - The caller owns every input and output buffer.  Each one may be host memory or CUDA device memory;
 *    the library tells them apart with cudaPointerGetAttributes.  Host buffers are read or written
 *    before the call returns.  Device buffers are read or written on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream); the call synchronises `stream` before returning, so outputs are
 *    complete on return either way.
 *  - The library owns the graph and all scratch memory (device memory held by the graph object and
 *    released by probesim_graph_destroy).
 *  - A graph object may be used from several threads.  Direct query calls on one graph share one workspace
 *    and are serialised internally; a server's workers each own a workspace and run queries on one graph
 *    concurrently.  An update batch builds the next version of the graph store beside the current one and
 *    publishes it: a query sees the version current when it started, and neither waits for the other.
 *  - All arithmetic on the GPU is FP32 or integer; FP64 is used only on the host (n_r, thresholds).
 */
#ifndef PROBESIM_H
#define PROBESIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct probesim_graph probesim_graph; /* opaque, owned by the library */

typedef enum {
    PROBESIM_OK = 0,
    PROBESIM_E_INVALID = 1,     /* null pointer, size or parameter out of its documented range */
    PROBESIM_E_RANGE = 2,       /* a node id outside [0, n) */
    PROBESIM_E_NOMEM = 3,       /* a device or host allocation failed; the graph is unchanged */
    PROBESIM_E_CUDA = 4,        /* a CUDA runtime error; the message names it */
    PROBESIM_E_TIMEOUT = 5,     /* reserved: no call of this version waits on the device without a bound */
    PROBESIM_E_BUSY = 6,        /* admission refused: not enough free slots or score-buffer memory */
    PROBESIM_E_UNSUPPORTED = 7  /* a valid request this build does not implement */
} probesim_status;

/* PROBE variants (probesim_config.probe_mode). */
enum {
    PROBESIM_PROBE_DETERMINISTIC = 0, /* Alg. 2 */
    PROBESIM_PROBE_RANDOMIZED = 1,    /* Alg. 3 */
    PROBESIM_PROBE_SWITCH = 2         /* Sec. 4.4: deterministic, then randomized above c0 * w * n */
};

/* Graph-wide parameters, fixed at creation. */
typedef struct {
    double c;           /* SimRank decay factor of Eq. 1, 0 < c < 1 (the paper uses 0.6) */
    double delta;       /* failure probability of Def. 1, 0 < delta < 1 */
    int32_t l_max;      /* Pruning Rule 1 (Sec. 4.1): a walk keeps at most l_max nodes, 1 <= l_max <= 255 */
    float eps_p;        /* Pruning Rule 2 (Sec. 4.1) threshold, >= 0; 0 disables the rule */
    float c0;           /* switch constant of Sec. 4.4, >= 0 (used by PROBESIM_PROBE_SWITCH) */
    int32_t probe_mode; /* PROBESIM_PROBE_* */
    uint32_t seed;      /* first Philox key word of every walk and every randomized PROBE draw */
    float shift;        /* added to every estimate s~(u, v), v != u (>= 0; 0 = none): the eps_t / 2 of Thm. 2 that
                           centres Pruning Rule 1's one-sided error (see probesim_split_error) */
} probesim_config;

/* One query.  Its Philox key is (config.seed, query_id): walk k, step s draws counter (k, s, 0, 0), so a
 * query's result does not depend on which other queries share its launch. */
typedef struct {
    int32_t node;       /* query node u */
    int32_t k;          /* number of results for probesim_topk, 1 <= k <= n-1; ignored by single_source */
    double eps;         /* sampling error of Alg. 1; n_r = ceil(3c/eps^2 * ln(n/delta)), 0 < eps < 1 */
    uint32_t query_id;  /* second Philox key word */
    int32_t walk_begin; /* use walks k in [walk_begin, walk_end) of the n_r walks (the estimate still */
    int32_t walk_end;   /* divides by n_r); walk_end <= 0 means n_r.  0/0 is the full estimator */
} probesim_query;

/* Fills *cfg with c = 0.6, delta = 0.01, l_max = 64, eps_p = 0, c0 = 1, deterministic PROBE, seed = 3, shift = 0. */
probesim_status probesim_config_default(probesim_config *cfg);

/* Thm. 2 (Sec. 4.1) bounds the error of Alg. 1 with both pruning rules, with probability 1 - delta, by
 *     eps + T_p + eps_t / 2   when every estimate is shifted up by eps_t / 2 (Rule 1's error is one-sided),
 *     eps + T_p + eps_t       without the shift,
 * where T_p is Rule 2's term.  The paper states T_p = (1+eps)/(1-sqrt(c)) * eps_p from a per-probe bound of eps_p;
 * that lemma's induction leaves out the score pruned at each later level, and the per-probe bound that holds is
 * (i-1) * eps_p for the prefix of length i.  Summed over a sqrt(c)-walk's probes (E[l(l-1)/2] = sqrt(c)/(1-sqrt(c))^2
 * for its geometric length l) it gives T_p = (1+eps) * sqrt(c)/(1-sqrt(c))^2 * eps_p.  This call splits a target
 * error eps_a (0 < eps_a < 1) with the corrected T_p: eps = eps_a/2, T_p = eps_a/4 and Rule 1's term eps_a/4; l_max
 * is the smallest walk length with sqrt(c)^l_max <= eps_t.  Pure host arithmetic (FP64). */
typedef struct {
    double eps;         /* sampling error of Alg. 1 (sets n_r) */
    double eps_t;       /* Pruning Rule 1's termination parameter */
    int32_t l_max;      /* nodes a walk keeps: ceil(ln eps_t / ln sqrt(c)), clamped to [1, 255] */
    float eps_p;        /* Pruning Rule 2's parameter, rounded down to FP32 (the config's type) */
    float shift;        /* eps_t / 2 with shift requested, else 0 (for probesim_config.shift) */
    double bound;       /* the guaranteed error with the corrected T_p: <= eps_a */
    double bound_paper; /* the same sum with the paper's T_p */
} probesim_error_split;
probesim_status probesim_split_error(double eps_a, double c, int32_t shift, probesim_error_split *out);

/* Builds the device graph store from m directed edges src[e] -> dst[e] (Sec. 2.1: a directed simple
 * graph).  src and dst may be host or device arrays (host arrays are copied to the device first); the build runs
 * on the device (radix sorts of the edge keys; it takes about 24 bytes of device memory per edge beyond the
 * store).  Self-loops and duplicate edges are dropped (a simple graph has neither) and the number kept is reported
 * by probesim_graph_info.  An id outside [0, n) gives E_RANGE and no graph.  n >= 1, 0 <= m < 2^31.  On success
 * *out owns the graph; the call synchronises `stream`. */
probesim_status probesim_graph_create(int32_t n, const int32_t *src, const int32_t *dst, int64_t m,
                                      const probesim_config *cfg, void *stream, probesim_graph **out);

/* Frees the graph and all its device memory.  NULL is accepted. */
probesim_status probesim_graph_destroy(probesim_graph *g);

/* Current node count, edge count, and update epoch (the number of update batches applied). */
probesim_status probesim_graph_info(const probesim_graph *g, int32_t *n, int64_t *m, uint64_t *epoch);

/* Dynamic updates (the paper's index-free design needs no rebuild, Sec. 1): apply k edge insertions or
 * deletions as one batch that advances the epoch.  Inserting an existing edge, deleting an absent edge and
 * self-loops are skipped; *applied (may be NULL) receives the number of edges actually changed.  Queries
 * issued after the call returns see the new edge set. */
probesim_status probesim_insert_edges(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k,
                                      int64_t *applied, void *stream);
probesim_status probesim_delete_edges(probesim_graph *g, const int32_t *src, const int32_t *dst, int64_t k,
                                      int64_t *applied, void *stream);

/* n_r = ceil(3c/eps^2 * ln(n/delta)) for this graph (Alg. 1 line 1), computed in FP64 on the host. */
probesim_status probesim_num_walks(const probesim_graph *g, double eps, int64_t *n_r);

/* The sqrt(c)-walks of the queries (Def. 3, truncated by Pruning Rule 1), for checking.  Walks are laid out
 * query by query, walk by walk (walk_begin..walk_end-1 of each): nodes[w * l_max + s] is node s+1 of walk w
 * (entries past its length are -1) and lens[w] its node count.  capacity is the number of walk rows the
 * buffers hold; PROBESIM_E_INVALID if the queries need more. */
probesim_status probesim_sample_walks(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t *nodes,
                                      int32_t *lens, int64_t capacity, void *stream);

/* Approximate single-source SimRank (Def. 1, Alg. 1 / Alg. 4): scores[i * n + v] = s~(q[i].node, v), with
 * s~(u, u) = 1.  scores holds nq * n floats. */
probesim_status probesim_single_source(probesim_graph *g, const probesim_query *q, int32_t nq, float *scores,
                                       void *stream);

/* Approximate top-k SimRank (Def. 2): for query i, ids[i * kmax + r] and vals[i * kmax + r], r < q[i].k, are
 * the nodes v != u with the largest s~(u, v), ordered by (s~ descending, id ascending); entries r >= q[i].k
 * are set to -1 and 0.  1 <= q[i].k <= kmax <= n-1. */
probesim_status probesim_topk(probesim_graph *g, const probesim_query *q, int32_t nq, int32_t kmax, int32_t *ids,
                              float *vals, void *stream);

/* Pairwise Monte Carlo SimRank (Sec. 2.2, Eq. 3), the single-pair estimator the paper uses as the "expert" that
 * gauges pooled top-k candidates: for pair i, r pairs of sqrt(c)-walks (Def. 3, at most l_max nodes each) from
 * u[i] and v[i]; meets[i] counts the walk pairs whose j-th nodes coincide for some j, and est[i] = meets[i] / r
 * (1 when u[i] = v[i]).  With r >= ln(1/delta) / (2 eps^2) the estimate is within eps of s(u, v) with probability
 * 1 - delta.  Walk t from u[i] draws Philox counter (t, s, 0, 0) under key (config.seed, key_u[i]) at step s, the
 * draws of walk t of a query with query_id key_u[i]; the walks from v[i] use key_v[i].  Inputs are host arrays of
 * npairs entries (1 <= npairs <= 65535, 1 <= r < 2^32); meets and est are host or device arrays (est may be
 * NULL). */
probesim_status probesim_pair_mc(probesim_graph *g, const int32_t *u, const int32_t *v, const uint32_t *key_u,
                                 const uint32_t *key_v, int32_t npairs, int64_t r, int64_t *meets, float *est,
                                 void *stream);

/* Per-call measurements of the last single_source/topk call on this graph.  When profiling is on, the
 * library records CUDA events around every launch of the PROBE level kernel (the dominant kernel) on the
 * call's stream; probe_ms is their summed duration and probe_launches their count.  probe_bytes is the
 * algorithmic byte count of those launches (see the field comments).  Profiling adds event records but
 * skips no work. */
typedef struct {
    int64_t walks;          /* walks generated */
    int64_t walk_nodes;     /* sum of walk lengths */
    int64_t tree_nodes;     /* reverse-reachability tree nodes (Alg. 4), the virtual super-roots included */
    int64_t vectors;        /* dense score vectors pushed (tree nodes with a subtree of height >= 2) */
    int64_t levels;         /* level-loop iterations */
    int64_t edge_gathers;   /* (edge, vector) pairs processed by the PROBE level kernel */
    int64_t probe_launches; /* launches of the PROBE level kernel */
    double probe_ms;        /* their summed CUDA-event duration (profiling on), else 0 */
    double probe_bytes;     /* algorithmic bytes of those launches: per launch 4 per in-edge index, 16 per
                               in-list piece record, 4 per vertex weight, and 4 per gathered-row score read
                               plus 4 per written score for each of the launch's S columns (4m + 16 pieces
                               + 4n + 8nS) */
    int64_t kernel_launches;/* all kernels this library launched in the call */
    double phase_ms[12];    /* profiling on: CUDA-event time per phase of the deterministic path: 0 walks,
                               1 walk tree and level schedule, 2 D accumulate, 3 gamma scatter, 4 split-row
                               zeroing, 5 pull, 6 push columns, 7 gamma, 8 estimates.  9 (always recorded):
                               host wall-clock time of the column schedule, during which the device waits;
                               10-11 unused */
    int64_t max_columns;    /* widest score matrix of the level loop, in columns (deterministic path) */
    int64_t probes;         /* walk prefixes probed one by one (Pruning Rule 2 or the switch) */
    int64_t switched;       /* of those, the probes the switch of Sec. 4.4 handed to Alg. 3 */
    int64_t table_passes;   /* passes over the frontier engine's per-level tables (more than one per level when
                               a table exceeds a quarter of the memory budget) */
    int64_t max_table_slots;/* largest per-level table, in slots of 12 bytes */
    int64_t deferred;       /* probe ranges the frontier engine set aside at a level and resumed later, so that
                               one level's frontier stays within an eighth of the memory budget */
} probesim_stats;

probesim_status probesim_set_profiling(probesim_graph *g, int32_t on);

/* Device memory that one call's working buffers on this graph may take, in bytes (0 restores the default, 60%
 * of the device's memory at graph creation).  A call whose queries need more is cut into smaller batches; the
 * frontier engine (Pruning Rule 2, the switch) also cuts a level's table into passes of a quarter of it.  A
 * single query that still does not fit fails with PROBESIM_E_NOMEM.  Results do not depend on the budget. */
probesim_status probesim_set_memory_budget(probesim_graph *g, double bytes);

/* Autotuner of the PROBE level kernel's launch shape on this graph.  It times the pull over the graph's own
 * in-lists for tile widths {1,2,4,8,16,32} columns and {2,4,8,16} blocks per SM (a constant-filled 64-column
 * score matrix, CUDA events, three runs after a warm-up), keeps the fastest shape per width and, for the
 * 32-column tiles of wide matrices, whichever of 32-column tiles, 16-column halves, 32-column tiles taken two
 * per pass (one read of the in-lists for both) and 32-column tiles gathered by the TMA takes less time.
 * Later queries on the graph use the choice.  Takes about a second; results do not depend on it (only the
 * summation order). */
probesim_status probesim_autotune(probesim_graph *g, void *stream);
/* The current choice: *wide_tile in {16, 32, 64, 96} (see probesim_set_tuning); blocks_per_sm[6] for tile widths
 * 1, 2, 4, 8, 16, 32. */
probesim_status probesim_get_tuning(const probesim_graph *g, int32_t *wide_tile, int32_t *blocks_per_sm);
/* Sets the launch shape by hand: wide_tile in {16, 32, 64, 96} (64: 32-column tiles two per pass; 96: 32-column
 * tiles whose rows the Tensor Memory Accelerator gathers into shared memory, E_UNSUPPORTED without a tensor-map
 * encoder in the driver); blocks_per_sm (may be null: keep the current ones) holds 8 entries in [1, 32], for tile
 * widths 1, 2, 4, 8, 16, 32, the pairs and the TMA launch (at most 3 fit).  Set it while no call runs on the graph
 * (the level loop reads the shape without a lock).  Results do not depend on it beyond rounding. */
probesim_status probesim_set_tuning(probesim_graph *g, int32_t wide_tile, const int32_t *blocks_per_sm);
probesim_status probesim_get_stats(const probesim_graph *g, probesim_stats *out);

/* ---------------------------------------------------------------------------------------------------------
 * Serving loop (continuous batching).  Queries and edge-update batches enter one FIFO.  `workers` threads,
 * each with its own scratch memory and CUDA stream, take the next batch of queries from the head as soon as
 * they are free: up to max_batch queries, admitted while the estimated memory of the batches in flight stays
 * within memory_budget_bytes (the deterministic engine's score buffers, about 12 * n * 0.25 * n_r bytes per
 * query; with Pruning Rule 2, the switch or the randomized PROBE, an estimate row and walk rows, 12 n + 8 l_max
 * n_r bytes, since those engines fit their level tables into each worker's share of the budget, 1/workers of
 * it).  Queries that arrive while other batches run are admitted by the next free worker, so the work of
 * several batches overlaps on the device.  An update batch at the head is applied between batches: queries
 * submitted after it see the new edge set, queries submitted before it the old one; it builds the next store
 * version while earlier batches still run.  Results are top-k lists (Def. 2).
 * --------------------------------------------------------------------------------------------------------- */
typedef struct probesim_server probesim_server;

typedef struct {
    int32_t workers;            /* concurrent batch pipelines, 1..8 (default 3) */
    int32_t max_batch;          /* queries per batch, 1..4096 (default 2) */
    int32_t kmax;               /* largest k a query may ask for, 1..min(4096, n-1) */
    int32_t queue_capacity;     /* queries waiting at once; submit beyond it fails with PROBESIM_E_BUSY */
    double memory_budget_bytes; /* score-buffer memory admitted at once; 0 = 60% of device memory */
} probesim_server_config;

typedef struct {
    uint64_t ticket;     /* returned by probesim_server_submit */
    uint32_t query_id;
    int32_t node, k;
    int32_t status;      /* probesim_status of the batch that ran the query */
    uint64_t epoch;      /* update epoch of the edge set the query saw */
    int32_t batch_size;  /* queries in its batch */
    int32_t worker;      /* worker that ran it */
    double queue_ms;     /* submit -> batch start */
    double latency_ms;   /* submit -> result ready */
} probesim_result;

typedef struct {
    int64_t submitted, completed, rejected, failed, batches, updates_applied;
    double mean_batch;   /* queries per batch */
    double p50_ms, p99_ms, mean_ms;  /* latency of completed queries */
    double qps;          /* completed queries / (last completion - first submit) */
} probesim_server_stats;

/* workers = 3, max_batch = 2, kmax = 100, queue_capacity = 100000, memory_budget_bytes = 0. */
probesim_status probesim_server_config_default(probesim_server_config *cfg);
/* Starts the workers over graph g (which must outlive the server). */
probesim_status probesim_server_create(probesim_graph *g, const probesim_server_config *cfg, probesim_server **out);
/* Enqueues nq queries (host array, k <= kmax); tickets (host, may be NULL) receives their tickets. */
probesim_status probesim_server_submit(probesim_server *s, const probesim_query *q, int32_t nq, uint64_t *tickets);
/* Enqueues an update batch of k edges (host arrays); insert != 0 inserts, 0 deletes (see probesim_insert_edges). */
probesim_status probesim_server_update(probesim_server *s, const int32_t *src, const int32_t *dst, int64_t k,
                                       int32_t insert);
/* Moves up to max_results finished results into res, with their top-k in ids/vals ([max_results][kmax], host),
 * waiting up to wait_ms for the first one; *count receives the number moved. */
probesim_status probesim_server_poll(probesim_server *s, int32_t max_results, int32_t kmax, probesim_result *res,
                                     int32_t *ids, float *vals, int32_t *count, int32_t wait_ms);
probesim_status probesim_server_get_stats(probesim_server *s, probesim_server_stats *out);
/* Stops the workers after their current batches; queries still waiting are dropped. */
probesim_status probesim_server_destroy(probesim_server *s);

/* Top-k selection that allocates no memory.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory while they run, such as a component that has reserved all device memory for its own
 * pool, or a serving loop that must not take the device-wide synchronisation cudaMalloc and cudaFree imply.
 * It selects, for each of nq score rows, the kmax-bounded top-k that probesim_topk returns (ordered by score
 * descending then id ascending, node u excluded, entries r >= ks[i] set to -1 / 0):
 *   scores  device memory, nq * n FP32 scores, row i for query node nodes[i] (e.g. probesim_single_source output)
 *   nodes   host array of nq query nodes in [0, n) (excluded from their row's ranking)
 *   ks      host array of nq result counts in [1, kmax]
 *   ids     device memory, nq * kmax int32 results;  vals  device memory, nq * kmax FP32 results
 * Limits: 1 <= nq <= 64, 1 <= kmax <= min(1024, n-1), n >= 2; larger requests fail with PROBESIM_E_INVALID
 * and a message naming the limit.  The scratch is one fixed __device__ array of 853,504 bytes in the library,
 * which every GPU that loads the library holds until the process exits.  No call allocates: no cudaMalloc,
 * cudaFree or allocating library routine is used.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current and loads the top-k kernels; module loading may
 * allocate device memory, so make that first call before reserving the device's memory for a pool, and before
 * any stream capture.
 * Every call shares the array, and calls serialise on the host and synchronise `stream` before they return;
 * calls that would overlap on the GPU (for instance from several processes sharing a context) race on it. */
probesim_status probesim_topk_select_noalloc(const float *scores, int32_t n, int32_t nq, const int32_t *nodes,
                                             const int32_t *ks, int32_t kmax, int32_t *ids, float *vals, void *stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char *probesim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PROBESIM_H */
