/*
 * ProbeSim CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of the method of
 *   Y. Liu, B. Zheng, X. He, Z. Wei, X. Xiao, K. Zheng, J. Lu,
 *   "ProbeSim: Scalable Single-Source and Top-k SimRank Computations on Dynamic Graphs",
 *   PVLDB 11(1), 2017 (arXiv 1709.06955).
 * It follows the paper's algorithms step by step in the paper's order and notation, with
 * dense FP64 arrays standing in for the paper's hash sets.  There is no blocking, fusion or
 * reordering beyond what each algorithm states.  It shares no code with the CUDA library: it has
 * its own Philox generator, its own graph arrays and its own arithmetic.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Contents (each function cites the passage it follows):
 *   orc_philox4x32_10   counter-based generator of Salmon et al. (SC'11), from its published definition
 *   orc_graph_*         in/out adjacency of a directed simple graph (Sec. 2.1)
 *   orc_num_walks       n_r = ceil(3c/eps^2 * ln(n/delta))              (Alg. 1, Thm. 1)
 *   orc_walk            one sqrt(c)-walk, truncated at l_max nodes          (Def. 3, Pruning Rule 1)
 *   orc_probe_det       deterministic PROBE with optional Pruning Rule 2     (Alg. 2, Sec. 4.1)
 *   orc_probe_rand      randomized PROBE levels                              (Alg. 3)
 *   orc_single_source   Basic ProbeSim                                       (Alg. 1)
 *   orc_single_source_batch  reverse-reachability tree + best-of-both switch (Alg. 4, Sec. 4.4)
 *   orc_topk            the k largest estimates, v != u                      (Def. 2, Sec. 3)
 *   orc_pair_mc         pairwise Monte Carlo meeting estimator              (Sec. 2.2, Eq. 3)
 *
 * Readings of points the paper leaves open:
 *   - the stop test of Def. 3 is applied at every visited node including u_1; a draw x0 below
 *     T_stop = floor((1 - sqrt(c)) * 2^32) stops the walk;
 *   - a walk at a node with no in-neighbour stops there;
 *   - the next node is entry floor(x1 * |I(v)| / 2^32) of I(v) sorted by ascending source id;
 *   - Philox key = (seed, query_id); walk k, step s uses counter (k, s, 0, 0);
 *     randomized PROBE of walk k on prefix length i, level j, candidate x uses counter
 *     (k, 2^24 | i << 8 | j, x, 0) (x0 picks the in-edge, x1 < T_keep = floor(sqrt(c) * 2^32) keeps);
 *   - level j of PROBE on (u_1..u_i) excludes u_{i-j-1};
 *   - Pruning Rule 2 drops x when Score(x) * sqrt(c)^(i-j-1) <= eps_p, and eps_p = 0 disables it;
 *   - in the switch of Sec. 4.4 a probe of weight w whose frontier H_j has out-degree sum above
 *     c0 * w * n is handed to the randomized PROBE algorithm: the deterministic levels run so far are
 *     dropped and Alg. 3 runs on the whole partial walk w times, once per walk sharing the prefix,
 *     each with that walk's own Philox stream (Sec. 4.4 states that the switched probe needs w
 *     independent randomized probes, averaged).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",     */
/* SC'11): ten rounds of two 32x32->64 multiplies on a 4-word counter, with a Weyl-sequence     */
/* key schedule between rounds.                                                                  */
/* ------------------------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += ORC_PHILOX_W0; k1 += ORC_PHILOX_W1; }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void orc_draw(uint32_t seed, uint32_t qid, uint32_t a, uint32_t b, uint32_t x, uint32_t out[4]) {
    uint32_t ctr[4] = {a, b, x, 0u};
    uint32_t key[2] = {seed, qid};
    orc_philox4x32_10(ctr, key, out);
}

/* multiply-shift index in [0, d): floor(x * d / 2^32) */
static int64_t orc_pick(uint32_t x, int64_t d) { return (int64_t)(((uint64_t)x * (uint64_t)d) >> 32); }

/* probability thresholds on 32-bit draws, computed in FP64 */
uint32_t orc_threshold_stop(double c) { return (uint32_t)floor((1.0 - sqrt(c)) * 4294967296.0); }
uint32_t orc_threshold_keep(double c) {
    double t = floor(sqrt(c) * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

/* ------------------------------------------------------------------------------------------ */
/* Graph (Sec. 2.1: a directed simple graph G=(V,E), |V|=n, |E|=m).                            */
/* I(v): in-neighbours of v sorted ascending; O(x): out-neighbours of x sorted ascending.        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    int64_t m;
    int64_t *in_off, *out_off; /* n+1 */
    int32_t *in_col, *out_col; /* m */
} orc_graph;

static int orc_cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_graph_free(orc_graph *g) {
    if (!g) return;
    free(g->in_off); free(g->out_off); free(g->in_col); free(g->out_col); free(g);
}

/* Returns NULL on a self-loop, a duplicate edge, an id outside [0,n) or allocation failure. */
orc_graph *orc_graph_new(int32_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    if (n <= 0 || m < 0) return NULL;
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    if (!g || !key) { free(key); free(g); return NULL; }
    g->n = n; g->m = m;
    g->in_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->out_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->in_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    g->out_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!g->in_off || !g->out_off || !g->in_col || !g->out_col) goto fail;
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || src[e] == dst[e]) goto fail;
    }
    /* in-lists: sort by (dst, src) */
    for (int64_t e = 0; e < m; ++e) key[e] = ((uint64_t)(uint32_t)dst[e] << 32) | (uint32_t)src[e];
    qsort(key, (size_t)m, sizeof(uint64_t), orc_cmp_u64);
    for (int64_t e = 0; e < m; ++e) {
        if (e > 0 && key[e] == key[e - 1]) goto fail;
        g->in_off[(key[e] >> 32) + 1]++;
        g->in_col[e] = (int32_t)(key[e] & 0xffffffffu);
    }
    for (int32_t v = 0; v < n; ++v) g->in_off[v + 1] += g->in_off[v];
    /* out-lists: sort by (src, dst) */
    for (int64_t e = 0; e < m; ++e) key[e] = ((uint64_t)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
    qsort(key, (size_t)m, sizeof(uint64_t), orc_cmp_u64);
    for (int64_t e = 0; e < m; ++e) {
        g->out_off[(key[e] >> 32) + 1]++;
        g->out_col[e] = (int32_t)(key[e] & 0xffffffffu);
    }
    for (int32_t v = 0; v < n; ++v) g->out_off[v + 1] += g->out_off[v];
    free(key);
    return g;
fail:
    free(key);
    orc_graph_free(g);
    return NULL;
}

int64_t orc_in_degree(const orc_graph *g, int32_t v) { return g->in_off[v + 1] - g->in_off[v]; }
int64_t orc_out_degree(const orc_graph *g, int32_t v) { return g->out_off[v + 1] - g->out_off[v]; }

/* ------------------------------------------------------------------------------------------ */
/* n_r = (3c / eps^2) * ln(n / delta), rounded up (Alg. 1 line 1; the natural log is the one   */
/* the Chernoff step of Thm. 1 needs).                                                          */
/* ------------------------------------------------------------------------------------------ */
int64_t orc_num_walks(double c, double eps, double delta, int64_t n) {
    return (int64_t)ceil(3.0 * c / (eps * eps) * log((double)n / delta));
}

/* ------------------------------------------------------------------------------------------ */
/* sqrt(c)-walk (Def. 3 and the generation procedure after it): at the current node v, stop     */
/* with probability 1 - sqrt(c), otherwise move to a uniformly chosen in-neighbour.  Pruning     */
/* Rule 1 keeps at most l_max nodes.  Writes the nodes into path[0..len) and returns len >= 1.  */
/* ------------------------------------------------------------------------------------------ */
int32_t orc_walk(const orc_graph *g, int32_t u, double c, int32_t l_max, uint32_t seed, uint32_t qid,
                 uint32_t k, int32_t *path) {
    const uint32_t t_stop = orc_threshold_stop(c);
    int32_t len = 0, v = u;
    path[len++] = u;
    for (uint32_t s = 0;; ++s) {
        if (len >= l_max) break; /* Pruning Rule 1 */
        uint32_t r[4];
        orc_draw(seed, qid, k, s, 0u, r);
        if (r[0] < t_stop) break; /* stop with probability 1 - sqrt(c) */
        int64_t d = orc_in_degree(g, v);
        if (d == 0) break; /* no in-neighbour to move to */
        v = g->in_col[g->in_off[v] + orc_pick(r[1], d)];
        path[len++] = v;
    }
    return len;
}

/* ------------------------------------------------------------------------------------------ */
/* A hash set H_j of (node, score) pairs, kept as a dense FP64 array plus a member list.        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n, size;
    double *score;   /* n */
    char *present;   /* n */
    int32_t *member; /* n */
} orc_set;

static int orc_set_init(orc_set *h, int32_t n) {
    h->n = n; h->size = 0;
    h->score = (double *)calloc((size_t)n, sizeof(double));
    h->present = (char *)calloc((size_t)n, 1);
    h->member = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    return (h->score && h->present && h->member) ? 0 : -1;
}
static void orc_set_free(orc_set *h) { free(h->score); free(h->present); free(h->member); }
static void orc_set_clear(orc_set *h) {
    for (int32_t t = 0; t < h->size; ++t) { h->score[h->member[t]] = 0.0; h->present[h->member[t]] = 0; }
    h->size = 0;
}
static void orc_set_add(orc_set *h, int32_t v, double s) {
    if (!h->present[v]) { h->present[v] = 1; h->member[h->size++] = v; }
    h->score[v] += s;
}
static void orc_set_put(orc_set *h, int32_t v, double s) {
    if (!h->present[v]) { h->present[v] = 1; h->member[h->size++] = v; }
    h->score[v] = s;
}
static void orc_set_swap(orc_set *a, orc_set *b) { orc_set t = *a; *a = *b; *b = t; }

typedef struct {
    int64_t edge_pushes;  /* (x -> v) traversals in deterministic PROBE levels */
    int64_t rand_samples; /* candidates sampled by randomized PROBE levels */
    int64_t probes;       /* PROBE invocations */
    int64_t walks;
    int64_t walk_nodes;   /* sum of walk lengths */
    int64_t tree_nodes;   /* reverse-reachability tree nodes below the root (Alg. 4) */
    int64_t switched;     /* probes that switched to randomized levels (Sec. 4.4) */
} orc_counters;

/* scratch for one PROBE: two level sets */
typedef struct { orc_set a, b, t; } orc_probe_ws;

static int orc_ws_init(orc_probe_ws *w, int32_t n) {
    if (orc_set_init(&w->a, n) || orc_set_init(&w->b, n) || orc_set_init(&w->t, n)) return -1;
    return 0;
}
static void orc_ws_free(orc_probe_ws *w) { orc_set_free(&w->a); orc_set_free(&w->b); orc_set_free(&w->t); }

/* Pruning Rule 2 (Sec. 4.1): before descending from H_j, drop every x with
 * Score(x) * sqrt(c)^(i-j-1) <= eps_p.  eps_p = 0 disables the rule. */
static void orc_prune(orc_set *h, double sqrt_c, int32_t i, int32_t j, double eps_p, orc_set *tmp) {
    if (!(eps_p > 0.0)) return;
    double f = pow(sqrt_c, (double)(i - j - 1));
    orc_set_clear(tmp);
    for (int32_t t = 0; t < h->size; ++t) {
        int32_t x = h->member[t];
        if (h->score[x] * f > eps_p) orc_set_put(tmp, x, h->score[x]);
    }
    orc_set_swap(h, tmp);
}

/* One deterministic level of Alg. 2 (lines 4-9): for each (x, Score(x)) in H_j and each
 * v in O(x) with v != excl, add sqrt(c)/|I(v)| * Score(x) to Score(v) in H_{j+1}. */
static void orc_det_level(const orc_graph *g, double sqrt_c, const orc_set *hj, int32_t excl, orc_set *hj1,
                          orc_counters *cnt) {
    orc_set_clear(hj1);
    for (int32_t t = 0; t < hj->size; ++t) {
        int32_t x = hj->member[t];
        double sx = hj->score[x];
        for (int64_t e = g->out_off[x]; e < g->out_off[x + 1]; ++e) {
            int32_t v = g->out_col[e];
            if (cnt) cnt->edge_pushes++;
            if (v == excl) continue;
            orc_set_add(hj1, v, sqrt_c / (double)orc_in_degree(g, v) * sx);
        }
    }
}

/* One randomized level of Alg. 3 (lines 4-11) for walk k on prefix length i, level j.
 * Candidates U are the union of O(y) over y in H_j when the out-degree sum is at most n, else V
 * (lines 4-7).  Each candidate x != excl samples one in-edge (v, x) of I(x) (line 9); if v is in
 * H_j, x joins H_{j+1} with probability sqrt(c) (lines 10-11) carrying Score(v). */
static void orc_rand_level(const orc_graph *g, double c, uint32_t seed, uint32_t qid, uint32_t k, int32_t i,
                           int32_t j, const orc_set *hj, int32_t excl, orc_set *hj1, orc_set *cand,
                           orc_counters *cnt) {
    const uint32_t t_keep = orc_threshold_keep(c);
    orc_set_clear(hj1);
    orc_set_clear(cand);
    int64_t degsum = 0;
    for (int32_t t = 0; t < hj->size; ++t) degsum += orc_out_degree(g, hj->member[t]);
    if (degsum <= (int64_t)g->n) {
        for (int32_t t = 0; t < hj->size; ++t) {
            int32_t y = hj->member[t];
            for (int64_t e = g->out_off[y]; e < g->out_off[y + 1]; ++e) orc_set_put(cand, g->out_col[e], 1.0);
        }
    } else {
        for (int32_t x = 0; x < g->n; ++x) orc_set_put(cand, x, 1.0);
    }
    for (int32_t t = 0; t < cand->size; ++t) {
        int32_t x = cand->member[t];
        if (x == excl) continue;
        int64_t d = orc_in_degree(g, x);
        if (d == 0) continue;
        if (cnt) cnt->rand_samples++;
        uint32_t r[4];
        orc_draw(seed, qid, k, (1u << 24) | ((uint32_t)i << 8) | (uint32_t)j, (uint32_t)x, r);
        int32_t v = g->in_col[g->in_off[x] + orc_pick(r[0], d)];
        if (hj->present[v] && r[1] < t_keep) orc_set_put(hj1, x, hj->score[v]);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Deterministic PROBE (Alg. 2) on the partial walk path[0..i) = (u_1..u_i), with Pruning     */
/* Rule 2 when eps_p > 0.  Adds weight * Score(v) of S = H_{i-1} into acc[v].                   */
/* ------------------------------------------------------------------------------------------ */
static void orc_probe_det_ws(const orc_graph *g, const int32_t *path, int32_t i, double c, double eps_p,
                             double weight, double *acc, orc_probe_ws *w, orc_counters *cnt) {
    const double sqrt_c = sqrt(c);
    orc_set *hj = &w->a, *hj1 = &w->b;
    orc_set_clear(hj);
    orc_set_put(hj, path[i - 1], 1.0); /* line 2: H_0 = {(u_i, 1)} */
    for (int32_t j = 0; j <= i - 2; ++j) {   /* line 3 */
        orc_prune(hj, sqrt_c, i, j, eps_p, &w->t);
        orc_det_level(g, sqrt_c, hj, path[i - j - 2] /* u_{i-j-1} */, hj1, cnt);
        orc_set_swap(hj, hj1);
    }
    for (int32_t t = 0; t < hj->size; ++t) acc[hj->member[t]] += weight * hj->score[hj->member[t]];
    orc_set_clear(hj);
    orc_set_clear(hj1);
    if (cnt) cnt->probes++;
}

/* Randomized PROBE (Alg. 3) for walk k on path[0..i); adds weight * Score(v) (= weight for
 * members of H_{i-1}) into acc. */
static void orc_probe_rand_ws(const orc_graph *g, const int32_t *path, int32_t i, double c, uint32_t seed,
                              uint32_t qid, uint32_t k, double weight, double *acc, orc_probe_ws *w,
                              orc_counters *cnt) {
    orc_set *hj = &w->a, *hj1 = &w->b;
    orc_set_clear(hj);
    orc_set_put(hj, path[i - 1], 1.0);
    for (int32_t j = 0; j <= i - 2; ++j) {
        orc_rand_level(g, c, seed, qid, k, i, j, hj, path[i - j - 2], hj1, &w->t, cnt);
        orc_set_swap(hj, hj1);
    }
    for (int32_t t = 0; t < hj->size; ++t) acc[hj->member[t]] += weight * hj->score[hj->member[t]];
    orc_set_clear(hj);
    orc_set_clear(hj1);
    orc_set_clear(&w->t);
    if (cnt) cnt->probes++;
}

/* Public single-probe entry points: out[n] receives S (zeroed first). */
int orc_probe_det(const orc_graph *g, const int32_t *path, int32_t i, double c, double eps_p, double *out) {
    orc_probe_ws w;
    if (i < 2 || orc_ws_init(&w, g->n)) return -1;
    memset(out, 0, sizeof(double) * (size_t)g->n);
    orc_probe_det_ws(g, path, i, c, eps_p, 1.0, out, &w, NULL);
    orc_ws_free(&w);
    return 0;
}

int orc_probe_rand(const orc_graph *g, const int32_t *path, int32_t i, double c, uint32_t seed, uint32_t qid,
                   uint32_t k, double *out) {
    orc_probe_ws w;
    if (i < 2 || orc_ws_init(&w, g->n)) return -1;
    memset(out, 0, sizeof(double) * (size_t)g->n);
    orc_probe_rand_ws(g, path, i, c, seed, qid, k, 1.0, out, &w, NULL);
    orc_ws_free(&w);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Parameters of one single-source query.                                                       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double c, eps, delta, eps_p, c0;
    int32_t l_max;
    int32_t probe_mode; /* 0 deterministic, 1 randomized, 2 switch (Alg. 4 only) */
    uint32_t seed, query_id;
    int64_t walk_begin, walk_end; /* walks k in [walk_begin, walk_end); walk_end <= 0 means n_r */
} orc_params;

static void orc_walk_range(const orc_params *p, int64_t n_r, int64_t *b, int64_t *e) {
    *b = p->walk_begin < 0 ? 0 : p->walk_begin;
    *e = p->walk_end <= 0 ? n_r : (p->walk_end < n_r ? p->walk_end : n_r);
    if (*b > *e) *b = *e;
}

/* ------------------------------------------------------------------------------------------ */
/* Basic ProbeSim (Alg. 1).  For each trial k: generate W_k(u) (line 3), probe every partial    */
/* walk W_k(u, i), i = 2..l (lines 5-6), and sum the scores into s_k (lines 7-11).  The final   */
/* estimator is (1/n_r) * sum_k s_k (the running average of lines 12-16 ends at this value),   */
/* and s(u,u) = 1.  out[n] receives the estimates.                                              */
/* ------------------------------------------------------------------------------------------ */
int orc_single_source(const orc_graph *g, int32_t u, const orc_params *p, double *out, orc_counters *cnt) {
    if (u < 0 || u >= g->n || p->l_max < 1 || p->l_max > 255) return -1;
    const int64_t n_r = orc_num_walks(p->c, p->eps, p->delta, g->n);
    int64_t kb, ke;
    orc_walk_range(p, n_r, &kb, &ke);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)p->l_max);
    double *sum = (double *)calloc((size_t)g->n, sizeof(double));
    orc_probe_ws w;
    if (!path || !sum || orc_ws_init(&w, g->n)) { free(path); free(sum); return -1; }
    for (int64_t k = kb; k < ke; ++k) {
        int32_t len = orc_walk(g, u, p->c, p->l_max, p->seed, p->query_id, (uint32_t)k, path);
        if (cnt) { cnt->walks++; cnt->walk_nodes += len; }
        for (int32_t i = 2; i <= len; ++i) {
            if (p->probe_mode == 1)
                orc_probe_rand_ws(g, path, i, p->c, p->seed, p->query_id, (uint32_t)k, 1.0, sum, &w, cnt);
            else
                orc_probe_det_ws(g, path, i, p->c, p->eps_p, 1.0, sum, &w, cnt);
        }
    }
    for (int32_t v = 0; v < g->n; ++v) out[v] = sum[v] / (double)n_r;
    out[u] = 1.0;
    orc_ws_free(&w);
    free(path);
    free(sum);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Batch algorithm (Alg. 4) with the best-of-both switch (Sec. 4.4).                           */
/* The reverse-reachability tree: node r_q holds a graph node and a weight (the number of walks */
/* sharing the prefix); children are kept in a plain sibling list.                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t node, weight, depth, parent;
    int32_t first_child, next_sibling;
    int32_t walk_head; /* list of walks through this tree node (for the randomized instances) */
} orc_tnode;

int orc_single_source_batch(const orc_graph *g, int32_t u, const orc_params *p, double *out, orc_counters *cnt) {
    if (u < 0 || u >= g->n || p->l_max < 1 || p->l_max > 255) return -1;
    const int64_t n_r = orc_num_walks(p->c, p->eps, p->delta, g->n);
    const double sqrt_c = sqrt(p->c);
    int64_t kb, ke;
    orc_walk_range(p, n_r, &kb, &ke);
    int64_t cap = 1 + (ke - kb) * (int64_t)p->l_max;
    orc_tnode *T = (orc_tnode *)malloc(sizeof(orc_tnode) * (size_t)cap);
    int32_t *walk_next = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap); /* per (tree node, walk) link */
    int32_t *walk_id = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)p->l_max);
    int32_t *prefix = (int32_t *)malloc(sizeof(int32_t) * (size_t)p->l_max);
    double *sum = (double *)calloc((size_t)g->n, sizeof(double));
    orc_probe_ws w;           /* deterministic levels: w.a = H_j, w.b = H_{j+1}, w.t = pruning scratch */
    orc_probe_ws rw;          /* randomized instances: rw.a = H_j, rw.b = H_{j+1}, rw.t = candidates */
    if (!T || !walk_next || !walk_id || !path || !prefix || !sum || orc_ws_init(&w, g->n) ||
        orc_ws_init(&rw, g->n)) {
        free(T); free(walk_next); free(walk_id); free(path); free(prefix); free(sum);
        return -1;
    }
    int64_t nt = 0, nl = 0;
    /* line 2: the root r with r.node = u */
    T[nt++] = (orc_tnode){u, 0, 1, -1, -1, -1, -1};
    /* lines 3-11: insert each walk, one tree level per walk node */
    for (int64_t k = kb; k < ke; ++k) {
        int32_t len = orc_walk(g, u, p->c, p->l_max, p->seed, p->query_id, (uint32_t)k, path);
        if (cnt) { cnt->walks++; cnt->walk_nodes += len; }
        int32_t r = 0;
        T[0].weight++;
        for (int32_t i = 2; i <= len; ++i) {
            int32_t ch = T[r].first_child;
            while (ch >= 0 && T[ch].node != path[i - 1]) ch = T[ch].next_sibling;
            if (ch >= 0) {
                T[ch].weight++; /* lines 7-8 */
            } else {           /* lines 9-10 */
                ch = (int32_t)nt++;
                T[ch] = (orc_tnode){path[i - 1], 1, i, r, -1, T[r].first_child, -1};
                T[r].first_child = ch;
            }
            walk_id[nl] = (int32_t)k; walk_next[nl] = T[ch].walk_head; T[ch].walk_head = (int32_t)nl; ++nl;
            r = ch;
        }
    }
    if (cnt) cnt->tree_nodes += nt - 1;
    /* lines 12-14: probe every root-to-node path (r_1..r_q), q >= 2, weighted by r_q.weight / n_r */
    for (int64_t t = 1; t < nt; ++t) {
        const int32_t q = T[t].depth;
        for (int32_t a = (int32_t)t, d = q; a >= 0; a = T[a].parent, --d) prefix[d - 1] = T[a].node;
        const double wq = (double)T[t].weight;
        orc_set *hj = &w.a, *hj1 = &w.b;
        orc_set_clear(hj);
        orc_set_put(hj, prefix[q - 1], 1.0);
        int switched = 0;
        for (int32_t j = 0; j <= q - 2; ++j) {
            orc_prune(hj, sqrt_c, q, j, p->eps_p, &w.t);
            if (p->probe_mode == 1 || p->probe_mode == 2) {
                int64_t degsum = 0;
                for (int32_t s = 0; s < hj->size; ++s) degsum += orc_out_degree(g, hj->member[s]);
                if (p->probe_mode == 1 || (double)degsum > p->c0 * wq * (double)g->n) {
                    /* Sec. 4.4: the probe switches to the randomized PROBE algorithm (Alg. 3) on the
                     * partial walk (r_1.node .. r_q.node), run once for each of the w walks sharing it */
                    for (int32_t l = T[t].walk_head; l >= 0; l = walk_next[l]) {
                        orc_set *ra = &rw.a, *rb = &rw.b;
                        orc_set_clear(ra);
                        orc_set_put(ra, prefix[q - 1], 1.0); /* Alg. 3 line 2: H_0 = {(u_q, 1)} */
                        for (int32_t jj = 0; jj <= q - 2; ++jj) {
                            orc_rand_level(g, p->c, p->seed, p->query_id, (uint32_t)walk_id[l], q, jj, ra,
                                           prefix[q - jj - 2], rb, &rw.t, cnt);
                            orc_set *tmp = ra; ra = rb; rb = tmp;
                        }
                        for (int32_t s = 0; s < ra->size; ++s) sum[ra->member[s]] += ra->score[ra->member[s]];
                        orc_set_clear(&rw.a);
                        orc_set_clear(&rw.b);
                        orc_set_clear(&rw.t);
                    }
                    switched = 1;
                    if (cnt) cnt->switched++;
                    break;
                }
            }
            orc_det_level(g, sqrt_c, hj, prefix[q - j - 2] /* u_{q-j-1} */, hj1, cnt);
            orc_set *tmp = hj; hj = hj1; hj1 = tmp;
        }
        if (!switched)
            for (int32_t s = 0; s < hj->size; ++s) sum[hj->member[s]] += wq * hj->score[hj->member[s]];
        orc_set_clear(&w.a);
        orc_set_clear(&w.b);
        orc_set_clear(&w.t);
        if (cnt) cnt->probes++;
    }
    for (int32_t v = 0; v < g->n; ++v) out[v] = sum[v] / (double)n_r;
    out[u] = 1.0;
    orc_ws_free(&w);
    orc_ws_free(&rw);
    free(T); free(walk_next); free(walk_id); free(path); free(prefix); free(sum);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Top-k (Def. 2, Sec. 3): the k nodes v != u with the largest estimates, by (estimate desc,    */
/* id asc).  Returns the number written (min(k, n-1)).                                         */
/* ------------------------------------------------------------------------------------------ */
static const double *orc_sort_key;
static int orc_cmp_rank(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (orc_sort_key[x] > orc_sort_key[y]) return -1;
    if (orc_sort_key[x] < orc_sort_key[y]) return 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int32_t orc_topk(const double *s, int32_t n, int32_t u, int32_t k, int32_t *ids, double *vals) {
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!idx) return -1;
    int32_t cnt = 0;
    for (int32_t v = 0; v < n; ++v)
        if (v != u) idx[cnt++] = v;
    orc_sort_key = s;
    qsort(idx, (size_t)cnt, sizeof(int32_t), orc_cmp_rank);
    int32_t kk = k < cnt ? k : cnt;
    for (int32_t t = 0; t < kk; ++t) { ids[t] = idx[t]; vals[t] = s[idx[t]]; }
    free(idx);
    return kk;
}

/* ------------------------------------------------------------------------------------------ */
/* Pairwise Monte Carlo (Sec. 2.2, Eq. 3): r pairs of sqrt(c)-walks from u and v; the fraction */
/* of pairs whose i-th nodes coincide for some i estimates s(u, v).  Walk pair t uses Philox    */
/* keys (seed, key_u) / (seed, key_v) with walk index t, so the pair walks are independent of   */
/* each other and of ProbeSim's own walks when the keys differ.                                */
/* ------------------------------------------------------------------------------------------ */
double orc_pair_mc(const orc_graph *g, int32_t u, int32_t v, double c, int32_t l_max, uint32_t seed, uint32_t key_u,
                   uint32_t key_v, int64_t r) {
    if (u == v) return 1.0;
    int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)l_max);
    int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)l_max);
    if (!pu || !pv) { free(pu); free(pv); return -1.0; }
    int64_t meet = 0;
    for (int64_t t = 0; t < r; ++t) {
        int32_t lu = orc_walk(g, u, c, l_max, seed, key_u, (uint32_t)t, pu);
        int32_t lv = orc_walk(g, v, c, l_max, seed, key_v, (uint32_t)t, pv);
        int32_t l = lu < lv ? lu : lv;
        for (int32_t i = 0; i < l; ++i)
            if (pu[i] == pv[i]) { ++meet; break; }
    }
    free(pu); free(pv);
    return (double)meet / (double)r;
}
