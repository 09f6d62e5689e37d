"""Accuracy measures of Sec. 6 and the pooling evaluation of its large-graph experiments.

Host-side numpy over estimates the library returns.  ``s_true`` is a ground truth: exact SimRank where it can be
computed (the Power Method on small graphs), otherwise the pooled expert scores below.

* ``abs_error``: max over v != u of |s(u, v) - s~(u, v)| (the AbsError of a single-source query).
* ``precision_at_k``: |V_k intersect V'_k| / k, V_k the returned top-k, V'_k the true top-k.
* ``ndcg_at_k``: (1/Z_k) sum_{i<=k} (2^{s(u, v_i)} - 1) / log2(i + 1), with Z_k the same sum over V'_k.  The paper
  prints the normaliser's gain as 2^{s-1}; the gain 2^s - 1 is used in both sums, so a perfect list scores 1.
* ``kendall_tau_k``: (concordant - discordant pairs) / (k(k-1)/2) over the pairs of the returned list, a pair
  concordant when the list orders it as the true scores do; pairs with equal true scores count as neither.
* ``pool``: the union of several methods' top-k lists (duplicates removed), gauged by a single-pair estimator
  (the pairwise Monte Carlo of Sec. 2.2 on the GPU) with r = ceil(ln(1/delta) / (2 eps^2)) walk pairs per node;
  its best k are the ground truth top-k the methods are measured against.
"""
import math

import numpy as np


def abs_error(s_true, s_est, u):
    d = np.abs(np.asarray(s_true, np.float64) - np.asarray(s_est, np.float64))
    d[u] = 0.0
    return float(d.max())


def true_topk(s_true, u, k):
    """The k nodes v != u with the largest true scores (ties by smaller id)."""
    s = np.asarray(s_true, np.float64)
    order = [int(v) for v in np.lexsort((np.arange(s.size), -s)) if v != u]
    return np.array(order[:k], np.int64)


def precision_at_k(returned, truth_topk):
    k = len(truth_topk)
    return len(set(int(x) for x in returned[:k]) & set(int(x) for x in truth_topk)) / float(k)


def ndcg_at_k(returned, truth_topk, s_of):
    """s_of(v) gives the true score of node v."""
    k = len(truth_topk)
    disc = [1.0 / math.log2(i + 2) for i in range(k)]
    dcg = sum((2.0 ** s_of(int(v)) - 1.0) * disc[i] for i, v in enumerate(returned[:k]))
    z = sum((2.0 ** s_of(int(v)) - 1.0) * disc[i] for i, v in enumerate(truth_topk[:k]))
    return dcg / z if z > 0 else 1.0


def kendall_tau_k(returned, s_of):
    r = [int(v) for v in returned]
    k = len(r)
    if k < 2:
        return 1.0
    con = dis = 0
    for i in range(k):
        for j in range(i + 1, k):
            a, b = s_of(r[i]), s_of(r[j])
            if a > b:
                con += 1
            elif a < b:
                dis += 1
    return (con - dis) / (k * (k - 1) / 2.0)


def mc_walk_pairs(eps, delta):
    """Walk pairs of the pairwise Monte Carlo for error eps with probability 1 - delta (Chernoff, Sec. 2.2)."""
    return int(math.ceil(math.log(1.0 / delta) / (2.0 * eps * eps)))


def pool(graph, u, lists, k, eps=2e-3, delta=1e-4, key_base=1 << 30):
    """Pooled ground truth for query node u: the union of the top-k ``lists`` gauged by the GPU pairwise Monte
    Carlo (``graph.pair_mc``).  Returns (truth top-k ids, dict node -> expert score)."""
    cand = sorted({int(v) for lst in lists for v in lst[:k] if int(v) != u and int(v) >= 0})
    r = mc_walk_pairs(eps, delta)
    cu = np.full(len(cand), u, np.int32)
    ku = np.full(len(cand), key_base, np.uint32)
    kv = (key_base + 1 + np.arange(len(cand))).astype(np.uint32)
    _, est = graph.pair_mc(cu, np.array(cand, np.int32), ku, kv, r)
    score = {v: float(e) for v, e in zip(cand, est)}
    order = sorted(cand, key=lambda v: (-score[v], v))
    return np.array(order[:k], np.int64), score


def evaluate(returned, truth_topk, s_of, s_true=None, s_est=None, u=None):
    """All measures of one top-k list; AbsError too when full score vectors are given."""
    out = {"precision": precision_at_k(returned, truth_topk), "ndcg": ndcg_at_k(returned, truth_topk, s_of),
           "tau": kendall_tau_k(returned, s_of)}
    if s_true is not None and s_est is not None:
        out["abs_error"] = abs_error(s_true, s_est, u)
    return out
