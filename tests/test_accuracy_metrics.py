"""The accuracy measures of Sec. 6 on hand-checked cases, and the harness on the oracle's ProbeSim against the
Power Method (CPU)."""
import math

import numpy as np

from oracle import core, power_method
from paper_1709_06955_gb300 import accuracy as A, synth


def test_precision_counts_common_members():
    assert A.precision_at_k([1, 2, 3, 4], [4, 3, 9, 8]) == 0.5
    assert A.precision_at_k([5, 6], [6, 5]) == 1.0


def test_ndcg_hand_example():
    s = {1: 0.5, 2: 0.25, 3: 0.0, 4: 0.75}
    got = A.ndcg_at_k([1, 2, 3], [4, 1, 2], s.get)
    g = lambda x: 2.0 ** x - 1.0  # noqa: E731
    dcg = g(0.5) / math.log2(2) + g(0.25) / math.log2(3) + g(0.0) / math.log2(4)
    z = g(0.75) / math.log2(2) + g(0.5) / math.log2(3) + g(0.25) / math.log2(4)
    assert abs(got - dcg / z) < 1e-15
    assert A.ndcg_at_k([4, 1, 2], [4, 1, 2], s.get) == 1.0


def test_kendall_tau_extremes_and_ties():
    s = {i: 1.0 - 0.1 * i for i in range(6)}
    assert A.kendall_tau_k([0, 1, 2, 3], s.get) == 1.0
    assert A.kendall_tau_k([3, 2, 1, 0], s.get) == -1.0
    assert abs(A.kendall_tau_k([0, 2, 1, 3], s.get) - (5 - 1) / 6.0) < 1e-15
    assert A.kendall_tau_k([7, 8], {7: 0.3, 8: 0.3}.get) == 0.0  # a tie is neither concordant nor discordant


def test_abs_error_skips_the_query_node():
    assert abs(A.abs_error([1.0, 0.2, 0.3], [0.0, 0.25, 0.1], 0) - 0.2) < 1e-15


def test_walk_pairs_follow_chernoff():
    r = A.mc_walk_pairs(0.01, 0.001)
    assert r == math.ceil(math.log(1000) / (2 * 1e-4))
    assert 2 * r * 0.01 ** 2 >= math.log(1000)


def test_harness_on_the_oracle_against_the_power_method():
    """Sec. 6's small-graph protocol on the 1,000-node Chung-Lu graph: ProbeSim (the oracle, eps = 0.1) against the
    Power Method: every query's AbsError within eps and high top-50 Precision, NDCG and Kendall tau."""
    n, s, d = synth.config_graph("chunglu-1k")
    g = core.Graph(n, s, d)
    S = power_method.simrank(n, s, d, 0.6, 30)
    res = []
    for t, u in enumerate(synth.queries(n, d, 5, seed=2)):
        u = int(u)
        est, _ = g.single_source(u, eps=0.1, seed=3, qid=t)
        ids, _ = core.topk(est, u, 50)
        truth = A.true_topk(S[u], u, 50)
        res.append(A.evaluate(ids, truth, lambda v, u=u: S[u, v], S[u], est, u))
    assert all(r["abs_error"] <= 0.1 for r in res)
    assert np.mean([r["precision"] for r in res]) >= 0.9
    assert np.mean([r["ndcg"] for r in res]) >= 0.99
    assert np.mean([r["tau"] for r in res]) >= 0.75
