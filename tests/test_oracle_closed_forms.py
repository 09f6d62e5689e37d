"""Pins the oracle's whole estimator (Alg. 1) on graphs where Eq. 1 has a closed form and where the
estimate is fixed exactly by the number of walks that take a step."""
import math

import numpy as np
import pytest

from oracle import core, power_method


def _moving_walks(g, u, c, n_r, l_max, seed, qid):
    return sum(1 for k in range(n_r) if len(g.walk(u, c, l_max, seed, qid, k)) >= 2)


@pytest.mark.parametrize("d", [1, 2, 5])
def test_shared_root_parents(d):
    """u and v with the same d in-neighbours, all of them roots: Eq. 1 gives s(u,v) = c/d.  Every walk
    from u that moves reaches a root x_i, and PROBE(u, x_i) gives v the score sqrt(c)/d, so
    s~(u,v) = sqrt(c)/d * (#moving walks)/n_r exactly."""
    c, eps, delta = 0.6, 0.1, 0.01
    n = d + 2
    u, v = d, d + 1
    src = [x for x in range(d) for _ in (0, 1)]
    dst = [u, v] * d
    g = core.Graph(n, src, dst)
    est, cnt = g.single_source(u, c=c, eps=eps, delta=delta, l_max=64, seed=7, qid=11)
    n_r = core.num_walks(c, eps, delta, n)
    moving = _moving_walks(g, u, c, n_r, 64, 7, 11)
    assert est[v] == pytest.approx(math.sqrt(c) / d * moving / n_r, abs=1e-14)
    assert est[u] == 1.0
    assert all(est[x] == 0.0 for x in range(d))  # roots: no in-neighbour, never scored
    S = power_method.simrank(n, src, dst, c, 40)
    assert S[u, v] == pytest.approx(c / d, abs=1e-12)
    # and the estimate is within eps of it (Thm. 1; here the error is binomial in the moving count)
    assert abs(est[v] - c / d) <= eps


def test_query_without_in_neighbours():
    """|I(u)| = 0: every walk is (u), no probe runs, s~(u, .) = e_u."""
    g = core.Graph(3, [0, 0], [1, 2])
    est, cnt = g.single_source(0)
    assert est.tolist() == [1.0, 0.0, 0.0]
    assert cnt["probes"] == 0


def test_self_similarity_and_range():
    from paper_1709_06955_gb300 import synth
    s, d = synth.chung_lu(200, 1500, seed=5)
    g = core.Graph(200, s, d)
    u = int(synth.queries(200, d, 1, seed=3)[0])
    est, _ = g.single_source(u, eps=0.2)
    assert est[u] == 1.0
    others = np.delete(est, u)
    assert np.all(others >= 0.0) and np.all(others <= 1.0)  # each trial's estimator is in [0,1] (Thm. 1 proof)


def test_num_walks_meets_chernoff_exactly():
    """n_r is the smallest integer with exp(-eps^2 n_r / (3c)) <= delta/n (the step in Thm. 1's proof)."""
    for (c, eps, delta, n) in [(0.6, 0.1, 0.01, 1000), (0.6, 0.1, 0.01, 1 << 20), (0.6, 0.05, 0.01, 1 << 22),
                               (0.6, 0.025, 0.01, 1 << 23), (0.8, 0.2, 0.1, 50)]:
        n_r = core.num_walks(c, eps, delta, n)
        assert math.exp(-eps * eps * n_r / (3 * c)) <= delta / n * (1 + 1e-12)
        assert math.exp(-eps * eps * (n_r - 1) / (3 * c)) > delta / n
    assert core.num_walks(0.6, 0.1, 0.01, 1000) == 2073
