"""Thm. 2's parameter split (probesim_split_error, host arithmetic) and the facts it rests on, pinned against
the oracle.

- The split satisfies Thm. 2's inequality: eps + T_p + (eps_t/2 with the shift, else eps_t) <= eps_a, with the
  corrected Rule-2 term T_p = (1+eps) sqrt(c)/(1-sqrt(c))^2 eps_p, and l_max is the shortest truncation with
  sqrt(c)^l_max <= eps_t.
- E[l(l-1)/2] = sqrt(c)/(1-sqrt(c))^2 for the length l of a sqrt(c)-walk (Def. 3: it stops at each node with
  probability 1 - sqrt(c)): checked on the oracle's walks over a graph where every node has an in-neighbour.
- Rule 2 removes at most (i-1) eps_p from the probe of a prefix of length i (the per-probe bound that holds,
  see the lemma in the proof of Thm. 2), so a query's pruned estimate lies below the unpruned one by at most
  eps_p times the mean over its walks of l(l-1)/2: checked exactly on the oracle with the same walks.
"""
import math

import numpy as np
import pytest

from oracle import core
from paper_1709_06955_gb300 import probesim, synth


@pytest.mark.parametrize("c", [0.36, 0.6, 0.8])
@pytest.mark.parametrize("shift", [True, False])
def test_split_satisfies_thm2(c, shift):
    sc = math.sqrt(c)
    for eps_a in (0.5, 0.2, 0.1, 0.05, 0.0125):
        r = probesim.split_error(eps_a, c, shift)
        tp = (1 + r["eps"]) * sc / (1 - sc) ** 2 * r["eps_p"]
        r1 = sc ** r["l_max"]
        assert r1 <= r["eps_t"] * (1 + 1e-12) and (r["l_max"] == 1 or sc ** (r["l_max"] - 1) > r["eps_t"])
        total = r["eps"] + tp + (r1 / 2 if shift else r1)
        assert abs(total - r["bound"]) <= 1e-12 and r["bound"] <= eps_a
        assert r["bound_paper"] <= r["bound"]  # the paper's T_p is the smaller term
        assert r["eps"] == eps_a / 2 and r["eps_p"] > 0
        assert (r["shift"] == np.float32(r["eps_t"] / 2)) if shift else r["shift"] == 0


def test_split_rejects_bad_arguments():
    for bad in ((0.0, 0.6), (1.0, 0.6), (0.1, 0.0), (0.1, 1.0)):
        with pytest.raises(probesim.ProbeSimError):
            probesim.split_error(*bad)


def test_walk_length_second_moment():
    """E[l(l-1)/2] of a sqrt(c)-walk equals sqrt(c)/(1-sqrt(c))^2 (geometric length, Def. 3)."""
    n = 64
    s = np.arange(n, dtype=np.int32)
    d = ((np.arange(n) + 1) % n).astype(np.int32)  # a directed cycle: every node has an in-neighbour
    s2, d2 = np.arange(0, n, 2, dtype=np.int32), ((np.arange(0, n, 2) + 5) % n).astype(np.int32)
    g = core.Graph(n, np.concatenate([s, s2]), np.concatenate([d, d2]))
    c = 0.6
    sc = math.sqrt(c)
    vals = np.array([(lambda w: w.size * (w.size - 1) / 2)(g.walk(3, c, 255, 11, 7, k)) for k in range(40000)])
    want = sc / (1 - sc) ** 2
    assert abs(vals.mean() - want) <= 5 * vals.std() / math.sqrt(vals.size)


def test_rule2_error_per_walk_bound():
    s, d = synth.chung_lu(300, 2500, seed=21)
    g = core.Graph(300, s, d)
    c, eps, lmax = 0.6, 0.2, 64
    nr = core.num_walks(c, eps, 0.01, 300)
    for u in synth.queries(300, d, 3, seed=23):
        u = int(u)
        mean_pairs = np.mean([(lambda w: w.size * (w.size - 1) / 2)(g.walk(u, c, lmax, 3, u, k)) for k in range(nr)])
        full, _ = g.single_source(u, eps=eps, qid=u, l_max=lmax)
        for eps_p in (1e-3, 1e-2):
            pruned, _ = g.single_source(u, eps=eps, qid=u, l_max=lmax, eps_p=eps_p)
            diff = np.delete(full - pruned, u)
            assert diff.min() >= -1e-12 and diff.max() <= eps_p * mean_pairs + 1e-12
