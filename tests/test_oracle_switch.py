"""The best-of-both switch of Sec. 4.4 in the oracle, composed by hand from pinned parts.

Alg. 4 probes every walk prefix (r_1..r_q), q >= 2, once with the weight w of its tree node.  Sec. 4.4 checks,
before each deterministic level j, whether the out-degree sum of H_j exceeds c0 * w * n; a probe that does is
handed to the randomized PROBE (Alg. 3), run once for each of the w walks through the prefix and averaged.
This test rebuilds that sum from the oracle's single-walk generator (Def. 3), its deterministic PROBE (Alg. 2,
pinned by Lemma 2) and its randomized PROBE (Alg. 3, pinned by its mean), deciding every switch with its own
level loop in Python, and requires the batch oracle to return the same estimate and the same switch count."""
import math

import numpy as np
import pytest

from oracle import core
from paper_1709_06955_gb300 import synth

C, SEED, QID, LMAX = 0.6, 3, 17, 64


@pytest.fixture(scope="module")
def small():
    n = 300
    s, d = synth.chung_lu(n, 2500, seed=21)
    outs = [[] for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        outs[a].append(b)
    indeg = np.bincount(d, minlength=n)
    return n, s, d, core.Graph(n, s, d), outs, indeg


def by_hand(n, g, outs, indeg, u, eps, c0, eps_p):
    nr = core.num_walks(C, eps, 0.01, n)
    sc = math.sqrt(C)
    prefixes = {}
    for k in range(nr):
        w = g.walk(u, C, LMAX, SEED, QID, k)
        for q in range(2, len(w) + 1):
            prefixes.setdefault(tuple(int(x) for x in w[:q]), []).append(k)
    total = np.zeros(n)
    switched = 0
    for pre, ks in prefixes.items():
        q, w = len(pre), len(ks)
        H = {pre[-1]: 1.0}
        sw = False
        for j in range(q - 1):
            if eps_p > 0:  # Pruning Rule 2 before descending
                H = {x: s for x, s in H.items() if s * sc ** (q - j - 1) > eps_p}
            if sum(len(outs[x]) for x in H) > c0 * w * n:
                sw = True
                break
            H2 = {}
            for x, s in H.items():
                for v in outs[x]:
                    if v != pre[q - j - 2]:
                        H2[v] = H2.get(v, 0.0) + sc / indeg[v] * s
            H = H2
        if sw:
            switched += 1
            for k in ks:
                total += g.probe_rand(list(pre), C, SEED, QID, k)
        else:
            total += w * g.probe(list(pre), C, eps_p)
    est = total / nr
    est[u] = 1.0
    return est, switched, len(prefixes)


@pytest.mark.parametrize("c0,eps_p", [(0.02, 0.0), (0.05, 0.0), (0.02, 2e-3)])
def test_switch_equals_hand_composition(small, c0, eps_p):
    n, s, d, g, outs, indeg = small
    for u in synth.queries(n, d, 2, seed=31):
        u = int(u)
        got, cnt = g.single_source(u, eps=0.25, seed=SEED, qid=QID, l_max=LMAX, probe_mode=2, c0=c0, eps_p=eps_p,
                                   batch=True)
        want, switched, probes = by_hand(n, g, outs, indeg, u, 0.25, c0, eps_p)
        assert cnt["switched"] == switched
        assert 0 < switched < probes  # both kinds of probe occur
        assert np.max(np.abs(got - want)) < 1e-12
