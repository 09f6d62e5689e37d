"""Pins the oracle against the paper's lemmas by exact enumeration on tiny graphs."""
import math

import numpy as np
import pytest

from oracle import core, enumerate as en, power_method


def _random_graph(rng, n, p):
    src, dst = [], []
    for x in range(n):
        for v in range(n):
            if x != v and rng.random() < p:
                src.append(x)
                dst.append(v)
    return src, dst


def _random_walk_path(rng, I, u, length):
    path = [u]
    while len(path) < length and I[path[-1]]:
        path.append(int(rng.choice(I[path[-1]])))
    return path


def test_lemma2_probe_is_first_meeting_probability():
    """Lemma 2: PROBE(u_1..u_i) gives every v != u_1 exactly P(v, (u_1..u_i)) of Def. 4."""
    rng = np.random.default_rng(0)
    checked = 0
    for trial in range(40):
        n = int(rng.integers(3, 8))
        src, dst = _random_graph(rng, n, 0.45)
        if not src:
            continue
        g = core.Graph(n, src, dst)
        I = en.in_lists(n, src, dst)
        c = float(rng.choice([0.25, 0.6, 0.8]))
        for _ in range(4):
            u = int(rng.integers(n))
            path = _random_walk_path(rng, I, u, int(rng.integers(2, 7)))
            if len(path) < 2:
                continue
            score = g.probe(path, c)
            for v in range(n):
                if v == path[0]:
                    assert score[v] == 0.0  # the last level excludes u_1 = u
                    continue
                assert score[v] == pytest.approx(en.first_meeting(I, c, v, path), abs=1e-13)
                checked += 1
    assert checked > 300


def test_lemma1_estimator_is_unbiased():
    """Lemma 1: summing Pr[W] * sum_{i>=2} PROBE(W(u,i)) over every walk W(u) gives s(u,v).  With walks
    cut at L nodes the gap is one-sided and at most sqrt(c)^L (Pruning Rule 1 lemma)."""
    rng = np.random.default_rng(1)
    c, L = 0.36, 11
    for trial in range(4):
        n = 5
        src, dst = _random_graph(rng, n, 0.5)
        g = core.Graph(n, src, dst)
        I = en.in_lists(n, src, dst)
        S = power_method.simrank(n, src, dst, c, 80)
        u = int(rng.integers(n))
        walks = en.walks(I, c, u, L)
        assert sum(p for _, p in walks) == pytest.approx(1.0, abs=1e-12)
        exp = np.zeros(n)
        for path, p in walks:
            for i in range(2, len(path) + 1):
                exp += p * g.probe(list(path[:i]), c)
        for v in range(n):
            if v == u:
                continue
            gap = S[u, v] - exp[v]
            assert -1e-12 <= gap <= math.sqrt(c) ** L + 1e-12, (trial, u, v, S[u, v], exp[v])


def test_pruning_rule2_is_one_sided_per_probe():
    """Pruning Rule 2 only removes score: 0 <= Score_i(x) - Score_i(x, eps_p).  The lemma in the proof
    of Thm. 2 states an upper bound of eps_p per probe, but its induction leaves out the score removed
    by pruning at each later level; each of the i-1 pruned levels removes at most eps_p of the final
    score (a walk from x is at one node per step), so the bound that holds is (i-1) * eps_p.  The
    oracle exceeds eps_p alone on this graph (about 1.3 eps_p at eps_p = 1e-2)."""
    from paper_1709_06955_gb300 import synth
    rng = np.random.default_rng(2)
    s, d = synth.chung_lu(300, 3000, seed=9)
    g = core.Graph(300, s, d)
    I = en.in_lists(300, s, d)
    worst = 0.0
    for _ in range(30):
        u = int(rng.integers(300))
        path = _random_walk_path(rng, I, u, int(rng.integers(2, 9)))
        if len(path) < 2:
            continue
        for eps_p in (1e-4, 1e-3, 1e-2):
            diff = g.probe(path, 0.6) - g.probe(path, 0.6, eps_p=eps_p)
            assert diff.min() >= -1e-15 and diff.max() <= (len(path) - 1) * eps_p + 1e-15
            worst = max(worst, diff.max() / eps_p)
    assert worst > 1.0  # the per-probe bound eps_p of the paper's lemma is exceeded


def test_pruning_rule1_is_one_sided_per_walk():
    """Lemma in the proof of Thm. 2: truncating a walk at l_t nodes changes its estimator by a value in
    [0, sqrt(c)^l_t]."""
    from paper_1709_06955_gb300 import synth
    s, d = synth.chung_lu(300, 3000, seed=9)
    g = core.Graph(300, s, d)
    c = 0.6
    u = int(synth.queries(300, d, 1, seed=4)[0])
    for k in range(200):
        full = g.walk(u, c, 64, 5, 6, k)
        for l_t in (2, 3, 4):
            if len(full) <= l_t:
                continue
            trunc = g.walk(u, c, l_t, 5, 6, k)
            assert list(trunc) == list(full[:l_t])  # the same draws: truncation is a prefix
            e_full = sum(g.probe(full[:i], c) for i in range(2, len(full) + 1))
            e_trunc = sum(g.probe(trunc[:i], c) for i in range(2, len(trunc) + 1)) if l_t >= 2 else 0
            diff = e_full - e_trunc
            assert diff.min() >= -1e-13 and diff.max() <= math.sqrt(c) ** l_t + 1e-13


def test_randomized_probe_mean_is_deterministic_probe():
    """Lemma in the proof of Thm. 3: the randomized PROBE sets Score(v) = 1 with probability
    P(v, W(u,i)) = the deterministic Score(v).  Mean over 4000 instances, within 5 sigma."""
    from paper_1709_06955_gb300 import synth
    s, d = synth.chung_lu(120, 900, seed=13)
    g = core.Graph(120, s, d)
    I = en.in_lists(120, s, d)
    rng = np.random.default_rng(3)
    c = 0.6
    N = 4000
    for _ in range(3):
        u = int(synth.queries(120, d, 1, seed=int(rng.integers(100)))[0])
        path = _random_walk_path(rng, I, u, 4)
        if len(path) < 3:
            continue
        det = g.probe(path, c)
        mean = np.zeros(120)
        for k in range(N):
            r = g.probe_rand(path, c, 17, 23, k)
            assert set(np.unique(r)) <= {0.0, 1.0}
            mean += r
        mean /= N
        sig = np.sqrt(np.maximum(det * (1 - det), 1.0 / N) / N)
        assert np.all(np.abs(mean - det) <= 5 * sig + 1e-12)
