"""Pins the oracle's Philox4x32-10 and walk sampler by their statistics (no published answer vectors
are available here), and the walk sampler by its first-step distribution (Def. 3)."""
import math

import numpy as np
import pytest

from oracle import core
from paper_1709_06955_gb300 import synth


def _words(n, key=(3, 5), hi=0):
    return np.array([core.philox([k, hi, 0, 0], key) for k in range(n)], dtype=np.uint64)


def test_uniform_bytes_chi2():
    w = _words(20000)
    b = np.concatenate([((w >> s) & 0xFF).ravel() for s in (0, 8, 16, 24)])
    counts = np.bincount(b.astype(np.int64), minlength=256)
    exp = b.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)  # mean 255, sd sqrt(510)


def test_no_collisions_across_counters_and_keys():
    a = _words(20000)
    b = _words(20000, key=(3, 6))
    c = _words(20000, key=(4, 5))
    d = _words(20000, hi=1)
    packed = [tuple(r) for x in (a, b, c, d) for r in x]
    assert len(set(packed)) == len(packed)


def test_avalanche():
    """Flipping one input bit flips about half of the 128 output bits (16 of 32 per word)."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(400):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        base = core.philox(ctr, key)
        which = int(rng.integers(6))
        bit = np.uint32(1 << int(rng.integers(32)))
        c2, k2 = ctr.copy(), key.copy()
        if which < 4:
            c2[which] ^= bit
        else:
            k2[which - 4] ^= bit
        out = core.philox(c2, k2)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(base, out)))
    assert 62 <= np.mean(flips) <= 66


def test_walk_first_step_distribution():
    """From u, a walk stops at once with probability 1 - sqrt(c); otherwise its second node is uniform
    over I(u) (Def. 3)."""
    c = 0.6
    s, d = synth.chung_lu(400, 4000, seed=2)
    g = core.Graph(400, s, d)
    indeg = np.bincount(d, minlength=400)
    u = int(np.argmax(indeg))
    nbrs = sorted(int(x) for x in s[d == u])
    N = 30000
    second = {}
    stops = 0
    for k in range(N):
        w = g.walk(u, c, 64, 11, 12, k)
        if len(w) == 1:
            stops += 1
        else:
            second[int(w[1])] = second.get(int(w[1]), 0) + 1
    p = 1 - math.sqrt(c)
    assert abs(stops / N - p) < 5 * math.sqrt(p * (1 - p) / N)
    assert set(second) <= set(nbrs)
    moved = N - stops
    exp = moved / len(nbrs)
    chi2 = sum((second.get(x, 0) - exp) ** 2 / exp for x in nbrs)
    dof = len(nbrs) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_walk_length_distribution():
    """On a graph where every node has an in-neighbour the length is geometric: P(l >= t) = sqrt(c)^(t-1)."""
    n = 50
    src = [(v + 1) % n for v in range(n)] + [(v + 7) % n for v in range(n)]
    dst = list(range(n)) * 2
    g = core.Graph(n, src, dst)
    c = 0.6
    N = 20000
    lens = np.array([len(g.walk(0, c, 64, 1, 2, k)) for k in range(N)])
    for t in (2, 3, 5, 8):
        p = math.sqrt(c) ** (t - 1)
        assert abs((lens >= t).mean() - p) < 5 * math.sqrt(p * (1 - p) / N)
    assert lens.max() <= 64
    assert (g.walk(0, c, 3, 1, 2, 0).size) <= 3
