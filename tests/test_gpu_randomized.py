"""Randomized PROBE (Alg. 3) on the GPU against the oracle.  Every decision is an integer comparison of
Philox words, so the member counts agree exactly: s~ * n_r is the same integer on both sides."""
import numpy as np
import pytest

from gpu_util import oracle_graph
from paper_1709_06955_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build
    from oracle import build as obuild
    build.build()
    obuild.build()


def _rand_graph(n, s, d, **kw):
    from paper_1709_06955_gb300 import probesim
    return probesim.Graph(n, s, d, probe_mode=probesim.PROBE_RANDOMIZED, **kw)


def _exact(gpu, ref, nr, u):
    cg = np.rint(np.delete(gpu.astype(np.float64), u) * nr)
    co = np.rint(np.delete(ref, u) * nr)
    assert np.array_equal(cg, co)
    assert np.max(np.abs(np.delete(gpu, u) - np.delete(ref, u))) <= 1e-6
    assert gpu[u] == 1.0


@pytest.mark.parametrize("graph,eps", [("chunglu-1k", 0.2), ("rmat-10", 0.2), ("rmat-12", 0.3)])
def test_randomized_counts_exact(graph, eps):
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.config_graph(graph)
    G, O = _rand_graph(n, s, d), oracle_graph(n, s, d)
    qs = synth.queries(n, d, 4, seed=21)
    out = G.single_source(probesim.make_queries(qs, eps=eps, query_ids=np.arange(4) + 40))
    nr = G.num_walks(eps)
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=eps, seed=3, qid=40 + t, probe_mode=1)
        _exact(out[t], ref, nr, int(u))


def test_randomized_alone_equals_mixed_exactly():
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.config_graph("chunglu-1k")
    G = _rand_graph(n, s, d)
    qs = synth.queries(n, d, 6, seed=22)
    eps = [0.2, 0.3, 0.25, 0.2, 0.3, 0.25]
    mix = G.single_source(probesim.make_queries(qs, eps=eps, query_ids=np.arange(6)))
    for i in range(6):
        alone = G.single_source(probesim.make_queries([qs[i]], eps=eps[i], query_ids=[i]))
        assert np.array_equal(alone[0], mix[i])


def test_randomized_edge_cases():
    from paper_1709_06955_gb300 import probesim
    n = 40
    rng = np.random.default_rng(9)
    s = rng.integers(0, n, 300).astype(np.int32)
    d = rng.integers(0, n, 300).astype(np.int32)
    d[d == 0] = 1
    from gpu_util import dedup
    ds, dd = dedup(n, s, d)
    O = oracle_graph(n, ds, dd)
    for lmax in (1, 2, 5, 64):
        G = _rand_graph(n, s, d, l_max=lmax)
        for u in (0, 3):
            out = G.single_source(probesim.make_queries([u], eps=0.3, query_ids=[u]))[0]
            ref, _ = O.single_source(u, eps=0.3, l_max=lmax, seed=3, qid=u, probe_mode=1)
            _exact(out, ref, G.num_walks(0.3), u)
