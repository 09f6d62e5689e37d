"""Full-size workload (R-MAT, n = 2^20, m = 2^24, eps = 0.1, n_r = 3,325) in the launch configuration
the benchmark times: walks and a walk subset's estimate against the oracle, and properties of the full
estimate that hold at any size."""
import numpy as np
import pytest

from gpu_util import TOL, oracle_graph
from paper_1709_06955_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build, probesim
    build.build()
    n, s, d = synth.config_graph("rmat-20")
    G = probesim.Graph(n, s, d)
    qs = synth.queries(n, d, 100, seed=2)
    return n, s, d, G, qs


def test_fullsize_walks_and_walk_subset(big):
    from paper_1709_06955_gb300 import probesim
    n, s, d, G, qs = big
    O = oracle_graph(n, s, d)
    nr = G.num_walks(0.1)
    assert nr == 3325
    for t in (0, 1):
        u = int(qs[t])
        nodes, lens = G.sample_walks(probesim.make_queries([u], eps=0.1, query_ids=[t]))
        for k in range(0, nr, 97):
            ref = O.walk(u, 0.6, 64, 3, t, k)
            assert lens[k] == ref.size and np.array_equal(nodes[k, :ref.size], ref)
        # estimate of walks [0, 12): the oracle runs Alg. 1 on them literally
        part = G.single_source(probesim.make_queries([u], eps=0.1, query_ids=[t], walk_begin=0, walk_end=12))[0]
        ref, _ = O.single_source(u, eps=0.1, seed=3, qid=t, walk_begin=0, walk_end=12)
        assert np.max(np.abs(part - ref)) <= TOL


def test_fullsize_properties(big):
    from paper_1709_06955_gb300 import probesim
    n, s, d, G, qs = big
    u = int(qs[3])
    full = G.single_source(probesim.make_queries([u], eps=0.1, query_ids=[3]))[0]
    assert full[u] == 1.0
    rest = np.delete(full, u)
    assert rest.min() >= 0.0 and rest.max() <= 1.0
    indeg = np.bincount(d, minlength=n)
    roots = np.nonzero(indeg == 0)[0]
    assert np.all(full[roots[roots != u]] == 0.0)  # a node without in-neighbours is in no out-list
    # linearity over walk ranges at full size
    a = G.single_source(probesim.make_queries([u], eps=0.1, query_ids=[3], walk_begin=0, walk_end=1600))[0]
    b = G.single_source(probesim.make_queries([u], eps=0.1, query_ids=[3], walk_begin=1600, walk_end=0))[0]
    tot = a + b
    tot[u] = 1.0
    assert np.max(np.abs(tot - full)) <= 3e-6
