"""Pairwise Monte Carlo on the GPU (Sec. 2.2, Eq. 3) against the oracle's restatement, and the accuracy harness of
Sec. 6 on the GPU's estimates: Power-Method ground truth on a small graph, and the pooling protocol with the GPU
pair estimator as the expert."""
import numpy as np
import pytest

from gpu_util import gpu_graph, oracle_graph
from paper_1709_06955_gb300 import accuracy as A, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build, probesim
    from oracle import build as obuild
    build.build()
    obuild.build()
    probesim.load()


@pytest.fixture(scope="module")
def cl1k():
    n, s, d = synth.config_graph("chunglu-1k")
    return n, s, d


def test_pair_mc_meets_bit_exact(cl1k):
    """The walk pairs follow the same Philox streams as the oracle's pairwise estimator: meet counts are equal."""
    n, s, d = cl1k
    G, O = gpu_graph(n, s, d), oracle_graph(n, s, d)
    rng = np.random.default_rng(5)
    us = synth.queries(n, d, 6, seed=6)
    vs = np.concatenate([rng.integers(0, n, 4), us[:2]]).astype(np.int32)  # two pairs with u = v
    ku = (1000 + np.arange(6)).astype(np.uint32)
    kv = (5000 + np.arange(6)).astype(np.uint32)
    for r, lmax in ((1, 64), (3000, 64), (20000, 3)):
        Gl = G if lmax == 64 else gpu_graph(n, s, d, l_max=lmax)
        meets, est = Gl.pair_mc(us, vs, ku, kv, r)
        for i in range(6):
            ref = O.pair_mc(int(us[i]), int(vs[i]), 0.6, lmax, 3, int(ku[i]), int(kv[i]), r)
            if us[i] == vs[i]:
                assert est[i] == 1.0 and meets[i] == r and ref == 1.0
            else:
                assert meets[i] == round(ref * r) and abs(est[i] - ref) < 1e-6


def test_pair_mc_estimates_simrank(cl1k):
    """r >= ln(1/delta) / (2 eps^2) walk pairs: within eps of the Power Method (Chernoff)."""
    from oracle import power_method
    n, s, d = cl1k
    G = gpu_graph(n, s, d)
    S = power_method.simrank(n, s, d, 0.6, 30)
    us = synth.queries(n, d, 8, seed=7)
    vs = np.array([int(np.argsort(-S[u])[1]) for u in us], np.int32)  # each node's most similar other node
    r = A.mc_walk_pairs(0.01, 1e-4)
    _, est = G.pair_mc(us, vs, np.full(8, 77, np.uint32), 100 + np.arange(8, dtype=np.uint32), r)
    assert np.max(np.abs(est - S[us, vs])) <= 0.01


def test_accuracy_harness_on_gpu(cl1k):
    """Sec. 6's measures of the GPU's top-50 lists (deterministic, switch and randomized PROBE, eps = 0.1) against
    the Power Method, and the pooling protocol (the pair estimator as the expert) measuring the lists about as the Power Method does."""
    from oracle import power_method
    from paper_1709_06955_gb300 import probesim
    n, s, d = cl1k
    S = power_method.simrank(n, s, d, 0.6, 30)
    qs = synth.queries(n, d, 5, seed=2)
    Q = probesim.make_queries(qs, eps=0.1, k=50, query_ids=np.arange(5))
    modes = {"det": {}, "switch": dict(probe_mode=probesim.PROBE_SWITCH, c0=0.01),
             "rand": dict(probe_mode=probesim.PROBE_RANDOMIZED)}
    lists, ests = {}, {}
    for name, kw in modes.items():
        G = gpu_graph(n, s, d, **kw)
        ests[name] = G.single_source(Q)
        lists[name] = G.topk(Q, kmax=50)[0]
        G.close()
    Gx = gpu_graph(n, s, d)
    for t, u in enumerate(qs):
        u = int(u)
        truth = A.true_topk(S[u], u, 50)
        ptruth, pscore = A.pool(Gx, u, [lists[m][t] for m in modes], 50, eps=3e-3, delta=1e-4)
        for name in modes:
            r = A.evaluate(lists[name][t], truth, lambda v, u=u: S[u, v], S[u], ests[name][t], u)
            assert r["abs_error"] <= 0.1 and r["precision"] >= 0.8 and r["ndcg"] >= 0.97
            # pooling can only rank what some method returned: its precision is close to the exact one
            pr = A.precision_at_k(lists[name][t], ptruth)
            assert abs(pr - r["precision"]) <= 0.12
        # the expert's scores follow the Power Method within its error
        assert max(abs(pscore[v] - S[u, v]) for v in pscore) <= 3e-3 * 2
