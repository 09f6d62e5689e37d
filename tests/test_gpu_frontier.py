"""The frontier engine through the C ABI: every walk prefix probed on its own (Alg. 4 running Alg. 2), with
Pruning Rule 2 (Sec. 4.1) and the best-of-both switch of Sec. 4.4, against the FP64 oracle.

Tolerances:
- eps_p = 0: the frontier sets are exact and every switch decision compares an integer out-degree sum with
  the same FP64 threshold, so the switch counts match exactly and the scores within 1e-5 (FP32 products
  summed in fixed point against FP64).
- eps_p > 0: a pruning decision taken in FP32 can differ from the FP64 one for a score within rounding of the
  threshold.  Each such flip moves the estimate by at most the pruned score mass, so the bound is
  1e-5 + (1+eps)/(1-sqrt(c)) * eps_p, the Rule-2 term of Thm. 2.  Round thresholds tie exactly in real
  arithmetic with products such as c/600 = 1e-3 (c = 0.6, in-degrees 20 and 30), and then the two roundings
  decide the tie; the thresholds below (1.1e-4, 1.3e-3, 1.7e-2) have no such ties, so flips stay rare.
"""
import math

import numpy as np
import pytest

from gpu_util import TOL, gpu_graph, oracle_graph
from paper_1709_06955_gb300 import synth

pytestmark = pytest.mark.gpu
C = 0.6


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


def _q(nodes, **kw):
    from paper_1709_06955_gb300 import probesim
    return probesim.make_queries(nodes, **kw)


def _f32(x):
    return float(np.float32(x))


def _prune_tol(eps, eps_p):
    return TOL + (1 + eps) / (1 - math.sqrt(C)) * eps_p


@pytest.fixture(scope="module")
def cl1k():
    n, s, d = synth.config_graph("chunglu-1k")
    return n, s, d, oracle_graph(n, s, d)


@pytest.fixture(scope="module")
def rmat12():
    n, s, d = synth.rmat(12, 16 << 12, seed=12)
    return n, s, d, oracle_graph(n, s, d)


@pytest.mark.parametrize("c0", [0.0, 0.002, 0.02, 1e30])
def test_switch_matches_oracle(cl1k, c0):
    """Sec. 4.4 at both extremes and in between: scores within 1e-5, switch counts exact."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = cl1k
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=c0)
    qs = synth.queries(n, d, 4, seed=41)
    out = G.single_source(_q(qs, eps=0.15, query_ids=np.arange(4) + 300))
    gsw = G.stats()["switched"]
    osw = 0
    for t, u in enumerate(qs):
        ref, cnt = O.single_source(int(u), eps=0.15, seed=3, qid=300 + t, probe_mode=2, c0=_f32(c0), batch=True)
        osw += cnt["switched"]
        assert out[t][u] == 1.0
        assert np.max(np.abs(out[t] - ref)) <= TOL
    assert gsw == osw
    if c0 == 1e30:
        assert gsw == 0
    if c0 == 0.02:
        assert 0 < gsw < G.stats()["probes"]
    G.close()


def test_switch_extremes_equal_the_other_engines(cl1k):
    """c0 = 0 hands every probe with out-edges to Alg. 3 at level 0: the randomized engine's result, bit for bit
    (integer member counts).  c0 = 1e30 never switches: the deterministic (regrouped) engine within 1e-5."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = cl1k
    qs = synth.queries(n, d, 3, seed=42)
    Q = _q(qs, eps=0.2, query_ids=[5, 6, 7])
    rand = gpu_graph(n, s, d, probe_mode=probesim.PROBE_RANDOMIZED).single_source(Q)
    sw0 = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.0).single_source(Q)
    assert np.array_equal(rand, sw0)
    det = gpu_graph(n, s, d).single_source(Q)
    swinf = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=1e30).single_source(Q)
    assert np.max(np.abs(det - swinf)) <= TOL


@pytest.mark.parametrize("eps_p", [1.1e-4, 1.3e-3, 1.7e-2])
def test_pruning_rule2_matches_oracle(cl1k, eps_p):
    """Deterministic PROBE with Rule 2 on the GPU against the oracle's Alg. 1 with the same eps_p.

    Pruning is monotone: a larger threshold drops a superset of entries, every score is a sum of nonnegative
    terms, so the estimate cannot grow with eps_p.  The GPU's FP32 comparisons act like FP64 comparisons
    against a threshold within a relative r of eps_p (a few roundings per level, far below r = 1e-5), so its
    estimate lies between the oracle's at eps_p (1 + r) and at eps_p (1 - r), up to 1e-5.  Near a large
    threshold that sandwich is wider than 1e-5 (at 1.7e-2 the oracle moves by ~2.5e-4 when eps_p moves by one
    part in a million), which is why the element-wise bound alone is the Rule-2 term of Thm. 2."""
    n, s, d, O = cl1k
    G = gpu_graph(n, s, d, eps_p=eps_p)
    qs = synth.queries(n, d, 4, seed=43)
    out = G.single_source(_q(qs, eps=0.15, query_ids=np.arange(4) + 400))
    e32, r = _f32(eps_p), 1e-5
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=0.15, seed=3, qid=400 + t, eps_p=e32)
        lo, _ = O.single_source(int(u), eps=0.15, seed=3, qid=400 + t, eps_p=e32 * (1 + r))
        hi, _ = O.single_source(int(u), eps=0.15, seed=3, qid=400 + t, eps_p=e32 * (1 - r))
        assert np.max(np.abs(out[t] - ref)) <= _prune_tol(0.15, eps_p)
        assert np.all(out[t] >= lo - TOL) and np.all(out[t] <= hi + TOL)
    # pruning removes score: the pruned estimate is below the unpruned one up to rounding (one-sided, Sec. 4.1)
    full = gpu_graph(n, s, d).single_source(_q(qs, eps=0.15, query_ids=np.arange(4) + 400))
    assert np.all(out <= full + TOL)
    G.close()


def test_switch_with_pruning_matches_oracle(rmat12):
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = rmat12
    eps_p = 1.3e-3
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.05, eps_p=eps_p)
    qs = synth.queries(n, d, 3, seed=44)
    out = G.single_source(_q(qs, eps=0.2, query_ids=[11, 12, 13]))
    gsw = G.stats()["switched"]
    osw = 0
    for t, u in enumerate(qs):
        ref, cnt = O.single_source(int(u), eps=0.2, seed=3, qid=11 + t, probe_mode=2, c0=_f32(0.05),
                                   eps_p=_f32(eps_p), batch=True)
        osw += cnt["switched"]
        assert np.max(np.abs(out[t] - ref)) <= _prune_tol(0.2, eps_p)
    assert abs(gsw - osw) <= max(1, osw // 100)


@pytest.mark.parametrize("scale,eps,c0", [(10, 0.1, 0.01), (12, 0.15, 0.1), (13, 0.2, 1.0)])
def test_switch_rmat(scale, eps, c0):
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.rmat(scale, 16 << scale, seed=scale)
    O = oracle_graph(n, s, d)
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=c0)
    qs = synth.queries(n, d, 2, seed=scale + 2)
    out = G.single_source(_q(qs, eps=eps, query_ids=[21, 22]))
    gsw = G.stats()["switched"]
    osw = 0
    for t, u in enumerate(qs):
        ref, cnt = O.single_source(int(u), eps=eps, seed=3, qid=21 + t, probe_mode=2, c0=_f32(c0), batch=True)
        osw += cnt["switched"]
        assert np.max(np.abs(out[t] - ref)) <= TOL
    assert gsw == osw


def test_batch_equals_alone_bit_for_bit(cl1k):
    """Fixed-point sums are exact in any order, so a query's estimate is the same bits alone and in a mixed
    batch with uneven eps (and n_r)."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = cl1k
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.02, eps_p=1e-4)
    qs = synth.queries(n, d, 9, seed=45)
    eps = np.where(np.arange(9) % 3 == 0, 0.1, np.where(np.arange(9) % 3 == 1, 0.2, 0.15))
    Q = _q(qs, eps=eps, query_ids=np.arange(9) * 7 + 2)
    mix = G.single_source(Q)
    again = G.single_source(Q)
    assert np.array_equal(mix, again)
    for i in (0, 4, 8):
        alone = G.single_source(_q([qs[i]], eps=eps[i], query_ids=[i * 7 + 2]))
        assert np.array_equal(alone[0], mix[i])


def test_level_table_in_passes(rmat12):
    """A small memory budget cuts every level's table into several passes (and the call into batches); the
    estimates do not change."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = rmat12
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=1.0, eps_p=1e-4)
    qs = synth.queries(n, d, 4, seed=46)
    Q = _q(qs, eps=0.2, query_ids=[31, 32, 33, 34])
    ref = G.single_source(Q)
    whole = G.stats()
    G.set_memory_budget(48 * 12 * n)  # passes of 12 n slots, frontiers of 6 n entries before a range is deferred
    cut = G.single_source(Q)
    parts = G.stats()
    G.set_memory_budget(0)
    assert whole["max_table_slots"] > 12 * n  # the default budget took each level in one pass
    assert whole["table_passes"] <= whole["levels"] and whole["deferred"] == 0
    assert parts["table_passes"] > 2 * whole["table_passes"]
    assert parts["deferred"] > 0
    assert np.array_equal(ref, cut)


def test_randomized_walk_ranges_under_a_small_budget(rmat12):
    """Alg. 3 for the switched probes (and for the all-randomized mode) is cut into walk ranges when a level's
    hash sets exceed the budget; the integer member counts, hence the estimates, do not change."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = rmat12
    qs = synth.queries(n, d, 3, seed=47)
    Q = _q(qs, eps=0.15, query_ids=[41, 42, 43])
    for kw in (dict(probe_mode=probesim.PROBE_SWITCH, c0=0.01), dict(probe_mode=probesim.PROBE_RANDOMIZED)):
        G = gpu_graph(n, s, d, **kw)
        ref = G.single_source(Q)
        G.set_memory_budget(64 * 1024)
        cut = G.single_source(Q)
        G.set_memory_budget(0)
        assert np.array_equal(ref, cut)
        G.close()


def test_edge_cases_frontier():
    """Queries without in-neighbours, l_max = 1 and 2, an edgeless node, with Rule 2 and the switch."""
    from paper_1709_06955_gb300 import probesim
    n = 60
    rng = np.random.default_rng(6)
    s = rng.integers(0, n - 1, 500).astype(np.int32)
    d = rng.integers(0, n - 1, 500).astype(np.int32)
    d[d == 3] = 4  # node 3 has no in-neighbours; node n-1 no edges at all
    keep = s != d
    key = np.unique(s[keep].astype(np.int64) * n + d[keep])
    s, d = (key // n).astype(np.int32), (key % n).astype(np.int32)
    O = oracle_graph(n, s, d)
    for lmax in (1, 2, 64):
        G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.05, eps_p=1.3e-3, l_max=lmax)
        Q = _q([3, n - 1, 7, 8], eps=0.3, query_ids=[1, 2, 3, 4])
        out = G.single_source(Q)
        for t, u in enumerate([3, n - 1, 7, 8]):
            ref, _ = O.single_source(u, eps=0.3, seed=3, qid=t + 1, l_max=lmax, probe_mode=2, c0=_f32(0.05),
                                     eps_p=_f32(1.3e-3), batch=True)
            assert np.max(np.abs(out[t] - ref)) <= _prune_tol(0.3, 1.3e-3)
            if u in (3, n - 1) or lmax == 1:
                expect = np.zeros(n, np.float32)
                expect[u] = 1
                assert np.array_equal(out[t], expect)
        G.close()


def test_switch_after_updates(cl1k):
    from paper_1709_06955_gb300 import probesim
    n, s, d, _ = cl1k
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.02)
    rng = np.random.default_rng(47)
    ins_s, ins_d = rng.integers(0, n, 300).astype(np.int32), rng.integers(0, n, 300).astype(np.int32)
    G.insert_edges(ins_s, ins_d)
    pick = rng.choice(s.size, 200, replace=False)
    G.delete_edges(s[pick], d[pick])
    key = set((s.astype(np.int64) * n + d).tolist())
    key |= {int(a) * n + int(b) for a, b in zip(ins_s, ins_d) if a != b}
    key -= {int(s[i]) * n + int(d[i]) for i in pick}
    k = np.array(sorted(key), np.int64)
    O = oracle_graph(n, (k // n).astype(np.int32), (k % n).astype(np.int32))
    qs = synth.queries(n, (k % n).astype(np.int32), 3, seed=48)
    out = G.single_source(_q(qs, eps=0.2, query_ids=[51, 52, 53]))
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=0.2, seed=3, qid=51 + t, probe_mode=2, c0=_f32(0.02), batch=True)
        assert np.max(np.abs(out[t] - ref)) <= TOL


def test_topk_in_switch_mode(cl1k):
    """Top-k over the switch engine's estimates: the exact top-k of the GPU's own scores."""
    from paper_1709_06955_gb300 import probesim
    n, s, d, O = cl1k
    G = gpu_graph(n, s, d, probe_mode=probesim.PROBE_SWITCH, c0=0.02, eps_p=1e-4)
    qs = synth.queries(n, d, 3, seed=49)
    Q = _q(qs, eps=0.15, k=[10, 50, 100], query_ids=[61, 62, 63])
    sc = G.single_source(Q)
    ids, vals = G.topk(Q, kmax=100)
    for i, u in enumerate(qs):
        k = [10, 50, 100][i]
        order = [int(v) for v in np.lexsort((np.arange(n), -sc[i].astype(np.float64))) if v != u][:k]
        assert ids[i, :k].tolist() == order
        assert np.array_equal(vals[i, :k], sc[i][order])


def test_error_split_drives_queries_within_eps_a():
    """Thm. 2's split of eps_a = 0.2 (eps, l_max, eps_p and the eps_t/2 shift) drives the GPU on the 1,000-node
    Chung-Lu graph: the estimates follow the oracle with the same parameters (Rule-2 bound), and at least a 1-delta
    fraction of 20 queries is within eps_a of the Power Method's SimRank (30 iterations)."""
    from oracle import power_method
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.config_graph("chunglu-1k")
    sp = probesim.split_error(0.2, C, True)
    G = gpu_graph(n, s, d, l_max=sp["l_max"], eps_p=sp["eps_p"], shift=sp["shift"])
    qs = synth.queries(n, d, 20, seed=2)
    out = G.single_source(_q(qs, eps=sp["eps"], query_ids=np.arange(20) + 600))
    S = power_method.simrank(n, s, d, C, 30)
    O = oracle_graph(n, s, d)
    ok = 0
    for t, u in enumerate(qs):
        if t < 3:
            ref, _ = O.single_source(int(u), eps=sp["eps"], seed=3, qid=600 + t, l_max=sp["l_max"], eps_p=sp["eps_p"])
            ref = ref + sp["shift"]
            ref[u] = 1.0
            assert np.max(np.abs(out[t] - ref)) <= _prune_tol(sp["eps"], sp["eps_p"])
        ok += np.max(np.abs(np.delete(out[t] - S[u], u))) <= 0.2
    assert ok >= 19
    G.close()
