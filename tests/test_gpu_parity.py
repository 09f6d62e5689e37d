"""GPU path vs the FP64 oracle through the C ABI: walks bit-exact, scores within 1e-5 max-abs."""
import numpy as np
import pytest

from gpu_util import TOL, dedup, gpu_graph, oracle_graph
from paper_1709_06955_gb300 import synth

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
def cfg1():
    n, s, d = synth.config_graph("chunglu-1k")
    return n, s, d, gpu_graph(n, s, d), oracle_graph(n, s, d)


def _q(nodes, **kw):
    from paper_1709_06955_gb300 import probesim
    return probesim.make_queries(nodes, **kw)


def test_walks_bit_exact(cfg1):
    n, s, d, G, O = cfg1
    qs = synth.queries(n, d, 5, seed=2)
    Q = _q(qs, eps=0.1, query_ids=np.arange(5) + 100)
    nodes, lens = G.sample_walks(Q)
    nr = G.num_walks(0.1)
    assert nr == 2073 and nodes.shape[0] == 5 * nr
    for b, u in enumerate(qs):
        for k in range(nr):
            ref = O.walk(int(u), 0.6, 64, 3, 100 + b, k)
            row = nodes[b * nr + k]
            assert lens[b * nr + k] == ref.size
            assert np.array_equal(row[:ref.size], ref) and np.all(row[ref.size:] == -1)


def test_config1_single_source(cfg1):
    """Chung-Lu n=1,000, m=10,000: 20 queries, eps=0.1, delta=0.01 (n_r=2,073)."""
    n, s, d, G, O = cfg1
    qs = synth.queries(n, d, 20, seed=2)
    Q = _q(qs, eps=0.1, query_ids=np.arange(20))
    out = G.single_source(Q)
    worst = 0.0
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=0.1, seed=3, qid=t)
        worst = max(worst, float(np.max(np.abs(out[t] - ref))))
        assert out[t][u] == 1.0
    assert worst <= TOL, worst


@pytest.mark.parametrize("scale,eps", [(10, 0.1), (12, 0.15), (13, 0.2)])
def test_rmat_single_source(scale, eps):
    n, s, d = synth.rmat(scale, 16 << scale, seed=scale)
    G, O = gpu_graph(n, s, d), oracle_graph(n, s, d)
    qs = synth.queries(n, d, 3, seed=scale + 1)
    out = G.single_source(_q(qs, eps=eps, query_ids=[7, 8, 9]))
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=eps, seed=3, qid=7 + t)
        assert np.max(np.abs(out[t] - ref)) <= TOL


def test_batched_equals_alone(cfg1):
    """A query's result is the same alone and in a mixed batch (uneven eps and n_r)."""
    n, s, d, G, O = cfg1
    qs = synth.queries(n, d, 12, seed=5)
    eps = np.where(np.arange(12) % 3 == 0, 0.1, np.where(np.arange(12) % 3 == 1, 0.2, 0.15))
    Q = _q(qs, eps=eps, query_ids=np.arange(12) * 3 + 1)
    mix = G.single_source(Q)
    for i in range(12):
        alone = G.single_source(_q([qs[i]], eps=eps[i], query_ids=[i * 3 + 1]))
        assert np.max(np.abs(alone[0] - mix[i])) <= 1e-6


def test_wide_batch_equals_alone():
    """256 queries in one call (R-MAT 2^14): the score matrices are over 24K columns wide (grouped layout with
    many 256-column groups); sampled queries match the same queries alone (node-major matrices)."""
    n, s, d = synth.rmat(14, 16 << 14, seed=14)
    G = gpu_graph(n, s, d)
    qs = synth.queries(n, d, 256, seed=15)
    Q = _q(qs, eps=0.1, query_ids=np.arange(256) + 1000)
    mix = G.single_source(Q)
    assert G.stats()["max_columns"] > 24 * 1024
    for i in (0, 77, 255):
        alone = G.single_source(_q([qs[i]], eps=0.1, query_ids=[1000 + i]))
        assert G.stats()["max_columns"] <= 24 * 1024
        assert np.max(np.abs(alone[0] - mix[i])) <= 1e-6


def test_walk_ranges_add_up(cfg1):
    """The estimator is linear in the walks: disjoint walk ranges sum to the full estimate."""
    n, s, d, G, O = cfg1
    u = int(synth.queries(n, d, 1, seed=9)[0])
    full = G.single_source(_q([u], eps=0.1, query_ids=[4]))[0]
    parts = [G.single_source(_q([u], eps=0.1, query_ids=[4], walk_begin=a, walk_end=b))[0]
             for a, b in [(0, 700), (700, 1500), (1500, 0)]]
    tot = sum(p for p in parts)
    tot[u] = 1.0
    assert np.max(np.abs(tot - full)) <= 3e-6
    ref, _ = O.single_source(u, eps=0.1, seed=3, qid=4, walk_begin=700, walk_end=1500)
    assert np.max(np.abs(parts[1] - ref)) <= TOL


def test_edge_cases():
    # query without in-neighbours; node with no edges; l_max = 1 and 2; duplicates and loops dropped
    n = 50
    rng = np.random.default_rng(4)
    s = rng.integers(0, n, 400).astype(np.int32)
    d = rng.integers(0, n, 400).astype(np.int32)
    s[:5] = d[:5]  # self-loops
    s[5:10], d[5:10] = s[10:15], d[10:15]  # duplicates
    d[d == 0] = 1  # node 0 has no in-neighbour
    ds, dd = dedup(n, s, d)
    O = oracle_graph(n, ds, dd)
    for lmax in (1, 2, 3, 64):
        G = gpu_graph(n, s, d, l_max=lmax)
        assert G.info()[1] == ds.size
        for u in (0, 1, 7):
            out = G.single_source(_q([u], eps=0.3, query_ids=[u]))[0]
            ref, _ = O.single_source(u, eps=0.3, l_max=lmax, seed=3, qid=u)
            assert np.max(np.abs(out - ref)) <= TOL
    G = gpu_graph(n, s, d)
    out = G.single_source(_q([0], eps=0.3))[0]
    assert out[0] == 1.0 and np.count_nonzero(out) == 1
    # a graph without edges
    G0 = gpu_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    out = G0.single_source(_q([3], eps=0.5))[0]
    assert out.tolist() == [0, 0, 0, 1, 0]


def _check_topk(ids, vals, k, u, scores, tol):
    """(ids, vals) is a valid top-k of ``scores`` (a second FP32 evaluation of the same estimate, so
    entries within ``tol`` of each other may swap): ordered by (value desc, id asc), u excluded, values
    match the scores, and nothing outside the set beats the k-th value."""
    assert len(set(ids.tolist())) == k and u not in ids.tolist()
    for a in range(k - 1):
        assert vals[a] > vals[a + 1] or (vals[a] == vals[a + 1] and ids[a] < ids[a + 1])
    assert np.max(np.abs(vals - scores[ids])) <= tol
    rest = np.ones(scores.size, bool)
    rest[ids] = False
    rest[u] = False
    assert np.all(scores[rest] <= vals[-1] + tol)


def test_device_buffers_and_topk(cfg1):
    """Host and device output buffers, and top-k against the scores and the oracle.  Two evaluations
    differ in the last bits: FP32 atomic adds make the summation order vary."""
    import torch
    n, s, d, G, O = cfg1
    qs = synth.queries(n, d, 6, seed=11)
    Q = _q(qs, eps=0.1, k=[10, 50, 100, 1, 5, 100], query_ids=np.arange(6))
    dev = torch.zeros((6, n), dtype=torch.float32, device="cuda")
    G.single_source(Q, out=dev)
    host = G.single_source(Q)
    assert np.max(np.abs(dev.cpu().numpy() - host)) <= 1e-6
    ids, vals = G.topk(Q, kmax=100)
    for i, u in enumerate(qs):
        k = Q[i].k
        _check_topk(ids[i, :k], vals[i, :k], k, int(u), host[i], 1e-6)
        assert np.all(ids[i, k:] == -1) and np.all(vals[i, k:] == 0)
        ref, _ = O.single_source(int(u), eps=0.1, seed=3, qid=i)
        _check_topk(ids[i, :k], vals[i, :k].astype(np.float64), k, int(u), ref, 2 * TOL)
    did = torch.zeros((6, 100), dtype=torch.int32, device="cuda")
    dval = torch.zeros((6, 100), dtype=torch.float32, device="cuda")
    G.topk(Q, kmax=100, ids=did, vals=dval)
    for i, u in enumerate(qs):
        k = Q[i].k
        _check_topk(did[i, :k].cpu().numpy(), dval[i, :k].cpu().numpy(), k, int(u), host[i], 1e-6)


def test_topk_ties_prefer_small_ids():
    """Nodes that no walk reaches score exactly 0; when k exceeds the nonzero count the tail is the
    smallest ids among the zeros."""
    n = 64
    s = np.array([1, 2, 3, 4], np.int32)
    d = np.array([0, 0, 5, 5], np.int32)  # 1,2 -> 0 ; 3,4 -> 5: s(0, v) = 0 for every v != 0
    G = gpu_graph(n, s, d)
    ids, vals = G.topk(_q([0], eps=0.2, k=10), kmax=10)
    assert ids[0].tolist() == list(range(1, 11)) and np.all(vals[0] == 0)


def test_updates_match_oracle(cfg1):
    n, s, d, _, _ = cfg1
    G = gpu_graph(n, s, d)
    rng = np.random.default_rng(12)
    ins_s = rng.integers(0, n, 300).astype(np.int32)
    ins_d = rng.integers(0, n, 300).astype(np.int32)
    applied = G.insert_edges(ins_s, ins_d)
    cur_s, cur_d = dedup(n, np.concatenate([s, ins_s]), np.concatenate([d, ins_d]))
    assert applied == cur_s.size - s.size
    pick = rng.choice(cur_s.size, 500, replace=False)
    removed = G.delete_edges(cur_s[pick], cur_d[pick])
    assert removed == 500
    keep = np.ones(cur_s.size, bool)
    keep[pick] = False
    cur_s, cur_d = cur_s[keep], cur_d[keep]
    assert G.info()[1] == cur_s.size and G.info()[2] == 2
    O = oracle_graph(n, cur_s, cur_d)
    for t, u in enumerate(synth.queries(n, cur_d, 3, seed=13)):
        out = G.single_source(_q([u], eps=0.15, query_ids=[t]))[0]
        ref, _ = O.single_source(int(u), eps=0.15, seed=3, qid=t)
        assert np.max(np.abs(out - ref)) <= TOL
        nodes, lens = G.sample_walks(_q([u], eps=0.15, query_ids=[t]))  # in-lists keep the source-id order
        for k in range(0, nodes.shape[0], 37):
            w = O.walk(int(u), 0.6, 64, 3, t, k)
            assert lens[k] == w.size and np.array_equal(nodes[k, :w.size], w)


def test_updates_on_a_hub_row():
    """One batch of many inserts into the in- and out-lists of a hub, then many deletes from its in-list."""
    n = 3000
    s, d = synth.chung_lu(n, 30000, seed=4)
    hub = int(np.argmax(np.bincount(d, minlength=n)))
    rng = np.random.default_rng(5)
    in_src = rng.choice(n, 1500, replace=False).astype(np.int32)
    out_dst = rng.choice(n, 700, replace=False).astype(np.int32)
    add_s = np.concatenate([in_src, np.full(700, hub, np.int32)])
    add_d = np.concatenate([np.full(1500, hub, np.int32), out_dst])
    G = gpu_graph(n, s, d)
    before = G.info()[1]
    added = G.insert_edges(add_s, add_d)
    cur_s, cur_d = dedup(n, np.concatenate([s, add_s]), np.concatenate([d, add_d]))
    assert added == cur_s.size - before and G.info()[1] == cur_s.size
    drop = rng.choice(np.nonzero(cur_d == hub)[0], 400, replace=False)
    assert G.delete_edges(cur_s[drop], cur_d[drop]) == 400
    keep = np.ones(cur_s.size, bool)
    keep[drop] = False
    cur_s, cur_d = cur_s[keep], cur_d[keep]
    assert G.info()[1] == cur_s.size
    O = oracle_graph(n, cur_s, cur_d)
    for t, u in enumerate([hub] + list(synth.queries(n, cur_d, 2, seed=6))):
        out = G.single_source(_q([u], eps=0.2, query_ids=[t]))[0]
        ref, _ = O.single_source(int(u), eps=0.2, seed=3, qid=t)
        assert np.max(np.abs(out - ref)) <= TOL
        nodes, lens = G.sample_walks(_q([u], eps=0.2, query_ids=[t]))
        for k in range(0, nodes.shape[0], 11):
            w = O.walk(int(u), 0.6, 64, 3, t, k)
            assert lens[k] == w.size and np.array_equal(nodes[k, :w.size], w)


def test_updates_give_out_edges_to_nodes_without_any():
    """Nodes without out-edges come last in the internal order, and the level loop skips their rows when it
    accumulates (nothing gathers them).  An update batch that gives forty of them out-edges into the most popular
    targets must bring their rows back: estimates and walks of queries at those targets match the oracle."""
    n = 2000
    s, d = synth.chung_lu(n, 12000, seed=8)
    quiet = np.nonzero(np.bincount(s, minlength=n) == 0)[0][:40]
    assert quiet.size == 40
    targets = np.argsort(-np.bincount(d, minlength=n), kind="stable")[:5]
    add_s = np.repeat(quiet, targets.size).astype(np.int32)
    add_d = np.tile(targets, quiet.size).astype(np.int32)
    G = gpu_graph(n, s, d)
    G.insert_edges(add_s, add_d)
    cur_s, cur_d = dedup(n, np.concatenate([s, add_s]), np.concatenate([d, add_d]))
    assert G.info()[1] == cur_s.size
    O = oracle_graph(n, cur_s, cur_d)
    for t, u in enumerate(targets[:3]):
        out = G.single_source(_q([int(u)], eps=0.15, query_ids=[t]))[0]
        ref, _ = O.single_source(int(u), eps=0.15, seed=3, qid=t)
        assert np.max(np.abs(out - ref)) <= TOL


def test_errors(cfg1):
    from paper_1709_06955_gb300 import probesim
    n, s, d, G, O = cfg1
    with pytest.raises(probesim.ProbeSimError) as e:
        G.single_source(_q([n], eps=0.1))
    assert e.value.status == probesim.E_RANGE
    with pytest.raises(probesim.ProbeSimError) as e:
        G.single_source(_q([0], eps=1.5))
    assert e.value.status == probesim.E_INVALID
    with pytest.raises(probesim.ProbeSimError) as e:
        G.topk(_q([0], eps=0.1, k=5), kmax=n)
    assert e.value.status == probesim.E_INVALID
    with pytest.raises(probesim.ProbeSimError) as e:
        G.insert_edges(np.array([0], np.int32), np.array([n + 3], np.int32))
    assert e.value.status == probesim.E_RANGE
    with pytest.raises(probesim.ProbeSimError) as e:
        probesim.Graph(10, np.array([0], np.int32), np.array([1], np.int32), l_max=0)
    assert e.value.status == probesim.E_INVALID


def test_autotune_keeps_results(cfg1):
    n, s, d, _, O = cfg1
    G = gpu_graph(n, s, d)
    tune = G.autotune()
    assert tune["wide_tile"] in (16, 32, 64) and all(b in (2, 4, 8, 16) for b in tune["blocks_per_sm"].values())
    qs = synth.queries(n, d, 3, seed=41)
    out = G.single_source(_q(qs, eps=0.1, query_ids=[1, 2, 3]))
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=0.1, seed=3, qid=1 + t)
        assert np.max(np.abs(out[t] - ref)) <= TOL


def test_every_pull_shape_gives_the_same_scores():
    """Full tiles as 16-column halves, 32-column tiles, 32-column tiles two per pass (with an odd tile count at
    some depths, so a pass holds one tile), or 32-column tiles gathered by the TMA: the first three add a piece's
    in-neighbours in the same order and the TMA pull in four interleaved partial sums, so the scores agree to
    rounding (rows cut into several pieces also add their pieces atomically, in any order), and within 1e-5 of the
    oracle.  R-MAT 2^12, eps 0.1: the widest depths have hundreds of columns."""
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.rmat(12, 16 << 12, seed=12)
    G, O = gpu_graph(n, s, d), oracle_graph(n, s, d)
    qs = synth.queries(n, d, 2, seed=13)
    Q = _q(qs, eps=0.1, query_ids=[21, 22])
    outs = {}
    for wide in (32, 16, 64, 96):
        G.set_tuning(wide, [8, 8, 8, 4, 4, 4, 3, 2])
        assert G.tuning()["wide_tile"] == wide
        outs[wide] = G.single_source(Q)
    for wide in (16, 64, 96):
        assert np.max(np.abs(outs[32] - outs[wide])) <= 1e-6
    for t, u in enumerate(qs):
        for wide in (64, 96):
            ref, _ = O.single_source(int(u), eps=0.1, seed=3, qid=21 + t)
            assert np.max(np.abs(outs[wide][t] - ref)) <= TOL
    with pytest.raises(probesim.ProbeSimError):
        G.set_tuning(48)
