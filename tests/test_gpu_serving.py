"""Serving loop (continuous batching): results in the mix equal the same query run alone, update batches
take effect in submission order, and a full queue refuses work with E_BUSY."""
import time

import numpy as np
import pytest

from paper_1709_06955_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-6  # two FP32 evaluations of the same estimate


@pytest.fixture(scope="module")
def graph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build, probesim
    build.build()
    n, s, d = synth.config_graph("chunglu-1k")
    return n, s, d, probesim.Graph(n, s, d)


def _same_topk(ids_a, vals_a, ids_b, vals_b, k):
    assert np.max(np.abs(vals_a[:k] - vals_b[:k])) <= TOL
    differ = ids_a[:k] != ids_b[:k]
    assert np.all(np.abs(vals_a[:k][differ] - vals_b[:k][differ]) <= TOL)  # only near-ties may swap


def test_results_in_the_mix_equal_alone(graph):
    from paper_1709_06955_gb300 import probesim
    n, s, d, G = graph
    qs = synth.queries(n, d, 24, seed=31)
    eps = np.array([0.1, 0.2, 0.3])[np.arange(24) % 3]
    ks = np.array([5, 20, 50, 100])[np.arange(24) % 4]
    S = probesim.Server(G, workers=2, max_batch=4, kmax=100)
    tickets = {}
    got = {}
    for wave in range(4):  # arrivals while earlier batches run
        sel = range(wave * 6, wave * 6 + 6)
        Q = probesim.make_queries(qs[list(sel)], eps=eps[list(sel)], k=ks[list(sel)], query_ids=list(sel))
        for i, t in zip(sel, S.submit(Q)):
            tickets[t] = i
        for r, ids, vals in S.poll(64, wait_ms=5):
            got[r.ticket] = (r, ids, vals)
        time.sleep(0.01)
    deadline = time.time() + 120
    while len(got) < 24 and time.time() < deadline:
        for r, ids, vals in S.poll(64, wait_ms=200):
            got[r.ticket] = (r, ids, vals)
    assert len(got) == 24
    st = S.stats()
    assert st["completed"] == 24 and st["failed"] == 0 and st["batches"] >= 6
    assert st["p99_ms"] >= st["p50_ms"] > 0
    workers = {r.worker for r, _, _ in got.values()}
    assert workers <= {0, 1}
    for t, (r, ids, vals) in got.items():
        i = tickets[t]
        assert r.status == 0 and r.node == qs[i] and r.k == ks[i] and r.query_id == i
        a_ids, a_vals = G.topk(probesim.make_queries([qs[i]], eps=eps[i], k=ks[i], query_ids=[i]), kmax=100)
        _same_topk(ids, vals, a_ids[0], a_vals[0], int(ks[i]))
        assert np.all(ids[ks[i]:] == -1)
    S.close()


def test_updates_apply_in_submission_order(graph):
    from paper_1709_06955_gb300 import probesim
    n, s, d, _ = graph
    G = probesim.Graph(n, s, d)
    S = probesim.Server(G, workers=2, max_batch=2, kmax=10)
    u = int(synth.queries(n, d, 1, seed=33)[0])
    Q = probesim.make_queries([u], eps=0.2, k=10, query_ids=[7])
    before = S.submit(Q)[0]
    rng = np.random.default_rng(3)
    ins_s = rng.integers(0, n, 2000).astype(np.int32)
    ins_d = rng.integers(0, n, 2000).astype(np.int32)
    S.update(ins_s, ins_d, insert=True)
    after = S.submit(Q)[0]
    got = {}
    deadline = time.time() + 60
    while len(got) < 2 and time.time() < deadline:
        for r, ids, vals in S.poll(8, wait_ms=200):
            got[r.ticket] = (r, ids, vals)
    assert S.stats()["updates_applied"] == 1
    assert got[before][0].epoch == 0 and got[after][0].epoch == 1
    # the query after the update matches a direct call on the updated graph, the one before it the old graph
    ref_old = probesim.Graph(n, s, d).topk(Q, kmax=10)
    ref_new = G.topk(Q, kmax=10)
    _same_topk(got[before][1], got[before][2], ref_old[0][0], ref_old[1][0], 10)
    _same_topk(got[after][1], got[after][2], ref_new[0][0], ref_new[1][0], 10)
    S.close()


def test_full_queue_is_refused(graph):
    from paper_1709_06955_gb300 import probesim
    n, s, d, G = graph
    S = probesim.Server(G, workers=1, max_batch=1, kmax=5, queue_capacity=3)
    qs = synth.queries(n, d, 40, seed=34)
    refused = 0
    for i in range(40):
        try:
            S.submit(probesim.make_queries([qs[i]], eps=0.3, k=5, query_ids=[i]))
        except probesim.ProbeSimError as e:
            assert e.status == probesim.E_BUSY
            refused += 1
    assert refused > 0 and S.stats()["rejected"] == refused
    S.close()


def test_update_does_not_wait_for_a_query_in_flight():
    """An update batch builds the next store version beside the current one: applied from another thread while a
    long query runs, it returns before the query ends, and the query's estimates are those of the graph it
    started on (the store version it holds)."""
    import threading
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.rmat(16, 16 << 16, seed=16)
    G = probesim.Graph(n, s, d)
    qs = synth.queries(n, d, 8, seed=161)
    Q = probesim.make_queries(qs, eps=0.02, query_ids=np.arange(8) + 90)  # long enough to outlast the update
    ref_old = probesim.Graph(n, s, d).single_source(Q)
    G.single_source(probesim.make_queries(qs[:1], eps=0.2, query_ids=[1]))  # warm up the workspace
    box = {}

    def run():
        box["t0"] = time.perf_counter()
        box["out"] = G.single_source(Q)
        box["t1"] = time.perf_counter()

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.2)
    rng = np.random.default_rng(4)
    t_upd0 = time.perf_counter()
    applied = G.insert_edges(rng.integers(0, n, 5000).astype(np.int32), rng.integers(0, n, 5000).astype(np.int32))
    t_upd1 = time.perf_counter()
    th.join()
    assert applied > 0 and G.info()[2] == 1
    assert t_upd1 < box["t1"], "the update waited for the query (%.3f s after it)" % (t_upd1 - box["t1"])
    assert np.max(np.abs(box["out"] - ref_old)) <= TOL
    new = G.single_source(Q)  # a query that starts after the update sees it
    assert np.max(np.abs(new - ref_old)) > 1e-3
    del t_upd0
