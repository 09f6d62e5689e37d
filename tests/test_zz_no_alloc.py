"""The allocation-free top-k entry point (probesim_topk_select_noalloc) against probesim_topk.

It is for callers that cannot allocate device memory while they run (a component that has reserved all
device memory for its own pool, or a serving loop that must not take cudaMalloc's device-wide
synchronisation): its scratch is a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1709_06955_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-6  # two FP32 evaluations of the same estimates (atomic summation order varies)


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build, probesim
    build.build()
    n, s, d = synth.config_graph("chunglu-1k")
    G = probesim.Graph(n, s, d)
    qs = synth.queries(n, d, 6, seed=11)
    ks = [10, 50, 100, 1, 5, 100]
    Q = probesim.make_queries(qs, eps=0.1, k=ks, query_ids=np.arange(6))
    return n, G, Q, qs, ks


def test_noalloc_topk_matches_topk_on_two_calls(setup):
    import torch
    from paper_1709_06955_gb300 import probesim
    n, G, Q, qs, ks = setup
    scores = torch.zeros((6, n), dtype=torch.float32, device="cuda")
    G.single_source(Q, out=scores)
    ref_ids, ref_vals = G.topk(Q, kmax=100)  # the existing entry point (recomputes the scores)
    sc = scores.cpu().numpy()
    first = None
    for call in range(2):
        ids = torch.full((6, 100), -7, dtype=torch.int32, device="cuda")
        vals = torch.full((6, 100), -7.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        probesim.topk_select_noalloc(scores, qs, ks, 100, ids, vals)
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # after the first call's set-up, a call takes no device memory
            assert free1 == free0
        ids, vals = ids.cpu().numpy(), vals.cpu().numpy()
        for i in range(6):
            k = ks[i]
            assert np.max(np.abs(vals[i, :k] - ref_vals[i, :k])) <= TOL
            same = ids[i, :k] == ref_ids[i, :k]
            # a position may differ only between entries whose scores tie within the tolerance
            assert np.all(same | (np.abs(sc[i][ids[i, :k]] - sc[i][ref_ids[i, :k]]) <= TOL))
            assert np.all(ids[i, k:] == -1) and np.all(vals[i, k:] == 0)
            assert np.array_equal(vals[i, :k], sc[i][ids[i, :k]])
        if first is None:
            first = (ids, vals)
        else:  # the same input gives the same output: nothing left in the shared scratch leaks into a call
            assert np.array_equal(first[0], ids) and np.array_equal(first[1], vals)


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    import torch
    from paper_1709_06955_gb300 import probesim
    n, G, Q, qs, ks = setup
    scores = torch.zeros((65, n), dtype=torch.float32, device="cuda")
    ids = torch.zeros((65, 10), dtype=torch.int32, device="cuda")
    vals = torch.zeros((65, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(probesim.ProbeSimError) as e:
        probesim.topk_select_noalloc(scores, [0] * 65, [5] * 65, 10, ids, vals)
    assert e.value.status == probesim.E_INVALID and "64" in str(e.value)
    big_ids = torch.zeros((1, 1025), dtype=torch.int32, device="cuda")
    big_vals = torch.zeros((1, 1025), dtype=torch.float32, device="cuda")
    with pytest.raises(probesim.ProbeSimError) as e:
        probesim.topk_select_noalloc(scores[:1], [0], [5], 1025, big_ids, big_vals)
    assert e.value.status == probesim.E_INVALID and "1024" in str(e.value)
