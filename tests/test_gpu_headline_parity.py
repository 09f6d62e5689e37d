"""Full-n_r parity at the headline eps on R-MAT graphs larger than the small cases: R-MAT 2^14 (m = 2^18, three
queries) and 2^16 (m = 2^20, two queries), eps = 0.1 (n_r = 2,576 and 2,826), every walk, element-wise within 1e-5
of the FP64 oracle (Alg. 1).
The estimate is linear in the walks, so the oracle's share is computed over walk ranges on all host cores (the C
oracle releases the GIL) and summed; the deterministic GPU path runs the full queries in one call, wide tiles,
grouped layout, accumulate and push heirs included."""
import concurrent.futures
import os

import numpy as np
import pytest

from gpu_util import TOL, gpu_graph, oracle_graph
from paper_1709_06955_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _oracle_full(O, u, qid, nr, eps):
    threads = len(os.sched_getaffinity(0))
    cuts = np.linspace(0, nr, 4 * threads + 1).astype(int)
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda ab: O.single_source(u, eps=eps, seed=3, qid=qid, walk_begin=int(ab[0]),
                                                        walk_end=int(ab[1]))[0],
                            [(cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1) if cuts[i + 1] > cuts[i]]))
    tot = np.sum(parts, axis=0)
    tot[u] = 1.0
    return tot


@pytest.mark.parametrize("scale,nq,nr_expected", [(14, 3, 2576), (16, 2, 2826)])
def test_rmat_full_walks_headline_eps(scale, nq, nr_expected):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06955_gb300 import build, probesim
    from oracle import build as obuild
    build.build()
    obuild.build()
    n, s, d = synth.rmat(scale, 16 << scale, seed=scale)
    G, O = gpu_graph(n, s, d), oracle_graph(n, s, d)
    nr = G.num_walks(0.1)
    assert nr == nr_expected
    qs = synth.queries(n, d, nq, seed=scale * 10 + 1)
    out = G.single_source(probesim.make_queries(qs, eps=0.1, query_ids=31 + np.arange(nq)))
    for t, u in enumerate(qs):
        ref = _oracle_full(O, int(u), 31 + t, nr, 0.1)
        assert np.max(np.abs(out[t] - ref)) <= TOL
