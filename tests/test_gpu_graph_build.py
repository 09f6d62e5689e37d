"""The device-side initial build of the graph store (radix-sorted edge keys, the out-degree renumbering, the CSR
lists, w and the pull pieces): a graph built from device arrays, from host arrays, and from a shuffled edge list with
repeats and loops holds the same store, read back through the walks (each step takes the k-th in-neighbour in the
caller's source order, Sec. 2.1) and the estimates against the oracle; ids outside [0, n) are refused."""
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


def _walks(G, qs, eps, qids):
    from paper_1709_06955_gb300 import probesim
    return G.sample_walks(probesim.make_queries(qs, eps=eps, query_ids=qids))


def _check_walks(G, O, qs, eps, qids, stride=1):
    nodes, lens = _walks(G, qs, eps, qids)
    nr = G.num_walks(eps)
    for b, u in enumerate(qs):
        for k in range(0, nr, stride):
            ref = O.walk(int(u), 0.6, G.config.l_max, 3, int(qids[b]), k)
            assert lens[b * nr + k] == ref.size
            assert np.array_equal(nodes[b * nr + k][:ref.size], ref)


def test_device_and_host_edge_lists_build_the_same_store():
    import torch
    from paper_1709_06955_gb300 import probesim
    n, s, d = synth.rmat(13, 16 << 13, seed=4)
    Gh = gpu_graph(n, s, d)
    Gd = probesim.Graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    assert Gh.info()[:2] == Gd.info()[:2] == (n, s.size)
    qs = synth.queries(n, d, 3, seed=5)
    wh, lh = _walks(Gh, qs, 0.2, [1, 2, 3])
    wd, ld = _walks(Gd, qs, 0.2, [1, 2, 3])
    assert np.array_equal(wh, wd) and np.array_equal(lh, ld)
    Q = probesim.make_queries(qs, eps=0.2, query_ids=[1, 2, 3])
    assert np.max(np.abs(Gh.single_source(Q) - Gd.single_source(Q))) <= 1e-6


@pytest.mark.parametrize("n,m,seed", [(4097, 3 * 4096 + 17, 1), ((1 << 16) + 3, 5 * 4096 - 1, 2), (37, 300, 3)])
def test_repeats_and_loops_are_dropped(n, m, seed):
    """A shuffled edge list with every fifth edge repeated and loops mixed in builds the simple graph: the edge
    count, the walks and the estimates are those of the deduplicated list."""
    import torch
    from paper_1709_06955_gb300 import probesim
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m).astype(np.int32)
    d = (rng.zipf(1.6, m) % n).astype(np.int32)  # skewed in-degrees: some long in-lists, many empty ones
    rep = rng.choice(m, m // 5, replace=False)
    loops = rng.integers(0, n, 50).astype(np.int32)
    S = np.concatenate([s, s[rep], loops])
    D = np.concatenate([d, d[rep], loops])
    perm = rng.permutation(S.size)
    S, D = S[perm], D[perm]
    cs, cd = dedup(n, S, D)
    G = probesim.Graph(n, torch.from_numpy(S).cuda(), torch.from_numpy(D).cuda())
    assert G.info()[1] == cs.size
    O = oracle_graph(n, cs, cd)
    qs = synth.queries(n, cd, 2, seed=seed + 7)
    _check_walks(G, O, qs, 0.2, [11, 12], stride=7)
    out = G.single_source(probesim.make_queries(qs, eps=0.2, query_ids=[11, 12]))
    for t, u in enumerate(qs):
        ref, _ = O.single_source(int(u), eps=0.2, seed=3, qid=11 + t)
        assert np.max(np.abs(out[t] - ref)) <= TOL


def test_small_and_empty_graphs():
    import torch
    from paper_1709_06955_gb300 import probesim
    G = probesim.Graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert G.info()[:2] == (1, 0)
    out = G.single_source(probesim.make_queries([0], eps=0.3))
    assert out.shape == (1, 1) and out[0, 0] == 1.0
    G = probesim.Graph(2, torch.tensor([0, 1, 1, 0], dtype=torch.int32).cuda(),
                       torch.tensor([1, 0, 0, 0], dtype=torch.int32).cuda())
    assert G.info()[1] == 2  # (0,1), (1,0); the repeat and the loop dropped


@pytest.mark.parametrize("bad", [-1, 1000])
def test_ids_outside_the_range_are_refused_on_the_device(bad):
    import torch
    from paper_1709_06955_gb300 import probesim
    s = torch.arange(0, 900, dtype=torch.int32, device="cuda") % 1000
    d = (s * 7 + 1) % 1000
    s[450] = bad
    with pytest.raises(probesim.ProbeSimError, match="outside"):
        probesim.Graph(1000, s, d)
    s[450] = 3
    assert probesim.Graph(1000, s, d).info()[0] == 1000  # the library is still usable
