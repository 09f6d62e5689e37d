"""Pins the oracle's PROBE (Alg. 2), its pruning rules (Sec. 4.1) and the Power Method (Eq. 6) to the
values the paper prints for its running example on the toy graph (tests/golden/)."""
import numpy as np
import pytest

from oracle import core, power_method

C_TOY = 0.25  # the running example uses c' = 0.25


@pytest.fixture(scope="module")
def g(toy):
    n, s, d = toy
    return core.Graph(n, s, d)


def test_probe_trace_matches_printed(g, printed):
    """S_2, S_3, S_4 of the walk (a,b,a,b) and H_2 of PROBE(a,b,a,b), Sec. 3.2 running example."""
    checked = 0
    for kind, path, node, val, tol in printed:
        if kind == "probe":
            got = g.probe(path, C_TOY)[node]
        elif kind == "level2":
            # H_2 of PROBE(u_1..u_4) is PROBE(u_2, u_3, u_4): the same two levels with the same exclusions
            got = g.probe(path[1:], C_TOY)[node]
        else:
            continue
        assert abs(got - val) <= tol, (kind, path, node, got, val)
        checked += 1
    assert checked == 14


def test_probe_support_matches_printed(g):
    """The printed score sets are the whole support: no other node gets a score."""
    a, b = 0, 1
    assert set(np.nonzero(g.probe([a, b], C_TOY))[0]) == {2, 3, 4}
    assert set(np.nonzero(g.probe([a, b, a], C_TOY))[0]) == {5, 6, 7}
    assert set(np.nonzero(g.probe([a, b, a, b], C_TOY))[0]) == {1, 2, 4, 5}


def test_printed_intermediate_arithmetic(g):
    """The running example spells out Score(c,1) = 0.5/3, Score(d,1) = 0.5/1, Score(e,1) = 0.5/2 and
    Score(f,2) = (Score(c,1)+Score(d,1)+Score(e,1)) * 0.5/4."""
    s2 = g.probe([0, 1], C_TOY)
    assert s2[2] == pytest.approx(0.5 / 3, abs=1e-15)
    assert s2[3] == pytest.approx(0.5 / 1, abs=1e-15)
    assert s2[4] == pytest.approx(0.5 / 2, abs=1e-15)
    h2 = g.probe([1, 0, 1], C_TOY)
    assert h2[5] == pytest.approx((0.5 / 3 + 0.5 + 0.25) * 0.5 / 4, abs=1e-15)


def test_single_walk_estimate_matches_printed(g, printed):
    """s~_k(a, .) for the walk (a,b,a,b) is the sum of its three probes (Alg. 1 lines 5-11)."""
    walk = [0, 1, 0, 1]
    est = sum(g.probe(walk[:i], C_TOY) for i in range(2, 5))
    for kind, path, node, val, tol in printed:
        if kind == "walk":
            assert abs(est[node] - val) <= tol, (node, est[node], val)


def test_power_method_matches_table2(toy, printed):
    n, s, d = toy
    S = power_method.simrank(n, s, d, C_TOY, 60)
    for kind, path, node, val, tol in printed:
        if kind == "simrank":
            assert abs(S[path[0], node] - val) <= tol, (node, S[path[0], node], val)


def test_pruning_example(g):
    """Sec. 4.1 example, eps_t = eps_p = 0.05 at sqrt(c') = 0.5: rule 1 keeps l_t = 4 nodes of (a,b,a,b,e);
    rule 2 drops c from H_1 of PROBE(a,b,a,b) because 0.167 * 0.5^2 = 0.042 <= 0.05."""
    import math
    l_t = math.floor(math.log(0.05) / math.log(math.sqrt(C_TOY)))
    assert l_t == 4
    full = g.probe([0, 1, 0, 1], C_TOY)
    pruned = g.probe([0, 1, 0, 1], C_TOY, eps_p=0.05)
    diff = full - pruned
    assert np.all(diff >= -1e-15) and np.all(diff <= 0.05)  # one-sided, at most eps_p
    # the subtree of c is what is dropped: the difference is what c's score 1/6 alone pushes through
    # levels 1 and 2 of PROBE(a,b,a,b) (exclusions b then a), i.e. 1/6 times PROBE(x, b, c)'s last two levels
    from_c = g.probe([0, 1, 2], C_TOY) / 1.0 * (1 / 6)
    # PROBE((a, b, c)) starts at c with score 1 and excludes b then a -- the same two levels
    assert np.allclose(diff, from_c, atol=1e-15)
