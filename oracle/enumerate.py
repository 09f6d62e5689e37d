"""Exact expectations on tiny graphs by enumerating sqrt(c)-walks -- test infrastructure only.

``first_meeting``: P(v, (u_1..u_i)) of Def. 4 by summing the probability of every walk prefix
(v_1..v_i) from v that ends at u_i and avoids u_t at step t for t < i.  Lemma 2 states that PROBE
returns exactly this.

``expected_estimate``: E[s~(u, v)] = sum over all walks W(u) of Pr[W] * sum_{i=2..l} P(v, W(u, i))
(the expansion in the proof of Lemma 1), enumerating every walk of at most ``max_len`` nodes.
Lemma 1 states that this equals s(u, v) as max_len grows.
"""
import math


def in_lists(n, src, dst):
    I = [[] for _ in range(n)]
    for x, v in zip(src, dst):
        I[int(v)].append(int(x))
    return [sorted(l) for l in I]


def first_meeting(I, c, v, path):
    """P(v, path) for path = (u_1..u_i), v != u_1, by enumerating the walk prefixes from v."""
    sc = math.sqrt(c)
    i = len(path)
    total = 0.0
    # frontier: dict node -> probability of being at that node at step t having avoided path[0..t-1]
    if v == path[0]:
        return 0.0
    cur = {v: 1.0}
    for t in range(1, i):  # move from step t to step t+1 (1-based steps)
        nxt = {}
        for x, p in cur.items():
            if not I[x]:
                continue
            q = p * sc / len(I[x])  # continue w.p. sqrt(c), uniform in-neighbour
            for y in I[x]:
                nxt[y] = nxt.get(y, 0.0) + q
        if t + 1 < i:
            nxt.pop(path[t], None)  # must avoid u_{t+1} at step t+1
        cur = nxt
    total = cur.get(path[-1], 0.0)
    return total


def walks(I, c, u, max_len):
    """Every sqrt(c)-walk from u of at most max_len nodes with its probability.  A walk that
    would continue past max_len nodes is cut there (its probability mass is kept)."""
    sc = math.sqrt(c)
    out = []

    def rec(path, p):
        x = path[-1]
        if not I[x] or len(path) == max_len:
            out.append((tuple(path), p))
            return
        out.append((tuple(path), p * (1.0 - sc)))
        q = p * sc / len(I[x])
        for y in I[x]:
            rec(path + [y], q)

    rec([u], 1.0)
    return out


def expected_estimate(I, c, u, v, max_len):
    """sum_W Pr[W] * sum_{i=2..l} P(v, W(u, i)) over the walks of ``walks``."""
    tot = 0.0
    for path, p in walks(I, c, u, max_len):
        for i in range(2, len(path) + 1):
            tot += p * first_meeting(I, c, v, list(path[:i]))
    return tot
