"""Seeded synthetic inputs: directed power-law graphs and query nodes.

These stand in for the paper's SNAP/LAW graphs (Sec. 6, Table 3), which are not available here.
The module holds input generation only -- none of ProbeSim's arithmetic -- and is the one module
that both the CUDA library's callers and the CPU oracle's tests use.

* ``chung_lu``: directed Chung-Lu graph.  Out- and in-weights w_i ~ (i+1)^(-1/(gamma-1)) under two
  independent random permutations; edges drawn with src ~ w_out, dst ~ w_in; self-loops and
  duplicates rejected until m distinct edges exist.
* ``rmat``: R-MAT (a, b, c, d) with 2^scale nodes; one quadrant choice per bit level; self-loops and
  duplicates removed, drawing until m distinct edges exist; a seeded node relabelling permutation.
* ``rmat_device``: the same R-MAT recipe drawn on a CUDA device (torch), for the large benchmark graphs.
* ``queries``: query nodes sampled uniformly from the nodes with in-degree >= 1 (Sec. 6.1).
"""
import numpy as np


def _dedup_keep_order(keys):
    _, first = np.unique(keys, return_index=True)
    return keys[np.sort(first)]


def chung_lu(n, m, gamma=2.1, seed=1):
    """Directed Chung-Lu graph with n nodes and exactly m distinct non-loop edges."""
    rng = np.random.default_rng(seed)
    base = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    w_out = base[rng.permutation(n)]
    w_in = base[rng.permutation(n)]
    p_out = w_out / w_out.sum()
    p_in = w_in / w_in.sum()
    if m > n * (n - 1):
        raise ValueError("m too large for a simple graph")
    keys = np.zeros(0, np.int64)
    while keys.size < m:
        need = m - keys.size
        k = max(1024, int(need * 1.5))
        s = rng.choice(n, size=k, p=p_out).astype(np.int64)
        d = rng.choice(n, size=k, p=p_in).astype(np.int64)
        ok = s != d
        keys = _dedup_keep_order(np.concatenate([keys, s[ok] * n + d[ok]]))
    keys = keys[:m]
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def rmat(scale, m, a=0.57, b=0.19, c=0.19, seed=1, relabel=True):
    """R-MAT graph on 2^scale nodes with exactly m distinct non-loop edges (int32 ids)."""
    n = 1 << scale
    if m > n * (n - 1):
        raise ValueError("m too large for a simple graph")
    rng = np.random.default_rng(seed)
    keys = np.zeros(0, np.int64)
    ab, abc = a + b, a + b + c
    while keys.size < m:
        need = m - keys.size
        k = max(4096, int(need * 1.25))
        src = np.zeros(k, np.int64)
        dst = np.zeros(k, np.int64)
        for bit in range(scale):
            r = rng.random(k, dtype=np.float32)
            # quadrants: a -> (0,0), b -> (0,1), c -> (1,0), d -> (1,1) for (src bit, dst bit)
            src |= (r >= ab).astype(np.int64) << bit
            dst |= (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64) << bit
        ok = src != dst
        new = src[ok] * n + dst[ok]
        keys = np.unique(np.concatenate([keys, new])) if keys.size else np.unique(new)
    # keys are sorted by np.unique: keep a seeded random subset of exactly m, in random order
    keys = keys[rng.permutation(keys.size)[:m]]
    src = keys // n
    dst = keys % n
    if relabel:
        perm = rng.permutation(n).astype(np.int64)
        src, dst = perm[src], perm[dst]
    return n, src.astype(np.int32), dst.astype(np.int32)


def rmat_device(scale, m, a=0.57, b=0.19, c=0.19, seed=1, device="cuda"):
    """The same R-MAT recipe as ``rmat``, drawn on a CUDA device with torch's seeded generator (for the large
    benchmark graphs, where the host generator takes minutes).  Returns (n, src, dst) as int32 CUDA tensors.
    The draws differ from ``rmat``'s, so the two give different graphs of the same distribution."""
    import torch
    n = 1 << scale
    if m > n * (n - 1):
        raise ValueError("m too large for a simple graph")
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    while keys.numel() < m:
        k = max(4096, int((m - keys.numel()) * 1.25))
        src = torch.zeros(k, dtype=torch.int64, device=device)
        dst = torch.zeros(k, dtype=torch.int64, device=device)
        for bit in range(scale):
            r = torch.rand(k, generator=gen, device=device)
            src |= (r >= ab).long() << bit
            dst |= (((r >= a) & (r < ab)) | (r >= abc)).long() << bit
        ok = src != dst
        keys = torch.unique(torch.cat([keys, src[ok] * n + dst[ok]]))
        del src, dst, ok
    keys = keys[torch.randperm(keys.numel(), generator=gen, device=device)[:m]]
    relabel = torch.randperm(n, generator=gen, device=device)
    return n, relabel[keys // n].int(), relabel[keys % n].int()


def queries(n, dst, count, seed=2):
    """``count`` query nodes drawn uniformly (without replacement when possible) from the nodes
    with at least one in-neighbour."""
    rng = np.random.default_rng(seed)
    if type(dst).__module__.startswith("torch"):  # counted where the edges live (10^9 of them at the largest size)
        import torch
        indeg = torch.bincount(dst.to(torch.int64), minlength=n).cpu().numpy()
    else:
        indeg = np.bincount(np.asarray(dst, dtype=np.int64), minlength=n)
    cand = np.nonzero(indeg > 0)[0]
    if cand.size == 0:
        raise ValueError("graph has no node with an in-neighbour")
    replace = count > cand.size
    return rng.choice(cand, size=count, replace=replace).astype(np.int32)


def config_graph(name):
    """The named synthetic workloads (sizes of the paper-shaped configurations).

    ``chunglu-1k``: Chung-Lu, gamma 2.1, n = 1,000, m = 10,000, seed 1.
    ``rmat-20``:    R-MAT (.57,.19,.19,.05), n = 2^20, m = 2^24, seed 1.
    ``rmat-22``:    R-MAT, n = 2^22, m = 2^26, seed 1.
    ``rmat-23``:    R-MAT, n = 2^23, m = 2^27, seed 1.
    Small variants for tests: ``rmat-<s>`` for any scale s uses m = 16 * 2^s.
    """
    if name == "chunglu-1k":
        s, d = chung_lu(1000, 10000, 2.1, seed=1)
        return 1000, s, d
    if name.startswith("rmat-"):
        scale = int(name.split("-")[1])
        return rmat(scale, 16 << scale, seed=1)
    raise KeyError(name)
