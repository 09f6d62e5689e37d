"""Helpers shared by the GPU parity tests."""
import numpy as np

TOL = 1e-5  # max-abs bound on scores: FP32 path vs FP64 oracle


def gpu_graph(n, s, d, **cfg):
    from paper_1709_06955_gb300 import probesim
    return probesim.Graph(n, s, d, **cfg)


def oracle_graph(n, s, d):
    from oracle import core
    return core.Graph(n, s, d)


def dedup(n, s, d):
    """The simple graph a multigraph edge list denotes: loops dropped, duplicates merged."""
    s = np.asarray(s, np.int64)
    d = np.asarray(d, np.int64)
    keep = s != d
    k = np.unique(s[keep] * n + d[keep])
    return (k // n).astype(np.int32), (k % n).astype(np.int32)
