"""All-pairs SimRank by the Power Method (Eq. 6: S = (c P^T S P) v I from S = I) -- test infrastructure only.

P is the transition matrix with P[x, v] = 1/|I(v)| for every edge x -> v, so (P^T S P)[u, v] is the average
of S[x, y] over x in I(u), y in I(v), which is Eq. 1 for u != v.  Dense FP64, O(n^2) memory: tiny graphs only.
"""
import numpy as np


def transition(n, src, dst):
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    indeg = np.bincount(dst, minlength=n).astype(np.float64)
    P = np.zeros((n, n), np.float64)
    P[src, dst] = 1.0 / indeg[dst]
    return P


def simrank(n, src, dst, c, iters):
    """S after ``iters`` iterations of S <- max(c P^T S P, I) elementwise, starting at S = I."""
    P = transition(n, src, dst)
    S = np.eye(n)
    for _ in range(iters):
        S = np.maximum(c * (P.T @ S @ P), np.eye(n))
    return S
