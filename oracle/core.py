"""ctypes wrapper of the C oracle (``probesim_oracle.c``) -- test infrastructure only.

Every function here forwards to the C routine that restates the cited passage of the paper.
"""
import ctypes as C
import numpy as np

from . import build as _build

_lib = None


class Counters(C.Structure):
    _fields_ = [("edge_pushes", C.c_int64), ("rand_samples", C.c_int64), ("probes", C.c_int64),
                ("walks", C.c_int64), ("walk_nodes", C.c_int64), ("tree_nodes", C.c_int64),
                ("switched", C.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Params(C.Structure):
    _fields_ = [("c", C.c_double), ("eps", C.c_double), ("delta", C.c_double), ("eps_p", C.c_double),
                ("c0", C.c_double), ("l_max", C.c_int32), ("probe_mode", C.c_int32), ("seed", C.c_uint32),
                ("query_id", C.c_uint32), ("walk_begin", C.c_int64), ("walk_end", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_threshold_stop.restype = C.c_uint32
        L.orc_threshold_stop.argtypes = [C.c_double]
        L.orc_threshold_keep.restype = C.c_uint32
        L.orc_threshold_keep.argtypes = [C.c_double]
        L.orc_graph_new.restype = C.c_void_p
        L.orc_graph_new.argtypes = [C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int32)]
        L.orc_graph_free.argtypes = [C.c_void_p]
        L.orc_in_degree.restype = C.c_int64
        L.orc_in_degree.argtypes = [C.c_void_p, C.c_int32]
        L.orc_out_degree.restype = C.c_int64
        L.orc_out_degree.argtypes = [C.c_void_p, C.c_int32]
        L.orc_num_walks.restype = C.c_int64
        L.orc_num_walks.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int64]
        L.orc_walk.restype = C.c_int32
        L.orc_walk.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_uint32, C.c_uint32, C.c_uint32,
                               P(C.c_int32)]
        L.orc_probe_det.restype = C.c_int
        L.orc_probe_det.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, C.c_double, C.c_double, P(C.c_double)]
        L.orc_probe_rand.restype = C.c_int
        L.orc_probe_rand.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, C.c_double, C.c_uint32, C.c_uint32,
                                     C.c_uint32, P(C.c_double)]
        for fn in (L.orc_single_source, L.orc_single_source_batch):
            fn.restype = C.c_int
            fn.argtypes = [C.c_void_p, C.c_int32, P(Params), P(C.c_double), P(Counters)]
        L.orc_topk.restype = C.c_int32
        L.orc_topk.argtypes = [P(C.c_double), C.c_int32, C.c_int32, C.c_int32, P(C.c_int32), P(C.c_double)]
        L.orc_pair_mc.restype = C.c_double
        L.orc_pair_mc.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_uint32, C.c_uint32,
                                  C.c_uint32, C.c_int64]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter under a 2-word key (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def threshold_stop(c):
    return int(lib().orc_threshold_stop(float(c)))


def threshold_keep(c):
    return int(lib().orc_threshold_keep(float(c)))


def num_walks(c, eps, delta, n):
    """n_r = ceil(3c / eps^2 * ln(n / delta)) (Alg. 1 line 1)."""
    return int(lib().orc_num_walks(float(c), float(eps), float(delta), int(n)))


class Graph:
    """In/out adjacency of a directed simple graph; in-lists and out-lists sorted by id."""

    def __init__(self, n, src, dst):
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.m = int(self.src.size)
        self._h = lib().orc_graph_new(self.n, self.m, _ptr(self.src, C.c_int32), _ptr(self.dst, C.c_int32))
        if not self._h:
            raise ValueError("not a directed simple graph on [0, n) (self-loop, duplicate or bad id)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_graph_free(h)
            self._h = None

    def in_degree(self, v):
        return int(lib().orc_in_degree(self._h, int(v)))

    def out_degree(self, v):
        return int(lib().orc_out_degree(self._h, int(v)))

    def walk(self, u, c, l_max, seed, qid, k):
        """One sqrt(c)-walk W_k(u) (Def. 3), at most l_max nodes."""
        buf = np.zeros(max(1, l_max), np.int32)
        ln = lib().orc_walk(self._h, int(u), float(c), int(l_max), int(seed), int(qid), int(k), _ptr(buf, C.c_int32))
        return buf[:ln].copy()

    def probe(self, path, c, eps_p=0.0):
        """Deterministic PROBE (Alg. 2) on the partial walk ``path``; returns Score over V."""
        p = np.ascontiguousarray(path, dtype=np.int32)
        out = np.zeros(self.n, np.float64)
        if lib().orc_probe_det(self._h, _ptr(p, C.c_int32), int(p.size), float(c), float(eps_p), _ptr(out, C.c_double)):
            raise ValueError("bad probe path")
        return out

    def probe_rand(self, path, c, seed, qid, k):
        """Randomized PROBE (Alg. 3) of walk k on ``path``; returns the 0/1 scores over V."""
        p = np.ascontiguousarray(path, dtype=np.int32)
        out = np.zeros(self.n, np.float64)
        if lib().orc_probe_rand(self._h, _ptr(p, C.c_int32), int(p.size), float(c), int(seed), int(qid), int(k),
                                _ptr(out, C.c_double)):
            raise ValueError("bad probe path")
        return out

    def single_source(self, u, c=0.6, eps=0.1, delta=0.01, l_max=64, seed=3, qid=0, eps_p=0.0,
                      probe_mode=0, c0=1.0, walk_begin=0, walk_end=0, batch=False):
        """s(u, .) by Basic ProbeSim (Alg. 1), or by the batch algorithm with the switch (Alg. 4,
        Sec. 4.4) when ``batch``.  Returns (estimates, counters)."""
        prm = Params(float(c), float(eps), float(delta), float(eps_p), float(c0), int(l_max), int(probe_mode),
                     int(seed), int(qid), int(walk_begin), int(walk_end))
        out = np.zeros(self.n, np.float64)
        cnt = Counters()
        fn = lib().orc_single_source_batch if batch else lib().orc_single_source
        if fn(self._h, int(u), C.byref(prm), _ptr(out, C.c_double), C.byref(cnt)):
            raise ValueError("bad query")
        return out, cnt.as_dict()

    def pair_mc(self, u, v, c, l_max, seed, key_u, key_v, r):
        """Pairwise Monte Carlo estimate of s(u, v) from r walk pairs (Sec. 2.2, Eq. 3)."""
        return float(lib().orc_pair_mc(self._h, int(u), int(v), float(c), int(l_max), int(seed), int(key_u),
                                       int(key_v), int(r)))


def topk(s, u, k):
    """The k nodes v != u with the largest estimates, by (estimate desc, id asc) (Def. 2)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    ids = np.zeros(max(1, k), np.int32)
    vals = np.zeros(max(1, k), np.float64)
    kk = lib().orc_topk(_ptr(s, C.c_double), int(s.size), int(u), int(k), _ptr(ids, C.c_int32), _ptr(vals, C.c_double))
    return ids[:kk].copy(), vals[:kk].copy()
