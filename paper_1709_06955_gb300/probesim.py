"""Thin ctypes binding of libprobesim.so (include/probesim.h).

Argument marshalling only: every step of a query runs in the library's CUDA kernels.  Buffers may be
numpy arrays (host) or torch tensors (host or CUDA); device outputs are torch tensors on the current
CUDA device.  ``load()`` raises if the library has not been built -- there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libprobesim.so")

OK, E_INVALID, E_RANGE, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUSY, E_UNSUPPORTED = range(8)
PROBE_DETERMINISTIC, PROBE_RANDOMIZED, PROBE_SWITCH = 0, 1, 2

EXPORTS = [
    "probesim_config_default", "probesim_graph_create", "probesim_graph_destroy", "probesim_graph_info",
    "probesim_insert_edges", "probesim_delete_edges", "probesim_num_walks", "probesim_sample_walks",
    "probesim_single_source", "probesim_topk", "probesim_set_profiling", "probesim_get_stats",
    "probesim_last_error", "probesim_topk_select_noalloc", "probesim_server_config_default",
    "probesim_server_create", "probesim_server_submit", "probesim_server_update", "probesim_server_poll",
    "probesim_server_get_stats", "probesim_server_destroy", "probesim_autotune", "probesim_get_tuning",
    "probesim_set_tuning",
    "probesim_set_memory_budget", "probesim_split_error", "probesim_pair_mc",
]


class Config(C.Structure):
    _fields_ = [("c", C.c_double), ("delta", C.c_double), ("l_max", C.c_int32), ("eps_p", C.c_float),
                ("c0", C.c_float), ("probe_mode", C.c_int32), ("seed", C.c_uint32), ("shift", C.c_float)]


class ErrorSplit(C.Structure):
    _fields_ = [("eps", C.c_double), ("eps_t", C.c_double), ("l_max", C.c_int32), ("eps_p", C.c_float),
                ("shift", C.c_float), ("bound", C.c_double), ("bound_paper", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Query(C.Structure):
    _fields_ = [("node", C.c_int32), ("k", C.c_int32), ("eps", C.c_double), ("query_id", C.c_uint32),
                ("walk_begin", C.c_int32), ("walk_end", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("walks", C.c_int64), ("walk_nodes", C.c_int64), ("tree_nodes", C.c_int64), ("vectors", C.c_int64),
                ("levels", C.c_int64), ("edge_gathers", C.c_int64), ("probe_launches", C.c_int64),
                ("probe_ms", C.c_double), ("probe_bytes", C.c_double), ("kernel_launches", C.c_int64),
                ("phase_ms", C.c_double * 12), ("max_columns", C.c_int64), ("probes", C.c_int64),
                ("switched", C.c_int64), ("table_passes", C.c_int64), ("max_table_slots", C.c_int64),
                ("deferred", C.c_int64)]

    PHASES = ["walks", "tree", "accumulate", "scatter", "zero_rows", "pull", "push", "gamma", "estimates",
              "host_schedule"]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_ms"}
        d["phase_ms"] = {name: self.phase_ms[i] for i, name in enumerate(self.PHASES)}
        return d


class ServerConfig(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_batch", C.c_int32), ("kmax", C.c_int32), ("queue_capacity", C.c_int32),
                ("memory_budget_bytes", C.c_double)]


class Result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("query_id", C.c_uint32), ("node", C.c_int32), ("k", C.c_int32),
                ("status", C.c_int32), ("epoch", C.c_uint64), ("batch_size", C.c_int32), ("worker", C.c_int32),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64), ("failed", C.c_int64),
                ("batches", C.c_int64), ("updates_applied", C.c_int64), ("mean_batch", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("qps", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProbeSimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("probesim status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load(path=None):
    """Loads libprobesim.so (built by ``paper_1709_06955_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libprobesim.so is not built (%s); run paper_1709_06955_gb300.build.build()" % path)
    L = C.CDLL(path)
    P = C.POINTER
    vp = C.c_void_p
    L.probesim_last_error.restype = C.c_char_p
    L.probesim_config_default.argtypes = [P(Config)]
    L.probesim_graph_create.argtypes = [C.c_int32, vp, vp, C.c_int64, P(Config), vp, P(vp)]
    L.probesim_graph_destroy.argtypes = [vp]
    L.probesim_graph_info.argtypes = [vp, P(C.c_int32), P(C.c_int64), P(C.c_uint64)]
    L.probesim_insert_edges.argtypes = [vp, vp, vp, C.c_int64, P(C.c_int64), vp]
    L.probesim_delete_edges.argtypes = [vp, vp, vp, C.c_int64, P(C.c_int64), vp]
    L.probesim_num_walks.argtypes = [vp, C.c_double, P(C.c_int64)]
    L.probesim_sample_walks.argtypes = [vp, P(Query), C.c_int32, vp, vp, C.c_int64, vp]
    L.probesim_single_source.argtypes = [vp, P(Query), C.c_int32, vp, vp]
    L.probesim_topk.argtypes = [vp, P(Query), C.c_int32, C.c_int32, vp, vp, vp]
    L.probesim_set_profiling.argtypes = [vp, C.c_int32]
    L.probesim_set_memory_budget.argtypes = [vp, C.c_double]
    L.probesim_split_error.argtypes = [C.c_double, C.c_double, C.c_int32, P(ErrorSplit)]
    L.probesim_pair_mc.argtypes = [vp, vp, vp, vp, vp, C.c_int32, C.c_int64, vp, vp, vp]
    L.probesim_get_stats.argtypes = [vp, P(Stats)]
    L.probesim_topk_select_noalloc.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, C.c_int32, vp, vp, vp]
    L.probesim_server_config_default.argtypes = [P(ServerConfig)]
    L.probesim_server_create.argtypes = [vp, P(ServerConfig), P(vp)]
    L.probesim_server_submit.argtypes = [vp, P(Query), C.c_int32, P(C.c_uint64)]
    L.probesim_server_update.argtypes = [vp, vp, vp, C.c_int64, C.c_int32]
    L.probesim_server_poll.argtypes = [vp, C.c_int32, C.c_int32, P(Result), vp, vp, P(C.c_int32), C.c_int32]
    L.probesim_server_get_stats.argtypes = [vp, P(ServerStats)]
    L.probesim_server_destroy.argtypes = [vp]
    L.probesim_autotune.argtypes = [vp, vp]
    L.probesim_get_tuning.argtypes = [vp, P(C.c_int32), P(C.c_int32)]
    L.probesim_set_tuning.argtypes = [vp, C.c_int32, P(C.c_int32)]
    for name in EXPORTS:
        if name != "probesim_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st):
    if st != OK:
        raise ProbeSimError(st, load().probesim_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(x.ctypes.data)


def _int32(x):
    if _is_torch(x):
        import torch
        return x.to(torch.int32).contiguous()
    return np.ascontiguousarray(x, dtype=np.int32)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001 -- a missing torch only means the default stream
        pass
    return C.c_void_p(0)


def default_config(**kw):
    cfg = Config()
    _check(load().probesim_config_default(C.byref(cfg)))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def split_error(eps_a, c=0.6, shift=True):
    """Thm. 2's split of a target error eps_a into eps, eps_t (l_max), eps_p and the eps_t/2 shift
    (probesim_split_error).  Returns a dict; its l_max, eps_p and shift go into the graph's config."""
    out = ErrorSplit()
    _check(load().probesim_split_error(float(eps_a), float(c), 1 if shift else 0, C.byref(out)))
    return out.as_dict()


def make_queries(nodes, eps=0.1, k=50, query_ids=None, walk_begin=0, walk_end=0):
    """Packs query nodes (and per-query eps/k/query_id, scalars or sequences) into a Query array."""
    nodes = np.asarray(nodes, dtype=np.int64).ravel()
    nq = nodes.size
    arr = (Query * nq)()
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (nq,))
    k = np.broadcast_to(np.asarray(k, dtype=np.int64), (nq,))
    qid = np.arange(nq, dtype=np.int64) if query_ids is None else np.broadcast_to(np.asarray(query_ids), (nq,))
    wb = np.broadcast_to(np.asarray(walk_begin), (nq,))
    we = np.broadcast_to(np.asarray(walk_end), (nq,))
    for i in range(nq):
        arr[i] = Query(int(nodes[i]), int(k[i]), float(eps[i]), int(qid[i]) & 0xFFFFFFFF, int(wb[i]), int(we[i]))
    return arr


def topk_select_noalloc(scores, nodes, ks, kmax, ids, vals, stream=None):
    """Top-k of caller-provided device score rows without any allocation (probesim_topk_select_noalloc).

    For callers that cannot allocate device memory while they run.  ``scores`` is a CUDA tensor [nq, n];
    ``ids`` / ``vals`` are CUDA tensors [nq, kmax] (int32 / float32) that receive the results; ``nodes`` and
    ``ks`` are host sequences of length nq.  At most 64 queries and kmax <= 1024 per call."""
    import torch
    if not (_is_torch(scores) and scores.dtype == torch.float32 and scores.dim() == 2):
        raise ValueError("scores must be a 2-d float32 tensor [nq, n]")
    nq, n = int(scores.shape[0]), int(scores.shape[1])
    nodes = np.ascontiguousarray(nodes, dtype=np.int32).ravel()
    ks = np.ascontiguousarray(ks, dtype=np.int32).ravel()
    if nodes.size != nq or ks.size != nq:
        raise ValueError("nodes and ks must hold one entry per score row (%d)" % nq)
    for name, t, dt in (("ids", ids, torch.int32), ("vals", vals, torch.float32)):
        if not (_is_torch(t) and t.dtype == dt and tuple(t.shape) == (nq, int(kmax))):
            raise ValueError("%s must be a %s tensor of shape (%d, %d)" % (name, dt, nq, int(kmax)))
    for name, t in (("scores", scores), ("ids", ids), ("vals", vals)):
        if not t.is_cuda or t.device != scores.device:
            raise ValueError("%s must be CUDA memory on one device" % name)
    _check(load().probesim_topk_select_noalloc(_ptr(scores), n, nq, _ptr(nodes), _ptr(ks), int(kmax), _ptr(ids),
                                               _ptr(vals), _stream(stream)))
    return ids, vals


class Graph:
    """A device-resident graph store with ProbeSim queries over it."""

    def __init__(self, n, src, dst, config=None, stream=None, **cfg_kw):
        L = load()
        self.n = int(n)
        cfg = config if config is not None else default_config(**cfg_kw)
        src = _int32(src)
        dst = _int32(dst)
        m = int(src.numel() if _is_torch(src) else src.size)
        h = C.c_void_p()
        _check(L.probesim_graph_create(self.n, _ptr(src), _ptr(dst), m, C.byref(cfg), _stream(stream), C.byref(h)))
        self._h = h
        self.config = cfg

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().probesim_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass

    def info(self):
        n, m, ep = C.c_int32(), C.c_int64(), C.c_uint64()
        _check(load().probesim_graph_info(self._h, C.byref(n), C.byref(m), C.byref(ep)))
        return n.value, m.value, ep.value

    def num_walks(self, eps):
        r = C.c_int64()
        _check(load().probesim_num_walks(self._h, float(eps), C.byref(r)))
        return r.value

    def insert_edges(self, src, dst, stream=None):
        src, dst = _int32(src), _int32(dst)
        k = int(src.numel() if _is_torch(src) else src.size)
        a = C.c_int64()
        _check(load().probesim_insert_edges(self._h, _ptr(src), _ptr(dst), k, C.byref(a), _stream(stream)))
        return a.value

    def delete_edges(self, src, dst, stream=None):
        src, dst = _int32(src), _int32(dst)
        k = int(src.numel() if _is_torch(src) else src.size)
        a = C.c_int64()
        _check(load().probesim_delete_edges(self._h, _ptr(src), _ptr(dst), k, C.byref(a), _stream(stream)))
        return a.value

    def sample_walks(self, queries, stream=None):
        """Walk node sequences of the queries: (nodes [W, l_max] int32 padded with -1, lens [W])."""
        W = 0
        for q in queries:
            nr = self.num_walks(q.eps)
            kb = max(0, q.walk_begin)
            ke = nr if q.walk_end <= 0 else min(q.walk_end, nr)
            W += max(0, ke - kb)
        lm = self.config.l_max
        nodes = np.zeros((max(1, W), lm), np.int32)
        lens = np.zeros(max(1, W), np.int32)
        _check(load().probesim_sample_walks(self._h, queries, len(queries), _ptr(nodes), _ptr(lens), W,
                                            _stream(stream)))
        return nodes[:W], lens[:W]

    def single_source(self, queries, out=None, stream=None):
        """s~(u, .) for every query: a [nq, n] float32 array (numpy) or the given ``out`` buffer."""
        nq = len(queries)
        if out is None:
            out = np.zeros((nq, self.n), np.float32)
        _check(load().probesim_single_source(self._h, queries, nq, _ptr(out), _stream(stream)))
        return out

    def topk(self, queries, kmax=None, ids=None, vals=None, stream=None):
        nq = len(queries)
        kmax = int(kmax or max(q.k for q in queries))
        if ids is None:
            ids = np.zeros((nq, kmax), np.int32)
        if vals is None:
            vals = np.zeros((nq, kmax), np.float32)
        _check(load().probesim_topk(self._h, queries, nq, kmax, _ptr(ids), _ptr(vals), _stream(stream)))
        return ids, vals

    def pair_mc(self, u, v, key_u, key_v, r, stream=None):
        """Pairwise Monte Carlo SimRank of the pairs (u[i], v[i]) from r walk pairs each (probesim_pair_mc):
        (meet counts int64, estimates float32)."""
        u, v = _int32(u).ravel(), _int32(v).ravel()
        ku = np.ascontiguousarray(key_u, dtype=np.uint32).ravel()
        kv = np.ascontiguousarray(key_v, dtype=np.uint32).ravel()
        npairs = u.size
        if not (v.size == ku.size == kv.size == npairs):
            raise ValueError("u, v, key_u and key_v must have one entry per pair")
        meets = np.zeros(npairs, np.int64)
        est = np.zeros(npairs, np.float32)
        _check(load().probesim_pair_mc(self._h, _ptr(u), _ptr(v), _ptr(ku), _ptr(kv), npairs, int(r), _ptr(meets),
                                       _ptr(est), _stream(stream)))
        return meets, est

    def autotune(self, stream=None):
        """Times the pull launch shapes on this graph and keeps the fastest (probesim_autotune)."""
        _check(load().probesim_autotune(self._h, _stream(stream)))
        return self.tuning()

    def tuning(self):
        wide = C.c_int32()
        bps = (C.c_int32 * 6)()
        _check(load().probesim_get_tuning(self._h, C.byref(wide), bps))
        return {"wide_tile": wide.value, "blocks_per_sm": {1 << i: bps[i] for i in range(6)}}

    def set_tuning(self, wide_tile, blocks_per_sm=None):
        """Sets the pull's launch shape by hand (probesim_set_tuning): wide_tile 16, 32, 64 (32-column tiles two per
        pass) or 96 (32-column tiles gathered by the TMA); blocks_per_sm, if given, 8 values for tile widths 1..32,
        the pairs and the TMA launch."""
        arr = None
        if blocks_per_sm is not None:
            vals = [int(b) for b in blocks_per_sm]
            if len(vals) != 8:
                raise ValueError("blocks_per_sm needs 8 values")
            arr = (C.c_int32 * 8)(*vals)
        _check(load().probesim_set_tuning(self._h, int(wide_tile), arr))

    def set_memory_budget(self, nbytes):
        """Device memory one call's working buffers may take (0 = the default, 60% of the device)."""
        _check(load().probesim_set_memory_budget(self._h, float(nbytes)))

    def set_profiling(self, on=True):
        _check(load().probesim_set_profiling(self._h, 1 if on else 0))

    def stats(self):
        s = Stats()
        _check(load().probesim_get_stats(self._h, C.byref(s)))
        return s.as_dict()


class Server:
    """Continuous-batching top-k server over a Graph (probesim_server_*)."""

    def __init__(self, graph, workers=3, max_batch=2, kmax=100, queue_capacity=100000, memory_budget_bytes=0.0):
        L = load()
        cfg = ServerConfig()
        _check(L.probesim_server_config_default(C.byref(cfg)))
        cfg.workers, cfg.max_batch, cfg.kmax = int(workers), int(max_batch), int(kmax)
        cfg.queue_capacity, cfg.memory_budget_bytes = int(queue_capacity), float(memory_budget_bytes)
        h = C.c_void_p()
        _check(L.probesim_server_create(graph._h, C.byref(cfg), C.byref(h)))
        self._h = h
        self.graph = graph
        self.kmax = int(kmax)

    def submit(self, queries):
        t = (C.c_uint64 * len(queries))()
        _check(load().probesim_server_submit(self._h, queries, len(queries), t))
        return list(t)

    def update(self, src, dst, insert=True):
        src, dst = _int32(src), _int32(dst)
        _check(load().probesim_server_update(self._h, _ptr(src), _ptr(dst), int(src.size), 1 if insert else 0))

    def poll(self, max_results=64, wait_ms=100):
        """Finished results: a list of (Result, ids[kmax], vals[kmax])."""
        res = (Result * max_results)()
        ids = np.zeros((max_results, self.kmax), np.int32)
        vals = np.zeros((max_results, self.kmax), np.float32)
        cnt = C.c_int32()
        _check(load().probesim_server_poll(self._h, max_results, self.kmax, res, _ptr(ids), _ptr(vals), C.byref(cnt),
                                           int(wait_ms)))
        return [(res[i], ids[i].copy(), vals[i].copy()) for i in range(cnt.value)]

    def stats(self):
        st = ServerStats()
        _check(load().probesim_server_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().probesim_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass
