"""CPU oracle for range retrieval on a proximity graph -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never loads it, and the
two share no code.  The arithmetic is in ``oracle.c`` (plain C, exact int64
distances for 8-bit data, fp64 for fp32 data); this module only marshals
numpy arrays through ctypes and adds Def. 2.2 (average precision), which is a
two-line set computation.

Paper: "Range Retrieval with Graph-Based Indices" (arXiv 2502.13245),
Def. 2.1, Def. 2.2, Alg. 1-6.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(HERE, "_oracle.so")

BEAM, BEAM_ES, DOUBLING, DOUBLING_ES, GREEDY, GREEDY_ES, DOUBLING_WARM, DOUBLING_WARM_ES = range(8)
# doubling_warm(_es): a variant of Alg. 3 that continues each round from the last instead of restarting
VARIANTS = {"beam": BEAM, "beam_es": BEAM_ES, "doubling": DOUBLING, "doubling_es": DOUBLING_ES,
            "greedy": GREEDY, "greedy_es": GREEDY_ES, "doubling_warm": DOUBLING_WARM,
            "doubling_warm_es": DOUBLING_WARM_ES}
U8, I8, F32 = 0, 1, 2
L2, IP = 0, 1


def build(force: bool = False) -> str:
    """gcc -O2 -fopenmp oracle.c -> _oracle.so (OpenMP only for Alg. 6's parallel for)."""
    src = os.path.join(HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", _SO + ".tmp", src])
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _Index(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("metric", ctypes.c_int32), ("R", ctypes.c_int32), ("adj", ctypes.c_void_p),
                ("start", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("beam", ctypes.c_int32), ("b_max", ctypes.c_int32),
                ("es_vl", ctypes.c_int32), ("es_radius", ctypes.c_double), ("es_metric", ctypes.c_int32),
                ("expand", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("visits_beam", ctypes.c_int64), ("visits_greedy", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("distinct", ctypes.c_int64), ("rounds", ctypes.c_int32), ("phase", ctypes.c_int32),
                ("early_stopped", ctypes.c_int32), ("truncated", ctypes.c_int32), ("final_beam", ctypes.c_int32),
                ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.or_range_search_one.restype = ctypes.c_int64
        lib.or_range_search_one.argtypes = [P, P, ctypes.c_double, P, P, P, ctypes.c_int64, P]
        lib.or_beam_search.restype = ctypes.c_int
        lib.or_beam_search.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_int32, P, P, P, P, P, P]
        lib.or_greedy_search.restype = ctypes.c_int64
        lib.or_greedy_search.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double, P, P, P]
        lib.or_brute_force.restype = ctypes.c_int64
        lib.or_brute_force.argtypes = [P, P, ctypes.c_double, P, P, ctypes.c_int64]
        lib.or_distances.restype = None
        lib.or_distances.argtypes = [P, P, P, ctypes.c_int64, P]
        lib.or_range_search_batch.restype = ctypes.c_int
        lib.or_range_search_batch.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int, P, P, P, P]
        lib.or_free.restype = None
        lib.or_free.argtypes = [P]
        _lib = lib
    return _lib


def _dt(a):
    return {np.dtype(np.uint8): U8, np.dtype(np.int8): I8, np.dtype(np.float32): F32}[a.dtype]


class Index:
    """Holds the arrays the oracle reads: X (n x d), adj (n x R uint32, 0xFFFFFFFF pads), start id."""

    def __init__(self, X, adj, start, metric=L2):
        self.X = np.ascontiguousarray(X)
        self.adj = np.ascontiguousarray(adj, dtype=np.uint32)
        assert self.X.shape[0] == self.adj.shape[0]
        self.metric = metric
        self.start = int(start)
        self._s = _Index(self.X.ctypes.data, self.X.shape[0], self.X.shape[1], _dt(self.X), metric,
                         self.adj.shape[1], self.adj.ctypes.data, self.start)

    @property
    def n(self):
        return self.X.shape[0]

    def _q(self, q):
        q = np.ascontiguousarray(q, dtype=self.X.dtype)
        assert q.shape == (self.X.shape[1],)
        return q


ES_METRICS = {"visited": 0, "top1": 1, "top10": 2, "top10_ratio": 3}


def range_search_one(idx: Index, q, r, variant="greedy_es", beam=64, b_max=32768, es_vl=20, es_radius=None,
                     es_metric="visited", expand=1):
    """One query through Alg. 6 / Alg. 3 / plain beam search.  Returns (ids, dists, stats dict)."""
    q = idx._q(q)
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    p = _Params(v, beam, b_max, es_vl, float(r if es_radius is None else es_radius), ES_METRICS[es_metric], expand)
    st = Stats()
    cap = 1024
    while True:
        ids = np.empty(cap, np.uint32)
        ds = np.empty(cap, np.float64)
        c = _L().or_range_search_one(ctypes.byref(idx._s), q.ctypes.data, float(r), ctypes.byref(p), ids.ctypes.data,
                                     ds.ctypes.data, cap, ctypes.byref(st))
        if c < 0:
            raise MemoryError("oracle allocation failed")
        if c <= cap:
            return ids[:c].copy(), ds[:c].copy(), st.as_dict()
        cap = int(c)


def range_search(idx: Index, Q, r, variant="greedy_es", beam=64, b_max=32768, es_vl=20, es_radius=None,
                 threads=1, es_metric="visited", expand=1):
    """Batch driver (Alg. 6's parallel for; threads=1 is the single-threaded reference).

    r: scalar or per-query array.  es_radius None means esr = r per query.  es_metric: the early-stopping
    metric M of Alg. 4 -- "visited" (Alg. 5), "top1", "top10" (thresholds in distance units, es_radius) or
    "top10_ratio" (d_top10 / d_start against the ratio es_radius).  expand > 1 selects the multi-parent
    variant of Alg. 1 (that many closest unvisited points of B visited per iteration; not in the paper).
    Returns (list of id arrays, list of dist arrays, list of stats dicts)."""
    Q = np.ascontiguousarray(Q, dtype=idx.X.dtype)
    nq = Q.shape[0]
    radii = np.ascontiguousarray(np.broadcast_to(np.asarray(r, dtype=np.float64), (nq,)))
    if es_radius is not None and np.ndim(es_radius) == 0 and np.any(float(es_radius) != radii):
        # one esr for the whole batch: the C batch driver takes it from params (Alg. 6's parallel for)
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        p = _Params(v, beam, b_max, es_vl, float(es_radius), ES_METRICS[es_metric], expand)
        return _batch(idx, Q, radii, p, threads)
    if es_radius is not None and np.any(np.asarray(es_radius) != radii):
        # per-call esr differs from r: fall back to one call per query
        ids, ds, sts = [], [], []
        esr = np.broadcast_to(np.asarray(es_radius, dtype=np.float64), (nq,))
        for i in range(nq):
            a, b, s = range_search_one(idx, Q[i], radii[i], variant, beam, b_max, es_vl, esr[i], es_metric, expand)
            ids.append(a); ds.append(b); sts.append(s)
        return ids, ds, sts
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    p = _Params(v, beam, b_max, es_vl, float("nan"), ES_METRICS[es_metric], expand)
    # esr = r per query: the C batch driver reads es_radius from params, so run per distinct radius
    out_ids, out_d, out_s = [None] * nq, [None] * nq, [None] * nq
    for rv in np.unique(radii):
        sel = np.nonzero(radii == rv)[0]
        p.es_radius = float(rv)
        a, b, c = _batch(idx, np.ascontiguousarray(Q[sel]), np.ascontiguousarray(radii[sel]), p, threads)
        for k, i in enumerate(sel):
            out_ids[i], out_d[i], out_s[i] = a[k], b[k], c[k]
    return out_ids, out_d, out_s


def _batch(idx: Index, Qs, rs, p, threads):
    """or_range_search_batch over queries Qs with radii rs and the given params (marshalling only)."""
    m = Qs.shape[0]
    counts = np.zeros(m, np.int64)
    pid = (ctypes.c_void_p * m)()
    pd = (ctypes.c_void_p * m)()
    stats = (Stats * m)()
    rc = _L().or_range_search_batch(ctypes.byref(idx._s), Qs.ctypes.data, m, rs.ctypes.data, ctypes.byref(p),
                                    int(threads), counts.ctypes.data, pid, pd, stats)
    out_ids, out_d, out_s = [], [], []
    for k in range(m):
        c = int(counts[k])
        if c > 0:
            out_ids.append(np.ctypeslib.as_array(ctypes.cast(pid[k], ctypes.POINTER(ctypes.c_uint32)), (c,)).copy())
            out_d.append(np.ctypeslib.as_array(ctypes.cast(pd[k], ctypes.POINTER(ctypes.c_double)), (c,)).copy())
        else:
            out_ids.append(np.zeros(0, np.uint32))
            out_d.append(np.zeros(0, np.float64))
        out_s.append(stats[k].as_dict())
        _L().or_free(pid[k])
        _L().or_free(pd[k])
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out_ids, out_d, out_s


def beam_search(idx: Index, q, S, r, b, use_es=False, es_vl=20, es_radius=None, es_metric="visited"):
    """Alg. 1 (+ Alg. 5 when use_es).  Returns (B ids sorted, B dists, V ids in visit order, stopped, stats)."""
    q = idx._q(q)
    S = np.ascontiguousarray(S, dtype=np.uint32)
    cap = len(S) + idx.n + idx.adj.shape[1] + 1
    bi = np.empty(cap, np.uint32)
    bd = np.empty(cap, np.float64)
    vi = np.empty(idx.n, np.uint32)
    nB = ctypes.c_int64()
    nV = ctypes.c_int64()
    st = Stats()
    esr = float(r if es_radius is None else es_radius)
    rc = _L().or_beam_search(ctypes.byref(idx._s), q.ctypes.data, S.ctypes.data, len(S), float(r), int(b),
                             int(bool(use_es)), int(es_vl), esr, ES_METRICS[es_metric], bi.ctypes.data, bd.ctypes.data, ctypes.byref(nB),
                             vi.ctypes.data, ctypes.byref(nV), ctypes.byref(st))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return bi[:nB.value].copy(), bd[:nB.value].copy(), vi[:nV.value].copy(), bool(rc), st.as_dict()


def greedy_search(idx: Index, q, S, r):
    """Alg. 2.  Returns (V ids in visit order, their dists, stats)."""
    q = idx._q(q)
    S = np.ascontiguousarray(S, dtype=np.uint32)
    oi = np.empty(idx.n, np.uint32)
    od = np.empty(idx.n, np.float64)
    st = Stats()
    c = _L().or_greedy_search(ctypes.byref(idx._s), q.ctypes.data, S.ctypes.data, len(S), float(r), oi.ctypes.data,
                              od.ctypes.data, ctypes.byref(st))
    if c < 0:
        raise MemoryError("oracle allocation failed")
    return oi[:c].copy(), od[:c].copy(), st.as_dict()


def brute_force(idx: Index, q, r):
    """Def. 2.1 by exhaustive scan: (ids, dists) of every point with d <= r, sorted by (dist, id)."""
    q = idx._q(q)
    cap = 1024
    while True:
        ids = np.empty(cap, np.uint32)
        ds = np.empty(cap, np.float64)
        c = _L().or_brute_force(ctypes.byref(idx._s), q.ctypes.data, float(r), ids.ctypes.data, ds.ctypes.data, cap)
        if c < 0:
            raise MemoryError("oracle allocation failed")
        if c <= cap:
            return ids[:c].copy(), ds[:c].copy()
        cap = int(c)


def distances(idx: Index, q, ids):
    q = idx._q(q)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.empty(len(ids), np.float64)
    _L().or_distances(ctypes.byref(idx._s), q.ctypes.data, ids.ctypes.data, len(ids), out.ctypes.data)
    return out


def average_precision(truth, found):
    """Def. 2.2: sum_q |K_q n K'_q| / sum_q |K_q|.  With no true results at all the ratio is
    0/0; it is reported as 1.0 (nothing was missed)."""
    num = 0
    den = 0
    for t, f in zip(truth, found):
        t = np.asarray(t)
        den += len(t)
        num += len(np.intersect1d(t, np.asarray(f)))
    return 1.0 if den == 0 else num / den
