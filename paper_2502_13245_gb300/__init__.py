"""GB300-native batched range retrieval on a proximity graph.

Python binding of ``librr.so`` (C ABI in ``include/rr.h``): argument
marshalling only, every step of the search runs in the library's CUDA
kernels.  The functions named ``rr_*`` mirror the C entry points one to one;
``Index`` is a small convenience wrapper over them.

Method: "Range Retrieval with Graph-Based Indices" (arXiv 2502.13245) --
Alg. 1 BeamSearch, Alg. 5 early stopping, Alg. 2 GreedySearch, Alg. 3
DoublingSearch and the Alg. 6 driver, over a Vamana-style graph.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB, build  # noqa: F401

RR_OK, RR_EINVAL, RR_ENOMEM, RR_ECUDA, RR_EFORMAT, RR_EOVERFLOW, RR_ETIMEOUT, RR_EBUSY, RR_EINTERNAL = range(9)
STATUS_NAMES = ["RR_OK", "RR_EINVAL", "RR_ENOMEM", "RR_ECUDA", "RR_EFORMAT", "RR_EOVERFLOW", "RR_ETIMEOUT",
                "RR_EBUSY", "RR_EINTERNAL"]
RR_BEAM, RR_BEAM_ES, RR_DOUBLING, RR_DOUBLING_ES, RR_GREEDY, RR_GREEDY_ES, RR_DOUBLING_WARM, RR_DOUBLING_WARM_ES = \
    range(8)
VARIANTS = {"beam": RR_BEAM, "beam_es": RR_BEAM_ES, "doubling": RR_DOUBLING, "doubling_es": RR_DOUBLING_ES,
            "greedy": RR_GREEDY, "greedy_es": RR_GREEDY_ES, "doubling_warm": RR_DOUBLING_WARM,
            "doubling_warm_es": RR_DOUBLING_WARM_ES}
RR_U8, RR_I8, RR_F32 = 0, 1, 2
RR_L2, RR_IP = 0, 1
RR_PREC_EXACT, RR_PREC_BF16, RR_PREC_FP8 = 0, 1, 2
RR_ES_VISITED, RR_ES_TOP1, RR_ES_TOP10, RR_ES_TOP10_RATIO = 0, 1, 2, 3
RR_ORDER_BFS = 1
RR_FLAG_TRUNCATED, RR_FLAG_EARLY_STOPPED, RR_FLAG_PHASE2, RR_FLAG_CANCELED = 1, 2, 4, 8

# every symbol include/rr.h declares (checked by the ABI test)
EXPORTS = ["rr_params_init", "rr_create_index", "rr_load_index", "rr_free_index", "rr_index_info_get",
           "rr_range_search", "rr_brute_force", "rr_result_free", "rr_last_error", "rr_last_profile",
           "rr_beam_search_noalloc", "rr_serve_cfg_init", "rr_serve_create", "rr_serve_submit", "rr_serve_poll",
           "rr_serve_collect", "rr_serve_cancel", "rr_serve_stats", "rr_serve_destroy", "rr_result_to_host",
           "rr_abi_sizes", "rr_debug_set", "rr_build_graph", "rr_index_relabel"]


class RRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("b_max", ctypes.c_int32), ("es_visit_limit", ctypes.c_int32),
                ("es_radius_mode", ctypes.c_int32), ("es_radius", ctypes.c_double), ("precision", ctypes.c_int32),
                ("recheck_eps", ctypes.c_float), ("persistent", ctypes.c_int32), ("collect_stats", ctypes.c_int32),
                ("max_results_total", ctypes.c_int64), ("tile_hint", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("seen_log2", ctypes.c_int32), ("es_metric", ctypes.c_int32),
                ("expand", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Profile(ctypes.Structure):
    _fields_ = [("beam_ms", ctypes.c_float), ("phase2_ms", ctypes.c_float), ("output_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("launches", ctypes.c_int32), ("phase2_steps", ctypes.c_int32),
                ("phase2_queries", ctypes.c_int32), ("valid", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeCfg(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("batch_wait_us", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("params", Params), ("result_budget_bytes", ctypes.c_int64),
                ("reserve_per_request", ctypes.c_int64), ("result_on_device", ctypes.c_int32),
                ("reserved_cfg", ctypes.c_int32 * 3)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("polled", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double), ("qps", ctypes.c_double),
                ("bytes_held", ctypes.c_int64), ("admission_waits", ctypes.c_int64), ("canceled", ctypes.c_int64),
                ("reserve_per_request", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class QueryStats(ctypes.Structure):
    _fields_ = [("visits_beam", ctypes.c_int32), ("visits_phase2", ctypes.c_int32), ("distinct", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("final_beam", ctypes.c_int32), ("evals", ctypes.c_int32)]


STATS_DTYPE = np.dtype([(n, np.int32) for n, _ in QueryStats._fields_])


class Result(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int64), ("total", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("ids", ctypes.c_void_p), ("dists", ctypes.c_void_p), ("dist_dtype", ctypes.c_int32),
                ("on_device", ctypes.c_int32), ("flags", ctypes.c_void_p), ("stats", ctypes.c_void_p),
                ("_stream", ctypes.c_void_p), ("_device", ctypes.c_int32), ("_pad", ctypes.c_int32)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("dtype", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("R", ctypes.c_int32), ("start", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("row_stride", ctypes.c_int32), ("device", ctypes.c_int32), ("scratch_bytes", ctypes.c_int64),
                ("order", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BuildInfo(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("repaired", ctypes.c_int64), ("gpu_seconds", ctypes.c_double),
                ("repair_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str | None = None):
    """Load librr.so.  There is no fallback: a missing or unloadable library raises."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError("librr.so is not built (%s); run paper_2502_13245_gb300.build()" % path)
    L = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.rr_params_init.restype = None
    L.rr_params_init.argtypes = [P]
    L.rr_create_index.restype = ctypes.c_int
    L.rr_create_index.argtypes = [P, I64, I32, I32, I32, P, I32, I64, I32, I32, P]
    L.rr_load_index.restype = ctypes.c_int
    L.rr_load_index.argtypes = [ctypes.c_char_p, I32, P]
    L.rr_free_index.restype = ctypes.c_int
    L.rr_free_index.argtypes = [P]
    L.rr_index_info_get.restype = ctypes.c_int
    L.rr_index_info_get.argtypes = [P, P]
    L.rr_index_relabel.restype = ctypes.c_int
    L.rr_index_relabel.argtypes = [P, I32]
    L.rr_range_search.restype = ctypes.c_int
    L.rr_range_search.argtypes = [P, P, I64, P, D, I32, P, P, I32, P]
    L.rr_brute_force.restype = ctypes.c_int
    L.rr_brute_force.argtypes = [P, P, I64, P, D, P, I32, P]
    L.rr_result_free.restype = ctypes.c_int
    L.rr_result_free.argtypes = [P]
    L.rr_last_error.restype = ctypes.c_char_p
    L.rr_last_error.argtypes = []
    L.rr_last_profile.restype = ctypes.c_int
    L.rr_last_profile.argtypes = [P, P]
    L.rr_beam_search_noalloc.restype = ctypes.c_int
    L.rr_beam_search_noalloc.argtypes = [P, P, I64, D, I32, P, P, P, P, P]
    L.rr_serve_cfg_init.restype = None
    L.rr_serve_cfg_init.argtypes = [P]
    L.rr_serve_create.restype = ctypes.c_int
    L.rr_serve_create.argtypes = [P, P, P]
    L.rr_serve_submit.restype = ctypes.c_int
    L.rr_serve_submit.argtypes = [P, P, I64, P, D, P]
    L.rr_serve_poll.restype = ctypes.c_int
    L.rr_serve_poll.argtypes = [P, ctypes.c_uint64, I32, P]
    L.rr_serve_collect.restype = ctypes.c_int
    L.rr_serve_collect.argtypes = [P, ctypes.c_uint64, I64, I32, P]
    L.rr_serve_cancel.restype = ctypes.c_int64
    L.rr_serve_cancel.argtypes = [P]
    L.rr_result_to_host.restype = ctypes.c_int
    L.rr_result_to_host.argtypes = [P, P]
    L.rr_abi_sizes.restype = None
    L.rr_abi_sizes.argtypes = [P]
    L.rr_serve_stats.restype = ctypes.c_int
    L.rr_serve_stats.argtypes = [P, P, I32]
    L.rr_serve_destroy.restype = ctypes.c_int
    L.rr_serve_destroy.argtypes = [P]
    L.rr_debug_set.restype = ctypes.c_int
    L.rr_debug_set.argtypes = [ctypes.c_char_p, I64]
    L.rr_build_graph.restype = ctypes.c_int
    L.rr_build_graph.argtypes = [P, I64, I32, I32, I32, I32, I32, D, I32, ctypes.c_uint64, I64, I32, P, P]
    _lib = L
    return L


def _check(status):
    if status != RR_OK:
        raise RRError(status, rr_last_error())


# ------------------------------------------------------------------------------------------------
# one-to-one entry points
# ------------------------------------------------------------------------------------------------

def rr_abi_sizes() -> dict:
    """sizeof of the public C structs as the library was compiled (layout check for this binding)."""
    out = (ctypes.c_int64 * 8)()
    load_library().rr_abi_sizes(out)
    names = ["rr_params", "rr_query_stats", "rr_result", "rr_index_info", "rr_profile", "rr_serve_cfg",
             "rr_serve_stats_t", "rr_build_info"]
    return dict(zip(names, list(out)))


def rr_last_error() -> str:
    return load_library().rr_last_error().decode("utf8", "replace")


def rr_params_init(**overrides) -> Params:
    p = Params()
    load_library().rr_params_init(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %s" % k)
        setattr(p, k, v)
    return p


def _ptr_and_device(a):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, False, a
    import torch
    if isinstance(a, torch.Tensor):
        a = a.contiguous()
        return a.data_ptr(), a.is_cuda, a
    raise TypeError("expected numpy array or torch tensor")


_DT = {np.dtype(np.uint8): RR_U8, np.dtype(np.int8): RR_I8, np.dtype(np.float32): RR_F32}


def _dtype_code(a):
    if isinstance(a, np.ndarray):
        return _DT[a.dtype]
    import torch
    return {torch.uint8: RR_U8, torch.int8: RR_I8, torch.float32: RR_F32}[a.dtype]


def rr_create_index(vectors, adjacency, start, metric=RR_L2, device=0, validate=True):
    """vectors: n x d (uint8/int8/float32), adjacency: n x R uint32 (0xFFFFFFFF pads), host or device."""
    vp, _, vk = _ptr_and_device(vectors)
    if isinstance(adjacency, np.ndarray):
        adjacency = np.ascontiguousarray(adjacency, dtype=np.uint32)
    ap, _, ak = _ptr_and_device(adjacency)
    n, d = vk.shape
    R = ak.shape[1]
    h = ctypes.c_void_p()
    _check(load_library().rr_create_index(vp, n, d, _dtype_code(vk), metric, ap, R, int(start), device,
                                          1 if validate else 0, ctypes.byref(h)))
    return h


def rr_build_graph(vectors, R, L, alpha, passes=2, seed=0, start=0, metric=RR_L2, device=0):
    """Proximity graph on the GPU (8-bit vectors, host or device): returns (adjacency uint32 [n, R], info dict)."""
    vp, _, vk = _ptr_and_device(vectors)
    n, d = vk.shape
    adj = np.empty((n, R), dtype=np.uint32)
    info = BuildInfo()
    _check(load_library().rr_build_graph(vp, n, d, _dtype_code(vk), metric, R, L, float(alpha), passes, int(seed),
                                         int(start), device, adj.ctypes.data, ctypes.byref(info)))
    return adj, info.as_dict()


def rr_load_index(path: str, device=0):
    h = ctypes.c_void_p()
    _check(load_library().rr_load_index(path.encode(), device, ctypes.byref(h)))
    return h


def rr_free_index(handle):
    _check(load_library().rr_free_index(handle))


def rr_index_info_get(handle) -> IndexInfo:
    info = IndexInfo()
    _check(load_library().rr_index_info_get(handle, ctypes.byref(info)))
    return info


def rr_index_relabel(handle, order=RR_ORDER_BFS):
    _check(load_library().rr_index_relabel(handle, order))


def _radii(nq, radius):
    if np.ndim(radius) == 0:
        return None, float(radius), None
    r = np.ascontiguousarray(np.asarray(radius, dtype=np.float64).reshape(-1))
    assert r.shape[0] == nq
    return r.ctypes.data, 0.0, r


def _stream_of(qdev, stream):
    if stream is not None:
        return stream
    if qdev:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return None


def rr_range_search(handle, queries, radius, variant=RR_GREEDY_ES, params: Params | None = None, stream=None,
                    result_on_device=False, check=True) -> tuple[int, Result]:
    """Returns (status, Result).  `radius`: scalar or one per query."""
    qp, qdev, qk = _ptr_and_device(queries)
    nq = qk.shape[0]
    rp, rs, rk = _radii(nq, radius)
    res = Result()
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    st = load_library().rr_range_search(handle, qp, nq, rp, rs, v, ctypes.byref(params) if params else None,
                                        _stream_of(qdev, stream), 1 if result_on_device else 0, ctypes.byref(res))
    if check and st not in (RR_OK, RR_EOVERFLOW):
        raise RRError(st, rr_last_error())
    return st, res


def rr_brute_force(handle, queries, radius, stream=None, result_on_device=False) -> Result:
    qp, qdev, qk = _ptr_and_device(queries)
    nq = qk.shape[0]
    rp, rs, rk = _radii(nq, radius)
    res = Result()
    _check(load_library().rr_brute_force(handle, qp, nq, rp, rs, _stream_of(qdev, stream),
                                         1 if result_on_device else 0, ctypes.byref(res)))
    return res


def rr_beam_search_noalloc(handle, queries, radius, variant, params, out_counts, out_ids, out_dists, stream=None):
    """Allocation-free beam search into caller-owned device arrays (torch CUDA tensors).

    For callers that may not allocate device memory while they run: the outputs
    must already exist (out_counts: nq int32, out_ids: nq x b int32/uint32,
    out_dists: nq x b int32 or float32) and the library uses only a fixed static
    scratch array.  Returns the status (raises on errors other than RR_OK)."""
    import torch
    qp, qdev, qk = _ptr_and_device(queries)
    nq = qk.shape[0]
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    info = rr_index_info_get(handle)
    beam = params.beam if params else rr_params_init().beam
    dist_ok = (torch.float32,) if info.dtype == RR_F32 else (torch.int32,)
    # the library cannot see the outputs' sizes: check them here, before anything is written
    for name, t, numel, dts in (("out_counts", out_counts, nq, (torch.int32,)),
                                ("out_ids", out_ids, nq * beam, (torch.int32, getattr(torch, "uint32", torch.int32))),
                                ("out_dists", out_dists, nq * beam, dist_ok)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.device.index != info.device:
            raise ValueError("%s is on cuda:%d, the index on cuda:%d" % (name, t.device.index, info.device))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() < numel:
            raise ValueError("%s holds %d elements, the call writes %d" % (name, t.numel(), numel))
        if t.dtype not in dts:
            raise ValueError("%s has dtype %s, expected one of %s" % (name, t.dtype, dts))
    st = load_library().rr_beam_search_noalloc(handle, qp, nq, float(radius), v,
                                               ctypes.byref(params) if params else None,
                                               _stream_of(qdev, stream), out_counts.data_ptr(), out_ids.data_ptr(),
                                               out_dists.data_ptr())
    _check(st)
    return st


def beam_hash_lg(beam: int) -> int:
    """log2 of the beam kernel's default seen-table size for beam b (what seen_log2 = 0 selects)."""
    return 10 if beam <= 256 else 11


def rr_debug_set(key: str, value: int):
    """Failure-path hooks for tests: "fail_alloc_after" (N-th next device allocation fails; -1 off),
    "beam_iteration_limit" (per-query iteration guard of the beam / doubling kernels; 0 default)."""
    _check(load_library().rr_debug_set(key.encode(), int(value)))


def rr_last_profile(handle) -> Profile:
    p = Profile()
    _check(load_library().rr_last_profile(handle, ctypes.byref(p)))
    return p


def rr_result_free(res: Result):
    _check(load_library().rr_result_free(ctypes.byref(res)))


def rr_serve_cfg_init(**overrides) -> ServeCfg:
    c = ServeCfg()
    load_library().rr_serve_cfg_init(ctypes.byref(c))
    for k, v in overrides.items():
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        if hasattr(c, k):
            setattr(c, k, v)
        elif hasattr(c.params, k):
            setattr(c.params, k, v)
        else:
            raise TypeError("unknown serving parameter %s" % k)
    return c


def rr_serve_create(handle, cfg: ServeCfg | None = None):
    s = ctypes.c_void_p()
    _check(load_library().rr_serve_create(handle, ctypes.byref(cfg) if cfg else None, ctypes.byref(s)))
    return s


def rr_serve_submit(server, queries, radius) -> int:
    """Queue len(queries) requests (host array); returns the first ticket."""
    qp, qdev, qk = _ptr_and_device(queries)
    if qdev:
        raise ValueError("rr_serve_submit takes host queries")
    n = qk.shape[0]
    rp, rs, rk = _radii(n, radius)
    t = ctypes.c_uint64()
    _check(load_library().rr_serve_submit(server, qp, n, rp, rs, ctypes.byref(t)))
    return t.value


def rr_serve_poll(server, ticket, timeout_ms=0):
    """(status, Result): RR_OK with the request's result, or RR_EBUSY while pending."""
    res = Result()
    st = load_library().rr_serve_poll(server, ticket, int(timeout_ms), ctypes.byref(res))
    if st not in (RR_OK, RR_EBUSY):
        msg = rr_last_error()
        if res.offsets:
            rr_result_free(res)
        raise RRError(st, msg)
    return st, res


def rr_serve_collect(server, first, n, timeout_ms=0):
    """(status, Result) for n consecutive tickets from `first`: RR_OK with one CSR, or RR_EBUSY."""
    res = Result()
    st = load_library().rr_serve_collect(server, int(first), int(n), int(timeout_ms), ctypes.byref(res))
    if st not in (RR_OK, RR_EBUSY):
        msg = rr_last_error()
        if res.offsets:
            rr_result_free(res)
        raise RRError(st, msg)
    return st, res


def rr_serve_cancel(server) -> int:
    """Drop every queued request (retired with RR_FLAG_CANCELED); returns how many."""
    return int(load_library().rr_serve_cancel(server))


def rr_result_to_host(res: Result) -> Result:
    """A host copy of a (host or device) result; free both with rr_result_free."""
    h = Result()
    _check(load_library().rr_result_to_host(ctypes.byref(res), ctypes.byref(h)))
    return h


def rr_serve_stats(server, reset=False) -> ServeStats:
    o = ServeStats()
    _check(load_library().rr_serve_stats(server, ctypes.byref(o), 1 if reset else 0))
    return o


def rr_serve_destroy(server):
    _check(load_library().rr_serve_destroy(server))


# ------------------------------------------------------------------------------------------------
# convenience
# ------------------------------------------------------------------------------------------------

class RangeResult:
    """Host copy of a result: offsets (nq+1), ids, dists, flags, optional stats."""

    def __init__(self, res: Result, status=RR_OK):
        self.status = status
        nq, tot = res.nq, res.total
        if res.on_device:
            raise ValueError("RangeResult wraps host results")

        def arr(p, ct, n, dt):
            if n == 0 or not p:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ct)), (n,)).copy()

        self.offsets = arr(res.offsets, ctypes.c_int64, nq + 1, np.int64)
        if nq + 1 > len(self.offsets):
            self.offsets = np.zeros(nq + 1, np.int64)
        self.ids = arr(res.ids, ctypes.c_uint32, tot, np.uint32)
        self.dists = arr(res.dists, ctypes.c_float if res.dist_dtype else ctypes.c_int32, tot,
                         np.float32 if res.dist_dtype else np.int32)
        self.flags = arr(res.flags, ctypes.c_uint8, nq, np.uint8)
        self.stats = None
        if res.stats:
            raw = np.ctypeslib.as_array(ctypes.cast(res.stats, ctypes.POINTER(ctypes.c_int32)), (nq * 6,)).copy()
            self.stats = raw.view(STATS_DTYPE)
        rr_result_free(res)

    def __len__(self):
        return len(self.offsets) - 1

    def query(self, i):
        s, e = self.offsets[i], self.offsets[i + 1]
        return self.ids[s:e], self.dists[s:e]

    def lists(self):
        return [self.ids[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self))]


class Index:
    """Owns an rr_index handle."""

    def __init__(self, handle):
        self.h = handle
        self.info = rr_index_info_get(handle)

    @classmethod
    def from_arrays(cls, X, adj, start, metric=RR_L2, device=0, validate=True):
        return cls(rr_create_index(X, adj, start, metric, device, validate))

    @classmethod
    def load(cls, path, device=0):
        return cls(rr_load_index(path, device))

    def relabel(self, order=RR_ORDER_BFS):
        """Renumber the points in breadth-first order from the start point (rr_index_relabel)."""
        rr_index_relabel(self.h, order)
        self.info = rr_index_info_get(self.h)
        return self

    def close(self):
        if self.h:
            rr_free_index(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def range_search(self, Q, radius, variant="greedy_es", stream=None, **params) -> RangeResult:
        p = rr_params_init(**params)
        st, res = rr_range_search(self.h, Q, radius, variant, p, stream=stream, result_on_device=False)
        return RangeResult(res, st)

    def brute_force(self, Q, radius, stream=None) -> RangeResult:
        return RangeResult(rr_brute_force(self.h, Q, radius, stream=stream))

    def serve(self, **cfg) -> "Server":
        return Server(self, rr_serve_cfg_init(**cfg))


class Server:
    """Continuous-batching server over an Index (rr_serve_*)."""

    def __init__(self, index: Index, cfg: ServeCfg):
        self.index = index  # keeps the index alive
        self.h = rr_serve_create(index.h, cfg)

    def submit(self, Q, radius) -> np.ndarray:
        t0 = rr_serve_submit(self.h, Q, radius)
        return np.arange(t0, t0 + len(Q), dtype=np.uint64)

    def _wrap(self, res):
        if res.on_device:  # a host copy for Python; the device arrays are freed here
            h = rr_result_to_host(res)
            rr_result_free(res)
            res = h
        return RangeResult(res)

    def poll(self, ticket, timeout_ms=0):
        """RangeResult of one request (nq = 1), or None while it is pending."""
        st, res = rr_serve_poll(self.h, int(ticket), timeout_ms)
        return self._wrap(res) if st == RR_OK else None

    def collect(self, first, n, timeout_ms=0):
        """RangeResult of the n requests first .. first+n-1 (one submit), or None while any is pending."""
        st, res = rr_serve_collect(self.h, int(first), int(n), timeout_ms)
        return self._wrap(res) if st == RR_OK else None

    def cancel(self) -> int:
        return rr_serve_cancel(self.h)

    def stats(self, reset=False) -> dict:
        return rr_serve_stats(self.h, reset).as_dict()

    def close(self):
        if self.h:
            rr_serve_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
