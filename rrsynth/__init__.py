"""Seeded synthetic inputs for range retrieval on a proximity graph.

This package is INPUT GENERATION shared by the oracle tests and the GPU
library's tests and benchmark.  It holds none of the range-search method's
arithmetic: it draws vectors and queries, picks a radius from exact 1-NN
distances (numpy), builds the proximity graph once (``vamana.c``), and writes
the ``.rrx`` index file.  The range search itself lives in ``oracle/`` (CPU
reference) and in ``paper_2502_13245_gb300`` (CUDA), which share no code.

The paper's datasets (BIGANN, SSNPP, Text2Image, ... in Table "Descriptions of
each dataset") are not available; the recipes below stand in for them with
their shapes: uint8 SIFT-like vectors in d=128/256, unit-norm fp32 vectors in
d=200 under inner product, and a heavy-tailed result-count distribution with
most queries matching nothing (Table "distribution of result sizes").
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(HERE, "_vamana.so")
SENTINEL = 0xFFFFFFFF

DT_U8, DT_I8, DT_F32 = 0, 1, 2
M_L2, M_IP = 0, 1


def build_lib(force: bool = False) -> str:
    """Compile vamana.c (gcc, OpenMP) into rrsynth/_vamana.so."""
    src = os.path.join(HERE, "vamana.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", _LIB + ".tmp", src]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB)
        lib.rrs_build_vamana.restype = ctypes.c_int
        lib.rrs_build_vamana.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
        lib.rrs_start_point.restype = ctypes.c_int64
        lib.rrs_start_point.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def _dtype_code(x: np.ndarray) -> int:
    return {np.dtype(np.uint8): DT_U8, np.dtype(np.int8): DT_I8, np.dtype(np.float32): DT_F32}[x.dtype]


def start_point(X: np.ndarray) -> int:
    """Point nearest (fp64 L2) to the coordinate-wise mean; ties to the smaller id."""
    X = np.ascontiguousarray(X)
    return int(_load().rrs_start_point(X.ctypes.data, X.shape[0], X.shape[1], _dtype_code(X)))


def build_graph(X: np.ndarray, R: int, L: int, alpha: float, metric: int = M_L2, passes: int = 2,
                seed: int = 0, threads: int = 0, start: int | None = None, builder: str = "cpu"):
    """Deterministic Vamana-style graph: returns (adj uint32 [n,R], start id).

    builder "cpu": vamana.c on the host cores.  builder "gpu": the same
    procedure run by the CUDA library's rr_build_graph (8-bit data only), which
    gives the same adjacency array (tested on C0, C1 and a d=256 sample of the
    C3 recipe); it is used where the host build would take the better part of
    an hour (C3)."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    if start is None:
        start = start_point(X)
    if builder == "gpu":
        import paper_2502_13245_gb300 as rr
        rr.build()
        adj, _ = rr.rr_build_graph(X, R, L, alpha, passes=passes, seed=seed, start=start,
                                   metric=rr.RR_IP if metric == M_IP else rr.RR_L2)
        return adj, int(start)
    adj = np.empty((n, R), dtype=np.uint32)
    rc = _load().rrs_build_vamana(X.ctypes.data, n, d, _dtype_code(X), metric, R, L, float(alpha), passes,
                                  seed, threads, adj.ctypes.data, start)
    if rc != 0:
        raise RuntimeError("rrs_build_vamana failed (%d)" % rc)
    return adj, int(start)


# ----------------------------------------------------------------------------------------------
# vectors
# ----------------------------------------------------------------------------------------------

def _grow_families(rng, X, n_base, sizes, dup_sigma, finish):
    """Near-duplicate families as random recursive trees: family f has a root
    (a random base point) and members m_1..m_s; member m_k copies a uniformly
    random earlier member of its family (the root included) and adds
    N(0, dup_sigma^2) noise.  Rows n_base.. of X are filled family-major."""
    nf = len(sizes)
    roots = rng.integers(0, n_base, size=nf)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]) + n_base
    d = X.shape[1]
    for k in range(int(sizes.max())):
        live = np.nonzero(sizes > k)[0]
        par = rng.integers(0, k + 1, size=len(live))  # 0 = root, j>0 = member m_j
        src = np.where(par == 0, roots[live], offs[live] + par - 1)
        v = X[src].astype(np.float64) + rng.normal(0.0, dup_sigma, size=(len(live), d))
        X[offs[live] + k] = finish(v)


def _family_sizes(rng, total, alpha, cap):
    sizes = []
    acc = 0
    while acc < total:
        s = int(min(cap, np.ceil(rng.pareto(alpha) + 1.0)))
        s = min(s, total - acc)
        sizes.append(s)
        acc += s
    return np.asarray(sizes, dtype=np.int64)


def mixture_u8(n, d, n_centres, sigma, seed, dup_frac=0.2, fam_alpha=1.0, fam_cap=500, dup_sigma=2.0,
               lo=40.0, hi=215.0, chunk=1 << 16, streams=0):
    """uint8 Gaussian mixture with Zipf(1) weights and near-duplicate families.

    Returns (X uint8 [n,d], centres float64, weights).  Rows are shuffled so ids
    carry no cluster order.  streams > 0 draws the noise of the base rows from
    that many independent seeded streams (chunks of rows, in threads)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(lo, hi, size=(n_centres, d))
    w = 1.0 / np.arange(1, n_centres + 1, dtype=np.float64)
    w /= w.sum()
    n_dup = int(round(dup_frac * n))
    sizes = _family_sizes(rng, n_dup, fam_alpha, fam_cap) if n_dup > 0 else np.zeros(0, np.int64)
    n_base = n - n_dup
    X = np.empty((n, d), dtype=np.uint8)
    assign = rng.choice(n_centres, size=n_base, p=w)
    if streams > 0:
        import concurrent.futures as cf
        kids = np.random.SeedSequence(seed).spawn(streams)
        bounds = np.linspace(0, n_base, streams + 1).astype(np.int64)

        def fill(j):
            g = np.random.Generator(np.random.PCG64(kids[j]))
            for s in range(int(bounds[j]), int(bounds[j + 1]), chunk):
                e = min(int(bounds[j + 1]), s + chunk)
                v = centres[assign[s:e]] + g.normal(0.0, sigma, size=(e - s, d))
                X[s:e] = np.clip(np.rint(v), 0, 255).astype(np.uint8)

        with cf.ThreadPoolExecutor(max_workers=min(streams, os.cpu_count() or 4)) as ex:
            list(ex.map(fill, range(streams)))
    else:
        for s in range(0, n_base, chunk):
            e = min(n_base, s + chunk)
            v = centres[assign[s:e]] + rng.normal(0.0, sigma, size=(e - s, d))
            X[s:e] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    if n_dup > 0:
        _grow_families(rng, X, n_base, sizes, dup_sigma, lambda v: np.clip(np.rint(v), 0, 255).astype(np.uint8))
    perm = rng.permutation(n)
    return X[perm], centres, w


def queries_u8(X, centres, w, nq, sigma, seed, near_frac=0.38, near_sigma=2.0):
    """Queries: near_frac perturbed copies of random base points, the rest fresh mixture draws."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n, d = X.shape
    n_near = int(round(near_frac * nq))
    ids = rng.integers(0, n, size=n_near)
    near = X[ids].astype(np.float64) + rng.normal(0.0, near_sigma, size=(n_near, d))
    a = rng.choice(len(centres), size=nq - n_near, p=w)
    fresh = centres[a] + rng.normal(0.0, sigma, size=(nq - n_near, d))
    Q = np.clip(np.rint(np.concatenate([near, fresh])), 0, 255).astype(np.uint8)
    return Q[rng.permutation(nq)]


def vmf_f32(n, d, n_centres, kappa_sigma, seed, dup_frac=0.2, fam_alpha=1.0, fam_cap=500, dup_sigma=0.01,
            chunk=1 << 16):
    """Unit-norm fp32 vectors around n_centres random directions (von Mises-Fisher-like):
    x = normalise(mu_k + N(0, kappa_sigma^2 I)), Zipf(1) weights, near-duplicate families."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.normal(size=(n_centres, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    w = 1.0 / np.arange(1, n_centres + 1, dtype=np.float64)
    w /= w.sum()
    n_dup = int(round(dup_frac * n))
    sizes = _family_sizes(rng, n_dup, fam_alpha, fam_cap) if n_dup > 0 else np.zeros(0, np.int64)
    n_base = n - n_dup
    X = np.empty((n, d), dtype=np.float32)
    assign = rng.choice(n_centres, size=n_base, p=w)
    for s in range(0, n_base, chunk):
        e = min(n_base, s + chunk)
        v = mu[assign[s:e]] + rng.normal(0.0, kappa_sigma, size=(e - s, d))
        X[s:e] = (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    if n_dup > 0:
        _grow_families(rng, X, n_base, sizes, dup_sigma,
                       lambda v: (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32))
    perm = rng.permutation(n)
    return X[perm], mu, w


def queries_f32(X, mu, w, nq, kappa_sigma, seed, near_frac=0.38, near_sigma=0.01):
    rng = np.random.Generator(np.random.PCG64(seed))
    n, d = X.shape
    n_near = int(round(near_frac * nq))
    ids = rng.integers(0, n, size=n_near)
    near = X[ids].astype(np.float64) + rng.normal(0.0, near_sigma, size=(n_near, d))
    a = rng.choice(len(mu), size=nq - n_near, p=w)
    fresh = mu[a] + rng.normal(0.0, kappa_sigma, size=(nq - n_near, d))
    Q = np.concatenate([near, fresh])
    Q = (Q / np.linalg.norm(Q, axis=1, keepdims=True)).astype(np.float32)
    return Q[rng.permutation(nq)]


# ----------------------------------------------------------------------------------------------
# radius picking (exact 1-NN distances, numpy; integer data is exact in fp32 GEMMs for d <= 256)
# ----------------------------------------------------------------------------------------------

def nn1_distances(X, Q, metric=M_L2, qblock=1024, xblock=1 << 16):
    """Nearest-neighbour distance per query (int64 for integer data, float64 otherwise).

    Integer data: ||x||^2 - 2<x,q> is formed in fp32, exact while every value
    stays below 2^24 (d <= 128 for uint8); larger d may round by a few units,
    which only moves the picked radius, never a search result."""
    n = X.shape[0]
    integer = X.dtype != np.float32
    Xf = X.astype(np.float32)
    xn = (Xf.astype(np.float64) ** 2).sum(1).astype(np.float32) if metric == M_L2 else None
    out = np.empty(Q.shape[0], dtype=np.int64 if integer else np.float64)
    for s in range(0, Q.shape[0], qblock):
        Qb = Q[s:s + qblock].astype(np.float32)
        best = np.full(Qb.shape[0], np.inf, dtype=np.float64)
        for xs in range(0, n, xblock):
            G = Qb @ Xf[xs:xs + xblock].T
            if metric == M_L2:
                G *= -2.0
                G += xn[None, xs:xs + xblock]
            else:
                G *= -1.0
            best = np.minimum(best, G.min(1).astype(np.float64))
        if metric == M_L2:
            best += (Qb.astype(np.float64) ** 2).sum(1)
        out[s:s + qblock] = np.rint(best).astype(np.int64) if integer else best
    return out


def nn1_distances_exact(X, Q, qblock=512, xblock=1 << 20):
    """Exact squared-L2 1-NN distance per query for 8-bit data (torch; a CUDA device when present).

    Products of 8-bit values are exact in TF32 and fp32, and their sums (< 2^24
    for d <= 256) exact in any order; the distance is formed from them in int64."""
    import torch
    dev = torch.device("cuda" if torch.cuda.is_available() else "cpu")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        Qf = torch.from_numpy(np.ascontiguousarray(Q)).to(dev).float()
        nq = (Qf * Qf).sum(1).to(torch.int64)
        best = torch.full((Q.shape[0],), np.iinfo(np.int64).max, dtype=torch.int64, device=dev)
        for xs in range(0, X.shape[0], xblock):
            Xb = torch.from_numpy(np.ascontiguousarray(X[xs:xs + xblock])).to(dev).float()
            nx = (Xb * Xb).sum(1).to(torch.int64)
            for s in range(0, Q.shape[0], qblock):
                G = (Qf[s:s + qblock] @ Xb.T).to(torch.int64)
                D = nq[s:s + qblock, None] + nx[None, :] - 2 * G
                best[s:s + qblock] = torch.minimum(best[s:s + qblock], D.min(1).values)
        return best.cpu().numpy()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def pick_radius(nn1, zero_frac=0.6):
    """Radius at the (1 - zero_frac) quantile of 1-NN distances (lower order statistic)."""
    srt = np.sort(nn1)
    k = int(np.floor((1.0 - zero_frac) * len(srt)))
    k = min(max(k, 0), len(srt) - 1)
    return srt[k]


# ----------------------------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    n: int
    d: int
    nq: int
    dtype: str          # "u8" or "f32"
    metric: int
    n_centres: int
    sigma: float
    fam_cap: int
    R: int
    L_build: int
    alpha: float
    passes: int
    seed: int
    near_sigma: float
    zero_frac: float = 0.6
    streams: int = 0           # > 0: base rows drawn from that many seeded streams in parallel
    builder: str = "cpu"       # graph builder: "cpu" (vamana.c) or "gpu" (the same procedure in librr)


CONFIGS = {
    # 10,000 x 128 uint8, 100 centres, 1,000 queries, R=32 L=64 alpha=1.2
    "c0": Config("c0", 10_000, 128, 1_000, "u8", M_L2, 100, 12.0, 500, 32, 64, 1.2, 2, 0, 2.0),
    # 1,000,000 x 128 uint8, 1,000 centres, 10,000 queries, R=64 L=128 alpha=1.2
    "c1": Config("c1", 1_000_000, 128, 10_000, "u8", M_L2, 1000, 12.0, 5000, 64, 128, 1.2, 2, 1, 2.0),
    # 1,000,000 x 200 fp32 unit vectors, inner product, 10,000 queries, R=64 L=128 alpha=1.0
    "c2": Config("c2", 1_000_000, 200, 10_000, "f32", M_IP, 1000, 0.06, 5000, 64, 128, 1.0, 1, 2, 0.01),
    # 10,000,000 x 256 uint8, 5,000 centres, families up to 20,000, 100,000 queries, R=64 L=48 alpha=1.2,
    # two construction passes, built on the GPU (the host build of this graph takes the better part of an hour).
    # L=48, not 128: on this recipe the more exact L=128 candidate pools give kNN-like rows inside the tight
    # near-duplicate families (alpha=1.2 prunes little where all distances are alike), their in-range subgraphs
    # fall apart, and greedy AP stays at 0.34 at b=128; with L=48 it is 0.9965 (20,000 queries)
    "c3": Config("c3", 10_000_000, 256, 100_000, "u8", M_L2, 5000, 12.0, 20000, 64, 48, 1.2, 2, 3, 2.0,
                 streams=64, builder="gpu"),
    # the same recipe at 2,000,000 points and 20,000 queries (1 GB of vectors + adjacency, well above L2): the
    # case that profiler captures of the 10^7-point workload's kernels run on
    "c3p": Config("c3p", 2_000_000, 256, 20_000, "u8", M_L2, 5000, 12.0, 20000, 64, 48, 1.2, 2, 3, 2.0,
                  streams=64, builder="gpu"),
}


def small_config(name, n, nq, d=128, R=32, L=64, seed=0, n_centres=20, fam_cap=200, passes=2, dtype="u8",
                 metric=M_L2, sigma=None, near_sigma=None, alpha=None):
    """Reduced configuration with the same recipe (tests)."""
    if dtype == "u8":
        return Config(name, n, d, nq, "u8", metric, n_centres, 12.0 if sigma is None else sigma, fam_cap, R, L,
                      1.2 if alpha is None else alpha, passes, seed, 2.0 if near_sigma is None else near_sigma)
    return Config(name, n, d, nq, "f32", metric, n_centres, 0.06 if sigma is None else sigma, fam_cap, R, L,
                  1.0 if alpha is None else alpha, passes, seed, 0.01 if near_sigma is None else near_sigma)


def config_hash(cfg: Config) -> str:
    src = open(os.path.join(HERE, "vamana.c"), "rb").read() + open(__file__, "rb").read()
    h = hashlib.sha1(json.dumps(dataclasses.asdict(cfg), sort_keys=True).encode() + src)
    return h.hexdigest()[:16]


@dataclasses.dataclass
class Dataset:
    cfg: Config
    X: np.ndarray
    Q: np.ndarray
    adj: np.ndarray
    start: int
    radius: float
    build_s: float = 0.0

    @property
    def R(self):
        return self.adj.shape[1]


def make_dataset(cfg: Config, cache_dir: str | None = None, threads: int = 0, verbose: bool = False) -> Dataset:
    """Generate (or load from cache) vectors, queries, graph and radius for a config."""
    path = None
    if cache_dir:
        os.makedirs(cache_dir, exist_ok=True)
        path = os.path.join(cache_dir, "%s_%s.npz" % (cfg.name, config_hash(cfg)))
        if os.path.exists(path):
            z = np.load(path)
            return Dataset(cfg, z["X"], z["Q"], z["adj"], int(z["start"]), z["radius"].item(), 0.0)
    t0 = time.time()
    if cfg.dtype == "u8":
        X, C, w = mixture_u8(cfg.n, cfg.d, cfg.n_centres, cfg.sigma, cfg.seed, fam_cap=cfg.fam_cap,
                             streams=cfg.streams)
        Q = queries_u8(X, C, w, cfg.nq, cfg.sigma, cfg.seed + 1, near_sigma=cfg.near_sigma)
    else:
        X, C, w = vmf_f32(cfg.n, cfg.d, cfg.n_centres, cfg.sigma, cfg.seed, fam_cap=cfg.fam_cap)
        Q = queries_f32(X, C, w, cfg.nq, cfg.sigma, cfg.seed + 1, near_sigma=cfg.near_sigma)
    t1 = time.time()
    # the radius comes from the 1-NN distances of (at most) 2,000 seeded queries
    sub = Q if cfg.nq <= 2000 else Q[np.random.Generator(np.random.PCG64(cfg.seed + 7)).choice(cfg.nq, 2000, replace=False)]
    if cfg.dtype == "u8" and cfg.d > 128:
        nn1 = nn1_distances_exact(X, sub)  # fp32 forms of ||x||^2 - 2<x,q> would round above d = 128
    else:
        nn1 = nn1_distances(X, sub, cfg.metric)
    radius = pick_radius(nn1, cfg.zero_frac)
    radius = int(radius) if cfg.dtype == "u8" else float(radius)
    t2 = time.time()
    adj, start = build_graph(X, cfg.R, cfg.L_build, cfg.alpha, cfg.metric, cfg.passes, cfg.seed, threads,
                             builder=cfg.builder)
    t3 = time.time()
    if verbose:
        print("[rrsynth] %s: gen %.1fs radius %.1fs graph %.1fs" % (cfg.name, t1 - t0, t2 - t1, t3 - t2),
              file=sys.stderr)
    ds = Dataset(cfg, X, Q, adj, start, radius, t3 - t2)
    if path:
        tmp = path + ".tmp.npz"
        np.savez(tmp, X=X, Q=Q, adj=adj, start=np.int64(start), radius=np.asarray(radius))
        os.replace(tmp, path)
    return ds


# ----------------------------------------------------------------------------------------------
# .rrx index file (written here, read by rr_load_index in the CUDA library)
# ----------------------------------------------------------------------------------------------

RRX_MAGIC = b"RRX1"
RRX_HEADER = 64


def write_rrx(path, X, adj, start, metric):
    """Header (64 bytes, little endian):
      0  magic 'RRX1'     4 u32 version=1   8 i64 n     16 i32 d     20 i32 dtype
      24 i32 metric      28 i32 R          32 i64 start 40 u64 checksum of the payload
      48 16 bytes zero
    then vectors (n*d*esz bytes) and adjacency (n*R uint32).  checksum: the
    payload as one byte stream, zero padded to 8 bytes, read as little-endian
    u64 words w_i; XOR over i of (w_i * 0x100000001B3 + i) mod 2^64."""
    import struct
    X = np.ascontiguousarray(X)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    payload = X.tobytes() + adj.tobytes()
    hdr = bytearray(RRX_HEADER)
    hdr[0:4] = RRX_MAGIC
    struct.pack_into("<I", hdr, 4, 1)
    struct.pack_into("<qiiiiqQ", hdr, 8, X.shape[0], X.shape[1], _dtype_code(X), metric, adj.shape[1], start,
                     rrx_checksum(payload))
    with open(path, "wb") as f:
        f.write(bytes(hdr))
        f.write(payload)


def rrx_checksum(buf: bytes) -> int:
    b = np.frombuffer(buf, dtype=np.uint8)
    pad = (-b.size) % 8
    if pad:
        b = np.concatenate([b, np.zeros(pad, np.uint8)])
    w = b.view("<u8")
    with np.errstate(over="ignore"):
        v = w * np.uint64(0x100000001B3) + np.arange(w.size, dtype=np.uint64)
    return int(np.bitwise_xor.reduce(v)) if v.size else 0
