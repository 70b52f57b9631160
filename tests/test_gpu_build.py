"""The GPU graph builder (rr_build_graph) against the CPU builder (rrsynth's vamana.c).

Both run the same deterministic procedure (batch-parallel Vamana insertion,
RobustPrune with alpha on the stored metric value, reverse edges merged per
target in batch order, a reachability repair), so on 8-bit data the adjacency
arrays must be identical, entry for entry: checked on tiny graphs of every
8-bit element type and metric, on padded rows (d not a multiple of 16), on the
10^4-point and 10^6-point configurations, and on a d=256 sample of the
10^7-point recipe whose full-size graph only the GPU builder makes."""
import dataclasses
import os

import numpy as np
import pytest

import rrsynth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")
SENT = 0xFFFFFFFF


@pytest.fixture(scope="module")
def rr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    return rr


def _invariants(adj, start, R):
    n = adj.shape[0]
    assert adj.shape[1] == R
    valid = adj != SENT
    # rows are filled from the left and hold distinct ids other than their own
    assert np.all(valid[:, :-1] | ~valid[:, 1:])
    for u in range(0, n, max(1, n // 2000)):
        row = adj[u][valid[u]]
        assert len(np.unique(row)) == len(row) and not np.any(row == u) and np.all(row < n)
    # every point is reachable from the start point
    seen = np.zeros(n, bool)
    seen[start] = True
    front = np.array([start])
    while len(front):
        nxt = adj[front].reshape(-1)
        nxt = nxt[nxt != SENT]
        nxt = np.unique(nxt[~seen[nxt]])
        seen[nxt] = True
        front = nxt
    assert seen.all()


def _compare(rr, X, R, L, alpha, passes, seed, metric):
    start = rrsynth.start_point(X)
    cpu, _ = rrsynth.build_graph(X, R, L, alpha, metric, passes, seed, start=start)
    gpu, info = rr.rr_build_graph(X, R, L, alpha, passes=passes, seed=seed, start=start,
                                  metric=rr.RR_IP if metric == rrsynth.M_IP else rr.RR_L2)
    diff = np.nonzero((cpu != gpu).any(1))[0]
    assert len(diff) == 0, "rows differ: %s (of %d), first: cpu %s gpu %s" % (
        diff[:10], len(diff), cpu[diff[0]], gpu[diff[0]])
    _invariants(gpu, start, R)
    return info


@pytest.mark.parametrize("case", [
    dict(n=600, d=16, R=12, L=24, passes=2, dtype="u8", metric="l2"),
    dict(n=2000, d=20, R=16, L=32, passes=1, dtype="u8", metric="l2"),
    dict(n=3000, d=32, R=16, L=32, passes=2, dtype="i8", metric="l2"),
    dict(n=3000, d=48, R=24, L=40, passes=2, dtype="i8", metric="ip"),
    dict(n=5000, d=64, R=32, L=64, passes=2, dtype="u8", metric="ip"),
])
def test_tiny_graphs_identical(rr, case):
    rng = np.random.default_rng(case["n"] + case["d"])
    centres = rng.uniform(40, 215, size=(8, case["d"]))
    X = np.clip(np.rint(centres[rng.integers(0, 8, case["n"])] + rng.normal(0, 12, (case["n"], case["d"]))), 0, 255)
    X = X.astype(np.uint8)
    # near-duplicates make ties and tight families (the repair's business)
    X[::7] = X[1::7][: len(X[::7])]
    if case["dtype"] == "i8":
        X = (X.astype(np.int16) - 128).astype(np.int8)
    metric = rrsynth.M_IP if case["metric"] == "ip" else rrsynth.M_L2
    alpha = 1.0 if metric == rrsynth.M_IP else 1.2
    _compare(rr, X, case["R"], case["L"], alpha, case["passes"], 7, metric)


def test_c0_graph_identical(rr):
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    cfg = ds.cfg
    gpu, info = rr.rr_build_graph(ds.X, cfg.R, cfg.L_build, cfg.alpha, passes=cfg.passes, seed=cfg.seed,
                                  start=ds.start)
    assert np.array_equal(gpu, ds.adj)
    assert info["batches"] > 0


def test_c1_graph_identical(rr):
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c1"], cache_dir=CACHE)
    cfg = ds.cfg
    gpu, info = rr.rr_build_graph(ds.X, cfg.R, cfg.L_build, cfg.alpha, passes=cfg.passes, seed=cfg.seed,
                                  start=ds.start)
    diff = np.nonzero((gpu != ds.adj).any(1))[0]
    assert len(diff) == 0, "%d rows differ, first %d" % (len(diff), diff[0])
    print("C1 GPU build: %.1f s (+ %.2f s repair, %d points attached), CPU build %.1f s" % (
        info["gpu_seconds"], info["repair_seconds"], info["repaired"], ds.build_s))


def test_c3_recipe_sample_identical(rr):
    """200,000 points of the 10^7-point recipe (d = 256, R = 64, alpha = 1.2, two passes), with the
    10^7-point graph's L = 48 and with L = 128."""
    for L in (48, 128):
        cfg = dataclasses.replace(rrsynth.CONFIGS["c3"], name="c3_sample_L%d" % L, n=200_000, nq=100,
                                  n_centres=500, fam_cap=2000, builder="cpu", streams=0, L_build=L)
        ds = rrsynth.make_dataset(cfg, cache_dir=CACHE)
        gpu, info = rr.rr_build_graph(ds.X, cfg.R, cfg.L_build, cfg.alpha, passes=cfg.passes, seed=cfg.seed,
                                      start=ds.start)
        diff = np.nonzero((gpu != ds.adj).any(1))[0]
        assert len(diff) == 0, "L=%d: %d rows differ, first %d" % (L, len(diff), diff[0])

