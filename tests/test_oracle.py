"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * hand-worked traces of Alg. 1/2/3/5/6 (tests/golden/hand_traces.json) and of
    Alg. 1 with the other early-stopping metrics of Sec. 3.2
    (tests/golden/es_metric_traces.json);
  * Def. 2.1 brute force on tiny inputs where the search must be exhaustive
    (b >= n on a graph whose every node is reachable from the start point);
  * an independent reachability closure (scipy BFS) for Alg. 2;
  * invariants: results within r, no duplicates, sorted by (dist, id), subset
    of the exact set, |beam result| <= b, early stop returns the non-ES result
    or nothing, greedy extends the beam result;
  * exact distances recomputed in numpy (int64 / fp64) for every element type
    and metric the oracle takes (uint8, int8, fp32; squared L2 and inner product);
  * Def. 2.2 on hand-computed values.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

import oracle
import rrsynth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")
SENT = 0xFFFFFFFF


def _gold_index():
    g = json.load(open(GOLD))
    X = np.asarray(g["points"], np.uint8)[:, None]
    adj = np.asarray([[SENT if v < 0 else v for v in row] for row in g["adjacency"]], np.uint32)
    return g, oracle.Index(X, adj, g["start"])


@pytest.mark.parametrize("case", [c["name"] for c in json.load(open(GOLD))["cases"]])
def test_hand_traces(case):
    g, idx = _gold_index()
    c = [c for c in g["cases"] if c["name"] == case][0]
    q = np.asarray([c["query"]], np.uint8)
    if "B" in c:
        B, Bd, V, stopped, st = oracle.beam_search(idx, q, [g["start"]], c["r"], c["b"], c.get("es", False),
                                                   c.get("vl", 20), c.get("esr", c["r"]))
        assert B.tolist() == c["B"]
        assert Bd.tolist() == c["B_dist"]
        assert V.tolist() == c["V"]
        assert stopped == c["stopped"]
        assert st["evals"] == c["evals"]
    elif "variant" in c:
        ids, ds, st = oracle.range_search_one(idx, q, c["r"], c["variant"], c["b"])
        assert ids.tolist() == c["result"]
        assert ds.tolist() == c["result_dist"]
        for k in ("visits_beam", "visits_greedy", "rounds", "final_beam", "evals", "distinct"):
            if k in c:
                assert st[k] == c[k], k
    else:
        ids, ds = oracle.brute_force(idx, q, c["r"])
        assert ids.tolist() == c["result"]
        assert ds.tolist() == c["result_dist"]


GOLD_ES = os.path.join(os.path.dirname(__file__), "golden", "es_metric_traces.json")


@pytest.mark.parametrize("case", [c["name"] for c in json.load(open(GOLD_ES))["cases"]])
def test_es_metric_hand_traces(case):
    """Alg. 1 + Alg. 4 with M = d_top1, d_top10 or d_top10 / d_start on a star built so that
    an off-by-one in the 10th-closest index, the farthest point in place of the 10th, or a
    ratio against the wrong distance each changes when the search stops."""
    g = json.load(open(GOLD_ES))
    X = np.asarray(g["points"], np.uint8)[:, None]
    adj = np.asarray([[SENT if v < 0 else v for v in row] for row in g["adjacency"]], np.uint32)
    idx = oracle.Index(X, adj, g["start"])
    c = [c for c in g["cases"] if c["name"] == case][0]
    q = np.asarray([g["query"]], np.uint8)
    B, Bd, V, stopped, st = oracle.beam_search(idx, q, [g["start"]], g["r"], c["b"], True, c["vl"], c["esr"],
                                               es_metric=c["metric"])
    assert B.tolist() == c["B"]
    assert Bd.tolist() == [float((g["query"] - g["points"][i]) ** 2) for i in c["B"]]
    assert V.tolist() == c["V"]
    assert stopped == c["stopped"]
    assert st["evals"] == c["evals"]


# ------------------------------------------------------------------------------------------------
# small synthetic datasets
# ------------------------------------------------------------------------------------------------

def _reachable(adj, start):
    n, R = adj.shape
    rows = np.repeat(np.arange(n), R)
    cols = adj.reshape(-1).astype(np.int64)
    ok = cols != SENT
    G = sp.csr_matrix((np.ones(ok.sum()), (rows[ok], cols[ok])), shape=(n, n))
    order = breadth_first_order(G, start, directed=True, return_predecessors=False)
    m = np.zeros(n, bool)
    m[order] = True
    return m


@pytest.fixture(scope="module")
def tiny():
    cfg = rrsynth.small_config("tiny", n=600, nq=40, d=16, R=12, L=24, n_centres=6, fam_cap=60, seed=3)
    ds = rrsynth.make_dataset(cfg)
    idx = oracle.Index(ds.X, ds.adj, ds.start)
    return ds, idx


@pytest.fixture(scope="module")
def small():
    cfg = rrsynth.small_config("small", n=3000, nq=120, d=32, R=16, L=32, n_centres=10, fam_cap=150, seed=5)
    ds = rrsynth.make_dataset(cfg)
    idx = oracle.Index(ds.X, ds.adj, ds.start)
    return ds, idx


def _exact(ds, q, r):
    diff = ds.X.astype(np.int64) - q.astype(np.int64)[None, :]
    d = (diff * diff).sum(1)
    ids = np.nonzero(d <= r)[0]
    order = np.lexsort((ids, d[ids]))
    return ids[order], d[ids][order]


def test_distances_exact_int64(tiny):
    ds, idx = tiny
    rng = np.random.default_rng(0)
    for qi in range(5):
        ids = rng.integers(0, ds.X.shape[0], 50).astype(np.uint32)
        got = oracle.distances(idx, ds.Q[qi], ids)
        diff = ds.X[ids].astype(np.int64) - ds.Q[qi].astype(np.int64)
        assert np.array_equal(got, (diff * diff).sum(1).astype(np.float64))


@pytest.mark.parametrize("dtype,metric", [("u8", "ip"), ("i8", "l2"), ("i8", "ip"), ("f32", "l2"), ("f32", "ip")])
def test_distances_every_branch(dtype, metric):
    """Every element type and metric of the distance (Sec. 2: squared L2, negative inner
    product), recomputed in numpy: int64 for 8-bit data (exact), fp64 for fp32 data."""
    rng = np.random.default_rng(17)
    n, d = 64, 37
    if dtype == "u8":
        X = rng.integers(0, 256, (n, d)).astype(np.uint8)
    elif dtype == "i8":
        X = rng.integers(-128, 128, (n, d)).astype(np.int8)
    else:
        X = rng.normal(size=(n, d)).astype(np.float32)
    adj = np.full((n, 4), SENT, np.uint32)
    idx = oracle.Index(X, adj, 0, metric=oracle.L2 if metric == "l2" else oracle.IP)
    wide = np.float64 if dtype == "f32" else np.int64
    for qi in range(5):
        q = X[qi * 7 + 3]
        ids = rng.integers(0, n, 40).astype(np.uint32)
        got = oracle.distances(idx, q, ids)
        x = X[ids].astype(wide)
        qq = q.astype(wide)
        want = ((x - qq) ** 2).sum(1) if metric == "l2" else -(x * qq).sum(1)
        if dtype == "f32":
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
        else:
            assert np.array_equal(got, want.astype(np.float64))
    # int8 extremes: |(-128) - 127|^2 * d and (-128)(-128) * d stay exact
    if dtype == "i8":
        lo = np.full(d, -128, np.int8)
        hi = np.full(d, 127, np.int8)
        X2 = np.stack([lo, hi])
        i2 = oracle.Index(X2, np.full((2, 1), SENT, np.uint32), 0, metric=oracle.L2 if metric == "l2" else oracle.IP)
        got = oracle.distances(i2, lo, np.array([0, 1], np.uint32))
        want = [0.0, float(255 * 255 * d)] if metric == "l2" else [-float(128 * 128 * d), float(128 * 127 * d)]
        assert got.tolist() == want


def test_brute_force_matches_numpy(tiny):
    ds, idx = tiny
    for qi in range(len(ds.Q)):
        ids, d = oracle.brute_force(idx, ds.Q[qi], ds.radius)
        eids, ed = _exact(ds, ds.Q[qi], ds.radius)
        assert np.array_equal(ids, eids)
        assert np.array_equal(d, ed)


@pytest.mark.parametrize("variant", ["beam", "greedy", "doubling"])
def test_exhaustive_beam_equals_brute_force(tiny, variant):
    """b >= n, no early stop, every node reachable: B is never trimmed, so the search
    visits the whole graph and N is the exact range result (Def. 2.1)."""
    ds, idx = tiny
    assert _reachable(ds.adj, ds.start).all()
    n = ds.X.shape[0]
    for r in (ds.radius, 2 * ds.radius, 4 * ds.radius):
        for qi in range(0, len(ds.Q), 4):
            ids, d, st = oracle.range_search_one(idx, ds.Q[qi], r, variant, beam=n + 1, b_max=4 * n)
            eids, ed = _exact(ds, ds.Q[qi], r)
            assert np.array_equal(ids, eids)
            assert np.array_equal(d, ed)
            assert st["visits_beam"] == n  # every node visited exactly once


def test_greedy_is_in_range_closure(small):
    """Alg. 2 returns S plus everything reachable from S through in-range nodes; the
    visit order does not matter.  Checked against scipy's BFS on the graph with edges
    kept only into in-range nodes, from a virtual source wired to S."""
    ds, idx = small
    n = ds.X.shape[0]
    rng = np.random.default_rng(1)
    for qi in range(0, len(ds.Q), 3):
        q = ds.Q[qi]
        r = 3 * ds.radius
        diff = ds.X.astype(np.int64) - q.astype(np.int64)
        dall = (diff * diff).sum(1)
        inr = dall <= r
        cand = np.nonzero(inr)[0]
        if len(cand) == 0:
            continue
        S = rng.choice(cand, size=min(3, len(cand)), replace=False)
        got, gd, _ = oracle.greedy_search(idx, q, S, r)
        rows = np.repeat(np.arange(n), ds.adj.shape[1])
        cols = ds.adj.reshape(-1).astype(np.int64)
        keep = (cols != SENT)
        keep[keep] &= inr[cols[keep]]
        rr = np.concatenate([rows[keep], np.full(len(S), n)])
        cc = np.concatenate([cols[keep], S])
        G = sp.csr_matrix((np.ones(len(rr)), (rr, cc)), shape=(n + 1, n + 1))
        order = breadth_first_order(G, n, directed=True, return_predecessors=False)
        want = np.sort(order[order != n])
        assert np.array_equal(np.sort(got), want)
        assert len(np.unique(got)) == len(got)
        assert np.array_equal(gd, dall[got].astype(np.float64))


VARS = ["beam", "beam_es", "greedy", "greedy_es", "doubling", "doubling_es"]


@pytest.fixture(scope="module")
def small_runs(small):
    ds, idx = small
    out = {}
    for v in VARS:
        for b in (8, 32):
            out[(v, b)] = oracle.range_search(idx, ds.Q, ds.radius, v, beam=b, b_max=4096)
    return out


@pytest.mark.parametrize("variant", VARS)
def test_invariants(small, small_runs, variant):
    ds, idx = small
    for b in (8, 32):
        ids_l, d_l, st_l = small_runs[(variant, b)]
        for qi, (ids, d, st) in enumerate(zip(ids_l, d_l, st_l)):
            eids, ed = _exact(ds, ds.Q[qi], ds.radius)
            assert np.all(d <= ds.radius)
            assert len(np.unique(ids)) == len(ids)
            assert np.all(np.isin(ids, eids))
            key = np.lexsort((ids, d))
            assert np.array_equal(key, np.arange(len(ids)))  # sorted by (dist, id)
            ex = dict(zip(eids.tolist(), ed.tolist()))
            assert all(ex[i] == dd for i, dd in zip(ids.tolist(), d.tolist()))
            if variant.startswith("beam"):
                assert len(ids) <= b
            if len(eids) == 0:
                assert len(ids) == 0
            if variant.endswith("_es") and st["early_stopped"]:
                assert len(ids) == 0


@pytest.mark.parametrize("base", ["beam", "greedy", "doubling"])
def test_early_stop_returns_full_result_or_nothing(small_runs, base):
    """Alg. 5 only fires while the closest point of B is outside r, so the result of
    an early-stopped search is empty; otherwise the search is identical."""
    for b in (8, 32):
        a_ids, _, a_st = small_runs[(base, b)]
        e_ids, _, e_st = small_runs[(base + "_es", b)]
        for x, y, s in zip(a_ids, e_ids, e_st):
            if len(y):
                assert np.array_equal(x, y)
            else:
                assert len(x) == 0 or s["early_stopped"]


def test_greedy_extends_beam(small_runs):
    for b in (8, 32):
        for x, y in zip(small_runs[("beam", b)][0], small_runs[("greedy", b)][0]):
            assert np.all(np.isin(x, y))
            if len(x) < b:
                assert np.array_equal(x, y)


def test_doubling_terminates_below_beam(small_runs):
    for b in (8, 32):
        for ids, st in zip(small_runs[("doubling", b)][0], small_runs[("doubling", b)][2]):
            assert st["truncated"] or len(ids) < st["final_beam"]
            assert st["final_beam"] == b * 2 ** (st["rounds"] - 1)


def test_average_precision_def22():
    truth = [np.array([1, 2, 3, 4]), np.array([], int), np.array([7])]
    found = [np.array([1, 2]), np.array([], int), np.array([7])]
    assert oracle.average_precision(truth, found) == pytest.approx(3 / 5)
    assert oracle.average_precision(truth, truth) == 1.0
    assert oracle.average_precision([np.array([], int)], [np.array([], int)]) == 1.0


def test_recall_improves_with_beam(small, small_runs):
    """More beam can only help on average (sanity of the whole pipeline)."""
    ds, idx = small
    truth = [_exact(ds, q, ds.radius)[0] for q in ds.Q]
    ap8 = oracle.average_precision(truth, small_runs[("greedy", 8)][0])
    ap32 = oracle.average_precision(truth, small_runs[("greedy", 32)][0])
    assert ap32 >= ap8 - 1e-12
    assert ap32 > 0.5


def test_inner_product_fp32_distances():
    cfg = rrsynth.small_config("ip", n=500, nq=10, d=24, R=12, L=24, n_centres=5, fam_cap=50, seed=9, dtype="f32",
                               metric=rrsynth.M_IP)
    ds = rrsynth.make_dataset(cfg)
    idx = oracle.Index(ds.X, ds.adj, ds.start, metric=oracle.IP)
    for qi in range(len(ds.Q)):
        ids, d = oracle.brute_force(idx, ds.Q[qi], ds.radius)
        want = -(ds.X.astype(np.float64) @ ds.Q[qi].astype(np.float64))
        sel = np.nonzero(want <= ds.radius)[0]
        assert set(ids.tolist()) == set(sel.tolist())
        np.testing.assert_allclose(d, want[ids], rtol=1e-12, atol=1e-12)
        n = ds.X.shape[0]
        if _reachable(ds.adj, ds.start).all():
            g, gd, _ = oracle.range_search_one(idx, ds.Q[qi], ds.radius, "beam", beam=n + 1)
            assert np.array_equal(np.sort(g), np.sort(ids))


def test_batch_threads_match_single(small):
    ds, idx = small
    a = oracle.range_search(idx, ds.Q[:40], ds.radius, "greedy_es", beam=16, threads=1)
    b = oracle.range_search(idx, ds.Q[:40], ds.radius, "greedy_es", beam=16, threads=4)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert a[2] == b[2]


# ---- early-stopping metrics of Sec. 3.2 (Alg. 4 with M = d_top1, d_top10, d_top10 / d_start)

def _run_es(idx, ds, metric, t, variant="greedy_es", b=8, vl=5):
    return oracle.range_search(idx, ds.Q, ds.radius, variant, beam=b, es_vl=vl, es_radius=t, es_metric=metric)


def _same(a, b):
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    for s, u in zip(a[2], b[2]):
        assert s == u


def test_es_top1_below_r_is_the_bare_closest_outside_r_test(small):
    """d_top1 > t with t <= r adds nothing to min_B d > r, so the stop rule reduces to
    'closest point outside r and vl visits' -- d_visited with an esr no distance is below."""
    ds, idx = small
    for t in (ds.radius, ds.radius / 3.0):
        _same(_run_es(idx, ds, "top1", t), _run_es(idx, ds, "visited", -1e300))


def test_es_ratio_at_zero_is_top10_at_zero(small):
    """d_top10 / d_start > 0 and d_top10 > 0 agree for squared L2 (d_start > 0 on these queries)."""
    ds, idx = small
    _same(_run_es(idx, ds, "top10_ratio", 0.0), _run_es(idx, ds, "top10", 0.0))


def test_es_top10_stops_no_later_than_top1(small):
    """d_top10 >= d_top1 at every step, so with one threshold the d_top10 rule fires no later."""
    ds, idx = small
    t = float(np.median([d for d in oracle.range_search(idx, ds.Q, 1e300, "beam", beam=8)[1][0]]))
    a = _run_es(idx, ds, "top10", t, variant="beam_es")
    b = _run_es(idx, ds, "top1", t, variant="beam_es")
    for sa, sb in zip(a[2], b[2]):
        assert sa["visits_beam"] <= sb["visits_beam"]
        assert sb["early_stopped"] <= sa["early_stopped"]


@pytest.mark.parametrize("metric", ["visited", "top1", "top10", "top10_ratio"])
def test_es_metrics_keep_full_result_or_nothing(small, small_runs, metric):
    """Any M only acts while the closest point of B is outside r: each result equals the
    search without early stopping, or is empty; an unreachable threshold never stops."""
    ds, idx = small
    t = 0.5 if metric == "top10_ratio" else ds.radius * 0.5
    full = small_runs[("greedy", 8)]
    es = _run_es(idx, ds, metric, t)
    for x, y, s in zip(full[0], es[0], es[2]):
        assert np.array_equal(x, y) or (len(y) == 0 and s["early_stopped"])
    never = _run_es(idx, ds, metric, 1e300)
    for x, y, s in zip(full[0], never[0], never[2]):
        assert np.array_equal(x, y) and not s["early_stopped"]


# ---- multi-parent beam search (expand parents per iteration; a variant of Alg. 1, not in the paper)

@pytest.mark.parametrize("expand", [2, 4])
@pytest.mark.parametrize("variant", ["beam", "greedy"])
def test_multi_parent_exhaustive_equals_brute_force(tiny, variant, expand):
    """With b >= n on a graph where every point is reachable, any number of parents per iteration
    still visits everything, so the result is the exact range (Def. 2.1)."""
    ds, idx = tiny
    assert _reachable(ds.adj, ds.start).all()
    n = ds.X.shape[0]
    for qi in range(len(ds.Q)):
        ids, d, st = oracle.range_search_one(idx, ds.Q[qi], ds.radius, variant, beam=n, b_max=n, expand=expand)
        eids, ed = _exact(ds, ds.Q[qi], ds.radius)
        assert np.array_equal(ids, eids) and np.array_equal(d.astype(np.int64), ed)


def test_multi_parent_with_one_parent_is_alg1(small, small_runs):
    ds, idx = small
    for v in ("beam_es", "greedy"):
        a = oracle.range_search(idx, ds.Q, ds.radius, v, beam=8, b_max=4096, expand=1)
        b = small_runs[(v, 8)]
        for x, y in zip(a[0], b[0]):
            assert np.array_equal(x, y)
        assert [s["visits_beam"] for s in a[2]] == [s["visits_beam"] for s in b[2]]


@pytest.mark.parametrize("expand", [2, 3, 8])
def test_multi_parent_invariants(small, small_runs, expand):
    """Results are in range, unique, sorted and exact-distance; plain beam keeps at most b; the early
    stop still returns the full result or nothing."""
    ds, idx = small
    for v in ("beam", "greedy", "greedy_es"):
        ids_l, d_l, st_l = oracle.range_search(idx, ds.Q, ds.radius, v, beam=16, expand=expand)
        for qi, (ids, d, st) in enumerate(zip(ids_l, d_l, st_l)):
            eids, ed = _exact(ds, ds.Q[qi], ds.radius)
            assert np.all(np.isin(ids, eids)) and len(np.unique(ids)) == len(ids)
            assert np.array_equal(np.lexsort((ids, d)), np.arange(len(ids)))
            ex = dict(zip(eids.tolist(), ed.tolist()))
            assert all(ex[i] == dd for i, dd in zip(ids.tolist(), d.tolist()))
            if v == "beam":
                assert len(ids) <= 16
            if v == "greedy_es" and st["early_stopped"]:
                assert len(ids) == 0


# ---- warm-restart doubling (rounds continue instead of restarting; a variant of Alg. 3, not in the paper)

def test_warm_doubling_equals_alg3_without_a_second_round(small, small_runs):
    """The first round of both is Alg. 1 from the start point: if it ends with |N| < b there is no
    second round, and the results agree."""
    ds, idx = small
    for v, w in (("doubling", "doubling_warm"), ("doubling_es", "doubling_warm_es")):
        lit = small_runs[(v, 8)]
        warm = oracle.range_search(idx, ds.Q, ds.radius, w, beam=8, b_max=4096)
        single = 0
        for x, y, sl, sw in zip(lit[0], warm[0], lit[2], warm[2]):
            if sl["rounds"] == 1:
                single += 1
                assert np.array_equal(x, y) and sw["rounds"] == 1
                assert sl["early_stopped"] == sw["early_stopped"]
        assert single > 0


@pytest.mark.parametrize("variant", ["doubling_warm", "doubling_warm_es"])
def test_warm_doubling_invariants(small, variant):
    """In range, unique, sorted, exact distances; no point visited twice; a stopped-early search is
    empty; the final beam is b * 2^(rounds - 1) and ends below b unless truncated."""
    ds, idx = small
    ids_l, d_l, st_l = oracle.range_search(idx, ds.Q, ds.radius, variant, beam=8, b_max=4096)
    for qi, (ids, d, st) in enumerate(zip(ids_l, d_l, st_l)):
        eids, ed = _exact(ds, ds.Q[qi], ds.radius)
        assert np.all(np.isin(ids, eids)) and len(np.unique(ids)) == len(ids)
        assert np.array_equal(np.lexsort((ids, d)), np.arange(len(ids)))
        ex = dict(zip(eids.tolist(), ed.tolist()))
        assert all(ex[i] == dd for i, dd in zip(ids.tolist(), d.tolist()))
        assert st["visits_beam"] <= ds.X.shape[0]
        assert st["final_beam"] == 8 * 2 ** (st["rounds"] - 1)
        assert st["truncated"] or len(ids) < st["final_beam"]
        if st["early_stopped"]:
            assert len(ids) == 0


def test_warm_doubling_exhaustive_equals_brute_force(tiny):
    ds, idx = tiny
    n = ds.X.shape[0]
    for qi in range(0, len(ds.Q), 3):
        ids, d, st = oracle.range_search_one(idx, ds.Q[qi], ds.radius, "doubling_warm", beam=n + 1, b_max=4 * n)
        eids, ed = _exact(ds, ds.Q[qi], ds.radius)
        assert np.array_equal(ids, eids) and np.array_equal(d.astype(np.int64), ed)
        assert st["visits_beam"] == n


def test_warm_doubling_evaluates_each_point_once(small):
    """Rounds never re-evaluate: the distance evaluations equal the distinct points evaluated."""
    ds, idx = small
    _, _, st_l = oracle.range_search(idx, ds.Q, ds.radius, "doubling_warm", beam=8, b_max=4096)
    for st in st_l:
        assert st["evals"] == st["distinct"]


def test_batch_with_one_early_stop_radius_matches_single_queries(small):
    """A constant esr different from r goes through the batch driver; it must agree with the
    one-query entry point called per query (the binding only marshals)."""
    ds, idx = small
    esr = 1.5 * ds.radius
    a = oracle.range_search(idx, ds.Q[:30], ds.radius, "greedy_es", beam=8, es_vl=5, es_radius=esr, threads=4)
    for i in range(30):
        ids, d, st = oracle.range_search_one(idx, ds.Q[i], ds.radius, "greedy_es", beam=8, es_vl=5, es_radius=esr)
        assert np.array_equal(a[0][i], ids) and np.array_equal(a[1][i], d) and a[2][i] == st
