"""Breadth-first relabeling of an index (rr_index_relabel).

The library renumbers the points in the queue order of a breadth-first
traversal from the start point (rows scanned in slot order, padding skipped,
unreached points last in id order) and searches the renamed graph.  The tests
compute that order themselves -- level by level with numpy, a formulation
pinned on the CPU against a plain queue traversal -- build the relabeled arrays
and run the oracle on them.  On 8-bit data the GPU's results on the relabeled
index equal, element by element, the oracle's results on the relabeled arrays
mapped back to the caller's ids (ties in distance come in internal order on
both sides).  Exhaustive search stays in (distance, id) order and equals the
un-relabeled index's."""
import collections
import os

import numpy as np
import pytest

import oracle
import rrsynth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")
SENT = 0xFFFFFFFF


def bfs_levels(adj, start):
    """old_of[new id] = caller's id: level-synchronous, each level in (parent position, slot) order with the
    first discovery of a point kept -- the queue order of a breadth-first traversal."""
    n = adj.shape[0]
    reached = np.zeros(n, bool)
    reached[start] = True
    frontier = np.array([start], dtype=np.int64)
    levels = [frontier]
    while len(frontier):
        nb = adj[frontier].reshape(-1)
        nb = nb[nb != SENT].astype(np.int64)
        nb = nb[~reached[nb]]
        _, first = np.unique(nb, return_index=True)
        frontier = nb[np.sort(first)]
        reached[frontier] = True
        levels.append(frontier)
    levels.append(np.nonzero(~reached)[0])
    return np.concatenate(levels).astype(np.int64)


def bfs_queue(adj, start):
    """The textbook queue traversal, one point at a time (small graphs only)."""
    n, R = adj.shape
    seen = [False] * n
    seen[start] = True
    q = collections.deque([start])
    order = []
    while q:
        v = q.popleft()
        order.append(v)
        for u in adj[v]:
            u = int(u)
            if u != SENT and not seen[u]:
                seen[u] = True
                q.append(u)
    order += [i for i in range(n) if not seen[i]]
    return np.array(order, dtype=np.int64)


def relabeled_arrays(X, adj, start, old_of):
    n = len(old_of)
    new_of = np.empty(n, np.int64)
    new_of[old_of] = np.arange(n)
    A = adj[old_of]
    A2 = np.where(A == SENT, SENT, new_of[np.where(A == SENT, 0, A)]).astype(np.uint32)
    return X[old_of], A2, int(new_of[start])


def test_level_bfs_equals_queue_bfs():
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(1, 60))
        R = int(rng.integers(1, 6))
        adj = rng.integers(0, n, size=(n, R)).astype(np.uint32)
        adj[rng.random((n, R)) < 0.3] = SENT  # padding anywhere in a row, some rows empty
        start = int(rng.integers(0, n))
        assert np.array_equal(bfs_levels(adj, start), bfs_queue(adj, start)), trial
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    order = bfs_levels(ds.adj, ds.start)
    assert np.array_equal(order, bfs_queue(ds.adj, ds.start))
    assert np.array_equal(np.sort(order), np.arange(len(ds.X)))  # a permutation
    assert order[0] == ds.start


def test_relabeled_arrays_are_the_same_graph():
    """Renaming commutes with the graph: the neighbours of new id i are the renamed neighbours of old_of[i]."""
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    old_of = bfs_levels(ds.adj, ds.start)
    X2, A2, s2 = relabeled_arrays(ds.X, ds.adj, ds.start, old_of)
    assert s2 == 0
    for i in range(0, len(old_of), 97):
        row = A2[i]
        back = np.where(row == SENT, SENT, old_of[np.where(row == SENT, 0, row)])
        assert np.array_equal(back.astype(np.uint32), ds.adj[old_of[i]])
        assert np.array_equal(X2[i], ds.X[old_of[i]])


def test_search_commutes_with_the_renaming_when_no_distances_tie():
    """With every distance distinct (fp32 data), no step of Alg. 1-3 depends on ids, so the oracle's search
    on the relabeled arrays returns the original search's results renamed, for every variant."""
    rng = np.random.default_rng(11)
    n, d = 1500, 12
    X = rng.standard_normal((n, d)).astype(np.float32)
    Q = rng.standard_normal((30, d)).astype(np.float32)
    adj, start = rrsynth.build_graph((X * 20 + 128).clip(0, 255).astype(np.uint8), 12, 24, 1.2, seed=3)
    d2 = ((Q[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    r = float(np.percentile(d2, 4))
    old_of = bfs_levels(adj, start)
    X2, A2, s2 = relabeled_arrays(X, adj, start, old_of)
    o1 = oracle.Index(X, adj, start)
    o2 = oracle.Index(X2, A2, s2)
    for v in ("beam", "beam_es", "greedy", "greedy_es", "doubling", "doubling_es"):
        ids1, d1, st1 = oracle.range_search(o1, Q, r, v, beam=8)
        ids2, dd2, st2 = oracle.range_search(o2, Q, r, v, beam=8)
        for i in range(len(Q)):
            assert np.array_equal(ids1[i], old_of[ids2[i]].astype(ids1[i].dtype)), (v, i)
            assert np.array_equal(d1[i], dd2[i]), (v, i)
            assert st1[i]["visits_beam"] == st2[i]["visits_beam"], (v, i)


# ------------------------------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def rr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    return rr


@pytest.fixture(scope="module")
def c0():
    return rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)


@pytest.fixture(scope="module")
def c0_relabeled(rr, c0):
    old_of = bfs_levels(c0.adj, c0.start)
    X2, A2, s2 = relabeled_arrays(c0.X, c0.adj, c0.start, old_of)
    gi = rr.Index.from_arrays(c0.X, c0.adj, c0.start).relabel()
    oi = oracle.Index(X2, A2, s2)
    return gi, oi, old_of


def _assert_mapped_equal(res, o_ids, o_d, old_of):
    for i in range(len(o_ids)):
        ids, d = res.query(i)
        want = old_of[o_ids[i]].astype(np.uint32) if len(o_ids[i]) else np.zeros(0, np.uint32)
        assert np.array_equal(ids, want), "query %d: ids differ (%d vs %d results)" % (i, len(ids), len(want))
        assert np.array_equal(d.astype(np.int64), o_d[i].astype(np.int64)), "query %d: distances differ" % i


@pytest.mark.gpu
def test_relabel_info_and_refusals(rr, c0):
    gi = rr.Index.from_arrays(c0.X, c0.adj, c0.start)
    assert gi.info.order == 0
    srv = gi.serve(workers=1)
    with pytest.raises(rr.RRError) as e:
        gi.relabel()
    assert e.value.status == rr.RR_EINVAL and "server" in str(e.value)
    srv.close()
    with pytest.raises(rr.RRError) as e:
        rr.rr_index_relabel(gi.h, 7)
    assert e.value.status == rr.RR_EINVAL
    before = gi.info.device_bytes
    gi.relabel()
    assert gi.info.order == rr.RR_ORDER_BFS
    assert gi.info.start == c0.start  # reported in the caller's ids
    assert gi.info.device_bytes == before + 4 * len(c0.X)
    with pytest.raises(rr.RRError) as e:
        gi.relabel()
    assert e.value.status == rr.RR_EINVAL and "already" in str(e.value)
    gi.close()


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["beam", "beam_es", "greedy", "greedy_es", "doubling", "doubling_es",
                                     "doubling_warm"])
@pytest.mark.parametrize("beam", [8, 32])
def test_relabel_c0_bit_exact(rr, c0, c0_relabeled, variant, beam):
    gi, oi, old_of = c0_relabeled
    o_ids, o_d, o_st = oracle.range_search(oi, c0.Q, c0.radius, variant, beam=beam, threads=os.cpu_count() or 4)
    res = gi.range_search(c0.Q, c0.radius, variant, beam=beam)
    assert res.status == rr.RR_OK
    _assert_mapped_equal(res, o_ids, o_d, old_of)
    es = np.array([s["early_stopped"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_EARLY_STOPPED) != 0, es)


@pytest.mark.gpu
def test_relabel_c0_multi_parent(rr, c0, c0_relabeled):
    gi, oi, old_of = c0_relabeled
    o_ids, o_d, _ = oracle.range_search(oi, c0.Q, c0.radius, "greedy", beam=16, expand=2,
                                        threads=os.cpu_count() or 4)
    res = gi.range_search(c0.Q, c0.radius, "greedy", beam=16, expand=2)
    _assert_mapped_equal(res, o_ids, o_d, old_of)


@pytest.mark.gpu
def test_relabel_brute_force_unchanged(rr, c0, c0_relabeled):
    gi, _, _ = c0_relabeled
    plain = rr.Index.from_arrays(c0.X, c0.adj, c0.start)
    a = plain.brute_force(c0.Q, c0.radius)
    b = gi.brute_force(c0.Q, c0.radius)
    assert np.array_equal(a.offsets, b.offsets)
    assert np.array_equal(a.ids, b.ids)  # (distance, id) order in the caller's ids on both
    assert np.array_equal(a.dists, b.dists)
    plain.close()


@pytest.mark.gpu
def test_relabel_noalloc_and_server(rr, c0, c0_relabeled):
    import torch
    gi, _, _ = c0_relabeled
    Qd = torch.from_numpy(c0.Q).cuda()
    nq, beam = len(c0.Q), 32
    want = gi.range_search(c0.Q, c0.radius, "beam_es", beam=beam)
    counts = torch.zeros((nq,), dtype=torch.int32, device="cuda")
    ids = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    dists = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    rr.rr_beam_search_noalloc(gi.h, Qd, c0.radius, "beam_es", rr.rr_params_init(beam=beam), counts, ids, dists)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    I = ids.cpu().numpy().view(np.uint32)
    assert np.array_equal(c, np.diff(want.offsets))
    for i in range(nq):
        assert np.array_equal(I[i, :c[i]], want.query(i)[0])
    g = gi.range_search(c0.Q, c0.radius, "greedy", beam=32)
    with gi.serve(workers=2, variant=rr.RR_GREEDY, beam=32) as srv:
        t0 = srv.submit(c0.Q[:200], c0.radius)[0]
        got = None
        for _ in range(200):
            got = srv.collect(t0, 200, timeout_ms=100)
            if got is not None:
                break
        assert got is not None
    for i in range(200):
        assert np.array_equal(got.query(i)[0], g.query(i)[0])


@pytest.mark.gpu
def test_relabel_precision_form_rebuilds_copies(rr):
    """A traversal copy built before the relabel is dropped and rebuilt in the new order: the FP8 search
    after the relabel returns exactly the points the exact search finds in range, mapped back."""
    cfg = rrsynth.small_config("relabel_ip", n=4000, nq=300, d=32, R=16, L=32, n_centres=8, fam_cap=200, seed=31,
                               dtype="f32", metric=rrsynth.M_IP)
    ds = rrsynth.make_dataset(cfg, cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start, metric=rr.RR_IP)
    before = gi.range_search(ds.Q, float(ds.radius), "greedy", beam=32, precision=2)
    gi.relabel()
    after = gi.range_search(ds.Q, float(ds.radius), "greedy", beam=32, precision=2)
    truth = gi.brute_force(ds.Q, float(ds.radius))
    r = float(ds.radius)
    for i in range(len(ds.Q)):
        ids, d = after.query(i)
        ex = -(ds.X[ids].astype(np.float64) @ ds.Q[i].astype(np.float64))
        np.testing.assert_allclose(d.astype(np.float64), ex, rtol=1e-5, atol=1e-6)
        assert np.all(ex <= r + 1e-5 * abs(r) + 1e-6)
        assert set(ids.tolist()) <= set(truth.query(i)[0].tolist())
    # the same points are found up to traversal order effects: totals within 2%
    assert abs(len(after.ids) - len(before.ids)) <= 0.02 * max(1, len(before.ids))
    gi.close()
