"""GPU parity: librr (through the C ABI) against the CPU oracle, element by element.

8-bit data must match bit-exactly: the same result ids, in the same (dist, id)
order, with the same int32 distances, and the same exact counters (|V| of
every phase, distinct ids evaluated)."""
import os

import numpy as np
import pytest

import oracle
import rrsynth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")
SENT = 0xFFFFFFFF
VARS = ["beam", "beam_es", "greedy", "greedy_es", "doubling", "doubling_es"]


@pytest.fixture(scope="module")
def rr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    rr.load_library()
    return rr


@pytest.fixture(scope="module")
def c0():
    return rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)


@pytest.fixture(scope="module")
def c0_index(rr, c0):
    return rr.Index.from_arrays(c0.X, c0.adj, c0.start)


@pytest.fixture(scope="module")
def c0_oracle(c0):
    return oracle.Index(c0.X, c0.adj, c0.start)


_ocache = {}


def oracle_run(oi, ds, variant, beam, Q=None, r=None, b_max=32768, key=None):
    k = (key or id(ds), variant, beam, b_max, None if r is None else float(np.sum(r)))
    if k not in _ocache:
        _ocache[k] = oracle.range_search(oi, ds.Q if Q is None else Q, ds.radius if r is None else r, variant,
                                         beam=beam, b_max=b_max, threads=os.cpu_count() or 4)
    return _ocache[k]


def assert_same(res, o_ids, o_d, nq):
    assert len(res) == nq
    for i in range(nq):
        ids, d = res.query(i)
        assert np.array_equal(ids, o_ids[i]), "query %d: ids differ (%d vs %d results)" % (i, len(ids), len(o_ids[i]))
        assert np.array_equal(d.astype(np.int64), o_d[i].astype(np.int64)), "query %d: distances differ" % i


@pytest.mark.parametrize("variant", VARS)
@pytest.mark.parametrize("beam", [8, 32, 64])
def test_c0_bit_exact(rr, c0, c0_index, c0_oracle, variant, beam):
    o_ids, o_d, o_st = oracle_run(c0_oracle, c0, variant, beam)
    res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam)
    assert res.status == rr.RR_OK
    assert_same(res, o_ids, o_d, len(c0.Q))
    es = np.array([s["early_stopped"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_EARLY_STOPPED) != 0, es)
    if variant.startswith(("greedy", "doubling")):
        ph = np.array([s["phase"] != 0 for s in o_st], bool)
        assert np.array_equal((res.flags & rr.RR_FLAG_PHASE2) != 0, ph)


@pytest.mark.parametrize("variant", VARS)
def test_c0_exact_counters(rr, c0, c0_index, c0_oracle, variant):
    """|V| of every phase and the number of distinct ids evaluated equal the oracle's."""
    beam = 32
    o_ids, o_d, o_st = oracle_run(c0_oracle, c0, variant, beam)
    res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, collect_stats=1)
    st = res.stats
    assert np.array_equal(st["visits_beam"], [s["visits_beam"] for s in o_st])
    assert np.array_equal(st["visits_phase2"], [s["visits_greedy"] for s in o_st])
    assert np.array_equal(st["distinct"], [s["distinct"] for s in o_st])
    assert np.array_equal(st["rounds"], [s["rounds"] for s in o_st])
    # the GPU never evaluates more than the paper's literal count, never fewer than the distinct ids
    assert np.all(st["evals"] >= st["distinct"])
    assert_same(res, o_ids, o_d, len(c0.Q))


@pytest.mark.parametrize("shape", [dict(persistent=1), dict(tile_hint=2, seen_log2=6), dict(tile_hint=8, seen_log2=12),
                                   dict(persistent=1, tile_hint=1, seen_log2=5)])
def test_launch_shapes_do_not_change_results(rr, c0, c0_index, c0_oracle, shape):
    """Warps per CTA, seen-table size and the persistent work queue are performance knobs only."""
    for variant, beam in (("greedy_es", 32), ("beam", 64), ("doubling", 16)):
        o_ids, o_d, _ = oracle_run(c0_oracle, c0, variant, beam)
        res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, **shape)
        assert_same(res, o_ids, o_d, len(c0.Q))


@pytest.mark.parametrize("metric,thr", [("top1", 1.5), ("top10", 1.5), ("top10_ratio", 0.9), ("visited", 1.2)])
@pytest.mark.parametrize("variant,beam", [("greedy_es", 16), ("beam_es", 32)])
def test_c0_early_stop_metrics_bit_exact(rr, c0, c0_index, c0_oracle, metric, thr, variant, beam):
    """Alg. 4 with the metrics of Sec. 3.2: same results, stop decisions and visit counts as the oracle."""
    m = {"visited": rr.RR_ES_VISITED, "top1": rr.RR_ES_TOP1, "top10": rr.RR_ES_TOP10,
         "top10_ratio": rr.RR_ES_TOP10_RATIO}[metric]
    t = thr if metric == "top10_ratio" else float(np.floor(c0.radius * thr))
    o_ids, o_d, o_st = oracle.range_search(c0_oracle, c0.Q, c0.radius, variant, beam=beam, es_vl=10, es_radius=t,
                                           es_metric=metric, threads=os.cpu_count() or 4)
    res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, es_visit_limit=10, es_radius_mode=1,
                                es_radius=t, es_metric=m, collect_stats=1)
    assert res.status == rr.RR_OK
    assert_same(res, o_ids, o_d, len(c0.Q))
    es = np.array([s["early_stopped"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_EARLY_STOPPED) != 0, es)
    assert np.array_equal(res.stats["visits_beam"], [s["visits_beam"] for s in o_st])
    assert es.any()  # the threshold makes the metric act on this workload


def test_early_stop_metric_arguments_are_checked(rr, c0, c0_index):
    for variant, kw in (("doubling_es", dict(es_metric=rr.RR_ES_TOP1)),
                        ("greedy_es", dict(es_metric=rr.RR_ES_TOP10_RATIO)),  # ratio needs es_radius_mode = 1
                        ("greedy_es", dict(es_metric=7))):
        p = rr.rr_params_init(beam=16, **kw)
        st, _ = rr.rr_range_search(c0_index.h, c0.Q[:4], c0.radius, variant, p, check=False)
        assert st == rr.RR_EINVAL


def test_ragged_and_tiny_batches(rr, c0, c0_index, c0_oracle):
    for nq in (1, 2, 37, 129):
        Q = c0.Q[:nq]
        o_ids, o_d, _ = oracle.range_search(c0_oracle, Q, c0.radius, "greedy_es", beam=16)
        res = c0_index.range_search(Q, c0.radius, "greedy_es", beam=16)
        assert_same(res, o_ids, o_d, nq)


def test_empty_batch(rr, c0, c0_index):
    res = c0_index.range_search(c0.Q[:0], c0.radius, "greedy_es", beam=16)
    assert len(res) == 0 and len(res.ids) == 0


def test_no_point_in_range(rr, c0, c0_index, c0_oracle):
    for v in ("beam", "greedy_es", "doubling_es"):
        res = c0_index.range_search(c0.Q[:50], -1, v, beam=16)
        assert len(res.ids) == 0
        o_ids, _, o_st = oracle.range_search(c0_oracle, c0.Q[:50], -1, v, beam=16)
        assert all(len(x) == 0 for x in o_ids)


def test_whole_graph_in_range(rr, c0, c0_index, c0_oracle):
    """r above every distance: the greedy phase floods the whole reachable graph."""
    r = 2 ** 31 - 1
    Q = c0.Q[:3]
    o_ids, o_d, _ = oracle.range_search(c0_oracle, Q, r, "greedy", beam=8, threads=3)
    res = c0_index.range_search(Q, r, "greedy", beam=8)
    assert_same(res, o_ids, o_d, 3)
    assert len(res.ids) == 3 * c0.X.shape[0]


def test_per_query_radii_and_device_queries(rr, c0, c0_index, c0_oracle):
    import torch
    rng = np.random.default_rng(3)
    radii = c0.radius * rng.choice([1.0, 1.5, 2.0], size=200)
    Q = c0.Q[:200]
    o_ids, o_d, _ = oracle.range_search(c0_oracle, Q, radii, "greedy_es", beam=32)
    Qd = torch.from_numpy(Q).cuda()
    res = c0_index.range_search(Qd, radii, "greedy_es", beam=32)
    torch.cuda.synchronize()
    assert_same(res, o_ids, o_d, 200)


def test_device_results(rr, c0, c0_index, c0_oracle):
    import ctypes
    import torch
    Qd = torch.from_numpy(c0.Q).cuda()
    p = rr.rr_params_init(beam=32)
    st, res = rr.rr_range_search(c0_index.h, Qd, c0.radius, "greedy_es", p, result_on_device=True)
    assert st == rr.RR_OK and res.on_device == 1
    torch.cuda.synchronize()
    nq, tot = res.nq, res.total
    # wrap the device arrays with torch through __cuda_array_interface__
    class _A:
        def __init__(self, ptr, n, typestr):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}
    off = torch.as_tensor(_A(res.offsets, nq + 1, "<i8"), device="cuda").cpu().numpy()
    ids = torch.as_tensor(_A(res.ids, tot, "<u4"), device="cuda").cpu().numpy() if tot else np.zeros(0, np.uint32)
    dd = torch.as_tensor(_A(res.dists, tot, "<i4"), device="cuda").cpu().numpy() if tot else np.zeros(0, np.int32)
    rr.rr_result_free(res)
    o_ids, o_d, _ = oracle_run(c0_oracle, c0, "greedy_es", 32)
    for i in range(nq):
        assert np.array_equal(ids[off[i]:off[i + 1]], o_ids[i])
        assert np.array_equal(dd[off[i]:off[i + 1]], o_d[i].astype(np.int32))


def _tiny_index(rr, X, adj, start):
    return rr.Index.from_arrays(X, adj, start), oracle.Index(X, adj, start)


def test_identical_points_tie_break(rr):
    """All points equal: every distance ties, only the id order decides."""
    n, d = 300, 16
    X = np.full((n, d), 7, np.uint8)
    adj, start = rrsynth.build_graph(X, 8, 16, 1.2, seed=1)
    gi, oi = _tiny_index(rr, X, adj, start)
    Q = np.stack([np.full(d, 7, np.uint8), np.full(d, 9, np.uint8), np.full(d, 0, np.uint8)])
    for v in ("beam", "greedy", "doubling", "greedy_es"):
        for r in (0, 64, 10 ** 6):
            print("identical points:", v, r, flush=True)
            o_ids, o_d, _ = oracle.range_search(oi, Q, r, v, beam=8)
            assert_same(gi.range_search(Q, r, v, beam=8), o_ids, o_d, 3)


def test_degree_zero_nodes_and_int8(rr):
    rng = np.random.default_rng(5)
    n, d = 800, 24
    X = rng.integers(-128, 128, size=(n, d), dtype=np.int8)
    adj, start = rrsynth.build_graph(X, 12, 24, 1.2, seed=2)
    adj = adj.copy()
    adj[rng.choice(n, 60, replace=False)] = SENT  # nodes with no out-edges
    gi, oi = _tiny_index(rr, X, adj, start)
    Q = rng.integers(-128, 128, size=(64, d), dtype=np.int8)
    d2 = ((X[None].astype(np.int64) - Q[:, None].astype(np.int64)) ** 2).sum(-1)
    r = float(np.percentile(d2, 2))
    for v in VARS:
        for b in (4, 16):
            o_ids, o_d, _ = oracle.range_search(oi, Q, r, v, beam=b)
            assert_same(gi.range_search(Q, r, v, beam=b), o_ids, o_d, 64)


def test_inner_product_int8(rr):
    rng = np.random.default_rng(6)
    n, d = 600, 32
    X = rng.integers(-100, 100, size=(n, d), dtype=np.int8)
    adj, start = rrsynth.build_graph(X, 12, 24, 1.0, metric=rrsynth.M_IP, seed=3)
    gi = rr.Index.from_arrays(X, adj, start, metric=rr.RR_IP)
    oi = oracle.Index(X, adj, start, metric=oracle.IP)
    Q = rng.integers(-100, 100, size=(40, d), dtype=np.int8)
    ip = -(X[None].astype(np.int64) * Q[:, None].astype(np.int64)).sum(-1)
    r = float(np.percentile(ip, 3))
    for v in ("beam", "greedy_es", "doubling"):
        o_ids, o_d, _ = oracle.range_search(oi, Q, r, v, beam=16)
        assert_same(gi.range_search(Q, r, v, beam=16), o_ids, o_d, 40)


def test_brute_force_matches_oracle(rr, c0, c0_index, c0_oracle):
    res = c0_index.brute_force(c0.Q, c0.radius)
    for i in range(len(c0.Q)):
        ids, d = oracle.brute_force(c0_oracle, c0.Q[i], c0.radius)
        g_ids, g_d = res.query(i)
        assert np.array_equal(g_ids, ids)
        assert np.array_equal(g_d.astype(np.int64), d.astype(np.int64))


def test_rrx_file_roundtrip(rr, c0, c0_oracle, tmp_path):
    p = str(tmp_path / "c0.rrx")
    rrsynth.write_rrx(p, c0.X, c0.adj, c0.start, rrsynth.M_L2)
    gi = rr.Index.load(p)
    assert gi.info.n == c0.X.shape[0] and gi.info.R == c0.adj.shape[1] and gi.info.start == c0.start
    o_ids, o_d, _ = oracle_run(c0_oracle, c0, "greedy_es", 32)
    assert_same(gi.range_search(c0.Q, c0.radius, "greedy_es", beam=32), o_ids, o_d, len(c0.Q))


@pytest.mark.parametrize("variant,beam", [("greedy", 32), ("doubling_es", 16), ("beam_es", 64)])
def test_profiled_calls_are_bit_exact(rr, c0, c0_index, c0_oracle, variant, beam):
    """profile = 1 records CUDA events between the phases and counts launches; the results are
    those of the unprofiled call (device queries, device results, the tuned launch shape)."""
    import torch
    Qd = torch.from_numpy(c0.Q).cuda()
    o_ids, o_d, _ = oracle_run(c0_oracle, c0, variant, beam)
    for prof in (1, 0):
        p = rr.rr_params_init(beam=beam, profile=prof, persistent=1, tile_hint=4, seen_log2=10)
        st, res = rr.rr_range_search(c0_index.h, Qd, c0.radius, variant, p, result_on_device=True)
        assert st == rr.RR_OK
        pr = rr.rr_last_profile(c0_index.h)
        h = rr.rr_result_to_host(res)
        rr.rr_result_free(res)
        assert_same(rr.RangeResult(h), o_ids, o_d, len(c0.Q))
        if prof:
            assert pr.valid == 1 and pr.launches >= 2
            assert pr.beam_ms > 0 and pr.total_ms >= pr.beam_ms
            if variant == "beam_es":
                assert pr.phase2_queries == 0 and pr.phase2_steps == 0
        else:
            assert pr.valid == 0


@pytest.mark.parametrize("expand", [2, 3, 4])
@pytest.mark.parametrize("variant,beam", [("beam", 32), ("beam_es", 16), ("greedy", 16), ("greedy_es", 32)])
def test_c0_multi_parent_bit_exact(rr, c0, c0_index, c0_oracle, variant, beam, expand):
    """Multi-parent beam search (expand parents per iteration, a variant of Alg. 1 that is not in the
    paper) against the oracle's own transcription of it: ids, distances, flags and exact counters."""
    o_ids, o_d, o_st = oracle.range_search(c0_oracle, c0.Q, c0.radius, variant, beam=beam, expand=expand,
                                           threads=os.cpu_count() or 4)
    res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, expand=expand, collect_stats=1)
    assert res.status == rr.RR_OK
    assert_same(res, o_ids, o_d, len(c0.Q))
    es = np.array([s["early_stopped"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_EARLY_STOPPED) != 0, es)
    assert np.array_equal(res.stats["visits_beam"], [s["visits_beam"] for s in o_st])
    assert np.array_equal(res.stats["distinct"], [s["distinct"] for s in o_st])
    # persistent launch in another shape: the same results
    res2 = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, expand=expand, persistent=1, tile_hint=2,
                                 seen_log2=7)
    assert_same(res2, o_ids, o_d, len(c0.Q))


def test_multi_parent_arguments_are_checked(rr, c0, c0_index):
    with pytest.raises(rr.RRError):
        c0_index.range_search(c0.Q[:4], c0.radius, "doubling", beam=16, expand=2)
    with pytest.raises(rr.RRError):
        c0_index.range_search(c0.Q[:4], c0.radius, "greedy", beam=16, expand=5)


@pytest.mark.parametrize("variant", ["doubling_warm", "doubling_warm_es"])
@pytest.mark.parametrize("beam", [4, 16])
def test_c0_warm_doubling_bit_exact(rr, c0, c0_index, c0_oracle, variant, beam):
    """Warm-restart doubling (a variant of Alg. 3 not in the paper: rounds continue from the kept
    evaluations and visits) against the oracle's transcription of it: ids, distances, flags and exact
    counters (every point is evaluated once, so evaluations equal distinct ids)."""
    o_ids, o_d, o_st = oracle.range_search(c0_oracle, c0.Q, c0.radius, variant, beam=beam, b_max=4096,
                                           threads=os.cpu_count() or 4)
    res = c0_index.range_search(c0.Q, c0.radius, variant, beam=beam, b_max=4096, collect_stats=1)
    assert res.status == rr.RR_OK
    assert_same(res, o_ids, o_d, len(c0.Q))
    es = np.array([s["early_stopped"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_EARLY_STOPPED) != 0, es)
    ph = np.array([s["phase"] != 0 for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_PHASE2) != 0, ph)
    tr = np.array([s["truncated"] for s in o_st], bool)
    assert np.array_equal((res.flags & rr.RR_FLAG_TRUNCATED) != 0, tr)
    assert np.array_equal(res.stats["visits_beam"], [s["visits_beam"] for s in o_st])
    assert np.array_equal(res.stats["rounds"], [s["rounds"] for s in o_st])
    assert np.array_equal(res.stats["final_beam"], [s["final_beam"] for s in o_st])
    assert np.array_equal(res.stats["distinct"], [s["distinct"] for s in o_st])
    # and it visits no more than the literal Alg. 3 at the same b
    lit = c0_index.range_search(c0.Q, c0.radius, variant.replace("_warm", ""), beam=beam, b_max=4096,
                                collect_stats=1)
    assert res.stats["visits_beam"].sum() <= lit.stats["visits_beam"].sum()


@pytest.mark.parametrize("d", [16, 32, 48, 64, 200, 512])
def test_greedy_levels_at_every_row_width(rr, d):
    """The greedy levels split a vector over 1 to 32 lanes (16 bytes each, rounded up to a power of two)
    and a writer lane ends with 8 / lanes candidates: every split is compared with the oracle bit for bit
    (graph degree 32 takes the row-major expand pass, 24 the per-pair one)."""
    rng = np.random.default_rng(d)
    n = 1500
    C = rng.integers(0, 256, size=(6, d))
    X = np.clip(C[rng.integers(0, 6, n)] + rng.integers(-12, 13, size=(n, d)), 0, 255).astype(np.uint8)
    Q = np.clip(C[rng.integers(0, 6, 40)] + rng.integers(-12, 13, size=(40, d)), 0, 255).astype(np.uint8)
    d2 = ((X[None].astype(np.int64) - Q[:, None].astype(np.int64)) ** 2).sum(-1)
    r = float(np.percentile(d2, 8))
    for R in (32, 24):
        adj, start = rrsynth.build_graph(X, R, 32, 1.2, seed=d)
        gi, oi = _tiny_index(rr, X, adj, start)
        for v in ("greedy", "greedy_es"):
            o_ids, o_d, _ = oracle.range_search(oi, Q, r, v, beam=8)
            res = gi.range_search(Q, r, v, beam=8)
            assert sum(len(x) for x in o_ids) > 40 * 8  # phase 2 runs
            assert_same(res, o_ids, o_d, len(Q))
        gi.close()


def test_degree_not_multiple_of_four(rr):
    """An odd degree (rows of 7 entries, 28 bytes): the per-warp shared-memory slices of the beam and
    doubling kernels hold R-sized arrays and must stay 8-byte aligned for every warp (a slice of
    2*KI*8 + 2*R*8 + R*4 bytes was not, and faulted); every variant gives the oracle's results."""
    rng = np.random.default_rng(77)
    n, d = 2000, 32
    C = rng.integers(0, 256, size=(5, d))
    X = np.clip(C[rng.integers(0, 5, n)] + rng.integers(-20, 21, size=(n, d)), 0, 255).astype(np.uint8)
    Q = np.clip(C[rng.integers(0, 5, 50)] + rng.integers(-20, 21, size=(50, d)), 0, 255).astype(np.uint8)
    d2 = ((X[None].astype(np.int64) - Q[:, None].astype(np.int64)) ** 2).sum(-1)
    r = float(np.percentile(d2, 3))
    adj, start = rrsynth.build_graph(X, 7, 24, 1.2, seed=7)
    gi, oi = _tiny_index(rr, X, adj, start)
    for v in VARS:
        for b in (8, 32):
            o_ids, o_d, _ = oracle.range_search(oi, Q, r, v, beam=b)
            assert_same(gi.range_search(Q, r, v, beam=b), o_ids, o_d, len(Q))
    gi.close()
