"""Serving (rr_serve_*): continuous batching of single requests.

Every query is searched independently, so a request's result must not depend
on which batch it landed in: results served from a concurrent mix of
submitters, radii and batch sizes must equal the oracle's bit for bit on 8-bit
data.  Admission by result memory must make progress under any budget, and a
request whose results the budget cut carries RR_FLAG_TRUNCATED and holds a
subset of the full answer."""
import os
import threading

import numpy as np
import pytest

import oracle
import rrsynth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    oi = oracle.Index(ds.X, ds.adj, ds.start)
    # mixed radii r, 1.5 r, 2 r (seeded), as a service would see them
    radii = ds.radius * np.random.default_rng(3).choice([1.0, 1.5, 2.0], len(ds.Q))
    radii = np.floor(radii)
    o_ids, o_d, _ = oracle.range_search(oi, ds.Q, radii, "greedy_es", beam=32, threads=os.cpu_count() or 4)
    return rr, ds, gi, radii, o_ids, o_d


def _submit_in_threads(srv, ds, radii, order, nthreads, chunk):
    tickets = np.zeros(len(ds.Q), np.uint64)
    parts = np.array_split(order, nthreads)

    def run(part):
        for s in range(0, len(part), chunk):
            idx = part[s:s + chunk]
            t = srv.submit(ds.Q[idx], radii[idx])
            tickets[idx] = t

    th = [threading.Thread(target=run, args=(p,)) for p in parts]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return tickets


@pytest.mark.parametrize("workers,max_batch,chunk", [(1, 4096, 1), (2, 64, 1), (4, 257, 7)])
def test_served_results_equal_the_oracle(env, workers, max_batch, chunk):
    rr, ds, gi, radii, o_ids, o_d = env
    order = np.random.default_rng(workers).permutation(len(ds.Q))
    with gi.serve(workers=workers, max_batch=max_batch, batch_wait_us=100, variant="greedy_es", beam=32) as srv:
        tickets = _submit_in_threads(srv, ds, radii, order, 3, chunk)
        for i in range(len(ds.Q)):
            r = srv.poll(tickets[i], timeout_ms=60_000)
            assert r is not None, "request %d not served within 60 s" % i
            ids, d = r.query(0)
            assert np.array_equal(ids, o_ids[i]), i
            assert np.array_equal(d.astype(np.int64), o_d[i].astype(np.int64)), i
            assert (r.flags[0] & rr.RR_FLAG_TRUNCATED) == 0
        st = srv.stats()
        assert st["completed"] == len(ds.Q) and st["polled"] == len(ds.Q)
        assert st["queued"] == 0 and st["in_flight"] == 0 and st["bytes_held"] == 0
        assert 1 <= st["mean_batch"] <= max_batch
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]


def test_poll_is_nonblocking_and_tickets_retire(env):
    rr, ds, gi, radii, o_ids, o_d = env
    with gi.serve(workers=1, batch_wait_us=0, beam=32) as srv:
        t = srv.submit(ds.Q[:5], radii[:5])
        for i in range(5):
            r = srv.poll(t[i], timeout_ms=60_000)
            assert r is not None and np.array_equal(r.query(0)[0], o_ids[i])
        with pytest.raises(rr.RRError):  # retired
            srv.poll(t[0])
        with pytest.raises(rr.RRError):  # never issued
            srv.poll(10 ** 9)
        with pytest.raises(rr.RRError):  # NaN radius
            srv.submit(ds.Q[:1], np.array([np.nan]))


def test_tiny_budget_makes_progress_and_flags_cuts(env):
    rr, ds, gi, radii, o_ids, o_d = env
    n = 300
    # 2 KB: at most a few requests in flight; results of a batch are cut to what the budget has left
    with gi.serve(workers=2, max_batch=64, batch_wait_us=0, beam=32, result_budget_bytes=2048,
                  reserve_per_request=256) as srv:
        t = srv.submit(ds.Q[:n], radii[:n])
        cut = 0
        for i in range(n):
            r = srv.poll(t[i], timeout_ms=60_000)
            assert r is not None
            ids, d = r.query(0)
            if r.flags[0] & rr.RR_FLAG_TRUNCATED:
                cut += 1
                assert np.all(np.isin(ids, o_ids[i])) and len(ids) < len(o_ids[i])
            else:
                assert np.array_equal(ids, o_ids[i]), i
        st = srv.stats()
        assert st["completed"] == n and st["bytes_held"] == 0
    big = sum(len(o_ids[i]) * 8 > 2048 for i in range(n))
    assert cut >= big  # a request whose answer exceeds the whole budget cannot come back whole


def test_destroy_with_unpolled_results(env):
    rr, ds, gi, radii, o_ids, o_d = env
    srv = gi.serve(workers=2, beam=16, result_budget_bytes=4096)
    srv.submit(ds.Q[:200], radii[:200])
    srv.close()  # drains the queue and frees what nobody polled


@pytest.mark.parametrize("prec", [1, 2])
def test_serving_precision_form(env, prec):
    rr, ds, gi, radii, o_ids, o_d = env
    rs = np.random.default_rng(9)
    X = rs.standard_normal((4000, 64)).astype(np.float32)
    Q = X[:64] + 0.05 * rs.standard_normal((64, 64)).astype(np.float32)
    adj, start = rrsynth.build_graph(X, R=24, L=48, alpha=1.2, metric=rrsynth.M_L2, passes=1, seed=0)
    fi = rr.Index.from_arrays(X, adj, start, metric=rr.RR_L2)
    r = 20.0
    ref = fi.range_search(Q, r, "greedy", beam=16, precision=prec)
    with fi.serve(workers=2, variant="greedy", beam=16, precision=prec) as srv:
        t = srv.submit(Q, r)
        for i in range(len(Q)):
            res = srv.poll(t[i], timeout_ms=60_000)
            assert np.array_equal(res.query(0)[0], ref.query(i)[0])
            assert np.array_equal(res.query(0)[1], ref.query(i)[1])


def test_collect_returns_a_submission_as_one_csr(env):
    rr, ds, gi, radii, o_ids, o_d = env
    with gi.serve(workers=3, max_batch=100, batch_wait_us=50, beam=32) as srv:
        firsts = [(s, srv.submit(ds.Q[s:s + 100], radii[s:s + 100])[0]) for s in range(0, 1000, 100)]
        for s, t0 in reversed(firsts):
            res = srv.collect(t0, 100, timeout_ms=60_000)
            assert res is not None and len(res) == 100
            for j in range(100):
                ids, d = res.query(j)
                assert np.array_equal(ids, o_ids[s + j]) and np.array_equal(d.astype(np.int64), o_d[s + j])
        assert srv.stats()["bytes_held"] == 0


def test_device_results_equal_the_oracle(env):
    rr, ds, gi, radii, o_ids, o_d = env
    with gi.serve(workers=3, max_batch=97, batch_wait_us=50, beam=32, result_on_device=1) as srv:
        firsts = [(s, srv.submit(ds.Q[s:s + 100], radii[s:s + 100])[0]) for s in range(0, 1000, 100)]
        for s, t0 in firsts[::2]:
            res = srv.collect(t0, 100, timeout_ms=60_000)  # gathered on the device, copied here for checking
            for j in range(100):
                ids, d = res.query(j)
                assert np.array_equal(ids, o_ids[s + j]) and np.array_equal(d.astype(np.int64), o_d[s + j])
        for s, t0 in firsts[1::2]:
            for j in range(100):
                r = srv.poll(t0 + j, timeout_ms=60_000)
                assert np.array_equal(r.query(0)[0], o_ids[s + j])
        st = srv.stats()
        assert st["bytes_held"] == 0 and st["completed"] == 1000


def test_cancel_drops_only_queued_requests(env):
    rr, ds, gi, radii, o_ids, o_d = env
    with gi.serve(workers=1, max_batch=8, batch_wait_us=0, beam=32) as srv:
        t0 = srv.submit(ds.Q, radii)[0]
        dropped = srv.cancel()
        res = srv.collect(t0, len(ds.Q), timeout_ms=60_000)
        canceled = (res.flags & rr.RR_FLAG_CANCELED) != 0
        assert int(canceled.sum()) == dropped
        for i in range(len(ds.Q)):
            ids, d = res.query(i)
            if canceled[i]:
                assert len(ids) == 0
            else:
                assert np.array_equal(ids, o_ids[i])
        st = srv.stats()
        assert st["canceled"] == dropped and st["queued"] == 0 and st["bytes_held"] == 0
