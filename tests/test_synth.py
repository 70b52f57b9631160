"""Input generation: determinism, graph invariants, result-count distribution (no GPU)."""
import numpy as np
import pytest

import rrsynth

SENT = 0xFFFFFFFF


@pytest.fixture(scope="module")
def c0():
    return rrsynth.make_dataset(rrsynth.CONFIGS["c0"])


def test_graph_invariants(c0):
    adj = c0.adj
    n, R = adj.shape
    assert R == 32
    for i in range(n):
        row = adj[i]
        valid = row[row != SENT]
        # padding only at the end of a row
        assert np.all(row[len(valid):] == SENT)
        assert np.all(valid < n)
        assert not np.any(valid == i)            # no self loops
        assert len(np.unique(valid)) == len(valid)  # no duplicate edges
    deg = (adj != SENT).sum(1)
    assert deg.max() <= R and deg.mean() > R / 3


def test_graph_reachable_from_start(c0):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    n, R = c0.adj.shape
    rows = np.repeat(np.arange(n), R)
    cols = c0.adj.reshape(-1).astype(np.int64)
    ok = cols != SENT
    G = sp.csr_matrix((np.ones(ok.sum()), (rows[ok], cols[ok])), shape=(n, n))
    order = breadth_first_order(G, c0.start, directed=True, return_predecessors=False)
    assert len(order) >= 0.999 * n


def test_builder_independent_of_threads():
    X, C, w = rrsynth.mixture_u8(3000, 32, 8, 12.0, 11, fam_cap=100)
    a1, s1 = rrsynth.build_graph(X, 16, 32, 1.2, passes=2, seed=4, threads=1)
    a4, s4 = rrsynth.build_graph(X, 16, 32, 1.2, passes=2, seed=4, threads=4)
    assert s1 == s4
    assert np.array_equal(a1, a4)


def test_start_point_is_nearest_to_mean():
    X, _, _ = rrsynth.mixture_u8(2000, 16, 4, 12.0, 2, fam_cap=50)
    m = X.astype(np.float64).mean(0)
    d = ((X.astype(np.float64) - m) ** 2).sum(1)
    assert rrsynth.start_point(X) == int(np.argmin(d))


def test_generator_deterministic():
    a = rrsynth.mixture_u8(1000, 16, 4, 12.0, 7, fam_cap=50)[0]
    b = rrsynth.mixture_u8(1000, 16, 4, 12.0, 7, fam_cap=50)[0]
    assert np.array_equal(a, b)


def test_c0_result_count_distribution(c0):
    """About 60% of queries match nothing and the tail reaches a few hundred
    (the shape of the paper's result-size table)."""
    X = c0.X.astype(np.int64)
    counts = []
    for q in c0.Q:
        d = ((X - q.astype(np.int64)) ** 2).sum(1)
        counts.append(int((d <= c0.radius).sum()))
    counts = np.asarray(counts)
    zero = (counts == 0).mean()
    assert 0.5 <= zero <= 0.7
    assert 250 <= counts.max() <= 1000


def test_rrx_roundtrip(tmp_path, c0):
    p = tmp_path / "c0.rrx"
    rrsynth.write_rrx(str(p), c0.X, c0.adj, c0.start, rrsynth.M_L2)
    raw = p.read_bytes()
    assert raw[:4] == b"RRX1"
    import struct
    n, d, dt, metric, R, start, ck = struct.unpack_from("<qiiiiqQ", raw, 8)
    assert (n, d, dt, metric, R, start) == (10000, 128, 0, 0, 32, c0.start)
    payload = raw[64:]
    assert len(payload) == n * d + n * R * 4
    assert rrsynth.rrx_checksum(payload) == ck
