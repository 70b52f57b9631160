"""Parity at full size: 1,000,000 uint8 vectors (d=128), 10,000 queries, R=64.

The GPU runs the whole batch in the benchmark's launch configuration (device
queries, library defaults); the oracle recomputes a seeded sample of queries
one by one -- the heaviest ones included -- and every sampled result must match
bit-exactly.  The exhaustive search (Def. 2.1) is checked the same way."""
import os

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
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c1"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    oi = oracle.Index(ds.X, ds.adj, ds.start)
    Qd = torch.from_numpy(ds.Q).cuda()
    gt = gi.brute_force(Qd, ds.radius)
    return rr, ds, gi, oi, Qd, gt


def _sample(gt, k_heavy, k_rand, seed):
    counts = np.diff(gt.offsets)
    heavy = np.argsort(-counts, kind="stable")[:k_heavy]
    rng = np.random.default_rng(seed)
    rest = np.setdiff1d(np.arange(len(counts)), heavy)
    return np.concatenate([heavy, rng.choice(rest, k_rand, replace=False)])


def test_c1_brute_force_sample(env):
    rr, ds, gi, oi, Qd, gt = env
    for i in _sample(gt, 5, 45, 1):
        ids, d = oracle.brute_force(oi, ds.Q[i], ds.radius)
        g_ids, g_d = gt.query(i)
        assert np.array_equal(g_ids, ids)
        assert np.array_equal(g_d.astype(np.int64), d.astype(np.int64))


@pytest.mark.parametrize("variant,beam,k_heavy,k_rand,expand", [("greedy_es", 16, 20, 80, 1), ("greedy", 64, 10, 40, 1),
                                                                 ("beam_es", 64, 5, 95, 1), ("doubling_es", 16, 6, 34, 1),
                                                                 ("greedy", 64, 10, 40, 2),
                                                                 ("doubling_warm_es", 16, 6, 34, 1)])
def test_c1_sampled_bit_exact(env, variant, beam, k_heavy, k_rand, expand):
    rr, ds, gi, oi, Qd, gt = env
    res = gi.range_search(Qd, ds.radius, variant, beam=beam, expand=expand)
    assert res.status == rr.RR_OK
    sel = _sample(gt, k_heavy, k_rand, 2)
    o_ids, o_d, o_st = oracle.range_search(oi, ds.Q[sel], ds.radius, variant, beam=beam, expand=expand,
                                           threads=os.cpu_count() or 4)
    for k, i in enumerate(sel):
        ids, d = res.query(i)
        assert np.array_equal(ids, o_ids[k]), "query %d: %d vs %d results" % (i, len(ids), len(o_ids[k]))
        assert np.array_equal(d.astype(np.int64), o_d[k].astype(np.int64))
        assert bool(res.flags[i] & rr.RR_FLAG_EARLY_STOPPED) == bool(o_st[k]["early_stopped"])
    # every returned point is truly in range (AP's precondition, Def. 2.2)
    assert np.all(res.dists <= ds.radius)
