"""Failure paths of the C ABI, made on the host or through a bounded device guard.

No test here faults, traps or hangs the GPU:
  * RR_EOVERFLOW: a small max_results_total cuts the result volume; every
    query keeps a subset of the oracle's answer and the cut ones carry
    RR_FLAG_TRUNCATED;
  * RR_ENOMEM: the library's next device allocation is made to fail (a host
    hook, rr_debug_set("fail_alloc_after")); the call fails cleanly and the
    next one is exact again;
  * RR_EINTERNAL: the beam and doubling kernels' per-query iteration guard is
    lowered (rr_debug_set("beam_iteration_limit")) so that it runs out; the
    kernel records the guard in its status word and returns, the call reports
    it, and the context stays usable."""
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
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    oi = oracle.Index(ds.X, ds.adj, ds.start)
    return rr, ds, oi


def _same_as_oracle(res, o_ids, o_d):
    for i in range(len(o_ids)):
        ids, d = res.query(i)
        assert np.array_equal(ids, o_ids[i]), i
        assert np.array_equal(d.astype(np.int64), o_d[i].astype(np.int64)), i


def test_overflow_keeps_a_truncated_subset(env):
    rr, ds, oi = env
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    beam = 16
    o_ids, o_d, _ = oracle.range_search(oi, ds.Q, ds.radius, "greedy", beam=beam, threads=os.cpu_count() or 4)
    full = sum(len(x) for x in o_ids)
    heavy = sum(1 for x in o_ids if len(x) >= beam)
    cap = heavy * beam + 50  # the first beams of the phase-2 queries plus a little of their expansion
    assert full > cap
    res = gi.range_search(ds.Q, ds.radius, "greedy", beam=beam, max_results_total=cap)
    assert res.status == rr.RR_EOVERFLOW
    trunc = (res.flags & rr.RR_FLAG_TRUNCATED) != 0
    assert trunc.any()
    # the cap bounds the greedy phase's results; every query keeps its first beam
    p2 = (res.flags & rr.RR_FLAG_PHASE2) != 0
    assert p2.sum() == heavy
    assert int(np.diff(res.offsets)[p2].sum()) <= max(cap, heavy * beam)
    for i in range(len(ds.Q)):
        ids, d = res.query(i)
        if trunc[i]:
            assert len(ids) < len(o_ids[i])
            assert np.all(np.isin(ids, o_ids[i]))
            assert np.all(d <= ds.radius)
        else:
            assert np.array_equal(ids, o_ids[i])
    # the same index answers exactly again without the cap
    _same_as_oracle(gi.range_search(ds.Q, ds.radius, "greedy", beam=beam), o_ids, o_d)
    gi.close()


@pytest.mark.parametrize("nth,on_device", [(0, False), (1, True), (3, True)])
def test_allocation_failure_is_reported_and_recovered(env, nth, on_device):
    import torch
    rr, ds, oi = env
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)  # fresh: its scratch is allocated on first use
    Qd = torch.from_numpy(ds.Q).cuda()
    o_ids, o_d, _ = oracle.range_search(oi, ds.Q, ds.radius, "greedy_es", beam=32, threads=os.cpu_count() or 4)
    p = rr.rr_params_init(beam=32)
    try:
        rr.rr_debug_set("fail_alloc_after", nth)
        st, res = rr.rr_range_search(gi.h, Qd, ds.radius, "greedy_es", p, result_on_device=on_device, check=False)
    finally:
        rr.rr_debug_set("fail_alloc_after", -1)
    assert st == rr.RR_ENOMEM, (st, rr.rr_last_error())
    assert "alloc" in rr.rr_last_error()
    torch.cuda.synchronize()
    _same_as_oracle(gi.range_search(Qd, ds.radius, "greedy_es", beam=32), o_ids, o_d)
    gi.close()


@pytest.mark.parametrize("variant", ["beam", "greedy", "doubling"])
def test_device_iteration_guard_returns_an_error(env, variant):
    import torch
    rr, ds, oi = env
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    try:
        rr.rr_debug_set("beam_iteration_limit", 3)  # every query needs more than 3 visits at b = 32
        st, res = rr.rr_range_search(gi.h, ds.Q, ds.radius, variant, rr.rr_params_init(beam=32), check=False)
    finally:
        rr.rr_debug_set("beam_iteration_limit", 0)
    assert st == rr.RR_EINTERNAL, (st, rr.rr_last_error())
    assert "guard" in rr.rr_last_error()
    torch.cuda.synchronize()  # the context is still usable
    o_ids, o_d, _ = oracle.range_search(oi, ds.Q, ds.radius, variant, beam=32, threads=os.cpu_count() or 4)
    _same_as_oracle(gi.range_search(ds.Q, ds.radius, variant, beam=32), o_ids, o_d)
    gi.close()


def test_debug_hook_rejects_unknown_keys(env):
    rr, ds, oi = env
    with pytest.raises(rr.RRError):
        rr.rr_debug_set("no_such_hook", 1)
