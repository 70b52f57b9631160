"""rr_beam_search_noalloc: the beam search for callers that may not allocate.

Some callers cannot allocate device memory while they run (a fixed memory
budget reserved up front, a host callback, a no-allocation policy after
start-up).  This entry point writes into arrays the caller already owns and
keeps its intermediate data in one static device array.  The test calls it
through the C ABI twice in a row -- different variants and beams, so a stale
leftover in the shared array would show -- and checks both outputs against
rr_range_search, exactly (8-bit data).  It must pass alone and after the other
tests, so it lives in the file pytest collects last."""
import os

import numpy as np
import pytest

import rrsynth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")


def test_noalloc_matches_range_search_twice_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    Qd = torch.from_numpy(ds.Q).cuda()
    nq = Qd.shape[0]
    for variant, beam in (("beam_es", 32), ("beam", 16)):
        p = rr.rr_params_init(beam=beam)
        counts = torch.full((nq,), -7, dtype=torch.int32, device="cuda")
        ids = torch.full((nq, beam), 123, dtype=torch.int32, device="cuda")
        dists = torch.full((nq, beam), -5, dtype=torch.int32, device="cuda")
        rr.rr_beam_search_noalloc(gi.h, Qd, ds.radius, variant, p, counts, ids, dists)
        torch.cuda.synchronize()
        want = gi.range_search(Qd, ds.radius, variant, beam=beam)
        c = counts.cpu().numpy()
        I = ids.cpu().numpy().view(np.uint32)
        D = dists.cpu().numpy()
        assert np.array_equal(c, np.diff(want.offsets))
        for i in range(nq):
            w_ids, w_d = want.query(i)
            assert np.array_equal(I[i, :c[i]], w_ids)
            assert np.array_equal(D[i, :c[i]], w_d)
            assert np.all(I[i, c[i]:] == 0xFFFFFFFF)
    gi.close()


def test_noalloc_rejects_a_batch_beyond_the_static_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    # 80,000 queries x beam 512 x 8 bytes is far above the static array; rejected before any launch
    Q = torch.from_numpy(np.repeat(ds.Q, 80, axis=0)).cuda()
    small = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = rr.rr_params_init(beam=512)
    with pytest.raises(rr.RRError) as e:
        rr.rr_beam_search_noalloc(gi.h, Q, ds.radius, "beam", p, small, small, small)
    assert e.value.status == rr.RR_EINVAL and "static scratch" in str(e.value)
    gi.close()
