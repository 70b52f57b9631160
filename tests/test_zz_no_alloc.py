"""rr_beam_search_noalloc: the beam search for callers that may not allocate.

Some callers cannot allocate device memory while they run (a fixed memory
budget reserved up front, a host callback, a no-allocation policy after
start-up).  This entry point writes into arrays the caller already owns and
keeps its intermediate data in one static device array.  The tests call it
through the C ABI twice in a row -- different variants and beams, so a stale
leftover in the shared array would show -- and check each output against
rr_range_search: exactly (the same kernels run on the same inputs), on an
8-bit L2 index, on an fp32 inner-product index, and on queries that need the
padded staging copy (d not a multiple of 16 bytes, an unaligned slice).  They
also check that a call allocates nothing: torch's allocator and the index's own
scratch stay as they were.  The file is collected last so that, if it fails, a
run that stops at the first failure has already run every other test; each
test also passes alone in a fresh process."""
import os

import numpy as np
import pytest

import rrsynth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.path.join(ROOT, "_cache")


def _rr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2502_13245_gb300 as rr
    rr.build()
    return rr, torch


def _check_against_range_search(rr, torch, gi, Qd, radius, variant, beam, is_float, **params):
    nq = Qd.shape[0]
    p = rr.rr_params_init(beam=beam, **params)
    counts = torch.full((nq,), -7, dtype=torch.int32, device="cuda")
    ids = torch.full((nq, beam), 123, dtype=torch.int32, device="cuda")
    dists = torch.full((nq, beam), -5, dtype=torch.float32 if is_float else torch.int32, device="cuda")
    rr.rr_beam_search_noalloc(gi.h, Qd, radius, variant, p, counts, ids, dists)
    torch.cuda.synchronize()
    want = gi.range_search(Qd, radius, variant, beam=beam, **params)
    c = counts.cpu().numpy()
    I = ids.cpu().numpy().view(np.uint32)
    D = dists.cpu().numpy()
    assert np.array_equal(c, np.diff(want.offsets))
    for i in range(nq):
        w_ids, w_d = want.query(i)
        assert np.array_equal(I[i, :c[i]], w_ids)
        assert np.array_equal(D[i, :c[i]], w_d)
        assert np.all(I[i, c[i]:] == 0xFFFFFFFF)
    return int(c.sum())


def test_noalloc_matches_range_search_twice_in_a_row():
    rr, torch = _rr()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    Qd = torch.from_numpy(ds.Q).cuda()
    total = 0
    for variant, beam, extra in (("beam_es", 32, {}), ("beam", 16, {}),
                                 ("beam_es", 24, {"es_metric": rr.RR_ES_TOP10, "es_radius_mode": 1,
                                                  "es_radius": float(ds.radius) * 1.5, "es_visit_limit": 10}),
                                 ("beam", 64, {"persistent": 1, "tile_hint": 2, "seen_log2": 9}),
                                 ("beam_es", 32, {"expand": 2})):
        total += _check_against_range_search(rr, torch, gi, Qd, ds.radius, variant, beam, False, **extra)
    assert total > 0
    gi.close()


def test_noalloc_allocates_nothing():
    """On a fresh index (no search has run, so it holds no scratch) two calls leave torch's
    allocator and the index's scratch exactly as they were."""
    rr, torch = _rr()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    Qd = torch.from_numpy(ds.Q).cuda()
    nq, beam = Qd.shape[0], 32
    counts = torch.zeros((nq,), dtype=torch.int32, device="cuda")
    ids = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    dists = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    before_torch = torch.cuda.memory_allocated()
    before_ix = rr.rr_index_info_get(gi.h).scratch_bytes
    assert before_ix == 0
    p = rr.rr_params_init(beam=beam)
    for variant in ("beam_es", "beam"):
        rr.rr_beam_search_noalloc(gi.h, Qd, ds.radius, variant, p, counts, ids, dists)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before_torch
    assert rr.rr_index_info_get(gi.h).scratch_bytes == before_ix
    assert int(counts.sum().item()) > 0
    gi.close()


def test_noalloc_fp32_inner_product_and_padded_queries():
    """fp32 distances come back as float (an inner-product index, d = 24); queries whose rows
    are not a multiple of 16 bytes (uint8, d = 20) or start unaligned are staged through the
    static array's padded copy first."""
    rr, torch = _rr()
    cfg = rrsynth.small_config("noalloc_ip", n=3000, nq=200, d=24, R=16, L=32, n_centres=8, fam_cap=100, seed=21,
                               dtype="f32", metric=rrsynth.M_IP)
    ds = rrsynth.make_dataset(cfg, cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start, metric=rr.RR_IP)
    Qd = torch.from_numpy(ds.Q).cuda()
    got = 0
    for variant, beam in (("beam", 32), ("beam_es", 16)):
        got += _check_against_range_search(rr, torch, gi, Qd, float(ds.radius), variant, beam, True)
    assert got > 0
    gi.close()

    cfg = rrsynth.small_config("noalloc_d20", n=3000, nq=200, d=20, R=16, L=32, n_centres=8, fam_cap=100, seed=22)
    ds = rrsynth.make_dataset(cfg, cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    assert rr.rr_index_info_get(gi.h).row_stride == 32  # 20-byte rows are padded on the device
    Qd = torch.from_numpy(ds.Q).cuda()
    got = _check_against_range_search(rr, torch, gi, Qd, ds.radius, "beam", 32, False)
    # an unaligned view: the rows start one byte into a larger buffer
    buf = torch.zeros(Qd.numel() + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = Qd.reshape(-1)
    Qu = buf[1:].view(Qd.shape)
    assert Qu.data_ptr() % 16 != 0
    got += _check_against_range_search(rr, torch, gi, Qu, ds.radius, "beam_es", 16, False)
    assert got > 0
    gi.close()


def test_noalloc_rejects_a_batch_beyond_the_static_scratch():
    rr, torch = _rr()
    ds = rrsynth.make_dataset(rrsynth.CONFIGS["c0"], cache_dir=CACHE)
    gi = rr.Index.from_arrays(ds.X, ds.adj, ds.start)
    # 80,000 queries x beam 512 x 8 bytes is far above the static array: rejected before any launch.
    # The outputs are full size, so no size check of the library is needed to keep writes in bounds.
    Q = torch.from_numpy(np.repeat(ds.Q, 80, axis=0)).cuda()
    nq, beam = Q.shape[0], 512
    counts = torch.zeros((nq,), dtype=torch.int32, device="cuda")
    ids = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    dists = torch.zeros((nq, beam), dtype=torch.int32, device="cuda")
    p = rr.rr_params_init(beam=beam)
    with pytest.raises(rr.RRError) as e:
        rr.rr_beam_search_noalloc(gi.h, Q, ds.radius, "beam", p, counts, ids, dists)
    assert e.value.status == rr.RR_EINVAL and "static scratch" in str(e.value)
    # the binding refuses outputs that are too small before the library sees them
    with pytest.raises(ValueError):
        rr.rr_beam_search_noalloc(gi.h, Q[:10], ds.radius, "beam", rr.rr_params_init(beam=16), counts[:5],
                                  ids, dists)
    # low-precision traversal would build (allocate) its copies: refused
    with pytest.raises(rr.RRError) as e:
        rr.rr_beam_search_noalloc(gi.h, Q[:10], ds.radius, "beam", rr.rr_params_init(beam=16, precision=1),
                                  counts, ids, dists)
    assert e.value.status == rr.RR_EINVAL
    gi.close()
