"""Autotuner for the launch shape of the beam phase.

The beam kernel's speed on a given index and batch depends on knobs that do not
change any result (the search is bit-exact for every setting): the warps per CTA
(`tile_hint`), the size of the per-warp seen table (`seen_log2`, which trades
shared memory -- and so resident warps -- against repeated distance
evaluations), and the persistent launch (a resident grid whose warps pull
queries from a device counter, versus one warp per query in a full grid).  `tune()` times every setting
on the caller's batch with CUDA events, re-times the three fastest and the library default in interleaved
rounds, and keeps a non-default setting only if its median beats the default's by more than 2% (single
timings of a few-millisecond batch differ by more than the settings do); results are cached per (index
shape, beam, variant).
"""
from __future__ import annotations

import itertools
import json
import os

TILES = (2, 4, 8)
SEEN_LOG2 = (9, 10, 11)
PERSISTENT = (0, 1)


def choose(runs, default, margin=0.98):
    """The setting to keep from interleaved re-timings `runs` ({setting: [ms, ...]}): the one with the
    lowest median, unless it is not the default and does not beat the default's median by more than
    1 - margin (single timings of a few-millisecond batch differ by more than the settings do)."""
    med = {c: sorted(v)[len(v) // 2] for c, v in runs.items()}
    best = min(runs, key=lambda c: med[c])
    if best != default and default in med and med[best] > margin * med[default]:
        best = default
    return best, med


def _key(info, variant, beam):
    return "n%d_d%d_R%d_dt%d_%s_b%d" % (info.n, info.d, info.R, info.dtype, variant, beam)


def tune(index, queries, radius, variant, beam, stream=None, reps=3, cache_path=None, base_params=None, log=None):
    """Return (best_params_dict, table).  `index` is a paper_2502_13245_gb300.Index."""
    import torch

    import paper_2502_13245_gb300 as rr
    key = _key(index.info, variant, beam)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return cache[key], []
    base = dict(base_params or {})
    base["beam"] = beam
    s = stream if stream is not None else torch.cuda.current_stream()

    def time_it(tile, sl, pers, n):
        p = rr.rr_params_init(tile_hint=tile, seen_log2=sl, persistent=pers, **base)
        with torch.cuda.stream(s):
            st, res = rr.rr_range_search(index.h, queries, radius, variant, p, stream=s.cuda_stream,
                                         result_on_device=True)
            rr.rr_result_free(res)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            for _ in range(n):
                st, res = rr.rr_range_search(index.h, queries, radius, variant, p, stream=s.cuda_stream,
                                             result_on_device=True)
                rr.rr_result_free(res)
            e1.record(s)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    table = []
    for tile, sl, pers in itertools.product(TILES, SEEN_LOG2, PERSISTENT):
        ms = time_it(tile, sl, pers, reps)
        table.append({"tile_hint": tile, "seen_log2": sl, "persistent": pers, "ms": ms})
        if log:
            log("tune %s b=%d tile=%d seen=2^%d persistent=%d: %.3f ms" % (variant, beam, tile, sl, pers, ms))
    # the library default (what tile_hint = seen_log2 = persistent = 0 selects)
    default = (4, rr.beam_hash_lg(beam), 0)
    top = [(t["tile_hint"], t["seen_log2"], t["persistent"]) for t in sorted(table, key=lambda t: t["ms"])[:3]]
    cands = list(dict.fromkeys(top + [default]))
    runs = {c: [] for c in cands}
    for _ in range(3):
        for c in cands:
            runs[c].append(time_it(*c, reps))
    best, med = choose(runs, default)
    if log:
        log("tune %s b=%d: default %.3f ms, chosen tile=%d seen=2^%d persistent=%d %.3f ms (medians)" % (
            variant, beam, med[default], best[0], best[1], best[2], med[best]))
    choice = {"tile_hint": best[0], "seen_log2": best[1], "persistent": best[2]}
    if cache_path:
        cache[key] = choice
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return choice, table
