// rr_search.cu -- orchestration of one batched range search on the caller's
// stream: stage queries and radii, the beam phase (Alg. 1 + Alg. 5), the
// phase-2 queue of Alg. 6 (GreedySearch, Alg. 2) or Alg. 3 (doubling), and
// the CSR assembly.  Also the exhaustive search of Def. 2.1.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rr_common.cuh"

using namespace rr;

namespace {

size_t ru(size_t x) { return (x + 255) & ~size_t(255); }

struct Search {
    rr_index *ix;
    cudaStream_t st;
    bool dev;
    rr_params P;
    int64_t nq;
    SearchArgs a;
    int32_t *hc = nullptr;      // pinned host words
    int64_t *offsets = nullptr; // device offsets (result array or arena)
    uint8_t *flags = nullptr;   // device flags (result array or arena)
    rr_query_stats *stats_res = nullptr;  // device stats result array (device results)
    // phase-2 per-slot arrays (arena): results per slot, truncation, scatter cursor, item tail
    int32_t *slot_count = nullptr, *slot_trunc = nullptr, *slot_cursor = nullptr;
    unsigned long long *tail = nullptr;
    int32_t phase2_steps = 0;   // greedy levels or doubling rounds run
    // result arrays allocated for device results (freed on failure)
    std::vector<void *> owned;

    void *res_alloc(size_t bytes) {
        void *p = nullptr;
        if (inject_alloc_failure() || cudaMallocAsync(&p, std::max<size_t>(bytes, 8), st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        owned.push_back(p);
        return p;
    }
    rr_status fail(rr_status s) {
        for (void *p : owned) cudaFreeAsync(p, st);
        owned.clear();
        return s;
    }
    int32_t *pinned(size_t bytes) {
        if (ix->pinned.cap < bytes) {
            if (ix->pinned.p) cudaFreeHost(ix->pinned.p);
            ix->pinned.p = nullptr;
            ix->pinned.cap = 0;
            if (cudaHostAlloc((void **)&ix->pinned.p, std::max<size_t>(bytes, 4096), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            ix->pinned.cap = std::max<size_t>(bytes, 4096);
        }
        return (int32_t *)ix->pinned.p;
    }
};

// Stage queries (padded to the index's row stride), radius keys and the
// beam-phase buffers in the index arena.  keys_only: brute force (no beam).
rr_status stage(Search &S, const void *queries, const double *radii, double radius, bool brute) {
    rr_index *ix = S.ix;
    const int64_t nq = S.nq;
    const size_t row_bytes = (size_t)ix->d * elem_size(ix->dtype);
    const bool qdev = nq > 0 && is_device_ptr(queries);
    const bool direct = qdev && row_bytes == (size_t)ix->row_stride && ((uintptr_t)queries % 16) == 0;
    const int b = brute ? 0 : S.P.beam;
    const bool stats = !brute && S.P.collect_stats;
    const int64_t words = (ix->n + 31) / 32;
    size_t need = 0;
    need += direct ? 0 : ru((size_t)nq * ix->row_stride);
    need += ru((size_t)nq * 8);                                  // radius keys
    need += ru((size_t)nq * b * 8);                              // beam results
    need += 3 * ru((size_t)nq * 4);                              // counts, queue/cursor, spare
    need += 3 * ru((size_t)nq * 4) + ru(64);                     // phase-2 slot arrays + tail
    need += ru(256);                                             // counters
    need += ru((size_t)nq) + ru((size_t)(nq + 1) * 8);           // flags, offsets (host results)
    need += ru((size_t)nq * sizeof(rr_query_stats));             // stats
    if (stats) need += ru((size_t)nq * words * 4);               // exact distinct bitmaps
    need += 4096;
    rr_status s = ix->arena.reserve(need);
    if (s != RR_OK) return s;
    ix->arena.reset();
    Arena &A = ix->arena;
    const uint8_t *qd = (const uint8_t *)queries;
    if (!direct && nq > 0) {
        uint8_t *q = (uint8_t *)A.take((size_t)nq * ix->row_stride);
        if (row_bytes != (size_t)ix->row_stride) RR_CUDA(cudaMemsetAsync(q, 0, (size_t)nq * ix->row_stride, S.st));
        RR_CUDA(cudaMemcpy2DAsync(q, ix->row_stride, queries, row_bytes, row_bytes, nq, cudaMemcpyDefault, S.st));
        qd = q;
    }
    uint32_t *kd = (uint32_t *)A.take((size_t)nq * 8);
    if (nq > 0) {
        uint32_t *hk = (uint32_t *)S.pinned((size_t)nq * 8 + 256);
        if (!hk) { set_error("pinned host allocation failed"); return RR_ENOMEM; }
        RR_CUDA(cudaStreamSynchronize(S.st));  // the pinned words may still be read by a previous copy
        for (int64_t i = 0; i < nq; i++) {
            double r = radii ? radii[i] : radius;
            double esr = S.P.es_radius_mode == 1 ? S.P.es_radius : r;
            if (!radius_key(r, ix->dtype, &hk[i]) || !radius_key(esr, ix->dtype, &hk[nq + i])) {
                set_error("radius of query %lld is NaN", (long long)i);
                return RR_EINVAL;
            }
        }
        RR_CUDA(cudaMemcpyAsync(kd, hk, (size_t)nq * 8, cudaMemcpyHostToDevice, S.st));
        RR_CUDA(cudaStreamSynchronize(S.st));
    }
    SearchArgs &a = S.a;
    memset(&a, 0, sizeof a);
    a.vec = ix->vec;
    a.adj = ix->adj;
    a.n = ix->n;
    a.R = ix->R;
    a.row_stride = ix->row_stride;
    a.row_chunks = ix->row_stride / 16;
    int lpv = 1;
    while (lpv < a.row_chunks && lpv < 32) lpv <<= 1;
    a.lpv = lpv;
    a.metric = ix->metric;
    a.start = (uint32_t)ix->start;
    a.queries = qd;
    a.nq = nq;
    a.rkey = kd;
    a.eskey = kd + nq;
    a.beam = b;
    a.res_keys = b ? (uint64_t *)A.take((size_t)nq * b * 8) : nullptr;
    a.res_count = (int32_t *)A.take((size_t)nq * 4);
    a.p2_list = (int32_t *)A.take((size_t)nq * 4);
    int32_t *counters = (int32_t *)A.take(256);
    a.p2_count = counters;
    a.error = counters + 1;
    RR_CUDA(cudaMemsetAsync(counters, 0, 256, S.st));
    uint8_t *flags_a = (uint8_t *)A.take((size_t)std::max<int64_t>(nq, 1));
    int64_t *offs_a = (int64_t *)A.take((size_t)(nq + 1) * 8);
    rr_query_stats *stats_a = (rr_query_stats *)A.take((size_t)std::max<int64_t>(nq, 1) * sizeof(rr_query_stats));
    if (stats) {
        a.stats = stats_a;
        a.count_bits = (uint32_t *)A.take((size_t)nq * words * 4);
        a.words_per_q = words;
        RR_CUDA(cudaMemsetAsync(a.count_bits, 0, (size_t)nq * words * 4, S.st));
    }
    S.slot_count = (int32_t *)A.take((size_t)std::max<int64_t>(nq, 1) * 4);
    S.slot_trunc = (int32_t *)A.take((size_t)std::max<int64_t>(nq, 1) * 4);
    S.slot_cursor = (int32_t *)A.take((size_t)std::max<int64_t>(nq, 1) * 4);
    S.tail = (unsigned long long *)A.take(64);
    if (!a.res_count || !offs_a || !stats_a || (stats && !a.count_bits) || !S.tail) {
        set_error("internal: arena sizing");
        return RR_EINTERNAL;
    }
    if (S.dev) {
        S.offsets = (int64_t *)S.res_alloc((size_t)(nq + 1) * 8);
        S.flags = (uint8_t *)S.res_alloc((size_t)nq);
        if (stats) S.stats_res = (rr_query_stats *)S.res_alloc((size_t)nq * sizeof(rr_query_stats));
        if (!S.offsets || !S.flags || (stats && !S.stats_res)) {
            set_error("result allocation failed");
            return S.fail(RR_ENOMEM);
        }
    } else {
        S.offsets = offs_a;
        S.flags = flags_a;
    }
    a.flags = S.flags;
    if (brute && nq > 0) {
        RR_CUDA(cudaMemsetAsync(a.res_count, 0, (size_t)nq * 4, S.st));
        RR_CUDA(cudaMemsetAsync(a.p2_list, 0, (size_t)nq * 4, S.st));
        RR_CUDA(cudaMemsetAsync(S.flags, 0, (size_t)nq, S.st));
    }
    S.hc = S.pinned((size_t)nq * 8 + 256);
    if (!S.hc) { set_error("pinned host allocation failed"); return RR_ENOMEM; }
    return RR_OK;
}

// Scan the final per-query counts, read the total (and the device status), allocate the id/dist arrays.
rr_status scan_and_alloc(Search &S, int64_t *total, uint32_t **ids, void **dists, size_t extra_keys) {
    rr_index *ix = S.ix;
    rr_status s;
    if ((s = launch_scan(S.a.res_count, S.nq, S.offsets, S.st)) != RR_OK) return s;
    int64_t *ht = (int64_t *)S.hc;
    RR_CUDA(cudaMemcpyAsync(ht, S.offsets + S.nq, 8, cudaMemcpyDeviceToHost, S.st));
    RR_CUDA(cudaMemcpyAsync(S.hc + 2, S.a.error, 4, cudaMemcpyDeviceToHost, S.st));
    RR_CUDA(cudaStreamSynchronize(S.st));
    *total = ht[0];
    if (S.hc[2] != 0) {
        set_error("a device-side guard tripped (code %d)", S.hc[2]);
        return RR_EINTERNAL;
    }
    const size_t t = (size_t)std::max<int64_t>(*total, 1);
    if (S.dev) {
        *ids = (uint32_t *)S.res_alloc(t * 4);
        *dists = S.res_alloc(t * 4);
        if (!*ids || !*dists) { set_error("result allocation failed"); return RR_ENOMEM; }
        if ((s = grow(ix->outbuf, extra_keys ? ru(t * 8) : 256, 0, S.st)) != RR_OK) return s;
    } else {
        // staging: [sort keys: t x 8][ids: t x 4][dists: t x 4], each region 256-byte aligned
        const size_t off_ids = ru(t * 8), off_d = off_ids + ru(t * 4), end = off_d + ru(t * 4);
        if ((s = grow(ix->outbuf, end, 0, S.st)) != RR_OK) return s;
        *ids = (uint32_t *)((uint8_t *)ix->outbuf.p + off_ids);
        *dists = (uint8_t *)ix->outbuf.p + off_d;
    }
    return RR_OK;
}

rr_status deliver(Search &S, int64_t total, uint32_t *ids, void *dists, rr_result *out) {
    rr_index *ix = S.ix;
    const int64_t nq = S.nq;
    out->nq = nq;
    out->total = total;
    out->dist_dtype = ix->dtype == RR_F32 ? 1 : 0;
    out->on_device = S.dev ? 1 : 0;
    out->_stream = (void *)S.st;
    out->_device = ix->device;
    // the output kernels refuse any write outside the result arrays; check that none was refused
    RR_CUDA(cudaMemcpyAsync(S.hc + 2, S.a.error, 4, cudaMemcpyDeviceToHost, S.st));
    RR_CUDA(cudaStreamSynchronize(S.st));
    if (S.hc[2] != 0) {
        set_error("a device-side guard tripped in the output stage (code %d)", S.hc[2]);
        return RR_EINTERNAL;
    }
    if (S.dev) {
        if (S.stats_res)
            RR_CUDA(cudaMemcpyAsync(S.stats_res, S.a.stats, (size_t)nq * sizeof(rr_query_stats),
                                    cudaMemcpyDeviceToDevice, S.st));
        out->offsets = S.offsets;
        out->ids = ids;
        out->dists = dists;
        out->flags = S.flags;
        out->stats = S.stats_res;
        S.owned.clear();
        return RR_OK;
    }
    if (!host_result_arrays(out, nq, total, S.a.stats != nullptr)) {
        rr_result_free(out);
        set_error("result: host allocation failed");
        return RR_ENOMEM;
    }
    RR_CUDA(cudaMemcpyAsync(out->offsets, S.offsets, (size_t)(nq + 1) * 8, cudaMemcpyDeviceToHost, S.st));
    if (total > 0) {
        RR_CUDA(cudaMemcpyAsync(out->ids, ids, (size_t)total * 4, cudaMemcpyDeviceToHost, S.st));
        RR_CUDA(cudaMemcpyAsync(out->dists, dists, (size_t)total * 4, cudaMemcpyDeviceToHost, S.st));
    }
    if (nq > 0) RR_CUDA(cudaMemcpyAsync(out->flags, S.flags, (size_t)nq, cudaMemcpyDeviceToHost, S.st));
    if (S.a.stats && nq > 0)
        RR_CUDA(cudaMemcpyAsync(out->stats, S.a.stats, (size_t)nq * sizeof(rr_query_stats), cudaMemcpyDeviceToHost, S.st));
    RR_CUDA(cudaStreamSynchronize(S.st));
    return RR_OK;
}

struct GreedyOut {
    int64_t nitems = 0;
    int32_t *slot_cursor = nullptr;
};

// Alg. 2 for the np2 queued queries, level by level (see k_greedy.cu).
rr_status run_greedy(Search &S, int32_t np2, GreedyOut &go) {
    rr_index *ix = S.ix;
    const SearchArgs &a = S.a;
    const int b = a.beam;
    const int64_t words = (ix->n + 31) / 32;
    rr_status s;
    if ((s = grow(ix->phase2, ru((size_t)np2 * words * 4), 0, S.st)) != RR_OK) return s;
    GreedyArgs g;
    memset(&g, 0, sizeof g);
    g.s = a;
    g.ng = np2;
    g.qlist = a.p2_list;
    g.seen = (uint32_t *)ix->phase2.p;
    g.seen_words = words;
    g.slot_count = S.slot_count;
    g.slot_trunc = S.slot_trunc;
    go.slot_cursor = S.slot_cursor;
    g.tail = S.tail;
    RR_CUDA(cudaMemsetAsync(g.seen, 0, (size_t)np2 * words * 4, S.st));
    RR_CUDA(cudaMemsetAsync(go.slot_cursor, 0, (size_t)np2 * 4, S.st));
    const int64_t init = (int64_t)np2 * b;
    const int64_t cap_limit = std::max<int64_t>(S.P.max_results_total, init);
    int64_t want = std::min<int64_t>(cap_limit, std::max<int64_t>(init * 8, (int64_t)1 << 20));
    if ((s = grow(ix->item_key, (size_t)want * 8, 0, S.st)) != RR_OK) return s;
    if ((s = grow(ix->item_slot, (size_t)want * 4, 0, S.st)) != RR_OK) return s;
    auto refresh = [&]() {
        g.item_key = (uint64_t *)ix->item_key.p;
        g.item_slot = (int32_t *)ix->item_slot.p;
        g.cap = std::min<int64_t>(cap_limit, (int64_t)std::min(ix->item_key.bytes / 8, ix->item_slot.bytes / 4));
    };
    refresh();
    unsigned long long *ht = (unsigned long long *)(S.hc + 4);
    *ht = (unsigned long long)init;
    RR_CUDA(cudaMemcpyAsync(g.tail, ht, 8, cudaMemcpyHostToDevice, S.st));
    if ((s = launch_greedy_init(g, S.st, ix->dtype)) != RR_OK) return s;
    const bool two_pass = greedy_two_pass(ix->dtype) && a.row_chunks <= 32;
    g.ccount = S.tail + 1;  // the second word of the tail block
    int64_t begin = 0, end = init, levels = 0;
    while (begin < end) {
        const int64_t need = end + (end - begin) * (int64_t)ix->R;
        if (need > g.cap && g.cap < cap_limit) {
            int64_t ncap = std::min<int64_t>(cap_limit, need);
            if ((s = grow(ix->item_key, (size_t)ncap * 8, (size_t)end * 8, S.st)) != RR_OK) return s;
            if ((s = grow(ix->item_slot, (size_t)ncap * 4, (size_t)end * 4, S.st)) != RR_OK) return s;
            refresh();
        }
        // 8-bit indexes: expand + evaluate passes over a candidate list of at most 2^27 entries (16 bytes
        // each), so a long level runs in chunks of items
        int64_t chunk = end - begin;
        if (two_pass) {
            const int64_t want_c = std::max<int64_t>(ix->R, std::min<int64_t>((end - begin) * (int64_t)ix->R,
                                                                            (int64_t)1 << 27));
            if ((s = grow(ix->cand, (size_t)want_c * 16, 0, S.st)) != RR_OK) return s;
            g.cand = (uint64_t *)ix->cand.p;
            g.ccap = (int64_t)(ix->cand.bytes / 16);
            chunk = std::max<int64_t>(1, g.ccap / ix->R);
        }
        for (int64_t cb = begin; cb < end; cb += chunk) {
            if (two_pass) RR_CUDA(cudaMemsetAsync(g.ccount, 0, 8, S.st));
            g.begin = cb;
            g.end = std::min(end, cb + chunk);
            if ((s = launch_greedy_level(g, S.st, ix->dtype)) != RR_OK) return s;
        }
        RR_CUDA(cudaMemcpyAsync(ht, g.tail, 8, cudaMemcpyDeviceToHost, S.st));
        RR_CUDA(cudaStreamSynchronize(S.st));
        begin = end;
        end = (int64_t)std::min<unsigned long long>(*ht, (unsigned long long)g.cap);
        S.phase2_steps++;
        if (++levels > ix->n + 1) {
            set_error("greedy phase: level guard tripped");
            return RR_EINTERNAL;
        }
    }
    go.nitems = end;
    RR_CUDA(cudaMemsetAsync(g.slot_count, 0, (size_t)np2 * 4, S.st));
    if ((s = launch_count_items(g.item_slot, end, g.slot_count, S.st)) != RR_OK) return s;
    return launch_set_counts(S.a.res_count, S.flags, a.p2_list, g.slot_count, g.slot_trunc, np2, S.st);
}

// Alg. 3 for the np2 queued queries: host-driven rounds over the still active ones.
rr_status run_doubling(Search &S, int32_t np2, GreedyOut &go, bool warm) {
    rr_index *ix = S.ix;
    const SearchArgs &a = S.a;
    const int64_t words = (ix->n + 31) / 32;
    const int b_max = S.P.b_max;
    rr_status s;
    go.slot_cursor = S.slot_cursor;
    if (warm) {
        // warm restart: one bitmap per query of every id it has evaluated, kept across the rounds
        if ((s = grow(ix->dbl_seen, ru((size_t)np2 * words * 4), 0, S.st)) != RR_OK) return s;
        if ((s = launch_zero_words((uint32_t *)ix->dbl_seen.p, (int64_t)np2 * words, S.st)) != RR_OK) return s;
    }
    RR_CUDA(cudaMemsetAsync(S.slot_cursor, 0, (size_t)np2 * 4, S.st));
    RR_CUDA(cudaMemsetAsync(S.slot_trunc, 0, (size_t)np2 * 4, S.st));
    RR_CUDA(cudaMemsetAsync(S.tail, 0, 8, S.st));
    std::vector<int32_t> act((size_t)np2);
    for (int32_t i = 0; i < np2; i++) act[(size_t)i] = i;
    const int64_t cap_limit = S.P.max_results_total;
    int64_t cap = 0;
    unsigned long long tail_h = 0;
    int b = a.beam;
    bool first = true;
    int cur = 0;            // which dbl_s buffer holds S
    int64_t s_cap = 1;
    int32_t *s_cnt = nullptr;
    for (int round = 0; !act.empty(); round++) {
        S.phase2_steps++;
        const int32_t na = (int32_t)act.size();
        const int64_t v_cap = 4 * (int64_t)b + 1024;
        // warm restart: every key the round evaluates is kept (at most R per visit)
        const int64_t ev_cap = warm ? v_cap * ix->R : 0;
        const bool last = (int64_t)b * 2 > b_max;
        // round scratch in phase2: act | status | nv | beam A | beam B | V | seen (| ev | nev)
        size_t off_status = ru((size_t)na * 4), off_nv = off_status + ru((size_t)na * 4);
        size_t off_bA = off_nv + ru((size_t)na * 4);
        size_t off_bB = off_bA + ru((size_t)na * b * 8);
        size_t off_v = off_bB + ru((size_t)na * b * 8);
        size_t off_seen = off_v + ru((size_t)na * v_cap * 8);
        size_t off_ev = off_seen + (warm ? 0 : ru((size_t)na * words * 4));
        size_t off_nev = off_ev + ru((size_t)na * ev_cap * 8);
        size_t total = off_nev + ru((size_t)na * 4);
        if ((s = grow(ix->phase2, total, 0, S.st)) != RR_OK) return s;
        uint8_t *base = (uint8_t *)ix->phase2.p;
        int32_t *act_d = (int32_t *)base;
        int32_t *hs = S.pinned((size_t)na * 4 + 256);
        if (!hs) { set_error("pinned host allocation failed"); return RR_ENOMEM; }
        S.hc = hs;
        RR_CUDA(cudaStreamSynchronize(S.st));
        memcpy(hs, act.data(), (size_t)na * 4);
        RR_CUDA(cudaMemcpyAsync(act_d, hs, (size_t)na * 4, cudaMemcpyHostToDevice, S.st));
        if (!warm && (s = launch_zero_words((uint32_t *)(base + off_seen), (int64_t)na * words, S.st)) != RR_OK)
            return s;
        // room for every active query to finish with a full beam this round
        int64_t need = (int64_t)tail_h + (int64_t)na * b;
        if (need > cap && cap < cap_limit) {
            int64_t ncap = std::min<int64_t>(cap_limit, std::max<int64_t>(need, cap * 2));
            if ((s = grow(ix->item_key, (size_t)ncap * 8, (size_t)tail_h * 8, S.st)) != RR_OK) return s;
            if ((s = grow(ix->item_slot, (size_t)ncap * 4, (size_t)tail_h * 4, S.st)) != RR_OK) return s;
            cap = std::min<int64_t>(cap_limit, (int64_t)std::min(ix->item_key.bytes / 8, ix->item_slot.bytes / 4));
        }
        DoublingRound d;
        memset(&d, 0, sizeof d);
        d.s = a;
        d.s.beam = b;
        d.na = na;
        d.act = act_d;
        d.qlist = a.p2_list;
        d.first = first ? 1 : 0;
        d.last = last ? 1 : 0;
        d.s_old = first ? nullptr : (const uint64_t *)ix->dbl_s[cur].p;
        d.s_cnt = s_cnt;
        d.s_cap = s_cap;
        d.bA = (uint64_t *)(base + off_bA);
        d.bB = (uint64_t *)(base + off_bB);
        d.v = (uint64_t *)(base + off_v);
        d.v_cap = v_cap;
        d.nv = (int32_t *)(base + off_nv);
        d.seen = warm ? (uint32_t *)ix->dbl_seen.p : (uint32_t *)(base + off_seen);
        d.seen_words = words;
        d.warm = warm ? 1 : 0;
        d.ev = warm ? (uint64_t *)(base + off_ev) : nullptr;
        d.ev_cap = ev_cap;
        d.nev = warm ? (int32_t *)(base + off_nev) : nullptr;
        d.status = (int32_t *)(base + off_status);
        d.item_key = (uint64_t *)ix->item_key.p;
        d.item_slot = (int32_t *)ix->item_slot.p;
        d.tail = S.tail;
        d.cap = cap;
        d.slot_count = S.slot_count;
        d.slot_trunc = S.slot_trunc;
        if ((s = launch_doubling_round(d, S.st, ix->dtype)) != RR_OK) return s;
        RR_CUDA(cudaMemcpyAsync(hs, d.status, (size_t)na * 4, cudaMemcpyDeviceToHost, S.st));
        RR_CUDA(cudaMemcpyAsync(hs + na + 16, S.tail, 8, cudaMemcpyDeviceToHost, S.st));
        RR_CUDA(cudaStreamSynchronize(S.st));
        memcpy(&tail_h, hs + na + 16, 8);
        tail_h = std::min<unsigned long long>(tail_h, (unsigned long long)cap);
        std::vector<int32_t> cont, nact;
        for (int32_t i = 0; i < na; i++)
            if (hs[i]) { cont.push_back(i); nact.push_back(act[(size_t)i]); }
        if (cont.empty()) break;
        // S <- S u V for the continuing queries, into the other buffer
        const int32_t nc = (int32_t)cont.size();
        const int64_t s_cap_new = std::min<int64_t>(b_max, (first ? 0 : s_cap) + ev_cap + v_cap);
        const int nxt = cur ^ 1;
        size_t sbytes = ru((size_t)nc * s_cap_new * 8) + ru((size_t)nc * 4) + ru((size_t)nc * 4);
        if ((s = grow(ix->dbl_s[nxt], sbytes, 0, S.st)) != RR_OK) return s;
        const int64_t tmp_row = (first ? 0 : s_cap) + ev_cap + v_cap;
        if ((s = grow(ix->dbl_tmp, (size_t)nc * tmp_row * 8 + 256, 0, S.st)) != RR_OK) return s;
        uint8_t *sb = (uint8_t *)ix->dbl_s[nxt].p;
        int32_t *cnt_new = (int32_t *)(sb + ru((size_t)nc * s_cap_new * 8));
        int32_t *cont_d = cnt_new + ru((size_t)nc * 4) / 4;
        memcpy(hs, cont.data(), (size_t)nc * 4);
        RR_CUDA(cudaMemcpyAsync(cont_d, hs, (size_t)nc * 4, cudaMemcpyHostToDevice, S.st));
        DoublingSUpdate u;
        memset(&u, 0, sizeof u);
        u.nc = nc;
        u.cont = cont_d;
        u.s_old = first ? nullptr : (const uint64_t *)ix->dbl_s[cur].p;
        u.s_cnt_old = s_cnt;
        u.s_cap_old = first ? 0 : s_cap;
        u.v = d.v;
        u.nv = d.nv;
        u.v_cap = v_cap;
        u.s_new = (uint64_t *)sb;
        u.s_cnt_new = cnt_new;
        u.s_cap_new = s_cap_new;
        u.tmp = (uint64_t *)ix->dbl_tmp.p;
        u.first = first ? 1 : 0;
        u.warm = warm ? 1 : 0;
        u.ev = d.ev;
        u.nev = d.nev;
        u.ev_cap = ev_cap;
        if ((s = launch_doubling_supdate(u, S.st)) != RR_OK) return s;
        RR_CUDA(cudaStreamSynchronize(S.st));  // hs is reused by the next round
        cur = nxt;
        s_cap = s_cap_new;
        s_cnt = cnt_new;
        act.swap(nact);
        b *= 2;
        first = false;
    }
    go.nitems = (int64_t)tail_h;
    return launch_set_counts(S.a.res_count, S.flags, a.p2_list, S.slot_count, S.slot_trunc, np2, S.st);
}

}  // namespace

extern "C" rr_status rr_range_search(rr_index *ix, const void *queries, int64_t nq, const double *radii, double radius,
                                     int32_t variant, const rr_params *params, void *stream, int32_t result_on_device,
                                     rr_result *out) {
    if (!out) { set_error("rr_range_search: out is NULL"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    if (!ix) { set_error("rr_range_search: index is NULL"); return RR_EINVAL; }
    if (nq < 0 || (nq > 0 && !queries)) { set_error("rr_range_search: bad queries"); return RR_EINVAL; }
    if (nq >= ((int64_t)1 << 31)) { set_error("rr_range_search: nq too large"); return RR_EINVAL; }
    if (variant < RR_BEAM || variant > RR_DOUBLING_WARM_ES) { set_error("rr_range_search: bad variant %d", variant); return RR_EINVAL; }
    Search S;
    S.ix = ix;
    S.st = (cudaStream_t)stream;
    S.dev = result_on_device != 0;
    S.nq = nq;
    if (params) S.P = *params;
    else rr_params_init(&S.P);
    rr_params &P = S.P;
    if (P.beam < 1 || P.beam > 512) { set_error("rr_range_search: beam=%d out of [1, 512]", P.beam); return RR_EINVAL; }
    if (P.max_results_total <= 0) P.max_results_total = (int64_t)1 << 28;
    if (P.es_visit_limit < 0) { set_error("rr_range_search: es_visit_limit < 0"); return RR_EINVAL; }
    const bool warm = variant == RR_DOUBLING_WARM || variant == RR_DOUBLING_WARM_ES;
    const bool doubling = variant == RR_DOUBLING || variant == RR_DOUBLING_ES || warm;
    const bool greedy = variant == RR_GREEDY || variant == RR_GREEDY_ES;
    const bool use_es = variant == RR_BEAM_ES || variant == RR_DOUBLING_ES || variant == RR_GREEDY_ES ||
                        variant == RR_DOUBLING_WARM_ES;
    if (P.es_metric < RR_ES_VISITED || P.es_metric > RR_ES_TOP10_RATIO) {
        set_error("rr_range_search: unknown early-stopping metric %d", P.es_metric);
        return RR_EINVAL;
    }
    if (use_es && doubling && P.es_metric != RR_ES_VISITED) {
        set_error("rr_range_search: the doubling variants stop early on d_visited only");
        return RR_EINVAL;
    }
    if (use_es && P.es_metric == RR_ES_TOP10_RATIO && (P.es_radius_mode != 1 || ix->metric != RR_L2)) {
        set_error("rr_range_search: the d_top10 / d_start metric takes its ratio from es_radius "
                  "(es_radius_mode = 1) and needs squared L2");
        return RR_EINVAL;
    }
    if (doubling && P.b_max < P.beam) { set_error("rr_range_search: b_max < beam"); return RR_EINVAL; }
    if (P.expand < 0 || P.expand > 4) { set_error("rr_range_search: expand=%d out of [0, 4]", P.expand); return RR_EINVAL; }
    if (P.expand > 1 && doubling) {
        set_error("rr_range_search: multi-parent expansion (expand > 1) is for the beam and greedy variants");
        return RR_EINVAL;
    }
    DeviceGuard dg(ix->device);
    rr_status s = stage(S, queries, radii, radius, false);
    if (s != RR_OK) return S.fail(s);
    SearchArgs &a = S.a;
    a.use_es = use_es ? 1 : 0;
    a.es_vl = P.es_visit_limit;
    a.es_metric = P.es_metric;
    a.es_ratio = P.es_radius;
    a.hash_lg = P.seen_log2;
    a.persistent = P.persistent ? 1 : 0;
    a.next_q = a.p2_count + 2;  // zeroed with the other counters in stage()
    a.iter_limit = beam_iteration_limit(ix->n);
    a.expand = std::max(1, P.expand);
    a.d = ix->d;
    a.prec = RR_PREC_EXACT;
    if (P.precision != RR_PREC_EXACT) {
        // precision form: traverse a BF16 / FP8 copy, decide membership in exact fp32
        if ((s = ensure_lowp(ix, P.precision, S.st)) != RR_OK) return S.fail(s);
        a.prec = P.precision;
        a.lp_vec = P.precision == RR_PREC_BF16 ? ix->lp_bf16 : ix->lp_fp8;
        a.lp_stride = P.precision == RR_PREC_BF16 ? ix->lp_bf16_stride : ix->lp_fp8_stride;
        a.lp_chunks = a.lp_stride / 16;
        if (a.lp_chunks > 32) {
            set_error("rr_range_search: %s traversal supports d <= %d", P.precision == RR_PREC_BF16 ? "BF16" : "FP8",
                      P.precision == RR_PREC_BF16 ? 256 : 512);
            return S.fail(RR_EINVAL);
        }
        int lpv = 1;
        while (lpv < a.lp_chunks) lpv <<= 1;
        a.lp_lpv = lpv;
        a.lp_info = ix->lp_fp8_info;
        slack_coefficients(ix, P.precision, &a.slackA, &a.slackB, &a.slackC);
        a.rel_eps = P.recheck_eps > 0.f ? P.recheck_eps : 0.f;
    }
    a.phase2 = greedy ? 1 : (doubling ? 2 : 0);
    const bool prof = P.profile != 0;
    const int64_t l0 = launches_so_far();
    ix->prof.valid = 0;
    if (prof) {
        for (int k = 0; k < 4; k++)
            if (!ix->ev[k]) RR_CUDA(cudaEventCreate(&ix->ev[k]));
        RR_CUDA(cudaEventRecord(ix->ev[0], S.st));
    }
    const int wpc = P.tile_hint > 0 ? std::min(8, P.tile_hint) : 4;
    if ((s = launch_beam(a, wpc, S.st, ix->dtype)) != RR_OK) return S.fail(s);
    if (prof) RR_CUDA(cudaEventRecord(ix->ev[1], S.st));

    int32_t np2 = 0;
    if (a.phase2 && nq > 0) {
        RR_CUDA(cudaMemcpyAsync(S.hc, a.p2_count, 4, cudaMemcpyDeviceToHost, S.st));
        RR_CUDA(cudaStreamSynchronize(S.st));
        np2 = S.hc[0];
    }
    GreedyOut go;
    if (greedy && np2 > 0) {
        if ((s = run_greedy(S, np2, go)) != RR_OK) return S.fail(s);
    }
    if (doubling && np2 > 0) {
        if ((s = run_doubling(S, np2, go, warm)) != RR_OK) return S.fail(s);
    }
    if (prof) RR_CUDA(cudaEventRecord(ix->ev[2], S.st));
    int64_t total = 0;
    uint32_t *ids = nullptr;
    void *dists = nullptr;
    const bool items = np2 > 0 && (greedy || doubling);
    if ((s = scan_and_alloc(S, &total, &ids, &dists, items ? 1 : 0)) != RR_OK) return S.fail(s);
    OutArgs o{nq, S.offsets, ix->dtype == RR_F32 ? 1 : 0, ids, dists, S.flags, total, S.a.error, ix->ext};
    if ((s = launch_copy_slots(o, a.res_keys, a.beam, a.res_count, nullptr, (int32_t)nq, S.st)) != RR_OK) return S.fail(s);
    if (items) {
        uint64_t *tmp = (uint64_t *)ix->outbuf.p;
        if ((s = launch_scatter_items(o, (const uint64_t *)ix->item_key.p, (const int32_t *)ix->item_slot.p, go.nitems,
                                      a.p2_list, go.slot_cursor, tmp, S.st)) != RR_OK)
            return S.fail(s);
        if ((s = launch_sort_segments(o, tmp, a.p2_list, np2, 0, S.st)) != RR_OK) return S.fail(s);
    }
    if (prof) {
        RR_CUDA(cudaEventRecord(ix->ev[3], S.st));
        memset(&ix->prof, 0, sizeof ix->prof);
        ix->prof.launches = (int32_t)(launches_so_far() - l0);
        ix->prof.phase2_steps = S.phase2_steps;
        ix->prof.phase2_queries = np2;
        ix->prof.valid = 1;
    }
    if ((s = deliver(S, total, ids, dists, out)) != RR_OK) return S.fail(s);
    for (int64_t i = 0; !S.dev && i < nq; i++) {
        if (out->flags[i] & RR_FLAG_TRUNCATED) return RR_EOVERFLOW;
    }
    return RR_OK;
}

extern "C" rr_status rr_brute_force(rr_index *ix, const void *queries, int64_t nq, const double *radii, double radius,
                                    void *stream, int32_t result_on_device, rr_result *out) {
    if (!out) { set_error("rr_brute_force: out is NULL"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    if (!ix) { set_error("rr_brute_force: index is NULL"); return RR_EINVAL; }
    if (nq < 0 || (nq > 0 && !queries)) { set_error("rr_brute_force: bad queries"); return RR_EINVAL; }
    if (nq >= ((int64_t)1 << 21)) { set_error("rr_brute_force: nq above 2^21, split the batch"); return RR_EINVAL; }
    Search S;
    S.ix = ix;
    S.st = (cudaStream_t)stream;
    S.dev = result_on_device != 0;
    S.nq = nq;
    rr_params_init(&S.P);
    DeviceGuard dg(ix->device);
    rr_status s = stage(S, queries, radii, radius, true);
    if (s != RR_OK) return S.fail(s);
    SearchArgs &a = S.a;
    a.ext = ix->ext;  // keys carry the caller's ids, so the sort below is by (distance, id)
    int32_t *counts = a.res_count, *cursor = a.p2_list;
    if ((s = launch_brute(a, counts, nullptr, nullptr, nullptr, 0, S.st, ix->dtype)) != RR_OK) return S.fail(s);
    int64_t total = 0;
    uint32_t *ids = nullptr;
    void *dists = nullptr;
    if ((s = scan_and_alloc(S, &total, &ids, &dists, 1)) != RR_OK) return S.fail(s);
    uint64_t *tmp = (uint64_t *)ix->outbuf.p;
    if ((s = launch_brute(a, counts, S.offsets, cursor, tmp, 1, S.st, ix->dtype)) != RR_OK) return S.fail(s);
    OutArgs o{nq, S.offsets, ix->dtype == RR_F32 ? 1 : 0, ids, dists, S.flags, total, S.a.error, nullptr};
    // every query is a segment to sort: list = identity
    int32_t *ident = (int32_t *)ix->arena.take((size_t)std::max<int64_t>(nq, 1) * 4);
    if (!ident) { set_error("internal: arena sizing"); return S.fail(RR_EINTERNAL); }
    std::vector<int32_t> h((size_t)nq);
    for (int64_t i = 0; i < nq; i++) h[(size_t)i] = (int32_t)i;
    if (nq > 0) {
        RR_CUDA(cudaMemcpyAsync(ident, h.data(), (size_t)nq * 4, cudaMemcpyHostToDevice, S.st));
        if ((s = launch_sort_segments(o, tmp, ident, (int32_t)nq, 0, S.st)) != RR_OK) return S.fail(s);
    }
    s = deliver(S, total, ids, dists, out);
    RR_CUDA(cudaStreamSynchronize(S.st));  // h must outlive the copy
    if (s != RR_OK) return S.fail(s);
    return RR_OK;
}

extern "C" rr_status rr_last_profile(rr_index *ix, rr_profile *out) {
    if (!ix || !out) { set_error("rr_last_profile: NULL argument"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    if (!ix->prof.valid) return RR_OK;
    DeviceGuard dg(ix->device);
    RR_CUDA(cudaEventSynchronize(ix->ev[3]));
    *out = ix->prof;
    RR_CUDA(cudaEventElapsedTime(&out->beam_ms, ix->ev[0], ix->ev[1]));
    RR_CUDA(cudaEventElapsedTime(&out->phase2_ms, ix->ev[1], ix->ev[2]));
    RR_CUDA(cudaEventElapsedTime(&out->output_ms, ix->ev[2], ix->ev[3]));
    RR_CUDA(cudaEventElapsedTime(&out->total_ms, ix->ev[0], ix->ev[3]));
    return RR_OK;
}
