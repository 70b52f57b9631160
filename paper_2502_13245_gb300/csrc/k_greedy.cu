// k_greedy.cu -- Alg. 2 GreedySearch for the queries whose beam phase filled
// the beam with in-range points (Alg. 6: |N| = b).
//
// Alg. 2 returns S plus every point reachable from S through out-edges whose
// endpoints lie within r; the argmin order only fixes the visit order, not the
// set.  So it runs here as a level-synchronous BFS over all greedy queries at
// once: an item is one (query slot, point) pair to visit; a level kernel
// expands every item of the current level with one warp each and appends the
// newly found in-range points to a global item list.  Each query slot owns an
// exact bitmap of n bits ("seen": ids already in F or already evaluated), so
// every point is evaluated at most once per query and enters F at most once.
// The items of a slot are exactly its result set V.
//
// 8-bit indexes run each level as two flat passes instead of one warp per
// item, so that the dependent chain of an item (its adjacency row, the seen
// bits of its neighbours, their vectors) is spread over many independent
// threads: the expand pass gives every (item, neighbour) pair a thread that
// tests-and-sets the neighbour's seen bit and appends the first-seen ones to
// a candidate list; the evaluate pass gives each candidate a lane group that
// gathers its vector and the query's, and appends the in-range ones as items
// of the next level.  The set of items is the same either way (the bitmap
// admits each point once per query, whichever pair claims it first).  Both
// passes append with one list reservation per warp iteration, and the
// per-query result counts are taken from the finished item list by a
// run-length pass, so no pass does an atomic per appended entry.
#include <algorithm>

#include "rr_common.cuh"

namespace rr {

namespace {

template <bool COUNT>
__global__ void greedy_init_kernel(GreedyArgs g) {
    const int b = g.s.beam;
    const int64_t total = (int64_t)g.ng * b;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t slot = (int32_t)(t / b);
        int32_t i = (int32_t)(t % b);
        int32_t qi = g.qlist[slot];
        uint64_t k = g.s.res_keys[(size_t)qi * b + i];
        g.item_key[t] = k;
        g.item_slot[t] = slot;
        mark_bit(g.seen + (size_t)slot * g.seen_words, key_id(k));
        if (i == 0) g.slot_trunc[slot] = 0;
    }
}

template <int DT, int CPL, bool COUNT>
__global__ void __launch_bounds__(256) greedy_level_kernel(GreedyArgs g) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    constexpr int UN = CPL == 1 ? 8 : (CPL == 2 ? 4 : 2);
    const SearchArgs &a = g.s;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int wpc = blockDim.x >> 5;
    const int R = a.R;
    uint64_t *ckey = reinterpret_cast<uint64_t *>(smem_raw) + (size_t)warp * R;
    uint32_t *cid = reinterpret_cast<uint32_t *>(reinterpret_cast<uint64_t *>(smem_raw) + (size_t)wpc * R) +
                    (size_t)warp * R;
    const int64_t nw = (int64_t)gridDim.x * wpc;
    for (int64_t it = g.begin + (int64_t)blockIdx.x * wpc + warp; it < g.end; it += nw) {
        const int32_t slot = g.item_slot[it];
        const uint32_t p = key_id(g.item_key[it]);
        const int32_t qi = g.qlist[slot];
        uint4 q[CPL];
        load_query<CPL>(a, a.queries + (size_t)qi * a.row_stride, q);
        const uint32_t rk = a.rkey[qi];
        uint32_t *seen = g.seen + (size_t)slot * g.seen_words;
        // f in N_out(p*) \ V, each evaluated once per query (exact bitmap)
        const uint32_t *row = a.adj + (size_t)p * R;
        int nc = 0;
        for (int e0 = 0; e0 < R; e0 += 32) {
            int e = e0 + lane;
            uint32_t j = e < R ? __ldg(row + e) : kSent;
            bool v = j < (uint32_t)a.n && mark_bit(seen, j);
            unsigned m = __ballot_sync(0xffffffffu, v);
            if (v) cid[nc + __popc(m & lanemask_lt())] = j;
            nc += __popc(m);
        }
        __syncwarp();
        if (nc > 0) {
            int dd = 0;
            if (COUNT) {
                uint32_t *cb = a.count_bits + (size_t)qi * a.words_per_q;
                for (int c = lane; c < nc; c += 32) dd += mark_bit(cb, cid[c]);
            }
            const int ne = nc;
            eval_candidates<DT, CPL, UN>(a, q, cid, nc, ckey);
            __syncwarp();
            // if d(f, q) <= r: F <- F u {f}
            for (int c0 = 0; c0 < ne; c0 += 32) {
                int c = c0 + lane;
                uint64_t k = c < ne ? ckey[c] : kEmpty;
                bool in = c < ne && key_dk(k) <= rk;
                unsigned m = __ballot_sync(0xffffffffu, in);
                int cnt = __popc(m);
                if (cnt == 0) continue;
                unsigned long long basepos = 0;
                if (lane == 0) basepos = atomicAdd(g.tail, (unsigned long long)cnt);
                basepos = __shfl_sync(0xffffffffu, basepos, 0);
                if (in) {
                    unsigned long long pos = basepos + __popc(m & lanemask_lt());
                    if (pos < (unsigned long long)g.cap) {
                        g.item_key[pos] = k;
                        g.item_slot[pos] = slot;
                    } else {
                        g.slot_trunc[slot] = 1;
                    }
                }
            }
            if (COUNT) {
                for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
            }
            if (lane == 0) {
                if (a.stats) {
                    atomicAdd(&a.stats[qi].evals, nc);
                    if (COUNT) atomicAdd(&a.stats[qi].distinct, dd);
                }
            }
        }
        if (lane == 0 && a.stats) atomicAdd(&a.stats[qi].visits_phase2, 1);
        __syncwarp();
    }
}

template <int DT, int CPL>
rr_status level_t(const GreedyArgs &g, cudaStream_t st) {
    const int wpc = 8;
    size_t smem = (size_t)wpc * g.s.R * 12;
    int64_t items = g.end - g.begin;
    int64_t blocks = (items + wpc - 1) / wpc;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (g.s.count_bits) {
        auto k = greedy_level_kernel<DT, CPL, true>;
        k<<<(unsigned)blocks, 32 * wpc, smem, st>>>(g);
    } else {
        auto k = greedy_level_kernel<DT, CPL, false>;
        k<<<(unsigned)blocks, 32 * wpc, smem, st>>>(g);
    }
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

// Expand pass: thread per (item, neighbour) of items [begin, end); first-seen neighbours become
// candidates {id, slot, query} (16 bytes).  A warp takes 32 x EU consecutive pairs per iteration and each lane
// issues the loads of its EU pairs together (item, then row entry, then bitmap word), so their
// latencies overlap.  Whole warps run the loop (ballot-aggregated appends).
template <bool COUNT>
__global__ void __launch_bounds__(256) greedy_expand_kernel(GreedyArgs g) {
    constexpr int EU = 4;
    const SearchArgs &a = g.s;
    const int lane = lane_id();
    const uint32_t R = (uint32_t)a.R;
    // pair index in 32 bits: the host splits a level into chunks of at most 2^27 candidates (pairs)
    const uint32_t total = (uint32_t)((g.end - g.begin) * (int64_t)R);
    const uint32_t warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = warp_g * 32 * EU; base < total; base += nwarps * 32 * EU) {
        int32_t slot[EU], qi[EU];
        uint32_t p[EU], j[EU], w[EU], k[EU];
        uint32_t *wp[EU];
#pragma unroll
        for (int u = 0; u < EU; u++) {
            const uint32_t x = base + u * 32 + lane;
            slot[u] = -1;
            k[u] = 0;
            if (x < total) {
                const uint32_t io = x / R;
                k[u] = x - io * R;
                const int64_t it = g.begin + io;
                slot[u] = g.item_slot[it];
                p[u] = key_id(g.item_key[it]);
            }
        }
#pragma unroll
        for (int u = 0; u < EU; u++) {
            j[u] = slot[u] >= 0 ? __ldg(a.adj + (size_t)p[u] * R + k[u]) : kSent;
            qi[u] = slot[u] >= 0 ? g.qlist[slot[u]] : 0;
            if (COUNT && slot[u] >= 0 && k[u] == 0 && a.stats) atomicAdd(&a.stats[qi[u]].visits_phase2, 1);
        }
#pragma unroll
        for (int u = 0; u < EU; u++) {
            wp[u] = nullptr;
            w[u] = 0xFFFFFFFFu;
            if (j[u] < (uint32_t)a.n) {
                wp[u] = g.seen + (size_t)slot[u] * g.seen_words + (j[u] >> 5);
                w[u] = *wp[u];  // bits only go from 0 to 1 during the phase: a set bit read here is final
            }
        }
        unsigned m[EU];
        int tot = 0;
#pragma unroll
        for (int u = 0; u < EU; u++) {
            const uint32_t bit = 1u << (j[u] & 31);
            bool fresh = false;
            if (wp[u] && !(w[u] & bit)) fresh = !(atomicOr(wp[u], bit) & bit);
            m[u] = __ballot_sync(0xffffffffu, fresh);
            tot += __popc(m[u]);
        }
        if (!tot) continue;
        // one reservation for the warp's first-seen neighbours of all EU rounds
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(g.ccount, (unsigned long long)tot);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
#pragma unroll
        for (int u = 0; u < EU; u++) {
            if ((m[u] >> lane) & 1u) {
                const unsigned long long pos = b0 + __popc(m[u] & lanemask_lt());
                if (pos < (unsigned long long)g.ccap)
                    reinterpret_cast<uint4 *>(g.cand)[pos] = make_uint4(j[u], (uint32_t)slot[u], (uint32_t)qi[u], 0u);
                else atomicExch(a.error, 7);  // the host sizes the list for the chunk: cannot happen
            }
            b0 += __popc(m[u]);
        }
    }
}

// Expand pass for R a multiple of 32 (RR = R / 32 row words per lane): a warp takes IW consecutive items
// per iteration and lane l the row entries l + 32 t of each, so no pair index is divided by R.  The
// items of the warp's next iteration are loaded before this iteration's seen words are read, so the
// item -> row -> seen-word chain of one iteration overlaps the item loads of the next.
template <bool COUNT, int RR>
__global__ void __launch_bounds__(256, 4) greedy_expand_rows_kernel(GreedyArgs g) {
    constexpr int IW = RR <= 2 ? 4 : 2;  // items per warp iteration: 4 to 8 row entries per lane
    constexpr int NP = IW * RR;          // pairs per lane and iteration
    const SearchArgs &a = g.s;
    const int lane = lane_id();
    const int R = 32 * RR;
    const int64_t nitems = g.end - g.begin;
    const int64_t warp_g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t step = (((int64_t)gridDim.x * blockDim.x) >> 5) * IW;
    int32_t slot[IW];
    uint32_t p[IW];
#pragma unroll
    for (int i = 0; i < IW; i++) {
        const int64_t it = warp_g * IW + i;
        slot[i] = it < nitems ? g.item_slot[g.begin + it] : -1;
        p[i] = it < nitems ? key_id(g.item_key[g.begin + it]) : 0u;
    }
    for (int64_t i0 = warp_g * IW; i0 < nitems; i0 += step) {
        uint32_t j[NP];
        int32_t qi[IW];
#pragma unroll
        for (int i = 0; i < IW; i++) {
            qi[i] = slot[i] >= 0 ? g.qlist[slot[i]] : 0;
#pragma unroll
            for (int t = 0; t < RR; t++)
                j[i * RR + t] = slot[i] >= 0 ? __ldg(a.adj + (size_t)p[i] * R + 32 * t + lane) : kSent;
            if (COUNT && slot[i] >= 0 && lane == 0 && a.stats) atomicAdd(&a.stats[qi[i]].visits_phase2, 1);
        }
        // the next iteration's items
        int32_t nslot[IW];
        uint32_t np[IW];
#pragma unroll
        for (int i = 0; i < IW; i++) {
            const int64_t it = i0 + step + i;
            nslot[i] = it < nitems ? g.item_slot[g.begin + it] : -1;
            np[i] = it < nitems ? key_id(g.item_key[g.begin + it]) : 0u;
        }
        uint32_t w[NP];
        uint32_t *wp[NP];
#pragma unroll
        for (int e = 0; e < NP; e++) {
            const int i = e / RR;  // compile-time
            wp[e] = nullptr;
            w[e] = 0xFFFFFFFFu;
            if (j[e] < (uint32_t)a.n) {
                wp[e] = g.seen + (size_t)slot[i] * g.seen_words + (j[e] >> 5);
                w[e] = *wp[e];  // bits only go from 0 to 1 during the phase: a set bit read here is final
            }
        }
        unsigned m[NP];
        int tot = 0;
#pragma unroll
        for (int e = 0; e < NP; e++) {
            const uint32_t bit = 1u << (j[e] & 31);
            bool fresh = false;
            if (wp[e] && !(w[e] & bit)) fresh = !(atomicOr(wp[e], bit) & bit);
            m[e] = __ballot_sync(0xffffffffu, fresh);
            tot += __popc(m[e]);
        }
        if (tot) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(g.ccount, (unsigned long long)tot);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
#pragma unroll
            for (int e = 0; e < NP; e++) {
                const int i = e / RR;
                if ((m[e] >> lane) & 1u) {
                    const unsigned long long pos = b0 + __popc(m[e] & lanemask_lt());
                    if (pos < (unsigned long long)g.ccap)
                        reinterpret_cast<uint4 *>(g.cand)[pos] =
                            make_uint4(j[e], (uint32_t)slot[i], (uint32_t)qi[i], 0u);
                    else atomicExch(a.error, 7);  // the host sizes the list for the chunk: cannot happen
                }
                b0 += __popc(m[e]);
            }
        }
#pragma unroll
        for (int i = 0; i < IW; i++) {
            slot[i] = nslot[i];
            p[i] = np[i];
        }
    }
}

template <bool COUNT>
void launch_expand(const GreedyArgs &g, int64_t pairs, cudaStream_t st) {
    const int R = g.s.R;
    if (R % 32 == 0 && R <= 128) {
        // a grid of resident CTAs that loops, so the next-iteration loads have an iteration to hide behind
        const int64_t per_warp = R <= 64 ? 4 : 2;
        const int64_t items = g.end - g.begin;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((items + 8 * per_warp - 1) / (8 * per_warp),
                                                                      152 * 4));
        switch (R / 32) {
            case 1: greedy_expand_rows_kernel<COUNT, 1><<<(unsigned)blocks, 256, 0, st>>>(g); return;
            case 2: greedy_expand_rows_kernel<COUNT, 2><<<(unsigned)blocks, 256, 0, st>>>(g); return;
            case 3: greedy_expand_rows_kernel<COUNT, 3><<<(unsigned)blocks, 256, 0, st>>>(g); return;
            default: greedy_expand_rows_kernel<COUNT, 4><<<(unsigned)blocks, 256, 0, st>>>(g); return;
        }
    }
    int64_t blocks = (pairs + 1023) / 1024;  // 4 pairs per thread and iteration
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 16));
    greedy_expand_kernel<COUNT><<<(unsigned)blocks, 256, 0, st>>>(g);
}

// Evaluate pass: each lane group of lpv lanes takes UN candidates at a time (their vectors gathered
// before any is reduced); in-range ones are appended to the item list.  8-bit sums are exact integers,
// so the UN partial sums of a group are combined by a reduce-scatter (each exchange with the partner
// lane halves the values a lane holds) and each writer lane ends with whole candidates, decided and
// appended by one ballot and one list reservation per warp iteration.
template <int DT, bool COUNT>
__global__ void __launch_bounds__(256, 3) greedy_eval_kernel(GreedyArgs g) {
    constexpr int UN = 8;
    using T = typename Acc<DT>::T;
    static_assert(std::is_integral<T>::value, "the two-pass levels run on 8-bit indexes");
    const SearchArgs &a = g.s;
    const int lane = lane_id();
    const int lpv = a.lpv, sub = lane & (lpv - 1), grp = lane >> (__ffs(lpv) - 1), ngrp = 32 >> (__ffs(lpv) - 1);
    const int64_t nc = (int64_t)min(*(volatile unsigned long long *)g.ccount, (unsigned long long)g.ccap);
    const int64_t warp_g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t per = (int64_t)ngrp * UN;
    const uint4 *cand = reinterpret_cast<const uint4 *>(g.cand);
    // the lane's chunk of the query of its last candidate: consecutive candidates mostly share a query
    // (the expand pass writes an item's first-seen neighbours together), so it is reloaded on change only
    int32_t qcur = -1;
    uint4 qv = make_uint4(0, 0, 0, 0);
    const int cnt = lpv >= UN ? 1 : UN / lpv;  // candidates a writer lane ends with
    const bool writer = lpv <= UN || (sub & (lpv / UN - 1)) == 0;
    for (int64_t c0 = warp_g * per; c0 < nc; c0 += nwarps * per) {
        uint4 v[UN];
        int32_t qi[UN];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int64_t c = c0 + grp + (int64_t)ngrp * u;
            const bool ok = c < nc;
            const uint4 e = ok ? cand[c] : make_uint4(0u, 0u, 0u, 0u);
            qi[u] = ok ? (int32_t)e.z : -1;
            v[u] = ok && sub < a.row_chunks ? ldg16(a.vec + (size_t)e.x * a.row_stride + (size_t)sub * 16)
                                            : make_uint4(0, 0, 0, 0);
        }
        T s[UN];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            if (qi[u] >= 0 && qi[u] != qcur) {
                qcur = qi[u];
                qv = sub < a.row_chunks ? ldg16(a.queries + (size_t)qcur * a.row_stride + (size_t)sub * 16)
                                        : make_uint4(0, 0, 0, 0);
            }
            s[u] = 0;
            if (a.metric == MET_L2) Acc<DT>::l2(s[u], qv, v[u]);
            else Acc<DT>::ip(s[u], qv, v[u]);
        }
        int base = 0, mk = lpv >> 1;
#pragma unroll
        for (int hh = UN >> 1; hh >= 1; hh >>= 1) {
            if (mk >= 1) {  // warp-uniform
                const bool up = (sub & mk) != 0;
#pragma unroll
                for (int i = 0; i < hh; i++) {
                    const T send = up ? s[i] : s[i + hh];
                    const T keep = up ? s[i + hh] : s[i];
                    s[i] = keep + __shfl_xor_sync(0xffffffffu, send, mk);
                }
                if (up) base += hh;
                mk >>= 1;
            }
        }
        for (; mk >= 1; mk >>= 1) s[0] += __shfl_xor_sync(0xffffffffu, s[0], mk);  // lpv > UN
        // lane holds the totals of candidates u = base .. base + cnt - 1 of its group (cnt = UN / lpv when
        // a row has fewer than UN chunks, up to UN for one-chunk rows); the candidate entries are read
        // again where needed (L1 hits) rather than kept in registers
        unsigned m[UN];
        int tot = 0;
#pragma unroll
        for (int i = 0; i < UN; i++) {
            m[i] = 0;
            if (i >= cnt) break;  // warp-uniform
            const int64_t c = c0 + grp + (int64_t)ngrp * (base + i);
            bool in = false;
            if (writer && c < nc) {
                const uint4 e = cand[c];
                in = finish_dk(s[i], a.metric) <= a.rkey[e.z];
                if (COUNT && a.stats) {
                    atomicAdd(&a.stats[e.z].evals, 1);
                    if (mark_bit(a.count_bits + (size_t)e.z * a.words_per_q, e.x)) atomicAdd(&a.stats[e.z].distinct, 1);
                }
            }
            m[i] = __ballot_sync(0xffffffffu, in);
            tot += __popc(m[i]);
        }
        if (!tot) continue;
        // one reservation for the warp's in-range points; per-query counts are taken from the item list
        // after the last level (count_items_kernel)
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(g.tail, (unsigned long long)tot);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
#pragma unroll
        for (int i = 0; i < UN; i++) {
            if (i >= cnt) break;
            if ((m[i] >> lane) & 1u) {
                const uint4 e = cand[c0 + grp + (int64_t)ngrp * (base + i)];
                const unsigned long long pos = b0 + __popc(m[i] & lanemask_lt());
                if (pos < (unsigned long long)g.cap) {
                    g.item_key[pos] = make_key(finish_dk(s[i], a.metric), e.x);
                    g.item_slot[pos] = (int32_t)e.y;
                } else {
                    g.slot_trunc[e.y] = 1;
                }
            }
            b0 += __popc(m[i]);
        }
    }
}

template <int DT>
rr_status two_pass_t(const GreedyArgs &g, cudaStream_t st) {
    const int64_t pairs = (g.end - g.begin) * (int64_t)g.s.R;
    if (g.s.count_bits) launch_expand<true>(g, pairs, st);
    else launch_expand<false>(g, pairs, st);
    RR_CUDA(cudaGetLastError());
    // the candidate count is read on the device; the grid covers a full level's worth of candidates
    int64_t eblocks = std::max<int64_t>(1, std::min<int64_t>((pairs + 255) / 256, 152 * 16));
    if (g.s.count_bits) greedy_eval_kernel<DT, true><<<(unsigned)eblocks, 256, 0, st>>>(g);
    else greedy_eval_kernel<DT, false><<<(unsigned)eblocks, 256, 0, st>>>(g);
    RR_CUDA(cudaGetLastError());
    note_launch(2);
    return RR_OK;
}

// slot_count[s] += the items of slot s among items [0, n).  Items are appended in runs of one slot (a
// warp's reservation holds consecutive pairs of one item, mostly), so each warp adds one count per run it
// sees rather than one per item.
__global__ void count_items_kernel(const int32_t *item_slot, int64_t n, int32_t *slot_count) {
    const int lane = lane_id();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < n; base += stride) {
        const int64_t t = base + lane;
        const int32_t s = t < n ? item_slot[t] : -1;
        const int32_t prev = __shfl_up_sync(0xffffffffu, s, 1);
        const bool head = t < n && (lane == 0 || prev != s);
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        if (head) {
            // the run ends at the next head of this warp, or after the warp's last item
            const unsigned later = hm & ~((2u << lane) - 1u);
            const int stop = later ? __ffs(later) - 1 : (n - base < 32 ? (int)(n - base) : 32);
            atomicAdd(slot_count + s, stop - lane);
        }
    }
}

__global__ void set_counts_kernel(int32_t *res_count, uint8_t *flags, const int32_t *qlist, const int32_t *slot_count,
                                  const int32_t *slot_trunc, int32_t n) {
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        int32_t q = qlist[s];
        res_count[q] = slot_count[s];
        if (slot_trunc && slot_trunc[s]) flags[q] |= RR_FLAG_TRUNCATED;
    }
}

}  // namespace

rr_status launch_greedy_init(const GreedyArgs &g, cudaStream_t st, int) {
    int64_t total = (int64_t)g.ng * g.s.beam;
    if (total == 0) return RR_OK;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    greedy_init_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(g);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

bool greedy_two_pass(int dtype_code) { return dtype_code == DT_U8 || dtype_code == DT_I8; }

rr_status launch_greedy_level(const GreedyArgs &g, cudaStream_t st, int dtype_code) {
    if (g.end <= g.begin) return RR_OK;
    const int cpl = (g.s.row_chunks + 31) / 32;
    switch (dtype_code) {
        case DT_U8:
            if (g.s.row_chunks > 32 || !g.cand || !g.ccount) break;
            return two_pass_t<DT_U8>(g, st);
        case DT_I8:
            if (g.s.row_chunks > 32 || !g.cand || !g.ccount) break;
            return two_pass_t<DT_I8>(g, st);
        case DT_F32:
            // the precision form too: nearly every candidate of the in-radius expansion is in range, and an
            // in-range point needs its exact fp32 distance anyway, so a low-precision first pass would only
            // add bytes; Alg. 2's levels evaluate in exact fp32 whatever the beam phase traversed in
            if (cpl <= 1) return level_t<DT_F32, 1>(g, st);
            if (cpl <= 2) return level_t<DT_F32, 2>(g, st);
            return level_t<DT_F32, 4>(g, st);
    }
    if (dtype_code == DT_U8 || dtype_code == DT_I8) {
        set_error("greedy phase: 8-bit levels need a candidate list and rows of at most 512 bytes");
        return RR_EINTERNAL;
    }
    set_error("greedy phase: unsupported element type %d", dtype_code);
    return RR_EINVAL;
}

rr_status launch_count_items(const int32_t *item_slot, int64_t n, int32_t *slot_count, cudaStream_t st) {
    if (n <= 0) return RR_OK;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    count_items_kernel<<<(unsigned)blocks, 256, 0, st>>>(item_slot, n, slot_count);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

rr_status launch_set_counts(int32_t *res_count, uint8_t *flags, const int32_t *qlist, const int32_t *slot_count,
                            const int32_t *slot_trunc, int32_t n, cudaStream_t st) {
    if (n <= 0) return RR_OK;
    set_counts_kernel<<<(n + 255) / 256, 256, 0, st>>>(res_count, flags, qlist, slot_count, slot_trunc, n);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

}  // namespace rr
