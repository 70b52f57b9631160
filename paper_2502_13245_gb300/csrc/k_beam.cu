// k_beam.cu -- the beam phase of every variant: Alg. 1 BeamSearch with the
// optional Alg. 5 early stop, then the range filter N = {n in B : d <= r} and
// the phase-2 classification of Alg. 6 / Alg. 3 (|N| = b -> greedy or
// doubling).  One warp per query.
//
// Per-warp shared memory: the beam B (keys sorted by (distance, id), the low
// bit marks V), the candidates of the current expansion, and a lossy two-way
// set-associative "seen" table (a set keeps its two most recent ids; a slot
// only ever holds an id that was evaluated).  The table only filters ids whose distance was
// evaluated before; that is exact because (a) B never holds an id twice
// (merges drop equal keys) and (b) an id that left B, or was refused by a full
// B, has b smaller keys in B from then on (B's b-th key only decreases), so
// offering it again changes nothing.  A table miss only costs a repeated
// distance evaluation, never a different B.  |V| is counted exactly.
//
// The merge of the (few) new keys into B is done in place: with the new keys
// sorted, old entry i moves right by the number of new keys below it, so only
// the suffix after the first insertion point is touched, chunk by chunk from
// the end.  The index of the first unvisited entry (p* of Alg. 1) is carried
// across iterations instead of rescanning B.
#include <algorithm>

#include "rr_common.cuh"

namespace rr {

namespace {

// per warp (R here counts the candidates of one iteration), rounded to 16 bytes so that every warp's
// 8-byte arrays stay aligned for any degree
__host__ __device__ inline size_t warp_smem_bytes(int bmax, int R, int hlg) {
    return ((size_t)bmax * 8 + (size_t)2 * R * 8 + (size_t)3 * R * 4 + ((size_t)4 << hlg) + 15) & ~(size_t)15;
}

// number of a[t] with (a[t] | 1) < k1
__device__ __forceinline__ int lower_bound_or1(const uint64_t *a, int n, uint64_t k1) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((a[mid] | 1ull) < k1) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// number of v[t] <= x (v non-decreasing)
__device__ __forceinline__ int upper_bound_i32(const int32_t *v, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (v[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// first index >= from with the visited bit clear, or n
__device__ __forceinline__ int next_unvisited(const uint64_t *B, int n, int from) {
    const int lane = lane_id();
    for (int b0 = from; b0 < n; b0 += 32) {
        int i = b0 + lane;
        unsigned m = __ballot_sync(0xffffffffu, i < n && !(B[i] & 1ull));
        if (m) return b0 + __ffs(m) - 1;
    }
    return n;
}

template <int DT, int CPL, int BMAX, bool COUNT, bool BUILD>
__device__ __forceinline__ void search_query(const SearchArgs &a, int hlg, int64_t qi, uint8_t *base);

// 8-bit searches fit 64 registers with a few bytes of spill and gain from the extra resident
// warps; the fp32 and low-precision forms keep 80 (they would spill 100-300 bytes).
template <int DT>
constexpr int kBeamMinBlocks = (DT == DT_U8 || DT == DT_I8) ? 4 : 3;

// One warp per query.  persistent = 0: warp w of CTA c takes query c*warps + w.
// persistent = 1: a grid sized to the resident capacity; every warp takes the
// next query from a device counter until the batch is done, so warps freed by
// cheap (e.g. early-stopped) queries move on to the rest of the batch.
template <int DT, int CPL, int BMAX, bool COUNT, bool BUILD = false>
__global__ void __launch_bounds__(256, kBeamMinBlocks<DT>) beam_kernel(SearchArgs a, int hlg, int persistent, int32_t *next_q) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    uint8_t *base = smem_raw + (size_t)warp * warp_smem_bytes(BMAX, a.R * (a.expand > 1 ? a.expand : 1), hlg);
    int64_t qi = 0;
    if (!persistent) qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    else if (lane == 0) qi = atomicAdd(next_q, 1);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    // whole warps leave together; the kernel has no block barriers
    while (qi < a.nq) {
        search_query<DT, CPL, BMAX, COUNT, BUILD>(a, hlg, qi, base);
        if (!persistent) break;
        __syncwarp();
        if (lane == 0) qi = atomicAdd(next_q, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
    }
}

template <int DT, int CPL, int BMAX, bool COUNT, bool BUILD>
__device__ __forceinline__ void search_query(const SearchArgs &a, int hlg, int64_t qi, uint8_t *base) {
    constexpr int UN = CPL == 1 ? 8 : (CPL == 2 ? 4 : 2);
    const int lane = lane_id();
    const int R = a.R;
    const int b = a.beam;
    const int H = 1 << hlg;
    const int E = a.expand > 1 ? a.expand : 1;  // parents per iteration (1: Alg. 1)
    const int ER = R * E;

    uint64_t *B = reinterpret_cast<uint64_t *>(base);
    uint64_t *ckey = B + BMAX;       // candidate keys, then the sorted survivors
    uint64_t *skey = ckey + ER;      // survivors before sorting
    uint32_t *cid = reinterpret_cast<uint32_t *>(skey + ER);
    int32_t *lbs = reinterpret_cast<int32_t *>(cid + ER);  // insertion point of each sorted survivor
    int32_t *slb = lbs + ER;                                // insertion point of each unsorted survivor
    uint32_t *hash = reinterpret_cast<uint32_t *>(slb + ER);

    constexpr bool LP = is_lowp(DT);
    uint4 q[CPL];
    float qf[16];
    float qn2 = 0.f;
    if constexpr (LP) {
        load_query_lp<DT>(a, reinterpret_cast<const float *>(a.queries + (size_t)qi * a.row_stride), qf);
        qn2 = query_norm2_lp(a, qf);
    } else if constexpr (BUILD) {
        load_query<CPL>(a, a.vec + (size_t)a.qids[qi] * a.row_stride, q);
    } else {
        load_query<CPL>(a, a.queries + (size_t)qi * a.row_stride, q);
    }
    const uint32_t rk = BUILD ? 0u : a.rkey[qi];
    const uint32_t ek = BUILD ? 0u : a.eskey[qi];
    // low precision: approximate distances above r + slack are certainly out of range
    const uint32_t rks = LP ? slack_key(a, rk, qn2) : rk;
    uint32_t *cbits = COUNT ? a.count_bits + (size_t)qi * a.words_per_q : nullptr;

    for (int i = lane; i < H; i += 32) hash[i] = kSent;
    // B <- S = {start}
    uint32_t dk0;
    if constexpr (LP) dk0 = eval_one_lp<DT>(a, qf, qn2, a.start);
    else dk0 = eval_one<DT, CPL>(a, q, a.start);
    int distinct = 0;
    __syncwarp();
    if (lane == 0) {
        B[0] = make_key(dk0, a.start);
        hash[hslot(a.start, hlg - 1) << 1] = a.start;
        if (COUNT) distinct += mark_bit(cbits, a.start);
    }
    __syncwarp();
    int nb = 1, cur = 0, nvis = 0, evals = 1;
    bool stopped = false;
    int64_t guard = 0;
    // adjacency row of the likely next p* (the next unvisited entry), loaded while the
    // current candidates are evaluated; used only if that entry is indeed chosen
    uint32_t pre[4];
    uint32_t pre_id = kSent;

    while (cur < nb) {
        // p* <- argmin over B \ V = B[cur] (B sorted, everything before cur visited)
        const uint64_t pk = B[cur];
        // Alg. 5 / Alg. 4: closest of B outside r, |V| >= vl, the metric above its threshold
        if (!BUILD && a.use_es && key_dk(B[0]) > rks && nvis >= a.es_vl) {
            bool fire;
            const uint32_t d10 = key_dk(B[min(nb, 10) - 1]);
            switch (a.es_metric) {
            case RR_ES_TOP1: fire = key_dk(B[0]) > ek; break;
            case RR_ES_TOP10: fire = d10 > ek; break;
            case RR_ES_TOP10_RATIO: {
                const bool fp = DT == DT_F32 || LP;
                fire = dkey_value(d10, fp) > a.es_ratio * dkey_value(dk0, fp);
                break;
            }
            default: fire = key_dk(pk) > ek;  // d_visited
            }
            if (fire) { stopped = true; break; }
        }
        const uint32_t p = key_id(pk);
        if (++guard > a.iter_limit || p >= (uint32_t)a.n) {  // cannot happen for a validated index
            if (lane == 0) atomicExch(a.error, p >= (uint32_t)a.n ? 3 : 1);
            break;
        }
        __syncwarp();
        // the parents of this iteration: p* and, with E > 1, the next E - 1 unvisited entries of B
        int par[3] = {-1, -1, -1};
        int np = 1;
        for (int b0 = cur + 1; b0 < nb && np < E; b0 += 32) {
            const int i = b0 + lane;
            unsigned m = __ballot_sync(0xffffffffu, i < nb && !(B[i] & 1ull));
            while (m && np < E) {
                const int pos = b0 + __ffs(m) - 1;
                m &= m - 1;
                par[np - 1] = pos;
                np++;
            }
        }
        uint32_t pid[3] = {kSent, kSent, kSent};
        for (int e = 1; e < np; e++) pid[e - 1] = key_id(B[par[e - 1]]);
        __syncwarp();
        if (lane == 0) {
            B[cur] = pk | 1ull;  // V <- V u {p*}
            if (BUILD && nvis < a.vis_cap) a.vis_out[(size_t)qi * a.vis_cap + nvis] = pk & ~1ull;
            for (int e = 1; e < np; e++) B[par[e - 1]] |= 1ull;
        }
        nvis += np;
        __syncwarp();
        const int nxt = next_unvisited(B, nb, cur + 1);
        // N_out of the parents minus ids seen before (see the file comment)
        uint32_t row4[4];
        if (p == pre_id) {
#pragma unroll
            for (int k = 0; k < 4; k++) row4[k] = pre[k];
        } else {
            const uint32_t *row = a.adj + (size_t)p * R;
#pragma unroll
            for (int k = 0; k < 4; k++) row4[k] = (32 * k + lane < R) ? __ldg(row + 32 * k + lane) : kSent;
        }
        pre_id = kSent;
        if (nxt < nb) {
            const uint32_t pn = key_id(B[nxt]);
            if (pn < (uint32_t)a.n) {
                const uint32_t *row = a.adj + (size_t)pn * R;
#pragma unroll
                for (int k = 0; k < 4; k++) pre[k] = (32 * k + lane < R) ? __ldg(row + 32 * k + lane) : kSent;
                pre_id = pn;
            }
        }
        int nc = 0;
        for (int e = 0; e < np; e++) {
            if (e > 0) {
                const uint32_t pe = pid[e - 1];
                if (pe >= (uint32_t)a.n) continue;  // cannot happen for a validated index
                const uint32_t *row = a.adj + (size_t)pe * R;
#pragma unroll
                for (int k = 0; k < 4; k++) row4[k] = (32 * k + lane < R) ? __ldg(row + 32 * k + lane) : kSent;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (32 * k >= R) break;  // warp-uniform
                uint32_t j = row4[k];
                bool v = j < (uint32_t)a.n;  // also drops the 0xFFFFFFFF padding
                uint32_t sl = 0, old = kSent;
                if (v) {
                    // two-way set: slot 2s holds the most recent id of the set, 2s+1 the one before
                    sl = hslot(j, hlg - 1) << 1;
                    old = hash[sl];
                    v = old != j && hash[sl + 1] != j;
                }
                unsigned m = __ballot_sync(0xffffffffu, v);
                __syncwarp();
                if (v) {
                    hash[sl + 1] = old;
                    hash[sl] = j;
                    cid[nc + __popc(m & lanemask_lt())] = j;
                }
                nc += __popc(m);
                __syncwarp();
            }
        }
        if (nc == 0) { cur = nxt; continue; }
        evals += nc;
        if constexpr (LP) {
            eval_candidates_lp<DT, DT == DT_FP8 ? 4 : 8>(a, qf, qn2, cid, nc, ckey);
        } else if constexpr (CPL == 1 && (DT == DT_U8 || DT == DT_I8)) {
            // few new candidates (late in a search): a shallower unroll wastes fewer lanes (exact integer
            // sums, so the keys do not depend on it)
            const int ngrp = 32 >> (__ffs(a.lpv) - 1);
            if (nc <= 2 * ngrp) eval_candidates<DT, CPL, 2>(a, q, cid, nc, ckey);
            else if (nc <= 4 * ngrp) eval_candidates<DT, CPL, 4>(a, q, cid, nc, ckey);
            else eval_candidates<DT, CPL, UN>(a, q, cid, nc, ckey);
        } else {
            eval_candidates<DT, CPL, UN>(a, q, cid, nc, ckey);
        }
        __syncwarp();
        if (COUNT) {
            int dd = 0;
            for (int c = lane; c < nc; c += 32) dd += mark_bit(cbits, cid[c]);
            distinct += dd;
        }
        // keys that can enter: below B[b-1] when B is full, and not already in B
        const uint64_t last = (nb == b) ? (B[b - 1] | 1ull) : kEmpty;
        int ns = 0;
        for (int c0 = 0; c0 < nc; c0 += 32) {
            int c = c0 + lane;
            uint64_t k = c < nc ? ckey[c] : kEmpty;
            bool keep = c < nc && (k | 1ull) < last;
            int lb = 0;
            if (keep) {
                lb = lower_bound_or1(B, nb, k | 1ull);
                keep = !(lb < nb && (B[lb] | 1ull) == (k | 1ull));
            }
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int o = ns + __popc(m & lanemask_lt());
                skey[o] = k;
                slb[o] = lb;
            }
            ns += __popc(m);
        }
        __syncwarp();
        if (ns == 0) { cur = nxt; continue; }
        int nsu = ns;
        if (E > 1) {
            // with several parents, a neighbour the lossy table forgot within this iteration can come
            // twice: keep the first copy of each key (B stays a set)
            nsu = 0;
            for (int c0 = 0; c0 < ns; c0 += 32) {
                const int c = c0 + lane;
                bool first = c < ns;
                if (first) {
                    const uint64_t k = skey[c];
                    for (int t = 0; t < c && first; t++) first = skey[t] != k;
                }
                nsu += __popc(__ballot_sync(0xffffffffu, first));
                if (c < ns && !first) slb[c] = -1;
            }
            __syncwarp();
        }
        // sort the survivors (distinct keys) by rank; each keeps its insertion point in B
        for (int c = lane; c < ns; c += 32) {
            const int lbc = slb[c];
            if (lbc < 0) continue;
            uint64_t k = skey[c];
            int r = 0;
            for (int t = 0; t < ns; t++) r += (skey[t] < k) && (E == 1 || slb[t] >= 0);
            ckey[r] = k;
            lbs[r] = lbc;
        }
        ns = nsu;
        __syncwarp();
        const int lb0 = lbs[0];
        // B <- top-b(B u survivors): shift the suffix [lb0, nb) right, last chunk first
        for (int hi = nb; hi > lb0;) {
            const int lo = max(lb0, hi - 32);
            const int i = lo + lane;
            uint64_t k = 0;
            int dst = b;
            if (i < hi) {
                k = B[i];
                dst = i + upper_bound_i32(lbs, ns, i);
            }
            __syncwarp();
            if (dst < b) B[dst] = k;
            __syncwarp();
            hi = lo;
        }
        for (int c = lane; c < ns; c += 32) {
            int pos = lbs[c] + c;
            if (pos < b) B[pos] = ckey[c];
        }
        __syncwarp();
        // first unvisited entry: the smallest survivor, or the old next one after its shift
        const int posn = nxt < nb ? nxt + upper_bound_i32(lbs, ns, nxt) : 0x7fffffff;
        nb = min(b, nb + ns);
        cur = min(min(posn, lb0), nb);
    }

    if constexpr (BUILD) {
        if (lane == 0) a.vis_count[qi] = min(nvis, a.vis_cap);
        return;
    }
    // N = {n in B : d(n, q) <= r}: a prefix of the sorted beam.  Low precision: the
    // prefix within r + slack is re-checked in exact fp32 and re-sorted by exact keys.
    int cnt = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        int i = b0 + lane;
        bool in = i < nb && key_dk(B[i]) <= rks;
        cnt += __popc(__ballot_sync(0xffffffffu, in));
    }
    if constexpr (LP) {
        evals += cnt;
        cnt = exact_filter_sort<CPL, UN>(a, qi, B, cnt, rk, cid, ckey, R);
    }
    uint64_t *out = a.res_keys + (size_t)qi * b;
    for (int i = lane; i < cnt; i += 32) out[i] = B[i] & ~1ull;
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
    }
    if (lane == 0) {
        a.res_count[qi] = cnt;
        uint8_t f = stopped ? RR_FLAG_EARLY_STOPPED : 0;
        if (a.phase2 && cnt == b) {
            f |= RR_FLAG_PHASE2;
            int slot = atomicAdd(a.p2_count, 1);
            a.p2_list[slot] = (int32_t)qi;
        }
        a.flags[qi] = f;
        if (a.stats) {
            rr_query_stats st;
            st.visits_beam = nvis;
            st.visits_phase2 = 0;
            st.distinct = distinct;
            st.rounds = 1;
            st.final_beam = b;
            st.evals = evals;
            a.stats[qi] = st;
        }
    }
}

template <int DT, int CPL, int BMAX, bool COUNT>
rr_status launch_k(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    auto k = beam_kernel<DT, CPL, BMAX, COUNT>;
    const size_t smem = (size_t)wpc * warp_smem_bytes(BMAX, a.R * std::max(1, a.expand), hlg);
    RR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (a.nq + wpc - 1) / wpc;
    if (a.persistent) {
        int dev = 0, sms = 0, per_sm = 0;
        RR_CUDA(cudaGetDevice(&dev));
        RR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        RR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * wpc, smem));
        blocks = std::min<int64_t>(blocks, (int64_t)std::max(1, per_sm) * sms);
    }
    k<<<(unsigned)blocks, 32 * wpc, smem, st>>>(a, hlg, a.persistent, a.next_q);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

template <int DT, int CPL, int BMAX>
rr_status launch_t(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    if (a.persistent && !a.next_q) {
        set_error("beam phase: persistent launch without a work counter");
        return RR_EINTERNAL;
    }
    if (a.count_bits) return launch_k<DT, CPL, BMAX, true>(a, wpc, hlg, st);
    return launch_k<DT, CPL, BMAX, false>(a, wpc, hlg, st);
}

template <int DT, int CPL>
rr_status launch_b(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    if (a.beam <= 32) return launch_t<DT, CPL, 32>(a, wpc, hlg, st);
    if (a.beam <= 64) return launch_t<DT, CPL, 64>(a, wpc, hlg, st);
    if (a.beam <= 128) return launch_t<DT, CPL, 128>(a, wpc, hlg, st);
    if (a.beam <= 256) return launch_t<DT, CPL, 256>(a, wpc, hlg, st);
    if (a.beam <= 512) return launch_t<DT, CPL, 512>(a, wpc, hlg, st);
    set_error("beam phase: b=%d exceeds the shared-memory beam limit 512", a.beam);
    return RR_EINVAL;
}

template <int DT, int BMAX>
rr_status launch_build_k(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    auto k = beam_kernel<DT, 1, BMAX, false, true>;
    const size_t smem = (size_t)wpc * warp_smem_bytes(BMAX, a.R, hlg);
    RR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = (a.nq + wpc - 1) / wpc;
    k<<<(unsigned)blocks, 32 * wpc, smem, st>>>(a, hlg, 0, nullptr);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

template <int DT>
rr_status launch_build_b(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    if (a.beam <= 32) return launch_build_k<DT, 32>(a, wpc, hlg, st);
    if (a.beam <= 64) return launch_build_k<DT, 64>(a, wpc, hlg, st);
    if (a.beam <= 128) return launch_build_k<DT, 128>(a, wpc, hlg, st);
    if (a.beam <= 256) return launch_build_k<DT, 256>(a, wpc, hlg, st);
    if (a.beam <= 512) return launch_build_k<DT, 512>(a, wpc, hlg, st);
    set_error("graph build: L=%d exceeds the shared-memory beam limit 512", a.beam);
    return RR_EINVAL;
}

}  // namespace

int beam_hash_lg(int beam) { return beam <= 256 ? 10 : 11; }

rr_status launch_build_search(const SearchArgs &a, int wpc, cudaStream_t st, int dtype_code) {
    if (a.nq == 0) return RR_OK;
    if (!a.qids || !a.vis_out || !a.vis_count || a.vis_cap < 1 || a.row_chunks > 32) {
        set_error("graph build: bad search arguments");
        return RR_EINTERNAL;
    }
    const int hlg = a.hash_lg > 0 ? a.hash_lg : beam_hash_lg(a.beam);
    switch (dtype_code) {
        case DT_U8: return launch_build_b<DT_U8>(a, wpc, hlg, st);
        case DT_I8: return launch_build_b<DT_I8>(a, wpc, hlg, st);
    }
    set_error("graph build: the GPU builder takes 8-bit vectors");
    return RR_EINVAL;
}

rr_status launch_beam(const SearchArgs &a, int wpc, cudaStream_t st, int dtype_code) {
    if (a.nq == 0) return RR_OK;
    const int hlg = a.hash_lg > 0 ? a.hash_lg : beam_hash_lg(a.beam);
    if (hlg < 5 || hlg > 14) {
        set_error("beam phase: seen-table size 2^%d out of [2^5, 2^14]", hlg);
        return RR_EINVAL;
    }
    const int cpl = (a.row_chunks + 31) / 32;
    switch (dtype_code) {
        case DT_U8: return launch_b<DT_U8, 1>(a, wpc, hlg, st);
        case DT_I8: return launch_b<DT_I8, 1>(a, wpc, hlg, st);
        case DT_F32:
            // low-precision traversal: the exact-recheck rows need CPL chunks per lane (2 up to d = 256,
            // 4 up to d = 512); the smaller instantiation keeps the FP8 kernel out of register spills
            if (a.prec == RR_PREC_BF16) return cpl <= 2 ? launch_b<DT_BF16, 2>(a, wpc, hlg, st) : launch_b<DT_BF16, 4>(a, wpc, hlg, st);
            if (a.prec == RR_PREC_FP8) return cpl <= 2 ? launch_b<DT_FP8, 2>(a, wpc, hlg, st) : launch_b<DT_FP8, 4>(a, wpc, hlg, st);
            if (cpl <= 1) return launch_b<DT_F32, 1>(a, wpc, hlg, st);
            if (cpl <= 2) return launch_b<DT_F32, 2>(a, wpc, hlg, st);
            return launch_b<DT_F32, 4>(a, wpc, hlg, st);
    }
    set_error("beam phase: unsupported element type %d", dtype_code);
    return RR_EINVAL;
}

}  // namespace rr
