// k_beam.cu -- the beam phase of every variant: Alg. 1 BeamSearch with the
// optional Alg. 5 early stop, then the range filter N = {n in B : d <= r} and
// the phase-2 classification of Alg. 6 / Alg. 3 (|N| = b -> greedy or
// doubling).  One warp per query.
//
// Per-warp shared memory: the beam B (sorted keys, double buffered), the
// candidate list of the current expansion, and a lossy direct-mapped "seen"
// table.  The table only filters ids that were inserted into B before; that is
// exact because (a) B never holds an id twice (merges drop equal keys) and (b)
// an id trimmed out of B has b smaller keys in B from then on, so re-inserting
// it is a no-op after the next trim.  A table miss therefore only costs a
// repeated distance evaluation, never a different B.  |V| is counted exactly.
#include "rr_common.cuh"

namespace rr {

namespace {

struct WarpSmem {
    uint64_t *bcur, *bnxt, *ckey, *skey;
    uint32_t *cid, *hash;
};

__host__ __device__ inline size_t warp_smem_bytes(int bmax, int R, int hlg) {
    return (size_t)2 * bmax * 8 + (size_t)2 * R * 8 + (size_t)R * 4 + ((size_t)4 << hlg);
}

__device__ __forceinline__ int lower_bound_or1(const uint64_t *a, int n, uint64_t k1) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((a[mid] | 1ull) < k1) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// B <- top-b(B u C): C = ckey[0..nc) (unsorted, visited bit clear).  Candidates
// that cannot enter (B full and not smaller than B[b-1]) or whose key is
// already in B are dropped first.  Writes the merged beam to Bn and returns
// its size, or -1 when nothing changed (Bn untouched).
__device__ int merge_into_beam(const uint64_t *B, uint64_t *Bn, int nb, int b, uint64_t *ckey, uint64_t *skey,
                               int nc) {
    const int lane = lane_id();
    const uint64_t last = (nb == b) ? (B[b - 1] | 1ull) : kEmpty;
    int ns = 0;
    for (int base = 0; base < nc; base += 32) {
        int c = base + lane;
        uint64_t k = c < nc ? ckey[c] : kEmpty;
        bool keep = c < nc && (k | 1ull) < last;
        if (keep) {
            int lb = lower_bound_or1(B, nb, k | 1ull);
            if (lb < nb && (B[lb] | 1ull) == (k | 1ull)) keep = false;
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) skey[ns + __popc(m & lanemask_lt())] = k;
        ns += __popc(m);
    }
    __syncwarp();
    if (ns == 0) return -1;
    // sort the survivors by rank (keys are distinct)
    for (int c = lane; c < ns; c += 32) {
        uint64_t k = skey[c];
        int r = 0;
        for (int t = 0; t < ns; t++) r += skey[t] < k;
        ckey[r] = k;
    }
    __syncwarp();
    for (int c = lane; c < ns; c += 32) {
        uint64_t k = ckey[c];
        int pos = c + lower_bound_or1(B, nb, k | 1ull);
        if (pos < b) Bn[pos] = k;
    }
    for (int i = lane; i < nb; i += 32) {
        uint64_t k = B[i];
        int pos = i + lower_bound_or1(ckey, ns, k | 1ull);
        if (pos < b) Bn[pos] = k;
    }
    __syncwarp();
    return min(b, nb + ns);
}

template <int DT, int CPL, int BMAX, bool COUNT>
__global__ void __launch_bounds__(256) beam_kernel(SearchArgs a, int hlg) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    constexpr int UN = CPL == 1 ? 8 : (CPL == 2 ? 4 : 2);
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (qi >= a.nq) return;  // whole warp leaves; the kernel has no block barriers
    const int R = a.R;
    const int b = a.beam;
    const int H = 1 << hlg;

    uint8_t *base = smem_raw + (size_t)warp * warp_smem_bytes(BMAX, R, hlg);
    WarpSmem s;
    s.bcur = reinterpret_cast<uint64_t *>(base);
    s.bnxt = s.bcur + BMAX;
    s.ckey = s.bnxt + BMAX;
    s.skey = s.ckey + R;
    s.cid = reinterpret_cast<uint32_t *>(s.skey + R);
    s.hash = s.cid + R;

    uint4 q[CPL];
    load_query<CPL>(a, a.queries + (size_t)qi * a.row_stride, q);
    const uint32_t rk = a.rkey[qi];
    const uint32_t ek = a.eskey[qi];
    uint32_t *cbits = COUNT ? a.count_bits + (size_t)qi * a.words_per_q : nullptr;

    for (int i = lane; i < H; i += 32) s.hash[i] = kSent;
    // B <- S = {start}
    const uint32_t dk0 = eval_one<DT, CPL>(a, q, a.start);
    int distinct = 0;
    if (lane == 0) {
        s.bcur[0] = make_key(dk0, a.start);
        if (COUNT) distinct += mark_bit(cbits, a.start);
    }
    __syncwarp();
    if (lane == 0) s.hash[hslot(a.start, hlg)] = a.start;
    int nb = 1, nvis = 0, evals = 1;
    bool stopped = false;
    int64_t guard = 0;
    __syncwarp();

    for (;;) {
        // p* <- argmin over B \ V: B is sorted, so the first unvisited entry
        int pidx = -1;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            int i = b0 + lane;
            bool un = i < nb && !(s.bcur[i] & 1ull);
            unsigned m = __ballot_sync(0xffffffffu, un);
            if (m) { pidx = b0 + __ffs(m) - 1; break; }
        }
        if (pidx < 0) break;
        const uint64_t pk = s.bcur[pidx];
        // Alg. 5: closest of B outside r, |V| >= vl, d(p*) outside esr
        if (a.use_es && key_dk(s.bcur[0]) > rk && nvis >= a.es_vl && key_dk(pk) > ek) { stopped = true; break; }
        if (++guard > a.n + 1) {  // every point is visited at most once
            if (lane == 0) atomicExch(a.error, 1);
            break;
        }
        __syncwarp();
        if (lane == 0) s.bcur[pidx] = pk | 1ull;  // V <- V u {p*}
        nvis++;
        const uint32_t p = key_id(pk);
        if (p >= (uint32_t)a.n) {  // cannot happen for a validated index; never index out of bounds
            if (lane == 0) atomicExch(a.error, 3);
            break;
        }
        // N_out(p*) minus ids seen before (see the file comment)
        const uint32_t *row = a.adj + (size_t)p * R;
        int nc = 0;
        for (int e0 = 0; e0 < R; e0 += 32) {
            int e = e0 + lane;
            uint32_t j = e < R ? __ldg(row + e) : kSent;
            bool v = j < (uint32_t)a.n;  // also drops the 0xFFFFFFFF padding
            uint32_t sl = 0;
            if (v) {
                sl = hslot(j, hlg);
                v = s.hash[sl] != j;
            }
            unsigned m = __ballot_sync(0xffffffffu, v);
            if (v) {
                s.hash[sl] = j;
                s.cid[nc + __popc(m & lanemask_lt())] = j;
            }
            nc += __popc(m);
            __syncwarp();
        }
        if (nc == 0) continue;
        evals += nc;
        eval_candidates<DT, CPL, UN>(a, q, s.cid, nc, s.ckey);
        __syncwarp();
        if (COUNT) {
            int dd = 0;
            for (int c = lane; c < nc; c += 32) dd += mark_bit(cbits, s.cid[c]);
            distinct += dd;
        }
        // B <- top-b(B u new)
        int nn = merge_into_beam(s.bcur, s.bnxt, nb, b, s.ckey, s.skey, nc);
        if (nn >= 0) {
            nb = nn;
            uint64_t *t = s.bcur;
            s.bcur = s.bnxt;
            s.bnxt = t;
        }
        __syncwarp();
    }

    // N = {n in B : d(n, q) <= r}: a prefix of the sorted beam
    int cnt = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        int i = b0 + lane;
        bool in = i < nb && key_dk(s.bcur[i]) <= rk;
        cnt += __popc(__ballot_sync(0xffffffffu, in));
    }
    uint64_t *out = a.res_keys + (size_t)qi * b;
    for (int i = lane; i < cnt; i += 32) out[i] = s.bcur[i] & ~1ull;
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

template <int DT, int CPL, int BMAX>
rr_status launch_t(const SearchArgs &a, int wpc, int hlg, cudaStream_t st) {
    size_t smem = (size_t)wpc * warp_smem_bytes(BMAX, a.R, hlg);
    dim3 grid((unsigned)((a.nq + wpc - 1) / wpc)), block(32 * wpc);
    if (a.count_bits) {
        auto k = beam_kernel<DT, CPL, BMAX, true>;
        RR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, block, smem, st>>>(a, hlg);
    } else {
        auto k = beam_kernel<DT, CPL, BMAX, false>;
        RR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, block, smem, st>>>(a, hlg);
    }
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
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

}  // namespace

int beam_hash_lg(int beam) { return beam <= 64 ? 10 : (beam <= 256 ? 11 : 12); }

rr_status launch_beam(const SearchArgs &a, int wpc, cudaStream_t st, int dtype_code) {
    if (a.nq == 0) return RR_OK;
    const int hlg = beam_hash_lg(a.beam);
    const int cpl = (a.row_chunks + 31) / 32;
    switch (dtype_code) {
        case DT_U8: return launch_b<DT_U8, 1>(a, wpc, hlg, st);
        case DT_I8: return launch_b<DT_I8, 1>(a, wpc, hlg, st);
        case DT_F32:
            if (cpl <= 1) return launch_b<DT_F32, 1>(a, wpc, hlg, st);
            if (cpl <= 2) return launch_b<DT_F32, 2>(a, wpc, hlg, st);
            return launch_b<DT_F32, 4>(a, wpc, hlg, st);
    }
    set_error("beam phase: unsupported element type %d", dtype_code);
    return RR_EINVAL;
}

}  // namespace rr
