// k_doubling.cu -- Alg. 3 DoublingSearch for the queries whose first beam
// search returned a full beam of in-range points (|N| = b, lambda = 1).
//
// Rounds are host-driven: round k runs Alg. 1 with beam b_k = b_0 * 2^(k-1)
// from B = S_k (trimming S_k to its b_k closest up front is equivalent: the
// first visit is the closest point of S_k either way, and top-b(S u X) =
// top-b(top-b(S) u X) at the first trim), with a fresh V.  Round 1 is
// re-run here from S = {start}, so the round kernel owns the whole per-query
// state.  Then S <- S u V (the b_max smallest keys are all any later round
// can use) and b <- 2b while |N| = b.
//
// Per query and round, one warp.  The beam can be tens of thousands of keys,
// so it lives in global memory (L2-resident) as a sorted array M, with a small
// sorted insertion buffer I in shared memory; the logical beam is the b
// smallest keys of M u I, tracked through their b-th key tau.  New keys enter
// I only if they are below tau; I is merged into M when full.  An exact
// per-round bitmap of evaluated ids replaces the visited filter (an id that is
// seen again is either in the beam or was trimmed, and a trimmed id can never
// re-enter: see the beam kernel), so no id is evaluated twice in a round.
#include "rr_common.cuh"

namespace rr {

namespace {

constexpr int KI = 256;  // insertion buffer entries

__device__ __forceinline__ int lb_or1(const uint64_t *a, int n, uint64_t k1) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((a[mid] | 1ull) < k1) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// number of a[t] with (a[t] | 1) <= k1
__device__ __forceinline__ int ub_or1(const uint64_t *a, int n, uint64_t k1) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((a[mid] | 1ull) <= k1) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// (key | 1) of the element of rank b-1 (0-based) of the sorted union M u I,
// or kEmpty when the union has fewer than b keys.  Serial (one lane).
__device__ uint64_t kth_or1(const uint64_t *M, int nM, const uint64_t *I, int nI, int b) {
    if (nM + nI < b) return kEmpty;
    int lo = max(0, b - nI), hi = min(b, nM);
    // largest i in [lo, hi] with: i == 0 || b - i >= nI || M[i-1] < I[b-i]
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        bool ok = (b - mid >= nI) || ((M[mid - 1] | 1ull) < (I[b - mid] | 1ull));
        if (ok) lo = mid;
        else hi = mid - 1;
    }
    int i = lo, j = b - lo;
    uint64_t x = i > 0 ? (M[i - 1] | 1ull) : 0ull;
    uint64_t y = j > 0 ? (I[j - 1] | 1ull) : 0ull;
    return x > y ? x : y;
}

struct RSmem {
    uint64_t *I, *I2, *ckey, *skey;
    uint32_t *cid;
};

// per warp, rounded to 16 bytes so that every warp's 8-byte arrays stay aligned for any degree R
__host__ __device__ inline size_t round_smem_bytes(int R) {
    return ((size_t)2 * KI * 8 + (size_t)2 * R * 8 + (size_t)R * 4 + 15) & ~(size_t)15;
}

template <int DT, int CPL>
__global__ void __launch_bounds__(128) round_kernel(DoublingRound d) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    constexpr int UN = CPL == 1 ? 8 : (CPL == 2 ? 4 : 2);
    const SearchArgs &a = d.s;
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= d.na) return;
    const int R = a.R;
    const int b = a.beam;
    uint8_t *base = smem_raw + (size_t)warp * round_smem_bytes(R);
    RSmem s;
    s.I = reinterpret_cast<uint64_t *>(base);
    s.I2 = s.I + KI;
    s.ckey = s.I2 + KI;
    s.skey = s.ckey + R;
    s.cid = reinterpret_cast<uint32_t *>(s.skey + R);

    const int32_t slot = d.act[i];
    const int32_t qi = d.qlist[slot];
    constexpr bool LP = is_lowp(DT);
    uint4 q[CPL];
    float qf[16];
    float qn2 = 0.f;
    if constexpr (LP) {
        load_query_lp<DT>(a, reinterpret_cast<const float *>(a.queries + (size_t)qi * a.row_stride), qf);
        qn2 = query_norm2_lp(a, qf);
    } else {
        load_query<CPL>(a, a.queries + (size_t)qi * a.row_stride, q);
    }
    const uint32_t rk = a.rkey[qi], ek = a.eskey[qi];
    const uint32_t rks = LP ? slack_key(a, rk, qn2) : rk;  // approximate keys above rks are out of range
    uint64_t *M = d.bA + (size_t)i * b;
    uint64_t *M2 = d.bB + (size_t)i * b;
    uint64_t *V = d.v + (size_t)i * d.v_cap;
    // warm restart: the bitmap of every id this query ever evaluated lives on across rounds (per slot)
    uint32_t *seen = d.seen + (size_t)(d.warm ? slot : i) * d.seen_words;
    uint64_t *EV = d.warm ? d.ev + (size_t)i * d.ev_cap : nullptr;
    int nev = 0;
    uint32_t *cbits = a.count_bits ? a.count_bits + (size_t)qi * a.words_per_q : nullptr;
    int evals = 0, distinct = 0;

    // B <- top-b(S)
    int nM;
    if (d.first) {
        uint32_t dk0;
        if constexpr (LP) dk0 = eval_one_lp<DT>(a, qf, qn2, a.start);
        else dk0 = eval_one<DT, CPL>(a, q, a.start);
        if (lane == 0) {
            M[0] = make_key(dk0, a.start);
            mark_bit(seen, a.start);
            if (EV) EV[0] = make_key(dk0, a.start);
        }
        nev = EV ? 1 : 0;
        nM = 1;
        evals = 1;
    } else if (d.warm) {
        // B <- the b closest points of E, visited ones still marked (they are not visited again); every id
        // of E is in seen already: one outside these b can never enter the beam of this round
        nM = min(b, d.s_cnt[i]);
        const uint64_t *S = d.s_old + (size_t)i * d.s_cap;
        for (int t = lane; t < nM; t += 32) M[t] = S[t];
    } else {
        nM = min(b, d.s_cnt[i]);
        const uint64_t *S = d.s_old + (size_t)i * d.s_cap;
        for (int t = lane; t < nM; t += 32) {
            uint64_t k = S[t] & ~1ull;
            M[t] = k;
            mark_bit(seen, key_id(k));
        }
    }
    __syncwarp();
    int nI = 0, cM = 0, nvis = 0;
    bool stopped = false, overflow = false;
    uint64_t tau = (nM >= b) ? (M[b - 1] | 1ull) : kEmpty;
    int64_t guard = 0;

    for (;;) {
        // first unvisited key of M from the cursor
        for (;;) {
            int t = cM + lane;
            bool un = t < nM && !(M[t] & 1ull);
            unsigned m = __ballot_sync(0xffffffffu, un);
            if (m) { cM += __ffs(m) - 1; break; }
            cM += 32;
            if (cM >= nM) { cM = nM; break; }
        }
        uint64_t kM = cM < nM ? M[cM] : kEmpty;
        int jI = -1;
        for (int b0 = 0; b0 < nI; b0 += 32) {
            int t = b0 + lane;
            bool un = t < nI && !(s.I[t] & 1ull);
            unsigned m = __ballot_sync(0xffffffffu, un);
            if (m) { jI = b0 + __ffs(m) - 1; break; }
        }
        uint64_t kI = jI >= 0 ? s.I[jI] : kEmpty;
        const bool fromI = (kI | 1ull) < (kM | 1ull);
        const uint64_t pk = fromI ? kI : kM;
        if (pk == kEmpty || (pk | 1ull) > tau) break;  // B \ V is empty
        if (a.use_es) {
            uint64_t mn = M[0] | 1ull;
            if (nI > 0 && (s.I[0] | 1ull) < mn) mn = s.I[0] | 1ull;
            if (key_dk(mn) > rks && nvis >= a.es_vl && key_dk(pk) > ek) { stopped = true; break; }
        }
        if (++guard > a.iter_limit) {
            if (lane == 0) atomicExch(a.error, 2);
            break;
        }
        if (nvis >= d.v_cap) { overflow = true; break; }
        __syncwarp();
        if (lane == 0) {
            if (fromI) s.I[jI] = pk | 1ull;
            else M[cM] = pk | 1ull;
            V[nvis] = pk & ~1ull;
        }
        nvis++;
        const uint32_t p = key_id(pk);
        const uint32_t *row = a.adj + (size_t)p * R;
        int nc = 0;
        for (int e0 = 0; e0 < R; e0 += 32) {
            int e = e0 + lane;
            uint32_t j = e < R ? __ldg(row + e) : kSent;
            bool v = j < (uint32_t)a.n && mark_bit(seen, j);
            unsigned m = __ballot_sync(0xffffffffu, v);
            if (v) s.cid[nc + __popc(m & lanemask_lt())] = j;
            nc += __popc(m);
        }
        __syncwarp();
        if (nc == 0) continue;
        evals += nc;
        if constexpr (LP) eval_candidates_lp<DT, DT == DT_FP8 ? 4 : 8>(a, qf, qn2, s.cid, nc, s.ckey);
        else eval_candidates<DT, CPL, UN>(a, q, s.cid, nc, s.ckey);
        __syncwarp();
        if (EV) {
            // E <- E u the new evaluations (kept for the rounds after this one)
            if (nev + nc > d.ev_cap) { overflow = true; break; }
            for (int c = lane; c < nc; c += 32) EV[nev + c] = s.ckey[c];
            nev += nc;
        }
        if (cbits) {
            int dd = 0;
            for (int c = lane; c < nc; c += 32) dd += mark_bit(cbits, s.cid[c]);
            distinct += dd;
        }
        // keys below tau enter the beam
        int ns = 0;
        for (int c0 = 0; c0 < nc; c0 += 32) {
            int c = c0 + lane;
            uint64_t k = c < nc ? s.ckey[c] : kEmpty;
            bool keep = c < nc && (k | 1ull) < tau;
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) s.skey[ns + __popc(m & lanemask_lt())] = k;
            ns += __popc(m);
        }
        __syncwarp();
        if (ns == 0) continue;
        for (int c = lane; c < ns; c += 32) {
            uint64_t k = s.skey[c];
            int r = 0;
            for (int t = 0; t < ns; t++) r += s.skey[t] < k;
            s.ckey[r] = k;  // survivors sorted
        }
        __syncwarp();
        if (nI + ns > KI) {
            // flush: M2 <- top-b(M u I)
            for (int t = lane; t < nM; t += 32) {
                uint64_t k = M[t];
                int pos = t + lb_or1(s.I, nI, k | 1ull);
                if (pos < b) M2[pos] = k;
            }
            for (int t = lane; t < nI; t += 32) {
                uint64_t k = s.I[t];
                int pos = t + lb_or1(M, nM, k | 1ull);
                if (pos < b) M2[pos] = k;
            }
            int posM = cM < nM ? cM + lb_or1(s.I, nI, M[cM] | 1ull) : 0x7fffffff;
            int jU = -1;
            for (int b0 = 0; b0 < nI; b0 += 32) {
                int t = b0 + lane;
                bool un = t < nI && !(s.I[t] & 1ull);
                unsigned m = __ballot_sync(0xffffffffu, un);
                if (m) { jU = b0 + __ffs(m) - 1; break; }
            }
            int posI = jU >= 0 ? jU + lb_or1(M, nM, s.I[jU] | 1ull) : 0x7fffffff;
            __syncwarp();
            nM = min(b, nM + nI);
            nI = 0;
            cM = min(min(posM, posI), nM);
            uint64_t *t = M;
            M = M2;
            M2 = t;
        }
        // I <- I u survivors (sorted merge into I2, then copy back)
        for (int t = lane; t < nI; t += 32) {
            uint64_t k = s.I[t];
            s.I2[t + lb_or1(s.ckey, ns, k | 1ull)] = k;
        }
        for (int t = lane; t < ns; t += 32) {
            uint64_t k = s.ckey[t];
            s.I2[t + lb_or1(s.I, nI, k | 1ull)] = k;
        }
        __syncwarp();
        nI += ns;
        for (int t = lane; t < nI; t += 32) s.I[t] = s.I2[t];
        __syncwarp();
        // tau <- b-th smallest of M u I; drop I keys beyond it
        uint64_t nt = 0;
        if (lane == 0) nt = kth_or1(M, nM, s.I, nI, b);
        tau = __shfl_sync(0xffffffffu, nt, 0);
        if (tau != kEmpty) nI = ub_or1(s.I, nI, tau);
        __syncwarp();
    }
    // final B = top-b(M u I)
    if (nI > 0) {
        for (int t = lane; t < nM; t += 32) {
            uint64_t k = M[t];
            int pos = t + lb_or1(s.I, nI, k | 1ull);
            if (pos < b) M2[pos] = k;
        }
        for (int t = lane; t < nI; t += 32) {
            uint64_t k = s.I[t];
            int pos = t + lb_or1(M, nM, k | 1ull);
            if (pos < b) M2[pos] = k;
        }
        __syncwarp();
        nM = min(b, nM + nI);
        uint64_t *t = M;
        M = M2;
        M2 = t;
    }
    // N = {n in B : d <= r} (low precision: exact fp32 recheck of the prefix within r + slack)
    int cnt = 0;
    for (int b0 = 0; b0 < nM; b0 += 32) {
        int t = b0 + lane;
        bool in = t < nM && key_dk(M[t]) <= rks;
        cnt += __popc(__ballot_sync(0xffffffffu, in));
    }
    if constexpr (LP) {
        evals += cnt;
        cnt = exact_filter_sort<CPL, UN>(a, qi, M, cnt, rk, s.cid, s.ckey, R);
    }
    const bool cont = !stopped && !overflow && cnt == b && !d.last;
    if (!cont) {
        // finished: append N to the result items
        unsigned long long basepos = 0;
        if (lane == 0 && cnt > 0) basepos = atomicAdd(d.tail, (unsigned long long)cnt);
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        int written = 0;
        for (int t = lane; t < cnt; t += 32) {
            unsigned long long pos = basepos + t;
            if (pos < (unsigned long long)d.cap) {
                d.item_key[pos] = M[t] & ~1ull;
                d.item_slot[pos] = slot;
                written++;
            }
        }
        for (int o = 16; o > 0; o >>= 1) written += __shfl_xor_sync(0xffffffffu, written, o);
        if (lane == 0) {
            d.slot_count[slot] = written;
            d.slot_trunc[slot] = (written < cnt || overflow || (d.last && cnt == b && !stopped)) ? 1 : 0;
        }
    }
    if (cbits) {
        for (int o = 16; o > 0; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
    }
    if (lane == 0) {
        d.status[i] = cont ? 1 : 0;
        d.nv[i] = nvis;
        if (d.nev) d.nev[i] = nev;
        if (a.stats) {
            rr_query_stats *st = a.stats + qi;
            if (d.first) {
                // round 1 repeats the beam phase exactly: replace its counters
                st->visits_beam = nvis;
                st->rounds = 1;
                st->evals = evals;  // distinct: the same ids as the beam phase, already counted
            } else {
                st->visits_beam += nvis;
                st->rounds += 1;
                st->evals += evals;
                st->distinct += distinct;
            }
            st->final_beam = b;
        }
    }
}

// CTA per continuing slot: S_new <- the s_cap_new smallest distinct keys of S_old u V.
__global__ void __launch_bounds__(1024) supdate_kernel(DoublingSUpdate u, int smem_cap) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
    __shared__ int wsum[32];
    for (int j = blockIdx.x; j < u.nc; j += gridDim.x) {
        const int i = u.cont[j];
        const int ns = u.first ? 0 : u.s_cnt_old[i];
        const int ne = u.warm ? u.nev[i] : 0;
        const int nv = u.nv[i];
        const int m = ns + ne + nv;
        uint64_t *a = m <= smem_cap ? sk : u.tmp + (size_t)j * (u.s_cap_old + (u.warm ? u.ev_cap : 0) + u.v_cap);
        const uint64_t *S = u.s_old + (size_t)i * u.s_cap_old;
        const uint64_t *EV = u.warm ? u.ev + (size_t)i * u.ev_cap : nullptr;
        const uint64_t *V = u.v + (size_t)i * u.v_cap;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            if (!u.warm) a[t] = (t < ns ? S[t] : V[t - ns]) & ~1ull;
            // warm restart: E's keys keep their visited bits, this round's visits get theirs
            else a[t] = t < ns ? S[t] : (t < ns + ne ? EV[t - ns] & ~1ull : V[t - ns - ne] | 1ull);
        }
        __syncthreads();
        // bitonic sort with flip stages (min to the lower index; virtual +inf padding)
        int P = 1;
        while (P < m) P <<= 1;
        for (int k = 2; k <= P; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const int lj = __ffs(jj) - 1;  // powers of two: shifts and masks
                for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                    const int off = t & (jj - 1);
                    const int lo = ((t >> lj) << (lj + 1)) + off;
                    const int hi = (jj == (k >> 1)) ? lo - off + (k - 1 - off) : lo + jj;
                    if (hi < m) {
                        uint64_t x = a[lo], y = a[hi];
                        if (y < x) { a[lo] = y; a[hi] = x; }
                    }
                }
                __syncthreads();
            }
        }
        // drop repeated keys (S and V share ids), keep the first s_cap_new distinct ones; warm restart: of the
        // copies of a key (with and without the visited bit) keep the last, which carries the bit if any does
        uint64_t *out = u.s_new + (size_t)j * u.s_cap_new;
        int carry = 0;
        for (int b0 = 0; b0 < m; b0 += blockDim.x) {
            int t = b0 + threadIdx.x;
            int keep;
            if (!u.warm) keep = (t < m && (t == 0 || a[t] != a[t - 1])) ? 1 : 0;
            else keep = (t < m && (t == m - 1 || (a[t] | 1ull) != (a[t + 1] | 1ull))) ? 1 : 0;
            unsigned bm = __ballot_sync(0xffffffffu, keep);
            int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            int pre = __popc(bm & ((1u << lane) - 1));
            if (lane == 0) wsum[w] = __popc(bm);
            __syncthreads();
            int wo = 0;
            for (int x = 0; x < w; x++) wo += wsum[x];
            int tot = 0;
            for (int x = 0; x < (int)(blockDim.x >> 5); x++) tot += wsum[x];
            int pos = carry + wo + pre;
            if (keep && pos < u.s_cap_new) out[pos] = a[t];
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) u.s_cnt_new[j] = carry < u.s_cap_new ? carry : (int)u.s_cap_new;
        __syncthreads();
    }
}

__global__ void zero_words_kernel(uint32_t *p, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) p[t] = 0;
}

template <int DT, int CPL>
rr_status round_t(const DoublingRound &d, cudaStream_t st) {
    const int wpc = 4;
    size_t smem = (size_t)wpc * round_smem_bytes(d.s.R);
    auto k = round_kernel<DT, CPL>;
    RR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<(unsigned)((d.na + wpc - 1) / wpc), 32 * wpc, smem, st>>>(d);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

}  // namespace

rr_status launch_doubling_round(const DoublingRound &d, cudaStream_t st, int dtype_code) {
    if (d.na <= 0) return RR_OK;
    const int cpl = (d.s.row_chunks + 31) / 32;
    switch (dtype_code) {
        case DT_U8: return round_t<DT_U8, 1>(d, st);
        case DT_I8: return round_t<DT_I8, 1>(d, st);
        case DT_F32:
            if (d.s.prec == RR_PREC_BF16) return cpl <= 2 ? round_t<DT_BF16, 2>(d, st) : round_t<DT_BF16, 4>(d, st);
            if (d.s.prec == RR_PREC_FP8) return cpl <= 2 ? round_t<DT_FP8, 2>(d, st) : round_t<DT_FP8, 4>(d, st);
            if (cpl <= 1) return round_t<DT_F32, 1>(d, st);
            if (cpl <= 2) return round_t<DT_F32, 2>(d, st);
            return round_t<DT_F32, 4>(d, st);
    }
    set_error("doubling phase: unsupported element type %d", dtype_code);
    return RR_EINVAL;
}

rr_status launch_doubling_supdate(const DoublingSUpdate &u, cudaStream_t st) {
    if (u.nc <= 0) return RR_OK;
    const int smem_cap = 16384;
    size_t smem = (size_t)smem_cap * 8;
    RR_CUDA(cudaFuncSetAttribute(supdate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int blocks = u.nc < 152 * 2 ? u.nc : 152 * 2;
    supdate_kernel<<<blocks, 1024, smem, st>>>(u, smem_cap);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

rr_status launch_zero_words(uint32_t *p, int64_t n, cudaStream_t st) {
    if (n <= 0) return RR_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    zero_words_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, n);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

}  // namespace rr
