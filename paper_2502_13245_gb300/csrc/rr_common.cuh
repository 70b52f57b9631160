// rr_common.cuh -- device helpers shared by the librr kernels (CUDA path only).
//
// Ordering keys.  Every ordered structure of the method (the beam B of Alg. 1,
// the argmin of Alg. 1/2, the trim to b, the output order) uses the pair
// (distance, id).  A key packs it into 64 bits so that one unsigned compare
// orders it:
//     key = dkey(dist) << 32 | id << 1 | visited
// dkey maps an int32 or fp32 distance to a uint32 with the same order.  The
// low "visited" bit marks V membership of beam entries; compares that must
// ignore it use (key | 1).  Ids are < 2^31.
#pragma once
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rr {

constexpr uint32_t kSent = 0xFFFFFFFFu;
constexpr uint64_t kEmpty = ~0ull;

enum { DT_U8 = 0, DT_I8 = 1, DT_F32 = 2, DT_BF16 = 3, DT_FP8 = 4 };
enum { MET_L2 = 0, MET_IP = 1 };

__host__ __device__ __forceinline__ uint32_t dkey_i32(int32_t d) { return (uint32_t)d ^ 0x80000000u; }
__host__ __device__ __forceinline__ int32_t dval_i32(uint32_t k) { return (int32_t)(k ^ 0x80000000u); }
__device__ __forceinline__ uint32_t dkey_f32(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float dval_f32(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
// The distance an order key encodes (exact for int32 distances).
__device__ __forceinline__ double dkey_value(uint32_t dk, bool fp) {
    if (!fp) return (double)(int32_t)(dk ^ 0x80000000u);
    const uint32_t b = (dk & 0x80000000u) ? (dk & 0x7fffffffu) : ~dk;
    return (double)__uint_as_float(b);
}

__host__ __device__ __forceinline__ uint64_t make_key(uint32_t dk, uint32_t id) {
    return ((uint64_t)dk << 32) | ((uint64_t)id << 1);
}
__host__ __device__ __forceinline__ uint32_t key_id(uint64_t k) { return ((uint32_t)k) >> 1; }
__host__ __device__ __forceinline__ uint32_t key_dk(uint64_t k) { return (uint32_t)(k >> 32); }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// -------------------------------------------------------------------------------------------
// distances over 16-byte chunks.  A lane accumulates the chunks it owns, then
// the lanes of a vector group (LPV lanes) are combined with xor shuffles.
// Integer data: exact int32 (dp4a on |a-b| for L2, dp4a on a*b for IP).
// fp32 data: FMA in fp32.
// -------------------------------------------------------------------------------------------
template <int DT>
struct Acc;

template <>
struct Acc<DT_U8> {
    using T = int32_t;
    __device__ __forceinline__ static void l2(T &s, const uint4 &a, const uint4 &b) {
        uint32_t x;
        x = __vabsdiffu4(a.x, b.x); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffu4(a.y, b.y); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffu4(a.z, b.z); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffu4(a.w, b.w); s = (T)__dp4a(x, x, (uint32_t)s);
    }
    __device__ __forceinline__ static void ip(T &s, const uint4 &a, const uint4 &b) {
        s = (T)__dp4a(a.x, b.x, (uint32_t)s);
        s = (T)__dp4a(a.y, b.y, (uint32_t)s);
        s = (T)__dp4a(a.z, b.z, (uint32_t)s);
        s = (T)__dp4a(a.w, b.w, (uint32_t)s);
    }
};

template <>
struct Acc<DT_I8> {
    using T = int32_t;
    __device__ __forceinline__ static void l2(T &s, const uint4 &a, const uint4 &b) {
        uint32_t x;
        x = __vabsdiffs4(a.x, b.x); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffs4(a.y, b.y); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffs4(a.z, b.z); s = (T)__dp4a(x, x, (uint32_t)s);
        x = __vabsdiffs4(a.w, b.w); s = (T)__dp4a(x, x, (uint32_t)s);
    }
    __device__ __forceinline__ static void ip(T &s, const uint4 &a, const uint4 &b) {
        s = __dp4a((int)a.x, (int)b.x, s);
        s = __dp4a((int)a.y, (int)b.y, s);
        s = __dp4a((int)a.z, (int)b.z, s);
        s = __dp4a((int)a.w, (int)b.w, s);
    }
};

template <>
struct Acc<DT_F32> {
    using T = float;
    __device__ __forceinline__ static void l2(T &s, const uint4 &a, const uint4 &b) {
        float t;
        t = __uint_as_float(a.x) - __uint_as_float(b.x); s = fmaf(t, t, s);
        t = __uint_as_float(a.y) - __uint_as_float(b.y); s = fmaf(t, t, s);
        t = __uint_as_float(a.z) - __uint_as_float(b.z); s = fmaf(t, t, s);
        t = __uint_as_float(a.w) - __uint_as_float(b.w); s = fmaf(t, t, s);
    }
    __device__ __forceinline__ static void ip(T &s, const uint4 &a, const uint4 &b) {
        s = fmaf(__uint_as_float(a.x), __uint_as_float(b.x), s);
        s = fmaf(__uint_as_float(a.y), __uint_as_float(b.y), s);
        s = fmaf(__uint_as_float(a.z), __uint_as_float(b.z), s);
        s = fmaf(__uint_as_float(a.w), __uint_as_float(b.w), s);
    }
};

// Final distance -> order key.  L2: the sum; IP: minus the sum (Sec. 2).
__device__ __forceinline__ uint32_t finish_dk(int32_t s, int metric) { return dkey_i32(metric == MET_L2 ? s : -s); }
__device__ __forceinline__ uint32_t finish_dk(float s, int metric) { return dkey_f32(metric == MET_L2 ? s : -s); }

template <typename T>
__device__ __forceinline__ T group_sum(T v, int lpv) {
    for (int o = lpv >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint4 ldg16(const uint8_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// Fibonacci hashing of an id into a table of 2^lg slots.
__device__ __forceinline__ uint32_t hslot(uint32_t id, int lg) { return (id * 2654435761u) >> (32 - lg); }

}  // namespace rr

#include "rr_internal.h"

namespace rr {

// Load the query chunks this lane owns (chunk sub + c*lpv for c < CPL).
template <int CPL>
__device__ __forceinline__ void load_query(const SearchArgs &a, const uint8_t *qp, uint4 (&q)[CPL]) {
    const int sub = lane_id() & (a.lpv - 1);
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        int ch = sub + c * a.lpv;
        q[c] = ch < a.row_chunks ? ldg16(qp + (size_t)ch * 16) : make_uint4(0, 0, 0, 0);
    }
}

// Evaluate d(q, cid[c]) for c in [0, nc) with the whole warp: lane groups of
// lpv lanes each take one candidate, UN candidates per group are loaded before
// any is reduced (memory-level parallelism).  Writes ckey[c] = key(dist, id).
// Every lane of the warp must call this (shuffles use the full mask).
template <int DT, int CPL, int UN>
__device__ __forceinline__ void eval_candidates(const SearchArgs &a, const uint4 (&q)[CPL], const uint32_t *cid,
                                                int nc, uint64_t *ckey) {
    using T = typename Acc<DT>::T;
    const int lane = lane_id();
    const int lpv = a.lpv, sub = lane & (lpv - 1), grp = lane >> (__ffs(lpv) - 1), ngrp = 32 >> (__ffs(lpv) - 1);
    for (int c0 = 0; c0 < nc; c0 += ngrp * UN) {
        uint4 v[UN][CPL];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            int c = c0 + grp + ngrp * u;
            const uint8_t *p = a.vec + (size_t)(c < nc ? cid[c] : 0u) * a.row_stride;
#pragma unroll
            for (int k = 0; k < CPL; k++) {
                int ch = sub + k * lpv;
                v[u][k] = (c < nc && ch < a.row_chunks) ? ldg16(p + (size_t)ch * 16) : make_uint4(0, 0, 0, 0);
            }
        }
        if constexpr (std::is_integral<T>::value) {
            // Integer sums do not depend on their order, so the UN partial sums of a lane group are
            // reduced by a reduce-scatter: each exchange with the partner lane halves the values a
            // lane holds, and lane `sub` ends with the totals of candidates base .. base + cnt - 1
            // (log2 UN shuffles per lane instead of UN * log2 lpv).
            T s[UN];
#pragma unroll
            for (int u = 0; u < UN; u++) {
                s[u] = 0;
#pragma unroll
                for (int k = 0; k < CPL; k++) {
                    if (a.metric == MET_L2) Acc<DT>::l2(s[u], q[k], v[u][k]);
                    else Acc<DT>::ip(s[u], q[k], v[u][k]);
                }
            }
            int base = 0, m = lpv >> 1;
#pragma unroll
            for (int hh = UN >> 1; hh >= 1; hh >>= 1) {
                if (m >= 1) {  // warp-uniform
                    const bool up = (sub & m) != 0;
#pragma unroll
                    for (int i = 0; i < hh; i++) {
                        const T send = up ? s[i] : s[i + hh];
                        const T keep = up ? s[i + hh] : s[i];
                        s[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                    }
                    if (up) base += hh;
                    m >>= 1;
                }
            }
            for (; m >= 1; m >>= 1) s[0] += __shfl_xor_sync(0xffffffffu, s[0], m);  // lpv > UN
            const int cnt = lpv >= UN ? 1 : UN / lpv;
            const bool writer = lpv <= UN || (sub & (lpv / UN - 1)) == 0;
#pragma unroll
            for (int i = 0; i < UN; i++) {
                if (i >= cnt) break;  // warp-uniform
                const int c = c0 + grp + ngrp * (base + i);
                if (writer && c < nc) ckey[c] = make_key(finish_dk(s[i], a.metric), cid[c]);
            }
        } else {
            // fp32: one fixed summation tree (the one eval_one uses), so an id evaluated twice gets
            // the same key
#pragma unroll
            for (int u = 0; u < UN; u++) {
                if (c0 + ngrp * u >= nc) break;  // warp-uniform
                T s = 0;
#pragma unroll
                for (int k = 0; k < CPL; k++) {
                    if (a.metric == MET_L2) Acc<DT>::l2(s, q[k], v[u][k]);
                    else Acc<DT>::ip(s, q[k], v[u][k]);
                }
                s = group_sum(s, lpv);
                int c = c0 + grp + ngrp * u;
                if (sub == 0 && c < nc) ckey[c] = make_key(finish_dk(s, a.metric), cid[c]);
            }
        }
    }
}

// Distance of q to one point, computed by every lane group (all get the same value).
template <int DT, int CPL>
__device__ __forceinline__ uint32_t eval_one(const SearchArgs &a, const uint4 (&q)[CPL], uint32_t id) {
    using T = typename Acc<DT>::T;
    const int sub = lane_id() & (a.lpv - 1);
    const uint8_t *p = a.vec + (size_t)id * a.row_stride;
    T s = 0;
#pragma unroll
    for (int k = 0; k < CPL; k++) {
        int ch = sub + k * a.lpv;
        uint4 v = ch < a.row_chunks ? ldg16(p + (size_t)ch * 16) : make_uint4(0, 0, 0, 0);
        if (a.metric == MET_L2) Acc<DT>::l2(s, q[k], v);
        else Acc<DT>::ip(s, q[k], v);
    }
    s = group_sum(s, a.lpv);
    return finish_dk(s, a.metric);
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Exact distinct-id accounting (stats mode): returns 1 if id was not marked yet.
__device__ __forceinline__ int mark_bit(uint32_t *bits, uint32_t id) {
    uint32_t m = 1u << (id & 31);
    return (atomicOr(bits + (id >> 5), m) & m) ? 0 : 1;
}

// -------------------------------------------------------------------------------------------
// Low-precision traversal (fp32 indexes).  A traversal row is split in 16-byte
// chunks over lp_lpv lanes: a chunk holds 8 BF16 or 16 FP8 values.  The lane
// keeps the fp32 query values of its chunk in qf[16] (one chunk per lane, so
// d <= 256 for BF16 and d <= 512 for FP8).  Products are accumulated in fp32.
// -------------------------------------------------------------------------------------------
__host__ __device__ constexpr bool is_lowp(int DT) { return DT == DT_BF16 || DT == DT_FP8; }

template <int DT>
__device__ __forceinline__ void load_query_lp(const SearchArgs &a, const float *qrow, float (&qf)[16]) {
    constexpr int E = DT == DT_BF16 ? 8 : 16;
    const int sub = lane_id() & (a.lp_lpv - 1);
#pragma unroll
    for (int j = 0; j < 16; j++) qf[j] = 0.f;
#pragma unroll
    for (int k = 0; k < 1; k++) {  // one chunk per lane: lp_chunks <= 32
        const int ch = sub + k * a.lp_lpv;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int e = ch * E + j;
            qf[k * E + j] = (ch < a.lp_chunks && e < a.d) ? qrow[e] : 0.f;
        }
    }
}

// ||q||^2 from the lane-distributed query values (every lane group holds the whole query)
__device__ __forceinline__ float query_norm2_lp(const SearchArgs &a, const float (&qf)[16]) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 16; j++) s = fmaf(qf[j], qf[j], s);
    return group_sum(s, a.lp_lpv);
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// one 16-byte chunk against 16 query values starting at qf[o]: BF16 -> L2 or dot, FP8 -> dot
template <int DT>
__device__ __forceinline__ void lp_chunk(const uint4 &v, const float *q, bool l2, float &acc) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    if (DT == DT_BF16) {
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const float x0 = bf16_lo(w[t]), x1 = bf16_hi(w[t]);
            if (l2) {
                const float d0 = q[2 * t] - x0, d1 = q[2 * t + 1] - x1;
                acc = fmaf(d0, d0, acc);
                acc = fmaf(d1, d1, acc);
            } else {
                acc = fmaf(q[2 * t], x0, acc);
                acc = fmaf(q[2 * t + 1], x1, acc);
            }
        }
    } else {
#pragma unroll
        for (int t = 0; t < 4; t++) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const __nv_fp8x2_storage_t pr = (__nv_fp8x2_storage_t)((w[t] >> (16 * h)) & 0xffffu);
                const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3);
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&hr));
                acc = fmaf(q[4 * t + 2 * h], f.x, acc);
                acc = fmaf(q[4 * t + 2 * h + 1], f.y, acc);
            }
        }
    }
}

// Approximate distances of q to cid[0..nc) through the traversal rows; writes key(d~, id).
template <int DT, int UN>
__device__ __forceinline__ void eval_candidates_lp(const SearchArgs &a, const float (&qf)[16], float qn2,
                                                   const uint32_t *cid, int nc, uint64_t *ckey) {
    constexpr int E = DT == DT_BF16 ? 8 : 16;
    constexpr int CH = 1;  // chunks per lane (lp_chunks <= 32)
    const int lane = lane_id();
    const int lpv = a.lp_lpv, sub = lane & (lpv - 1), grp = lane >> (__ffs(lpv) - 1), ngrp = 32 >> (__ffs(lpv) - 1);
    const bool l2 = a.metric == MET_L2;
    for (int c0 = 0; c0 < nc; c0 += ngrp * UN) {
        uint4 v[UN][CH];
        float2 inf[UN];
#pragma unroll
        for (int u = 0; u < UN; u++) {
            const int c = c0 + grp + ngrp * u;
            const uint32_t id = c < nc ? cid[c] : 0u;
            const uint8_t *p = a.lp_vec + (size_t)id * a.lp_stride;
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int ch = sub + k * lpv;
                v[u][k] = (c < nc && ch < a.lp_chunks) ? ldg16(p + (size_t)ch * 16) : make_uint4(0, 0, 0, 0);
            }
            inf[u] = (DT == DT_FP8 && c < nc) ? __ldg(a.lp_info + id) : make_float2(1.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < UN; u++) {
            if (c0 + ngrp * u >= nc) break;  // warp-uniform
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < CH; k++) lp_chunk<DT>(v[u][k], qf + k * E, DT == DT_BF16 && l2, s);
            s = group_sum(s, lpv);
            float dist;
            if (DT == DT_BF16) dist = l2 ? s : -s;
            else dist = l2 ? (qn2 - 2.f * inf[u].x * s + inf[u].y) : -(inf[u].x * s);
            const int c = c0 + grp + ngrp * u;
            if (sub == 0 && c < nc) ckey[c] = make_key(dkey_f32(dist), cid[c]);
        }
    }
}

// Approximate distance to one point, every lane group gets the value.
template <int DT>
__device__ __forceinline__ uint32_t eval_one_lp(const SearchArgs &a, const float (&qf)[16], float qn2, uint32_t id) {
    constexpr int E = DT == DT_BF16 ? 8 : 16;
    constexpr int CH = 1;
    const int sub = lane_id() & (a.lp_lpv - 1);
    const bool l2 = a.metric == MET_L2;
    const uint8_t *p = a.lp_vec + (size_t)id * a.lp_stride;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CH; k++) {
        const int ch = sub + k * a.lp_lpv;
        const uint4 v = ch < a.lp_chunks ? ldg16(p + (size_t)ch * 16) : make_uint4(0, 0, 0, 0);
        lp_chunk<DT>(v, qf + k * E, DT == DT_BF16 && l2, s);
    }
    s = group_sum(s, a.lp_lpv);
    if (DT == DT_BF16) return dkey_f32(l2 ? s : -s);
    const float2 inf = __ldg(a.lp_info + id);
    return dkey_f32(l2 ? (qn2 - 2.f * inf.x * s + inf.y) : -(inf.x * s));
}

// Key of r + slack: an approximate distance above it proves the exact one is above r.
__device__ __forceinline__ uint32_t slack_key(const SearchArgs &a, uint32_t rk, float qn2) {
    const float r = dval_f32(rk);
    const float qn = sqrtf(qn2);
    const float slack = a.rel_eps > 0.f ? a.rel_eps * fabsf(r) : (a.slackA * qn + a.slackB * qn2 + a.slackC);
    return dkey_f32(r + slack);
}

// Sort keys[0..m) (shared or global memory) ascending with the warp: bitonic
// network with flip stages, virtual +inf padding past m.
__device__ __forceinline__ void warp_sort_keys(uint64_t *keys, int m) {
    const int lane = lane_id();
    int P = 1;
    while (P < m) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int lj = __ffs(j) - 1;  // powers of two: shifts and masks
            for (int i = lane; i < P / 2; i += 32) {
                const int off = i & (j - 1);
                const int lo = ((i >> lj) << (lj + 1)) + off;
                const int hi = (j == (k >> 1)) ? lo - off + (k - 1 - off) : lo + j;
                if (hi < m) {
                    const uint64_t x = keys[lo], y = keys[hi];
                    if (y < x) {
                        keys[lo] = y;
                        keys[hi] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The exact recheck of the precision form: keys[0..m) hold approximate keys
// (visited bits ignored); replace them, in place, by the exact keys of the
// points whose exact fp32 distance is <= r (rk), sorted by (dist, id).
// cid/ckey are R-entry scratch.  Returns the count.  Whole warp.
template <int CPL, int UN>
__device__ int exact_filter_sort(const SearchArgs &a, int64_t qi, uint64_t *keys, int m, uint32_t rk, uint32_t *cid,
                                 uint64_t *ckey, int R) {
    const int lane = lane_id();
    uint4 q32[CPL];
    load_query<CPL>(a, a.queries + (size_t)qi * a.row_stride, q32);
    int cnt = 0;
    for (int base = 0; base < m; base += R) {
        const int mm = min(R, m - base);
        for (int t = lane; t < mm; t += 32) cid[t] = key_id(keys[base + t]);
        __syncwarp();
        eval_candidates<DT_F32, CPL, UN>(a, q32, cid, mm, ckey);
        __syncwarp();
        for (int t0 = 0; t0 < mm; t0 += 32) {
            const int t = t0 + lane;
            const uint64_t k = t < mm ? ckey[t] : kEmpty;
            const bool in = t < mm && key_dk(k) <= rk;
            const unsigned msk = __ballot_sync(0xffffffffu, in);
            if (in) keys[cnt + __popc(msk & lanemask_lt())] = k;  // cnt <= base + t0: never ahead of the reads
            cnt += __popc(msk);
        }
        __syncwarp();
    }
    warp_sort_keys(keys, cnt);
    return cnt;
}

}  // namespace rr
