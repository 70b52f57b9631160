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
    const int lpv = a.lpv, sub = lane & (lpv - 1), grp = lane / lpv, ngrp = 32 / lpv;
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

}  // namespace rr
