// k_output.cu -- assembly of the per-query results into one CSR (the output
// of Alg. 6 / Alg. 3 for the whole batch): count -> exclusive scan -> copy or
// scatter -> per-query sort by (distance, id) -> decode keys into ids and
// distances.
#include <algorithm>

#include "rr_common.cuh"

namespace rr {

namespace {

// Exclusive scan of int32 counts into int64 offsets[0..n], one CTA, chunked.
__global__ void __launch_bounds__(1024) scan_kernel(const int32_t *counts, int64_t n, int64_t *offsets) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t i = base + t;
        int64_t v = i < n ? (int64_t)counts[i] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;  // inclusive prefix of warp sums
        }
        __syncthreads();
        int64_t incl = x + (w > 0 ? wsum[w - 1] : 0) + carry;
        if (i < n) offsets[i] = incl - v;
        __syncthreads();
        if (t == 1023) carry = incl;
        __syncthreads();
    }
    if (t == 0) offsets[n] = carry;
}

__device__ __forceinline__ void decode_to(const OutArgs &o, int64_t pos, uint64_t k) {
    if (pos < 0 || pos >= o.total) {  // never write outside the result arrays
        atomicExch(o.error, 4);
        return;
    }
    const uint32_t id = key_id(k);
    o.ids[pos] = o.ext ? __ldg(o.ext + id) : id;
    uint32_t dk = key_dk(k);
    if (o.dist_is_float) reinterpret_cast<float *>(o.dists)[pos] = dval_f32(dk);
    else reinterpret_cast<int32_t *>(o.dists)[pos] = dval_i32(dk);
}

// Warp per listed slot: copy `count[slot]` sorted keys from keys[slot*stride]
// to the CSR range of query qlist[slot] (qlist == nullptr: slot = query, and
// queries flagged RR_FLAG_PHASE2 are skipped -- their results come later).
__global__ void copy_slots_kernel(OutArgs o, const uint64_t *keys, int64_t stride, const int32_t *count,
                                  const int32_t *qlist, int32_t nlist) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nlist; s += nw) {
        int64_t q = qlist ? qlist[s] : s;
        if (!qlist && (o.flags[q] & RR_FLAG_PHASE2)) continue;
        int32_t c = count[s];
        int64_t off = o.offsets[q];
        const uint64_t *src = keys + (size_t)s * stride;
        for (int i = lane; i < c; i += 32) decode_to(o, off + i, src[i]);
    }
}

// Items to the CSR segments of their queries (unsorted within a segment).  Items come in runs of one
// slot, so the first lane of each run in a warp reserves the run's positions with one atomic.
__global__ void scatter_items_kernel(OutArgs o, const uint64_t *item_key, const int32_t *item_slot, int64_t nitems,
                                     const int32_t *qlist, int32_t *cursor, uint64_t *tmp) {
    const int lane = lane_id();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < nitems; base += stride) {
        const int64_t t = base + lane;
        const bool ok = t < nitems;
        const int32_t s = ok ? item_slot[t] : -1;
        const int32_t prev = __shfl_up_sync(0xffffffffu, s, 1);
        const bool head = ok && (lane == 0 || prev != s);
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        int32_t r0 = 0;
        if (head) {
            const unsigned later = hm & ~((2u << lane) - 1u);
            const int stop = later ? __ffs(later) - 1 : (nitems - base < 32 ? (int)(nitems - base) : 32);
            r0 = atomicAdd(cursor + s, stop - lane);
        }
        // the head of this lane's run: the last head at or before the lane (lane 0 is one when ok)
        const unsigned upto = hm & ((2u << lane) - 1u);
        const int h = upto ? 31 - __clz(upto) : 0;
        r0 = __shfl_sync(0xffffffffu, r0, h);
        if (!ok) continue;
        const int64_t q = qlist[s];
        const int64_t pos = o.offsets[q] + r0 + (lane - h);
        if (pos < 0 || pos >= o.offsets[q + 1]) {
            atomicExch(o.error, 4);
            continue;
        }
        tmp[pos] = item_key[t];
    }
}

// Bitonic sort with "flip" first stages, so every compare puts the smaller key
// at the lower index and a virtual +inf padding past m never moves.  The
// stages whose pairs lie inside one 64-key region (every stage of the levels
// k <= 64, and the j <= 32 stages of every later level) run in registers: a
// warp holds a region as keys r + lane and r + 32 + lane and exchanges them by
// shuffles, so only the j >= 64 stages go through memory with a block barrier.

// one stage on a warp's 64-key region (x = key lane, y = key 32 + lane)
__device__ __forceinline__ void region_stage(uint64_t &x, uint64_t &y, int lane, int k, int j) {
    const bool flip = j == (k >> 1);
    if (j == 32) {
        if (flip) {  // k = 64: key lane pairs with key 63 - lane, the y of lane 31 - lane
            const uint64_t oy = __shfl_xor_sync(0xffffffffu, y, 31);
            const uint64_t ox = __shfl_xor_sync(0xffffffffu, x, 31);
            x = oy < x ? oy : x;
            y = ox > y ? ox : y;
        } else {
            const uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
            x = lo;
            y = hi;
        }
    } else {
        const int partner = flip ? k - 1 : j;  // pair (t, t ^ (k-1)) or (t, t + j), both within 32 keys
        const uint64_t ox = __shfl_xor_sync(0xffffffffu, x, partner);
        const uint64_t oy = __shfl_xor_sync(0xffffffffu, y, partner);
        const bool upper = (lane & j) != 0;  // the higher index of the pair keeps the larger key
        x = upper ? (ox > x ? ox : x) : (ox < x ? ox : x);
        y = upper ? (oy > y ? oy : y) : (oy < y ? oy : y);
    }
}

// stages (k, j) for j from j_hi down to 1 on every 64-key region (keys past m read as +inf, not stored)
__device__ __forceinline__ void region_pass(uint64_t *a, int m, int P, int k, int j_hi, bool levels_upto_64) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < (P >> 6); r += nw) {
        const int i0 = (r << 6) + lane, i1 = i0 + 32;
        uint64_t x = i0 < m ? a[i0] : ~0ull, y = i1 < m ? a[i1] : ~0ull;
        if (levels_upto_64) {
#pragma unroll
            for (int kk = 2; kk <= 64; kk <<= 1)
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) region_stage(x, y, lane, kk, j);
        } else {
#pragma unroll
            for (int j = 32; j > 0; j >>= 1)
                if (j <= j_hi) region_stage(x, y, lane, k, j);
        }
        if (i0 < m) a[i0] = x;
        if (i1 < m) a[i1] = y;
    }
}

__device__ void bitonic_sort_smem(uint64_t *a, int m) {
    int P = 64;
    while (P < m) P <<= 1;
    region_pass(a, m, P, 64, 32, true);
    __syncthreads();
    for (int k = 128; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 64; j >>= 1) {
            const int lj = __ffs(j) - 1;  // j and k are powers of two: shifts and masks, no divisions
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                // i-th compare pair of this stage
                const int off = i & (j - 1);
                const int lo = ((i >> lj) << (lj + 1)) + off;
                // flip stage: pair (x, x ^ (k-1)) inside each k-block; otherwise (x, x + j)
                const int hi = (j == (k >> 1)) ? lo - off + (k - 1 - off) : lo + j;
                if (hi < m) {
                    uint64_t x = a[lo], y = a[hi];
                    if (y < x) { a[lo] = y; a[hi] = x; }
                }
            }
            __syncthreads();
        }
        region_pass(a, m, P, k, 32, false);
        __syncthreads();
    }
}

// CTA per listed query: sort its CSR segment of tmp keys and decode it.
// Segments up to smem_cap keys are sorted in shared memory, longer ones in
// place in global memory with the same network.
__global__ void __launch_bounds__(1024) sort_segments_kernel(OutArgs o, uint64_t *tmp, const int32_t *qlist,
                                                             int32_t nlist, int smem_cap) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
    for (int32_t s = blockIdx.x; s < nlist; s += gridDim.x) {
        int64_t q = qlist[s];
        int64_t off = o.offsets[q];
        int m = (int)(o.offsets[q + 1] - off);
        if (m <= 0) continue;
        uint64_t *seg = tmp + off;
        uint64_t *a = seg;
        if (m <= smem_cap) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) sk[i] = seg[i];
            __syncthreads();
            a = sk;
        }
        bitonic_sort_smem(a, m);
        for (int i = threadIdx.x; i < m; i += blockDim.x) decode_to(o, off + i, a[i]);
        __syncthreads();
    }
}

}  // namespace

rr_status launch_scan(const int32_t *counts, int64_t n, int64_t *offsets, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(counts, n, offsets);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

rr_status launch_copy_slots(const OutArgs &o, const uint64_t *keys, int64_t stride, const int32_t *count,
                            const int32_t *qlist, int32_t nlist, cudaStream_t st) {
    if (nlist <= 0) return RR_OK;
    int64_t blocks = (nlist + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    copy_slots_kernel<<<(unsigned)blocks, 256, 0, st>>>(o, keys, stride, count, qlist, nlist);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

rr_status launch_scatter_items(const OutArgs &o, const uint64_t *item_key, const int32_t *item_slot, int64_t nitems,
                               const int32_t *qlist, int32_t *cursor, uint64_t *tmp, cudaStream_t st) {
    if (nitems <= 0) return RR_OK;
    int64_t blocks = (nitems + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    scatter_items_kernel<<<(unsigned)blocks, 256, 0, st>>>(o, item_key, item_slot, nitems, qlist, cursor, tmp);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

rr_status launch_sort_segments(const OutArgs &o, uint64_t *tmp, const int32_t *qlist, int32_t nlist, int64_t,
                               cudaStream_t st) {
    if (nlist <= 0) return RR_OK;
    // keys: the largest shared-memory block a CTA may take (227 KB), so segments of up to 29,056 results
    // are sorted on chip; longer ones in place in global memory.  (Size classes in three launches with
    // smaller blocks for short segments measured slower: each launch has its own tail.)
    int dev = 0, optin = 0;
    RR_CUDA(cudaGetDevice(&dev));
    RR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int smem_cap = std::max(4096, optin / 8);
    size_t smem = (size_t)smem_cap * 8;
    RR_CUDA(cudaFuncSetAttribute(sort_segments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int blocks = nlist < 152 * 2 ? nlist : 152 * 2;
    sort_segments_kernel<<<blocks, 1024, smem, st>>>(o, tmp, qlist, nlist, smem_cap);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

}  // namespace rr
