// k_brute.cu -- exact range search by exhaustive scan (Def. 2.1), the ground
// truth against which average precision (Def. 2.2) is measured.
//
// A CTA takes QT queries (kept in shared memory) and 256 points (one per
// thread, streamed from HBM in 16-byte chunks); every thread accumulates QT
// distances in registers.  8-bit data use exact integer arithmetic (dp4a),
// fp32 data FMA in fp32.  Two passes: count matches per query, then (after a
// scan) write keys at per-query cursors; the per-query sort happens in the
// output stage.
#include "rr_common.cuh"

namespace rr {

namespace {

constexpr int QT = 32;

template <int DT>
__global__ void __launch_bounds__(256) brute_kernel(SearchArgs a, int32_t *counts, const int64_t *offsets,
                                                    int32_t *cursor, uint64_t *keys, int fill) {
    using T = typename Acc<DT>::T;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint4 *qs = reinterpret_cast<uint4 *>(smem_raw);  // QT x row_chunks
    const int64_t q0 = (int64_t)blockIdx.y * QT;
    const int nqt = (int)((a.nq - q0) < QT ? (a.nq - q0) : QT);
    for (int i = threadIdx.x; i < QT * a.row_chunks; i += blockDim.x) {
        int qq = i / a.row_chunks, ch = i % a.row_chunks;
        qs[i] = qq < nqt ? ldg16(a.queries + (size_t)(q0 + qq) * a.row_stride + (size_t)ch * 16)
                         : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    T acc[QT];
#pragma unroll
    for (int qq = 0; qq < QT; qq++) acc[qq] = 0;
    const uint8_t *pv = a.vec + (size_t)p * a.row_stride;
    for (int ch = 0; ch < a.row_chunks; ch++) {
        uint4 v = ldg16(pv + (size_t)ch * 16);
#pragma unroll
        for (int qq = 0; qq < QT; qq++) {
            if (a.metric == MET_L2) Acc<DT>::l2(acc[qq], qs[qq * a.row_chunks + ch], v);
            else Acc<DT>::ip(acc[qq], qs[qq * a.row_chunks + ch], v);
        }
    }
#pragma unroll
    for (int qq = 0; qq < QT; qq++) {
        if (qq >= nqt) break;
        const int64_t qi = q0 + qq;
        uint32_t dk = finish_dk(acc[qq], a.metric);
        if (dk <= a.rkey[qi]) {
            if (!fill) {
                atomicAdd(counts + qi, 1);
            } else {
                int64_t pos = offsets[qi] + atomicAdd(cursor + qi, 1);
                if (pos >= offsets[qi + 1]) continue;  // never write past the query's segment
                keys[pos] = make_key(dk, a.ext ? __ldg(a.ext + p) : (uint32_t)p);
            }
        }
    }
}

}  // namespace

rr_status launch_brute(const SearchArgs &a, int32_t *counts, const int64_t *offsets, int32_t *cursor, uint64_t *keys,
                       int fill, cudaStream_t st, int dtype_code) {
    if (a.nq == 0 || a.n == 0) return RR_OK;
    dim3 grid((unsigned)((a.n + 255) / 256), (unsigned)((a.nq + QT - 1) / QT));
    if (grid.y > 65535) {
        set_error("brute force: batch too large for one launch (nq=%lld)", (long long)a.nq);
        return RR_EINVAL;
    }
    size_t smem = (size_t)QT * a.row_chunks * 16;
    switch (dtype_code) {
        case DT_U8:
            RR_CUDA(cudaFuncSetAttribute(brute_kernel<DT_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            brute_kernel<DT_U8><<<grid, 256, smem, st>>>(a, counts, offsets, cursor, keys, fill);
            break;
        case DT_I8:
            RR_CUDA(cudaFuncSetAttribute(brute_kernel<DT_I8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            brute_kernel<DT_I8><<<grid, 256, smem, st>>>(a, counts, offsets, cursor, keys, fill);
            break;
        case DT_F32:
            RR_CUDA(cudaFuncSetAttribute(brute_kernel<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            brute_kernel<DT_F32><<<grid, 256, smem, st>>>(a, counts, offsets, cursor, keys, fill);
            break;
        default:
            set_error("brute force: unsupported element type %d", dtype_code);
            return RR_EINVAL;
    }
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

}  // namespace rr
