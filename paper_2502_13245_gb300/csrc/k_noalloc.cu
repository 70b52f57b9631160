// k_noalloc.cu -- rr_beam_search_noalloc: the beam search of rr_range_search
// (RR_BEAM / RR_BEAM_ES) for callers that must not allocate memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// host callback, on a thread that works under a fixed, pre-reserved memory
// budget owned by someone else (an inference server's allocator), or under a
// policy that forbids any allocation after start-up.
// rr_range_search allocates its result arrays and grows per-index scratch, so
// those callers cannot use it.  This entry point writes into output arrays the
// caller already owns and keeps its intermediate data in one file-scope device
// array, g_scratch, of fixed size.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// The array is a static __device__ variable: every GPU that loads librr.so
// holds kNoAllocScratchBytes of it until the process exits.  In host code the
// name g_scratch is only a stand-in, not a device address, so the host looks
// its address up once per device with cudaGetSymbolAddress (with that device
// current) and passes that pointer to the kernels.  The first call on a device
// does this look-up; make that first call before any stream capture.
//
// All calls share the array and it keeps the last call's contents, so every
// call re-initialises what must start from zero.  Calls whose work overlaps
// on the GPU (different streams, or different host threads) race on the array
// and must be serialised by the caller.  Before returning, the call waits for
// its stream to finish the work (it reads the device guard word back).
//
// Parameters are those of rr_range_search for RR_BEAM / RR_BEAM_ES: the beam,
// the Alg. 5 / Alg. 4 early-stop settings (every metric), the launch shape
// (tile_hint, seen_log2, persistent); results are equal for equal settings.
// Low-precision traversal is refused (its traversal copies are allocated on
// first use), as are per-query radii.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "rr_common.cuh"

namespace rr {

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
uint8_t *g_addr[kMaxDevices] = {};

rr_status scratch_address(int dev, uint8_t **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("rr_beam_search_noalloc: device %d out of range", dev);
        return RR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);  // the caller made `dev` current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
        g_addr[dev] = (uint8_t *)p;
    }
    *out = g_addr[dev];
    return RR_OK;
}

size_t ru(size_t x) { return (x + 255) & ~size_t(255); }

// radius keys for every query, and the counters that must start at zero
__global__ void init_kernel(uint32_t *rkey, uint32_t *eskey, int64_t nq, uint32_t rk, uint32_t ek, int32_t *counters) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        rkey[i] = rk;
        eskey[i] = ek;
    }
    if (blockIdx.x == 0 && threadIdx.x < 64) counters[threadIdx.x] = 0;
}

// N of every query (sorted keys) -> the caller's fixed-stride outputs; slots past
// the count get id 0xFFFFFFFF and distance 0.
__global__ void emit_kernel(const uint64_t *keys, const int32_t *count, int64_t nq, int b, int is_float,
                            const uint32_t *ext, int32_t *out_counts, uint32_t *out_ids, void *out_dists) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nq; q += nw) {
        const int c = count[q];
        if (lane == 0) out_counts[q] = c;
        for (int i = lane; i < b; i += 32) {
            const size_t o = (size_t)q * b + i;
            uint64_t k = i < c ? keys[o] : 0;
            out_ids[o] = i < c ? (ext ? __ldg(ext + key_id(k)) : key_id(k)) : kSent;
            if (is_float) reinterpret_cast<float *>(out_dists)[o] = i < c ? dval_f32(key_dk(k)) : 0.f;
            else reinterpret_cast<int32_t *>(out_dists)[o] = i < c ? dval_i32(key_dk(k)) : 0;
        }
    }
}

}  // namespace

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_beam_search_noalloc(rr_index *ix, const void *queries, int64_t nq, double radius,
                                            int32_t variant, const rr_params *params, void *stream,
                                            int32_t *out_counts, uint32_t *out_ids, void *out_dists) {
    if (!ix) { set_error("rr_beam_search_noalloc: index is NULL"); return RR_EINVAL; }
    if (variant != RR_BEAM && variant != RR_BEAM_ES) {
        set_error("rr_beam_search_noalloc: variant must be RR_BEAM or RR_BEAM_ES");
        return RR_EINVAL;
    }
    if (nq < 0 || nq >= ((int64_t)1 << 31)) { set_error("rr_beam_search_noalloc: bad nq"); return RR_EINVAL; }
    if (nq == 0) return RR_OK;
    if (!queries || !out_counts || !out_ids || !out_dists) {
        set_error("rr_beam_search_noalloc: NULL array");
        return RR_EINVAL;
    }
    rr_params P;
    if (params) P = *params;
    else rr_params_init(&P);
    if (P.beam < 1 || P.beam > 512) { set_error("rr_beam_search_noalloc: beam=%d out of [1, 512]", P.beam); return RR_EINVAL; }
    if (P.es_visit_limit < 0) { set_error("rr_beam_search_noalloc: es_visit_limit < 0"); return RR_EINVAL; }
    if (P.es_metric < RR_ES_VISITED || P.es_metric > RR_ES_TOP10_RATIO) {
        set_error("rr_beam_search_noalloc: unknown early-stopping metric %d", P.es_metric);
        return RR_EINVAL;
    }
    if (variant == RR_BEAM_ES && P.es_metric == RR_ES_TOP10_RATIO && (P.es_radius_mode != 1 || ix->metric != RR_L2)) {
        set_error("rr_beam_search_noalloc: the d_top10 / d_start metric takes its ratio from es_radius "
                  "(es_radius_mode = 1) and needs squared L2");
        return RR_EINVAL;
    }
    if (P.expand < 0 || P.expand > 4) {
        set_error("rr_beam_search_noalloc: expand=%d out of [0, 4]", P.expand);
        return RR_EINVAL;
    }
    if (P.precision != RR_PREC_EXACT) {
        // the BF16 / FP8 traversal copies are built (allocated) on first use
        set_error("rr_beam_search_noalloc: only exact traversal (precision = RR_PREC_EXACT) allocates nothing");
        return RR_EINVAL;
    }
    DeviceGuard dg(ix->device);
    if (!is_device_ptr(queries) || !is_device_ptr(out_counts) || !is_device_ptr(out_ids) || !is_device_ptr(out_dists)) {
        set_error("rr_beam_search_noalloc: queries and outputs must be device memory");
        return RR_EINVAL;
    }
    const size_t row_bytes = (size_t)ix->d * elem_size(ix->dtype);
    const bool direct = row_bytes == (size_t)ix->row_stride && ((uintptr_t)queries % 16) == 0;
    const int b = P.beam;
    // scratch layout: radius keys | counts | counters | flags | padded queries | beam results
    const size_t off_rk = 0, off_ek = off_rk + ru((size_t)nq * 4), off_cnt = off_ek + ru((size_t)nq * 4);
    const size_t off_ctr = off_cnt + ru((size_t)nq * 4), off_flags = off_ctr + 256;
    const size_t off_q = off_flags + ru((size_t)nq);
    const size_t off_keys = off_q + (direct ? 0 : ru((size_t)nq * ix->row_stride));
    const size_t need = off_keys + ru((size_t)nq * b * 8);
    if (need > kNoAllocScratchBytes) {
        set_error("rr_beam_search_noalloc: nq=%lld with beam %d needs %zu bytes of scratch; the static scratch "
                  "holds %zu bytes (split the batch)", (long long)nq, b, need, kNoAllocScratchBytes);
        return RR_EINVAL;
    }
    uint8_t *S = nullptr;
    rr_status s = scratch_address(ix->device, &S);
    if (s != RR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t rk, ek;
    const double esr = P.es_radius_mode == 1 ? P.es_radius : radius;
    if (!radius_key(radius, ix->dtype, &rk) || !radius_key(esr, ix->dtype, &ek)) {
        set_error("rr_beam_search_noalloc: radius is NaN");
        return RR_EINVAL;
    }
    int32_t *counters = (int32_t *)(S + off_ctr);
    const uint8_t *qd = (const uint8_t *)queries;
    if (!direct) {
        uint8_t *q = S + off_q;
        RR_CUDA(cudaMemsetAsync(q, 0, (size_t)nq * ix->row_stride, st));
        RR_CUDA(cudaMemcpy2DAsync(q, ix->row_stride, queries, row_bytes, row_bytes, nq, cudaMemcpyDeviceToDevice, st));
        qd = q;
    }
    int blocks = (int)std::min<int64_t>((nq + 255) / 256, 1024);
    init_kernel<<<blocks, 256, 0, st>>>((uint32_t *)(S + off_rk), (uint32_t *)(S + off_ek), nq, rk, ek, counters);
    RR_CUDA(cudaGetLastError());
    note_launch();

    SearchArgs a;
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
    a.rkey = (const uint32_t *)(S + off_rk);
    a.eskey = (const uint32_t *)(S + off_ek);
    a.beam = b;
    a.use_es = variant == RR_BEAM_ES ? 1 : 0;
    a.es_vl = P.es_visit_limit;
    a.es_metric = P.es_metric;
    a.es_ratio = P.es_radius;
    a.hash_lg = P.seen_log2;
    a.persistent = P.persistent ? 1 : 0;
    a.next_q = counters + 2;  // zeroed by init_kernel
    a.d = ix->d;
    a.prec = RR_PREC_EXACT;
    a.iter_limit = beam_iteration_limit(ix->n);
    a.expand = std::max(1, P.expand);
    a.phase2 = 0;
    a.res_keys = (uint64_t *)(S + off_keys);
    a.res_count = (int32_t *)(S + off_cnt);
    a.p2_list = nullptr;
    a.p2_count = counters;
    a.error = counters + 1;
    a.flags = S + off_flags;
    const int wpc = P.tile_hint > 0 ? std::min(8, P.tile_hint) : 4;
    if ((s = launch_beam(a, wpc, st, ix->dtype)) != RR_OK) return s;
    int eb = (int)std::min<int64_t>((nq + 7) / 8, 152 * 16);
    emit_kernel<<<eb, 256, 0, st>>>(a.res_keys, a.res_count, nq, b, ix->dtype == RR_F32 ? 1 : 0, ix->ext, out_counts, out_ids,
                                    out_dists);
    RR_CUDA(cudaGetLastError());
    note_launch();
    // the device guard word: a plain copy into a host variable (no staging buffer is allocated)
    int32_t err = 0;
    RR_CUDA(cudaMemcpyAsync(&err, counters + 1, 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (err != 0) {
        set_error("rr_beam_search_noalloc: a device-side guard tripped (code %d)", err);
        return RR_EINTERNAL;
    }
    return RR_OK;
}
