// k_relabel.cu -- rr_index_relabel: renumber an index's points in
// breadth-first order from the start point.
//
// A layout step of this library, not part of the paper's method: the range
// search (Alg. 1, 2, 3, 6) runs unchanged on the renamed graph.  Points that
// are close in the graph get close internal ids, so a query's visited bitmap
// (Alg. 2's expansion) and its vector and adjacency gathers hit fewer distinct
// DRAM sectors.  The order is computed on the host (one pass over the
// adjacency); the rows move on the device with two gather kernels.
#include <memory>
#include <new>

#include "rr_common.cuh"

namespace rr {

namespace {

// new row i <- old row old_of[i]; rows are `chunks` 16-byte words (padding included)
__global__ void gather_rows_kernel(const uint4 *src, uint4 *dst, const uint32_t *old_of, int64_t n, int chunks) {
    const int64_t total = n * chunks;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / chunks;
        const int c = (int)(t - i * chunks);
        dst[t] = src[(int64_t)old_of[i] * chunks + c];
    }
}

// new adjacency row i <- old row old_of[i], every entry renamed through new_of,
// slot order and padding kept (entries were checked on the host to be < n or padding)
__global__ void relabel_adj_kernel(const uint32_t *src, uint32_t *dst, const uint32_t *old_of,
                                   const uint32_t *new_of, int64_t n, int R) {
    const int64_t total = n * R;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / R;
        const int k = (int)(t - i * R);
        const uint32_t u = src[(int64_t)old_of[i] * R + k];
        dst[t] = u == kSent ? kSent : new_of[u];
    }
}

// Breadth-first numbering: old_of doubles as the queue.  Returns false if an
// adjacency entry is neither padding nor a valid id.
bool bfs_order(const uint32_t *adj, int64_t n, int R, uint32_t start, uint32_t *old_of, uint8_t *reached) {
    memset(reached, 0, (size_t)n);
    int64_t head = 0, tail = 0;
    old_of[tail++] = start;
    reached[start] = 1;
    while (head < tail) {
        const uint32_t v = old_of[head++];
        const uint32_t *row = adj + (size_t)v * R;
        for (int k = 0; k < R; k++) {
            const uint32_t u = row[k];
            if (u == kSent) continue;
            if ((int64_t)u >= n) return false;
            if (!reached[u]) {
                reached[u] = 1;
                old_of[tail++] = u;
            }
        }
    }
    for (int64_t i = 0; i < n; i++)
        if (!reached[i]) {
            // an unreached row is never scanned above: check its entries here
            const uint32_t *row = adj + (size_t)i * R;
            for (int k = 0; k < R; k++)
                if (row[k] != kSent && (int64_t)row[k] >= n) return false;
            old_of[tail++] = (uint32_t)i;
        }
    return tail == n;
}

struct DevFree {
    void operator()(void *p) const {
        if (p) cudaFree(p);
    }
};
using DevPtr = std::unique_ptr<void, DevFree>;

void *dev_alloc(size_t bytes) {
    void *p = nullptr;
    if (inject_alloc_failure() || cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

}  // namespace

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_index_relabel(rr_index *ix, int32_t order) {
    if (!ix) { set_error("rr_index_relabel: index is NULL"); return RR_EINVAL; }
    if (order != RR_ORDER_BFS) { set_error("rr_index_relabel: unknown order %d", order); return RR_EINVAL; }
    if (ix->shared_data) { set_error("rr_index_relabel: a worker view cannot be relabeled"); return RR_EINVAL; }
    if (ix->live_views > 0) {
        set_error("rr_index_relabel: a server is running on this index (relabel before rr_serve_create)");
        return RR_EINVAL;
    }
    if (ix->order != 0) { set_error("rr_index_relabel: the index is already relabeled"); return RR_EINVAL; }
    DeviceGuard dg(ix->device);
    const int64_t n = ix->n;
    const int R = ix->R;
    const int chunks = ix->row_stride / 16;
    std::unique_ptr<uint32_t[]> h_adj(new (std::nothrow) uint32_t[(size_t)n * R]);
    std::unique_ptr<uint32_t[]> old_of(new (std::nothrow) uint32_t[(size_t)n]);
    std::unique_ptr<uint32_t[]> new_of(new (std::nothrow) uint32_t[(size_t)n]);
    std::unique_ptr<uint8_t[]> reached(new (std::nothrow) uint8_t[(size_t)n]);
    if (!h_adj || !old_of || !new_of || !reached) {
        set_error("rr_index_relabel: host allocation failed");
        return RR_ENOMEM;
    }
    RR_CUDA(cudaDeviceSynchronize());  // work on the index from earlier calls, on any stream
    RR_CUDA(cudaMemcpy(h_adj.get(), ix->adj, (size_t)n * R * 4, cudaMemcpyDeviceToHost));
    if (!bfs_order(h_adj.get(), n, R, (uint32_t)ix->start, old_of.get(), reached.get())) {
        set_error("rr_index_relabel: an adjacency entry is neither padding nor < n");
        return RR_EINVAL;
    }
    for (int64_t i = 0; i < n; i++) new_of[old_of[i]] = (uint32_t)i;
    h_adj.reset();
    reached.reset();

    DevPtr d_old(dev_alloc((size_t)n * 4)), d_new(dev_alloc((size_t)n * 4));
    DevPtr vec2(dev_alloc((size_t)n * ix->row_stride)), adj2(dev_alloc((size_t)n * R * 4));
    if (!d_old || !d_new || !vec2 || !adj2) {
        set_error("rr_index_relabel: device allocation failed");
        return RR_ENOMEM;
    }
    RR_CUDA(cudaMemcpy(d_old.get(), old_of.get(), (size_t)n * 4, cudaMemcpyHostToDevice));
    RR_CUDA(cudaMemcpy(d_new.get(), new_of.get(), (size_t)n * 4, cudaMemcpyHostToDevice));
    gather_rows_kernel<<<152 * 16, 256>>>((const uint4 *)ix->vec, (uint4 *)vec2.get(), (const uint32_t *)d_old.get(),
                                          n, chunks);
    RR_CUDA(cudaGetLastError());
    note_launch();
    relabel_adj_kernel<<<152 * 16, 256>>>(ix->adj, (uint32_t *)adj2.get(), (const uint32_t *)d_old.get(),
                                          (const uint32_t *)d_new.get(), n, R);
    RR_CUDA(cudaGetLastError());
    note_launch();
    RR_CUDA(cudaDeviceSynchronize());

    // swap in the relabeled arrays; traversal copies of the old order are dropped (rebuilt on next use)
    cudaFree(ix->vec);
    cudaFree(ix->adj);
    ix->vec = (uint8_t *)vec2.release();
    ix->adj = (uint32_t *)adj2.release();
    ix->ext = (uint32_t *)d_old.release();
    ix->device_bytes += n * 4;
    if (ix->lp_bf16) {
        cudaFree(ix->lp_bf16);
        ix->lp_bf16 = nullptr;
        ix->device_bytes -= n * ix->lp_bf16_stride;
    }
    if (ix->lp_fp8) {
        cudaFree(ix->lp_fp8);
        cudaFree(ix->lp_fp8_info);
        ix->lp_fp8 = nullptr;
        ix->lp_fp8_info = nullptr;
        ix->device_bytes -= n * (ix->lp_fp8_stride + 8);
    }
    ix->start_ext = ix->start;
    ix->start = new_of[ix->start];  // 0: the traversal starts there
    ix->order = order;
    return RR_OK;
}
