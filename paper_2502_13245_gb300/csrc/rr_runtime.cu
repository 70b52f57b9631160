// rr_runtime.cu -- host side of librr: errors, index creation and loading,
// and the orchestration of one batched range search (Alg. 6 / Alg. 3 / plain
// beam search over a batch, Sec. 4) on the caller's CUDA stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "rr_common.cuh"

namespace rr {

static thread_local std::string g_err;
static thread_local int64_t g_launches = 0;

void note_launch(int k) { g_launches += k; }
int64_t launches_so_far() { return g_launches; }

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

rr_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return RR_ECUDA;
}

// Failure-path hooks (rr_debug_set): process-wide, off by default.
static std::atomic<int64_t> g_fail_alloc_after{-1};
static std::atomic<int64_t> g_beam_iteration_limit{0};

bool inject_alloc_failure() {
    int64_t v = g_fail_alloc_after.load();
    while (v >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

int64_t beam_iteration_limit(int64_t n) {
    const int64_t v = g_beam_iteration_limit.load();
    return v > 0 ? v : n + 1;
}

rr_status Arena::reserve(size_t bytes) {
    if (bytes <= cap) return RR_OK;
    if (base) {
        cudaError_t e = cudaFree(base);
        base = nullptr;
        cap = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(arena)");
    }
    size_t want = std::max(bytes, (size_t)1 << 24);
    cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        set_error("device scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return RR_ENOMEM;
    }
    cap = want;
    return RR_OK;
}

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

int elem_size(int dtype) { return dtype == RR_F32 ? 4 : 1; }

static uint32_t host_dkey_f32(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Radius in the metric's units -> order key with d <= r  <=>  dkey(d) <= key.
bool radius_key(double r, int dtype, uint32_t *key) {
    if (isnan(r)) return false;
    if (dtype == RR_F32) {
        if (r >= 3.4e38) { *key = host_dkey_f32(INFINITY); return true; }
        if (r <= -3.4e38) { *key = host_dkey_f32(-INFINITY); return true; }
        float f = (float)r;
        if ((double)f > r) f = nextafterf(f, -INFINITY);  // largest float <= r
        *key = host_dkey_f32(f);
        return true;
    }
    double fl = floor(r);
    if (fl > 2147483647.0) fl = 2147483647.0;
    if (fl < -2147483648.0) fl = -2147483648.0;
    *key = dkey_i32((int32_t)fl);
    return true;
}

// Grow a device buffer to at least `need` bytes, keeping `keep` bytes of content.
rr_status grow(Grow &g, size_t need, size_t keep, cudaStream_t st) {
    if (need <= g.bytes) return RR_OK;
    size_t want = std::max(need, g.bytes + g.bytes / 2);
    void *np = nullptr;
    cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&np, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return RR_ENOMEM;
    }
    if (g.p && keep) RR_CUDA(cudaMemcpyAsync(np, g.p, std::min(keep, g.bytes), cudaMemcpyDeviceToDevice, st));
    if (g.p) {
        RR_CUDA(cudaStreamSynchronize(st));
        RR_CUDA(cudaFree(g.p));
    }
    g.p = np;
    g.bytes = want;
    return RR_OK;
}

void grow_free(Grow &g) {
    if (g.p) cudaFree(g.p);
    g.p = nullptr;
    g.bytes = 0;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace rr

using namespace rr;

extern "C" {

void rr_params_init(rr_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->beam = 64;
    p->b_max = 32768;
    p->es_visit_limit = 20;
    p->es_radius_mode = 0;
    p->es_radius = 0.0;
    p->precision = RR_PREC_EXACT;
    p->recheck_eps = 0.f;
    p->persistent = 0;
    p->collect_stats = 0;
    p->max_results_total = (int64_t)1 << 28;
    p->tile_hint = 0;
}

const char *rr_last_error(void) { return g_err.c_str(); }

rr_status rr_create_index(const void *vectors, int64_t n, int32_t d, int32_t dtype, int32_t metric,
                          const uint32_t *adjacency, int32_t R, int64_t start, int32_t device, int32_t validate,
                          rr_index **out) {
    if (!out) { set_error("rr_create_index: out is NULL"); return RR_EINVAL; }
    *out = nullptr;
    if (!vectors || !adjacency) { set_error("rr_create_index: NULL array"); return RR_EINVAL; }
    if (n < 1 || n >= ((int64_t)1 << 31)) { set_error("rr_create_index: n=%lld out of [1, 2^31)", (long long)n); return RR_EINVAL; }
    if (dtype != RR_U8 && dtype != RR_I8 && dtype != RR_F32) { set_error("rr_create_index: bad dtype %d", dtype); return RR_EINVAL; }
    if (metric != RR_L2 && metric != RR_IP) { set_error("rr_create_index: bad metric %d", metric); return RR_EINVAL; }
    if (d < 1 || d > 512) { set_error("rr_create_index: d=%d out of [1, 512]", d); return RR_EINVAL; }
    if (R < 1 || R > 128) { set_error("rr_create_index: R=%d out of [1, 128]", R); return RR_EINVAL; }
    if (start < 0 || start >= n) { set_error("rr_create_index: start=%lld out of range", (long long)start); return RR_EINVAL; }
    DeviceGuard dg(device);
    const int esz = elem_size(dtype);
    const int64_t row_bytes = (int64_t)d * esz;
    const int64_t row_stride = (row_bytes + 15) & ~(int64_t)15;
    if (validate) {
        std::vector<uint32_t> tmp;
        const uint32_t *h = adjacency;
        if (is_device_ptr(adjacency)) {
            tmp.resize((size_t)n * R);
            RR_CUDA(cudaMemcpy(tmp.data(), adjacency, (size_t)n * R * 4, cudaMemcpyDeviceToHost));
            h = tmp.data();
        }
        for (int64_t i = 0; i < n * (int64_t)R; i++) {
            if (h[i] != kSent && (int64_t)h[i] >= n) {
                set_error("rr_create_index: adjacency[%lld][%d] = %u is not a point id", (long long)(i / R),
                          (int)(i % R), h[i]);
                return RR_EINVAL;
            }
        }
    }
    rr_index *ix = new (std::nothrow) rr_index();
    if (!ix) { set_error("rr_create_index: host allocation failed"); return RR_ENOMEM; }
    ix->n = n; ix->d = d; ix->dtype = dtype; ix->metric = metric; ix->R = R; ix->start = start;
    ix->device = device; ix->row_stride = (int32_t)row_stride;
    cudaError_t e = cudaMalloc(&ix->vec, (size_t)n * row_stride);
    if (e == cudaSuccess) e = cudaMalloc(&ix->adj, (size_t)n * R * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ix->vec) cudaFree(ix->vec);
        delete ix;
        set_error("rr_create_index: device allocation failed: %s", cudaGetErrorString(e));
        return RR_ENOMEM;
    }
    ix->device_bytes = n * row_stride + n * (int64_t)R * 4;
    e = cudaSuccess;
    if (row_stride != row_bytes) e = cudaMemset(ix->vec, 0, (size_t)n * row_stride);
    if (e == cudaSuccess)
        e = cudaMemcpy2D(ix->vec, row_stride, vectors, row_bytes, row_bytes, n, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(ix->adj, adjacency, (size_t)n * R * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        rr_free_index(ix);
        return cuda_fail(e, "rr_create_index: copy to device");
    }
    *out = ix;
    return RR_OK;
}

static uint64_t rrx_checksum(const uint8_t *p, size_t nbytes) {
    uint64_t h = 0;
    size_t nw = (nbytes + 7) / 8;
    for (size_t i = 0; i < nw; i++) {
        uint64_t w = 0;
        size_t take = std::min((size_t)8, nbytes - i * 8);
        memcpy(&w, p + i * 8, take);  // little-endian hosts (x86-64, aarch64)
        h ^= w * 0x100000001B3ull + (uint64_t)i;
    }
    return h;
}

rr_status rr_load_index(const char *path, int32_t device, rr_index **out) {
    if (!path || !out) { set_error("rr_load_index: NULL argument"); return RR_EINVAL; }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("rr_load_index: cannot open %s", path); return RR_EINVAL; }
    uint8_t hdr[64];
    if (fread(hdr, 1, 64, f) != 64 || memcmp(hdr, "RRX1", 4) != 0) {
        fclose(f);
        set_error("rr_load_index: %s is not an .rrx file", path);
        return RR_EFORMAT;
    }
    uint32_t ver; int64_t n, start; int32_t d, dtype, metric, R; uint64_t ck;
    memcpy(&ver, hdr + 4, 4); memcpy(&n, hdr + 8, 8); memcpy(&d, hdr + 16, 4); memcpy(&dtype, hdr + 20, 4);
    memcpy(&metric, hdr + 24, 4); memcpy(&R, hdr + 28, 4); memcpy(&start, hdr + 32, 8); memcpy(&ck, hdr + 40, 8);
    if (ver != 1 || n < 1 || d < 1 || d > 512 || R < 1 || R > 128 || (dtype != RR_U8 && dtype != RR_I8 && dtype != RR_F32)) {
        fclose(f);
        set_error("rr_load_index: bad header in %s", path);
        return RR_EFORMAT;
    }
    size_t payload = (size_t)n * d * elem_size(dtype) + (size_t)n * R * 4;
    fseek(f, 0, SEEK_END);
    long long fsz = ftell(f);
    if (fsz < 0 || (size_t)fsz != 64 + payload) {
        fclose(f);
        set_error("rr_load_index: %s has %lld bytes, header implies %zu", path, fsz, 64 + payload);
        return RR_EFORMAT;
    }
    fseek(f, 64, SEEK_SET);
    uint8_t *buf = (uint8_t *)malloc(payload);
    if (!buf) { fclose(f); set_error("rr_load_index: host allocation failed"); return RR_ENOMEM; }
    size_t got = fread(buf, 1, payload, f);
    fclose(f);
    if (got != payload) { free(buf); set_error("rr_load_index: short read"); return RR_EFORMAT; }
    if (rrx_checksum(buf, payload) != ck) { free(buf); set_error("rr_load_index: checksum mismatch in %s", path); return RR_EFORMAT; }
    size_t vb = (size_t)n * d * elem_size(dtype);
    rr_status s = rr_create_index(buf, n, d, dtype, metric, (const uint32_t *)(buf + vb), R, start, device, 1, out);
    free(buf);
    return s;
}

rr_status rr_free_index(rr_index *ix) {
    if (!ix) return RR_OK;
    DeviceGuard dg(ix->device);
    if (ix->shared_data) {  // a worker view: the data belong to the parent index
        ix->vec = nullptr;
        ix->adj = nullptr;
        ix->lp_bf16 = ix->lp_fp8 = nullptr;
        ix->lp_fp8_info = nullptr;
        ix->lp_stats = nullptr;
        ix->ext = nullptr;
        if (ix->parent) ix->parent->live_views--;
    }
    if (ix->vec) cudaFree(ix->vec);
    if (ix->ext) cudaFree(ix->ext);
    if (ix->adj) cudaFree(ix->adj);
    if (ix->arena.base) cudaFree(ix->arena.base);
    if (ix->pinned.p) cudaFreeHost(ix->pinned.p);
    grow_free(ix->phase2);
    grow_free(ix->item_key);
    grow_free(ix->item_slot);
    grow_free(ix->outbuf);
    grow_free(ix->dbl_s[0]);
    grow_free(ix->dbl_s[1]);
    grow_free(ix->dbl_tmp);
    grow_free(ix->cand);
    grow_free(ix->dbl_seen);
    for (int k = 0; k < 4; k++)
        if (ix->ev[k]) cudaEventDestroy(ix->ev[k]);
    if (ix->lp_bf16) cudaFree(ix->lp_bf16);
    if (ix->lp_fp8) cudaFree(ix->lp_fp8);
    if (ix->lp_fp8_info) cudaFree(ix->lp_fp8_info);
    if (ix->lp_stats) cudaFree(ix->lp_stats);
    delete ix;
    return RR_OK;
}

rr_status rr_index_info_get(const rr_index *ix, rr_index_info *info) {
    if (!ix || !info) { set_error("rr_index_info_get: NULL argument"); return RR_EINVAL; }
    info->n = ix->n; info->d = ix->d; info->dtype = ix->dtype; info->metric = ix->metric; info->R = ix->R;
    info->start = ix->order ? ix->start_ext : ix->start; info->device_bytes = ix->device_bytes; info->row_stride = ix->row_stride;
    info->device = ix->device;
    info->scratch_bytes = (int64_t)ix->arena.cap + (int64_t)ix->phase2.bytes + (int64_t)ix->item_key.bytes +
                          (int64_t)ix->item_slot.bytes + (int64_t)ix->outbuf.bytes + (int64_t)ix->dbl_s[0].bytes +
                          (int64_t)ix->dbl_s[1].bytes + (int64_t)ix->dbl_tmp.bytes + (int64_t)ix->cand.bytes + (int64_t)ix->dbl_seen.bytes +
                          (int64_t)ix->pinned.cap;
    info->order = ix->order;
    info->reserved = 0;
    return RR_OK;
}

rr_status rr_debug_set(const char *key, int64_t value) {
    if (!key) { set_error("rr_debug_set: key is NULL"); return RR_EINVAL; }
    if (!strcmp(key, "fail_alloc_after")) {
        g_fail_alloc_after.store(value < 0 ? -1 : value);
        return RR_OK;
    }
    if (!strcmp(key, "beam_iteration_limit")) {
        g_beam_iteration_limit.store(value < 0 ? 0 : value);
        return RR_OK;
    }
    set_error("rr_debug_set: unknown key '%s'", key);
    return RR_EINVAL;
}

void rr_abi_sizes(int64_t out[8]) {
    if (!out) return;
    out[7] = sizeof(rr_build_info);
    out[0] = sizeof(rr_params);
    out[1] = sizeof(rr_query_stats);
    out[2] = sizeof(rr_result);
    out[3] = sizeof(rr_index_info);
    out[4] = sizeof(rr_profile);
    out[5] = sizeof(rr_serve_cfg);
    out[6] = sizeof(rr_serve_stats_t);
}

rr_status rr_result_to_host(const rr_result *r, rr_result *h) {
    if (!r || !h) { set_error("rr_result_to_host: NULL argument"); return RR_EINVAL; }
    memset(h, 0, sizeof *h);
    const int64_t nq = r->nq, tot = r->total;
    h->nq = nq;
    h->total = tot;
    h->dist_dtype = r->dist_dtype;
    if (!rr::host_result_arrays(h, nq, tot, r->stats != nullptr)) {
        rr_result_free(h);
        set_error("rr_result_to_host: allocation failed");
        return RR_ENOMEM;
    }
    struct { void *dst; const void *src; size_t bytes; } parts[5] = {
        {h->offsets, r->offsets, (size_t)(nq + 1) * 8}, {h->ids, r->ids, (size_t)tot * 4},
        {h->dists, r->dists, (size_t)tot * 4}, {h->flags, r->flags, (size_t)nq},
        {h->stats, r->stats, r->stats ? (size_t)nq * sizeof(rr_query_stats) : 0}};
    if (!r->on_device) {
        for (auto &p : parts)
            if (p.bytes) memcpy(p.dst, p.src, p.bytes);
        return RR_OK;
    }
    DeviceGuard dg(r->_device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)r->_stream);
    for (auto &p : parts)
        if (e == cudaSuccess && p.bytes) e = cudaMemcpy(p.dst, p.src, p.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        rr_result_free(h);
        return cuda_fail(e, "rr_result_to_host");
    }
    return RR_OK;
}

rr_status rr_result_free(rr_result *r) {
    if (!r) return RR_OK;
    if (r->on_device) {
        DeviceGuard dg(r->_device);
        cudaStream_t st = (cudaStream_t)r->_stream;
        if (r->offsets) cudaFreeAsync(r->offsets, st);
        if (r->ids) cudaFreeAsync(r->ids, st);
        if (r->dists) cudaFreeAsync(r->dists, st);
        if (r->flags) cudaFreeAsync(r->flags, st);
        if (r->stats) cudaFreeAsync(r->stats, st);
    } else if (!rr::host_pool_give(r->offsets)) {  // one pooled block holds every array; else separate mallocs
        free(r->offsets); free(r->ids); free(r->dists); free(r->flags); free(r->stats);
    }
    memset(r, 0, sizeof *r);
    return RR_OK;
}

}  // extern "C"

namespace rr {

// Pinned host blocks for host results: a device -> host copy into pinned memory runs at the link's
// speed, one into fresh pageable memory pays for faulting and pinning its pages on every call.  Blocks
// are reused after rr_result_free; at most kHostPoolBlocks are kept (held until the process exits), and
// a result that finds none free falls back to malloc.
namespace {
constexpr int kHostPoolBlocks = 4;
struct HostBlock {
    void *p;
    size_t cap;
    bool busy;
};
std::mutex g_host_mu;
std::vector<HostBlock> g_host_pool;
}  // namespace

void *host_pool_take(size_t bytes) {
    std::lock_guard<std::mutex> lock(g_host_mu);
    int best = -1, idle = -1;
    for (int i = 0; i < (int)g_host_pool.size(); i++) {
        const HostBlock &b = g_host_pool[(size_t)i];
        if (b.busy) continue;
        if (b.cap >= bytes && (best < 0 || b.cap < g_host_pool[(size_t)best].cap)) best = i;
        if (idle < 0 || b.cap > g_host_pool[(size_t)idle].cap) idle = i;
    }
    if (best >= 0) {
        g_host_pool[(size_t)best].busy = true;
        return g_host_pool[(size_t)best].p;
    }
    if (idle < 0 && (int)g_host_pool.size() >= kHostPoolBlocks) return nullptr;
    // a new block (replacing the largest idle one, which is too small), with a quarter of headroom
    const size_t cap = std::max<size_t>(bytes + bytes / 4, (size_t)1 << 20);
    void *p = nullptr;
    if (cudaHostAlloc(&p, cap, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (idle >= 0) {
        cudaFreeHost(g_host_pool[(size_t)idle].p);
        g_host_pool[(size_t)idle] = HostBlock{p, cap, true};
    } else {
        g_host_pool.push_back(HostBlock{p, cap, true});
    }
    return p;
}

bool host_pool_give(void *p) {
    if (!p) return false;
    std::lock_guard<std::mutex> lock(g_host_mu);
    for (HostBlock &b : g_host_pool)
        if (b.p == p) {
            b.busy = false;
            return true;
        }
    return false;
}

bool host_result_arrays(rr_result *out, int64_t nq, int64_t total, bool stats) {
    const size_t t = (size_t)std::max<int64_t>(total, 1), q = (size_t)std::max<int64_t>(nq, 1);
    auto up = [](size_t x) { return (x + 63) & ~(size_t)63; };
    // offsets first (the block's base: rr_result_free returns the block through it)
    const size_t o_st = up((size_t)(nq + 1) * 8), o_ids = o_st + up(stats ? q * sizeof(rr_query_stats) : 0);
    const size_t o_d = o_ids + up(t * 4), o_f = o_d + up(t * 4), end = o_f + q;
    if (uint8_t *b = (uint8_t *)host_pool_take(end)) {
        out->offsets = (int64_t *)b;
        out->stats = stats ? (rr_query_stats *)(b + o_st) : nullptr;
        out->ids = (uint32_t *)(b + o_ids);
        out->dists = b + o_d;
        out->flags = b + o_f;
        return true;
    }
    out->offsets = (int64_t *)malloc((size_t)(nq + 1) * 8);
    out->ids = (uint32_t *)malloc(t * 4);
    out->dists = malloc(t * 4);
    out->flags = (uint8_t *)malloc(q);
    out->stats = stats ? (rr_query_stats *)malloc(q * sizeof(rr_query_stats)) : nullptr;
    return out->offsets && out->ids && out->dists && out->flags && (!stats || out->stats);
}

rr_index *index_worker_view(rr_index *p) {
    rr_index *v = new (std::nothrow) rr_index();
    if (!v) return nullptr;
    v->n = p->n; v->d = p->d; v->dtype = p->dtype; v->metric = p->metric; v->R = p->R; v->start = p->start;
    v->device = p->device; v->row_stride = p->row_stride; v->vec = p->vec; v->adj = p->adj;
    v->lp_bf16 = p->lp_bf16; v->lp_bf16_stride = p->lp_bf16_stride;
    v->lp_fp8 = p->lp_fp8; v->lp_fp8_stride = p->lp_fp8_stride; v->lp_fp8_info = p->lp_fp8_info;
    v->lp_stats = p->lp_stats; v->max_norm = p->max_norm; v->max_abs = p->max_abs;
    v->ext = p->ext; v->start_ext = p->start_ext; v->order = p->order;
    v->shared_data = true;
    v->parent = p;
    p->live_views++;
    return v;
}
}  // namespace rr
