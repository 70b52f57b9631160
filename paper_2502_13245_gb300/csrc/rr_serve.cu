// rr_serve.cu -- continuous batching of single range queries (serving).
//
// The paper evaluates batched search (Sec. 4); a service sees queries one at a
// time.  Worker threads turn the arrival stream into batches: each owns a CUDA
// stream and a scratch view of the index (shared vectors and graph), takes
// whatever is queued when it becomes free, and searches it with the batched
// path of rr_range_search.  The batch's CSR stays where the search left it
// (host memory, or device memory with result_on_device) and is shared by the
// batch's requests; a request's row is copied out once, when it is collected
// (for device results: consecutive rows of a batch as one copy-engine transfer,
// or one gather kernel when the rows are scattered).  With two or more workers one batch's
// host-side work overlaps the next batch's kernels.  Admission is by result
// memory: the match counts of range queries are heavy-tailed (Sec. 3), so a
// count of requests is no bound on memory.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rr_internal.h"

using namespace rr;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket;
    size_t qoff;  // byte offset of the query in the server's arrival buffer
    double radius;
    Clock::time_point t0;
};

// One search's result, shared by the requests of its batch until the last is collected.
struct Batch {
    rr_result res;                 // host or device CSR of the batch
    std::vector<int64_t> off;      // host copy of the offsets (device results)
    std::vector<uint8_t> flags;    // host copy of the flags (device results)
    std::vector<rr_query_stats> stats;
    Batch() { memset(&res, 0, sizeof res); }
    ~Batch() { rr_result_free(&res); }
    int64_t lo(int64_t i) const { return res.on_device ? off[i] : res.offsets[i]; }
    int64_t count(int64_t i) const { return lo(i + 1) - lo(i); }
    uint8_t flag(int64_t i) const { return res.on_device ? flags[i] : res.flags[i]; }
    rr_query_stats stat(int64_t i) const {
        if (res.on_device) return stats.empty() ? rr_query_stats{} : stats[i];
        return res.stats ? res.stats[i] : rr_query_stats{};
    }
};

struct Done {
    rr_status status = RR_OK;
    std::string err;
    std::shared_ptr<Batch> batch;  // null for a failed or canceled request
    int64_t idx = 0;               // the request's row in the batch
    int64_t bytes = 0;             // held against the budget until collected
    uint8_t flag = 0;
};

struct Worker {
    std::thread th;
    rr_index *view = nullptr;
    cudaStream_t st = nullptr;
    uint8_t *qpin = nullptr;  // pinned batch of queries
    size_t qpin_cap = 0;
};

// segment copy for device results: row i of the output comes from src[i]
struct Seg {
    const uint32_t *ids;
    const uint32_t *dists;
    int64_t len;
    int64_t dst;
};

__global__ void gather_segments_kernel(const Seg *segs, int64_t n, uint32_t *ids, uint32_t *dists) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n; s += nw) {
        const Seg g = segs[s];
        for (int64_t k = lane; k < g.len; k += 32) {
            ids[g.dst + k] = g.ids[k];
            dists[g.dst + k] = g.dists[k];
        }
    }
}

}  // namespace

struct rr_server {
    rr_index *ix = nullptr;
    rr_serve_cfg cfg;
    size_t row_bytes = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers: requests queued, budget freed, stop
    std::condition_variable cv_done;  // pollers: a request finished
    std::deque<Request> queue;
    // arrival buffer: queries are appended at the back; consumed from the front
    std::vector<uint8_t> qbuf;
    size_t qbuf_head = 0;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> live;  // queued or in flight or done-not-collected
    uint64_t next_ticket = 1;
    int64_t bytes_held = 0;
    int64_t in_flight = 0;
    double reserve = 0;       // bytes reserved per admitted request (fixed, or a running mean)
    bool adaptive = false;
    bool stop = false;
    // statistics since the last reset
    int64_t submitted = 0, completed = 0, polled = 0, batches = 0, batched = 0, admission_waits = 0, canceled = 0;
    std::vector<float> lat_us;
    Clock::time_point t_reset;
    std::vector<Worker> workers;
    // collection of device results (one collector at a time)
    std::mutex cmu;
    cudaStream_t cst = nullptr;
    uint8_t *cpin = nullptr;
    size_t cpin_cap = 0;
};

namespace {

int64_t result_bytes(int64_t count, bool stats) {
    return 8 * count + 16 + 1 + (stats ? (int64_t)sizeof(rr_query_stats) : 0);
}

void worker_loop(rr_server *S, Worker *W) {
    DeviceGuard dg(S->ix->device);
    const rr_serve_cfg &C = S->cfg;
    const bool stats = C.params.collect_stats != 0;
    const bool dev = C.result_on_device != 0;
    std::vector<Request> batch;
    std::vector<double> radii;
    for (;;) {
        int64_t reserved = 0, budget_left = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->queue.empty()) return;  // stopping, nothing left
            if ((int64_t)S->queue.size() < C.max_batch && !S->stop && C.batch_wait_us > 0) {
                auto until = Clock::now() + std::chrono::microseconds(C.batch_wait_us);
                S->cv_work.wait_until(lk, until, [&] { return S->stop || (int64_t)S->queue.size() >= C.max_batch; });
                if (S->queue.empty()) continue;  // another worker took them
            }
            // admission: each request reserves S->reserve bytes of the budget
            const int64_t per = (int64_t)S->reserve;
            batch.clear();
            while (!S->queue.empty() && (int64_t)batch.size() < C.max_batch) {
                bool fits = S->bytes_held + reserved + per <= C.result_budget_bytes;
                // always admit one when nothing is held; a stopping server drains its queue regardless
                bool progress = S->bytes_held + reserved == 0 || S->stop;
                if (!fits && !progress) break;
                batch.push_back(S->queue.front());
                S->queue.pop_front();
                reserved += per;
            }
            if (batch.empty()) {
                S->admission_waits++;
                // wait for a collection to free budget (or stop); re-check from the top
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            if (!S->queue.empty()) S->cv_work.notify_one();  // more for another worker
            budget_left = C.result_budget_bytes - S->bytes_held;
            S->bytes_held += reserved;
            S->in_flight += (int64_t)batch.size();
            // copy the batch's queries to pinned memory while the arrival buffer is locked
            const size_t need = batch.size() * S->row_bytes;
            if (need > W->qpin_cap) {
                if (W->qpin) cudaFreeHost(W->qpin);
                W->qpin = nullptr;
                W->qpin_cap = 0;
                if (cudaMallocHost(&W->qpin, std::max(need, (size_t)1 << 20)) == cudaSuccess)
                    W->qpin_cap = std::max(need, (size_t)1 << 20);
                else
                    cudaGetLastError();
            }
            if (W->qpin)
                for (size_t j = 0; j < batch.size(); j++)
                    memcpy(W->qpin + j * S->row_bytes, S->qbuf.data() + batch[j].qoff, S->row_bytes);
            S->qbuf_head = S->queue.empty() ? 0 : S->queue.front().qoff;
            if (S->queue.empty()) S->qbuf.clear();
        }
        const int64_t k = (int64_t)batch.size();
        radii.resize(k);
        for (int64_t j = 0; j < k; j++) radii[j] = batch[j].radius;
        rr_params P = C.params;
        // a batch may fill what the budget has left (8 bytes per result: id + distance)
        int64_t cap = std::max<int64_t>(budget_left, reserved) / 8;
        if (P.max_results_total > 0) cap = std::min<int64_t>(cap, P.max_results_total);
        P.max_results_total = std::max<int64_t>(cap, 1);
        auto B = std::make_shared<Batch>();
        rr_status s = W->qpin ? rr_range_search(W->view, W->qpin, k, radii.data(), 0.0, C.variant, &P, W->st,
                                                dev ? 1 : 0, &B->res)
                              : RR_ENOMEM;
        if (s == RR_EOVERFLOW) s = RR_OK;  // truncated results are flagged per query
        if (s == RR_OK && dev) {
            // row bounds, flags (and counters) of the device CSR, for collection and accounting
            B->off.resize((size_t)k + 1);
            B->flags.resize((size_t)k);
            cudaError_t e = cudaMemcpyAsync(B->off.data(), B->res.offsets, (size_t)(k + 1) * 8, cudaMemcpyDeviceToHost, W->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(B->flags.data(), B->res.flags, (size_t)k, cudaMemcpyDeviceToHost, W->st);
            if (e == cudaSuccess && stats && B->res.stats) {
                B->stats.resize((size_t)k);
                e = cudaMemcpyAsync(B->stats.data(), B->res.stats, (size_t)k * sizeof(rr_query_stats),
                                    cudaMemcpyDeviceToHost, W->st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(W->st);
            if (e != cudaSuccess) s = cuda_fail(e, "rr_serve: reading a batch's row bounds");
        }
        std::string err = s == RR_OK ? std::string() : std::string(rr_last_error());
        std::vector<Done> out((size_t)k);
        int64_t batch_bytes = 0;
        for (int64_t j = 0; j < k; j++) {
            Done &d = out[(size_t)j];
            d.status = s;
            d.err = err;
            if (s == RR_OK) {
                d.batch = B;
                d.idx = j;
                d.flag = B->flag(j);
                d.bytes = result_bytes(B->count(j), stats);
                batch_bytes += d.bytes;
            }
        }
        B.reset();
        const Clock::time_point t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->bytes_held -= reserved;
            S->in_flight -= k;
            for (int64_t j = 0; j < k; j++) {
                S->bytes_held += out[(size_t)j].bytes;
                S->lat_us.push_back((float)std::chrono::duration<double, std::micro>(t1 - batch[j].t0).count());
                S->done.emplace(batch[j].ticket, std::move(out[(size_t)j]));
            }
            if (S->adaptive && s == RR_OK && k > 0) {
                // running mean of the bytes a request turns out to hold (never below the beam's share)
                const double floor_b = 8.0 * C.params.beam + 32.0;
                S->reserve = std::max(floor_b, 0.8 * S->reserve + 0.2 * ((double)batch_bytes / (double)k));
            }
            S->completed += k;
            S->batches += 1;
            S->batched += k;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // budget may have shrunk or grown
    }
}

// Take tickets first .. first+n-1 out of the done table (all must be done); caller holds S->mu.
void take_done(rr_server *S, uint64_t first, int64_t n, std::vector<Done> &got) {
    got.resize((size_t)n);
    int64_t freed = 0;
    for (int64_t i = 0; i < n; i++) {
        auto it = S->done.find(first + (uint64_t)i);
        got[(size_t)i] = std::move(it->second);
        S->done.erase(it);
        S->live.erase(first + (uint64_t)i);
        freed += got[(size_t)i].bytes;
    }
    S->bytes_held -= freed;
    S->polled += n;
}

// Build one CSR (host or device) from collected requests.
rr_status assemble(rr_server *S, std::vector<Done> &got, rr_result *out) {
    const int64_t n = (int64_t)got.size();
    const bool stats = S->cfg.params.collect_stats != 0;
    const bool dev = S->cfg.result_on_device != 0;
    std::vector<int64_t> off((size_t)n + 1);
    std::vector<uint8_t> fl((size_t)n);
    std::vector<rr_query_stats> st(stats ? (size_t)n : 0);
    int64_t total = 0;
    for (int64_t i = 0; i < n; i++) {
        const Done &d = got[(size_t)i];
        off[(size_t)i] = total;
        fl[(size_t)i] = d.flag;
        if (d.batch) {
            total += d.batch->count(d.idx);
            if (stats) st[(size_t)i] = d.batch->stat(d.idx);
        }
    }
    off[(size_t)n] = total;
    memset(out, 0, sizeof *out);
    out->nq = n;
    out->total = total;
    out->dist_dtype = S->ix->dtype == RR_F32 ? 1 : 0;
    if (!dev) {
        out->offsets = (int64_t *)malloc((size_t)(n + 1) * 8);
        out->ids = (uint32_t *)malloc((size_t)std::max<int64_t>(total, 1) * 4);
        out->dists = malloc((size_t)std::max<int64_t>(total, 1) * 4);
        out->flags = (uint8_t *)malloc((size_t)std::max<int64_t>(n, 1));
        if (stats) out->stats = (rr_query_stats *)malloc((size_t)std::max<int64_t>(n, 1) * sizeof(rr_query_stats));
        if (!out->offsets || !out->ids || !out->dists || !out->flags || (stats && !out->stats)) {
            rr_result_free(out);
            set_error("rr_serve: result allocation failed");
            return RR_ENOMEM;
        }
        memcpy(out->offsets, off.data(), (size_t)(n + 1) * 8);
        if (n) memcpy(out->flags, fl.data(), (size_t)n);
        if (stats && n) memcpy(out->stats, st.data(), (size_t)n * sizeof(rr_query_stats));
        for (int64_t i = 0; i < n; i++) {
            const Done &d = got[(size_t)i];
            const int64_t c = d.batch ? d.batch->count(d.idx) : 0;
            if (!c) continue;
            const int64_t lo = d.batch->lo(d.idx);
            memcpy(out->ids + off[(size_t)i], d.batch->res.ids + lo, (size_t)c * 4);
            memcpy((uint8_t *)out->dists + off[(size_t)i] * 4, (const uint8_t *)d.batch->res.dists + lo * 4, (size_t)c * 4);
        }
        return RR_OK;
    }
    // device results: one gather launch on the server's collection stream
    std::lock_guard<std::mutex> ck(S->cmu);
    DeviceGuard dg(S->ix->device);
    cudaStream_t cs = S->cst;
    int64_t nseg = 0;
    for (auto &d : got) nseg += d.batch && d.batch->count(d.idx) > 0;
    const size_t seg_bytes = (size_t)nseg * sizeof(Seg);
    const size_t head = (size_t)(n + 1) * 8 + (size_t)n + (stats ? (size_t)n * sizeof(rr_query_stats) : 0);
    const size_t pin_need = ((head + 15) & ~(size_t)15) + seg_bytes;
    if (pin_need > S->cpin_cap) {
        if (S->cpin) { cudaStreamSynchronize(cs); cudaFreeHost(S->cpin); }
        S->cpin = nullptr;
        S->cpin_cap = 0;
        if (cudaMallocHost(&S->cpin, std::max(pin_need, (size_t)1 << 20)) != cudaSuccess) {
            cudaGetLastError();
            set_error("rr_serve: pinned staging allocation failed");
            return RR_ENOMEM;
        }
        S->cpin_cap = std::max(pin_need, (size_t)1 << 20);
    }
    RR_CUDA(cudaStreamSynchronize(cs));  // the staging may still feed the previous collection's copies
    uint8_t *hp = S->cpin;
    memcpy(hp, off.data(), (size_t)(n + 1) * 8);
    if (n) memcpy(hp + (size_t)(n + 1) * 8, fl.data(), (size_t)n);
    if (stats && n) memcpy(hp + (size_t)(n + 1) * 8 + (size_t)n, st.data(), (size_t)n * sizeof(rr_query_stats));
    Seg *hs = reinterpret_cast<Seg *>(hp + ((head + 15) & ~(size_t)15));
    // consecutive requests of one batch are consecutive rows of its CSR: one run each
    int64_t k = 0;
    const Batch *prev_b = nullptr;
    int64_t prev_idx = -2;
    for (int64_t i = 0; i < n; i++) {
        const Done &d = got[(size_t)i];
        const int64_t c = d.batch ? d.batch->count(d.idx) : 0;
        if (!c) continue;
        const int64_t lo = d.batch->lo(d.idx);
        if (k > 0 && d.batch.get() == prev_b && d.idx == prev_idx + 1 && hs[k - 1].dst + hs[k - 1].len == off[(size_t)i]) {
            hs[k - 1].len += c;
        } else {
            hs[k++] = Seg{d.batch->res.ids + lo, (const uint32_t *)d.batch->res.dists + lo, c, off[(size_t)i]};
        }
        prev_b = d.batch.get();
        prev_idx = d.idx;
    }
    nseg = k;
    // a few long runs go to the copy engines; many short ones to one gather launch
    const bool by_copy = nseg <= 8;
    out->on_device = 1;
    out->_stream = (void *)cs;
    out->_device = S->ix->device;
    Seg *dsegs = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&out->offsets, (size_t)(n + 1) * 8, cs);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out->ids, (size_t)std::max<int64_t>(total, 1) * 4, cs);
    if (e == cudaSuccess) e = cudaMallocAsync(&out->dists, (size_t)std::max<int64_t>(total, 1) * 4, cs);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out->flags, (size_t)std::max<int64_t>(n, 1), cs);
    if (e == cudaSuccess && stats)
        e = cudaMallocAsync((void **)&out->stats, (size_t)std::max<int64_t>(n, 1) * sizeof(rr_query_stats), cs);
    if (e == cudaSuccess && nseg && !by_copy) e = cudaMallocAsync((void **)&dsegs, seg_bytes, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->offsets, hp, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(out->flags, hp + (size_t)(n + 1) * 8, (size_t)n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && stats && n)
        e = cudaMemcpyAsync(out->stats, hp + (size_t)(n + 1) * 8 + (size_t)n, (size_t)n * sizeof(rr_query_stats),
                            cudaMemcpyHostToDevice, cs);
    for (int64_t j = 0; by_copy && e == cudaSuccess && j < nseg; j++) {
        e = cudaMemcpyAsync(out->ids + hs[j].dst, hs[j].ids, (size_t)hs[j].len * 4, cudaMemcpyDeviceToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((uint32_t *)out->dists + hs[j].dst, hs[j].dists, (size_t)hs[j].len * 4,
                                cudaMemcpyDeviceToDevice, cs);
    }
    if (e == cudaSuccess && nseg && !by_copy)
        e = cudaMemcpyAsync(dsegs, hs, (size_t)nseg * sizeof(Seg), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && nseg && !by_copy) {
        const int blocks = (int)std::min<int64_t>((nseg + 7) / 8, 152 * 16);
        gather_segments_kernel<<<blocks, 256, 0, cs>>>(dsegs, nseg, out->ids, (uint32_t *)out->dists);
        note_launch();
        e = cudaGetLastError();
    }
    if (dsegs) cudaFreeAsync(dsegs, cs);
    // the batches' arrays are released when the caller drops them: finish reading them first
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        rr_result_free(out);
        return cuda_fail(e, "rr_serve: gathering device results");
    }
    return RR_OK;
}

rr_status collect_impl(rr_server *S, uint64_t first, int64_t n, int32_t timeout_ms, rr_result *out, const char *who) {
    std::vector<Done> got;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        for (int64_t i = 0; i < n; i++)
            if (!S->live.count(first + (uint64_t)i)) {
                set_error("%s: unknown or retired ticket %llu", who, (unsigned long long)(first + i));
                return RR_EINVAL;
            }
        auto ready = [&] {
            for (int64_t i = 0; i < n; i++)
                if (!S->done.count(first + (uint64_t)i)) return false;
            return true;
        };
        if (!ready()) {
            if (timeout_ms <= 0) return RR_EBUSY;
            if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return RR_EBUSY;
        }
        take_done(S, first, n, got);
    }
    S->cv_work.notify_all();
    rr_status bad = RR_OK;
    std::string err;
    for (auto &g : got)
        if (g.status != RR_OK && bad == RR_OK) { bad = g.status; err = g.err; }
    rr_status s = assemble(S, got, out);
    got.clear();  // drops the batch references (after any gather has finished reading them)
    if (s != RR_OK) return s;
    if (bad != RR_OK) {  // the requests are retired either way; report the first failure
        set_error("%s", err.c_str());
        return bad;
    }
    return RR_OK;
}

}  // namespace

extern "C" {

void rr_serve_cfg_init(rr_serve_cfg *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->workers = 2;
    c->max_batch = 4096;
    c->batch_wait_us = 200;
    c->variant = RR_GREEDY_ES;
    rr_params_init(&c->params);
    c->result_budget_bytes = (int64_t)4 << 30;
    c->reserve_per_request = 0;  // 0: a running mean of the bytes requests hold
    c->result_on_device = 0;
}

rr_status rr_serve_create(rr_index *ix, const rr_serve_cfg *cfg, rr_server **out) {
    if (!ix || !out) { set_error("rr_serve_create: NULL argument"); return RR_EINVAL; }
    *out = nullptr;
    rr_serve_cfg C;
    if (cfg) C = *cfg; else rr_serve_cfg_init(&C);
    if (C.workers < 1 || C.workers > 64 || C.max_batch < 1 || C.batch_wait_us < 0 || C.result_budget_bytes <= 0 ||
        C.reserve_per_request < 0 || C.variant < RR_BEAM || C.variant > RR_DOUBLING_WARM_ES || C.params.beam < 1 ||
        (C.result_on_device != 0 && C.result_on_device != 1)) {
        set_error("rr_serve_create: invalid configuration");
        return RR_EINVAL;
    }
    if (C.params.precision != RR_PREC_EXACT && ix->dtype != RR_F32) {
        set_error("rr_serve_create: the precision form needs an fp32 index");
        return RR_EINVAL;
    }
    DeviceGuard dg(ix->device);
    if (C.params.precision != RR_PREC_EXACT) {
        // build the traversal copy once on the shared index: the worker views borrow it
        rr_status s = ensure_lowp(ix, C.params.precision, nullptr);
        if (s != RR_OK) return s;
        RR_CUDA(cudaDeviceSynchronize());
    }
    rr_server *S = new (std::nothrow) rr_server();
    if (!S) { set_error("rr_serve_create: out of memory"); return RR_ENOMEM; }
    S->ix = ix;
    S->cfg = C;
    S->adaptive = C.reserve_per_request == 0;
    S->reserve = S->adaptive ? 8.0 * C.params.beam + 32.0 : (double)C.reserve_per_request;
    S->row_bytes = (size_t)ix->d * elem_size(ix->dtype);
    S->t_reset = Clock::now();
    S->workers.resize(C.workers);
    // collection runs at the highest stream priority: its gathers are short and should not queue
    // behind the workers' search kernels
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    bool ok = cudaStreamCreateWithPriority(&S->cst, cudaStreamNonBlocking, hi_prio) == cudaSuccess;
    for (auto &W : S->workers) {
        W.view = index_worker_view(ix);
        ok = ok && W.view && cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        for (auto &V : S->workers) {
            if (V.view) rr_free_index(V.view);
            if (V.st) cudaStreamDestroy(V.st);
        }
        if (S->cst) cudaStreamDestroy(S->cst);
        delete S;
        set_error("rr_serve_create: worker set-up failed");
        return RR_ENOMEM;
    }
    for (auto &W : S->workers) W.th = std::thread(worker_loop, S, &W);
    *out = S;
    return RR_OK;
}

rr_status rr_serve_submit(rr_server *S, const void *queries, int64_t n, const double *radii, double radius,
                          uint64_t *first_ticket) {
    if (!S || (n > 0 && !queries) || n < 0) { set_error("rr_serve_submit: bad argument"); return RR_EINVAL; }
    if (n > 0 && is_device_ptr(queries)) {
        set_error("rr_serve_submit: queries must be in host memory");
        return RR_EINVAL;
    }
    for (int64_t i = 0; i < n; i++) {
        uint32_t key;
        if (!radius_key(radii ? radii[i] : radius, S->ix->dtype, &key)) {
            set_error("rr_serve_submit: radius of request %lld is NaN", (long long)i);
            return RR_EINVAL;
        }
    }
    const Clock::time_point t0 = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { set_error("rr_serve_submit: server is stopping"); return RR_EINVAL; }
        if (first_ticket) *first_ticket = S->next_ticket;
        // drop the consumed prefix of the arrival buffer once it dominates
        if (S->qbuf_head > 0 && S->qbuf_head * 2 > S->qbuf.size()) {
            S->qbuf.erase(S->qbuf.begin(), S->qbuf.begin() + S->qbuf_head);
            for (auto &r : S->queue) r.qoff -= S->qbuf_head;
            S->qbuf_head = 0;
        }
        const size_t base = S->qbuf.size();
        const uint8_t *q = (const uint8_t *)queries;
        S->qbuf.insert(S->qbuf.end(), q, q + (size_t)n * S->row_bytes);
        for (int64_t i = 0; i < n; i++) {
            uint64_t t = S->next_ticket++;
            S->queue.push_back(Request{t, base + (size_t)i * S->row_bytes, radii ? radii[i] : radius, t0});
            S->live.emplace(t, 1);
        }
        S->submitted += n;
    }
    S->cv_work.notify_all();
    return RR_OK;
}

rr_status rr_serve_poll(rr_server *S, uint64_t ticket, int32_t timeout_ms, rr_result *out) {
    if (!S || !out) { set_error("rr_serve_poll: NULL argument"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    return collect_impl(S, ticket, 1, timeout_ms, out, "rr_serve_poll");
}

rr_status rr_serve_collect(rr_server *S, uint64_t first, int64_t n, int32_t timeout_ms, rr_result *out) {
    if (!S || !out || n < 0) { set_error("rr_serve_collect: bad argument"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    return collect_impl(S, first, n, timeout_ms, out, "rr_serve_collect");
}

int64_t rr_serve_cancel(rr_server *S) {
    if (!S) return 0;
    int64_t k = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->queue.empty()) {
            Done d;
            d.flag = RR_FLAG_CANCELED;
            S->done.emplace(S->queue.front().ticket, std::move(d));
            S->queue.pop_front();
            k++;
        }
        S->qbuf.clear();
        S->qbuf_head = 0;
        S->canceled += k;
    }
    S->cv_done.notify_all();
    return k;
}

rr_status rr_serve_stats(rr_server *S, rr_serve_stats_t *o, int32_t reset) {
    if (!S || !o) { set_error("rr_serve_stats: NULL argument"); return RR_EINVAL; }
    memset(o, 0, sizeof *o);
    std::lock_guard<std::mutex> lk(S->mu);
    o->submitted = S->submitted;
    o->completed = S->completed;
    o->polled = S->polled;
    o->queued = (int64_t)S->queue.size();
    o->in_flight = S->in_flight;
    o->batches = S->batches;
    o->mean_batch = S->batches ? (double)S->batched / S->batches : 0.0;
    o->bytes_held = S->bytes_held;
    o->admission_waits = S->admission_waits;
    o->canceled = S->canceled;
    o->reserve_per_request = (int64_t)S->reserve;
    const double secs = std::chrono::duration<double>(Clock::now() - S->t_reset).count();
    o->qps = secs > 0 ? S->completed / secs : 0.0;
    if (!S->lat_us.empty()) {
        std::vector<float> v = S->lat_us;
        auto pct = [&](double p) {
            size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * v.size() - 1e-9));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return (double)v[k];
        };
        o->p50_us = pct(0.50);
        o->p99_us = pct(0.99);
        double sum = 0, mx = 0;
        for (float x : S->lat_us) { sum += x; mx = std::max<double>(mx, x); }
        o->mean_us = sum / S->lat_us.size();
        o->max_us = mx;
    }
    if (reset) {
        S->submitted = S->completed = S->polled = S->batches = S->batched = S->admission_waits = S->canceled = 0;
        S->lat_us.clear();
        S->t_reset = Clock::now();
    }
    return RR_OK;
}

rr_status rr_serve_destroy(rr_server *S) {
    if (!S) return RR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &W : S->workers)
        if (W.th.joinable()) W.th.join();
    DeviceGuard dg(S->ix->device);
    S->done.clear();  // releases the batches nobody collected
    for (auto &W : S->workers) {
        if (W.st) cudaStreamSynchronize(W.st);
        if (W.view) rr_free_index(W.view);
        if (W.st) cudaStreamDestroy(W.st);
        if (W.qpin) cudaFreeHost(W.qpin);
    }
    if (S->cst) {
        cudaStreamSynchronize(S->cst);
        cudaStreamDestroy(S->cst);
    }
    if (S->cpin) cudaFreeHost(S->cpin);
    delete S;
    return RR_OK;
}

}  // extern "C"
