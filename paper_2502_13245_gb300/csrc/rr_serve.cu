// rr_serve.cu -- continuous batching of single range queries (serving).
//
// The paper evaluates batched search (Sec. 4); a service sees queries one at a
// time.  Worker threads turn the arrival stream into batches: each owns a CUDA
// stream and a scratch view of the index (shared vectors and graph), takes
// whatever is queued when it becomes free, searches it with the batched path
// of rr_range_search, and splits the CSR into per-request results.  With two
// or more workers one batch's host-side assembly overlaps the next batch's
// kernels.  Admission is by result memory: the match counts of range queries
// are heavy-tailed (Sec. 3), so a count of requests is no bound on memory.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
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

struct Done {
    rr_status status;
    std::string err;
    rr_result res;  // nq = 1, host arrays
    int64_t bytes;  // held against the budget until polled
};

struct Worker {
    std::thread th;
    rr_index *view = nullptr;
    cudaStream_t st = nullptr;
    uint8_t *qpin = nullptr;  // pinned batch of queries
    size_t qpin_cap = 0;
};

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
    std::unordered_map<uint64_t, int> live;  // queued or in flight or done-not-polled
    uint64_t next_ticket = 1;
    int64_t bytes_held = 0;
    int64_t in_flight = 0;
    bool stop = false;
    // statistics since the last reset
    int64_t submitted = 0, completed = 0, polled = 0, batches = 0, batched = 0, admission_waits = 0;
    std::vector<float> lat_us;
    Clock::time_point t_reset;
    std::vector<Worker> workers;
};

namespace {

int64_t result_bytes(int64_t count, bool stats) {
    return 8 * count + 16 + 1 + (stats ? (int64_t)sizeof(rr_query_stats) : 0);
}

// Split a host CSR result into single-query results (one per request).
rr_status split_one(const rr_result &b, int64_t i, bool stats, rr_result *o) {
    memset(o, 0, sizeof *o);
    const int64_t lo = b.offsets[i], cnt = b.offsets[i + 1] - lo;
    o->nq = 1;
    o->total = cnt;
    o->dist_dtype = b.dist_dtype;
    o->offsets = (int64_t *)malloc(2 * sizeof(int64_t));
    o->ids = (uint32_t *)malloc((size_t)std::max<int64_t>(cnt, 1) * 4);
    o->dists = malloc((size_t)std::max<int64_t>(cnt, 1) * 4);
    o->flags = (uint8_t *)malloc(1);
    if (stats) o->stats = (rr_query_stats *)malloc(sizeof(rr_query_stats));
    if (!o->offsets || !o->ids || !o->dists || !o->flags || (stats && !o->stats)) {
        rr_result_free(o);
        return RR_ENOMEM;
    }
    o->offsets[0] = 0;
    o->offsets[1] = cnt;
    if (cnt) {
        memcpy(o->ids, b.ids + lo, (size_t)cnt * 4);
        memcpy(o->dists, (const uint8_t *)b.dists + lo * 4, (size_t)cnt * 4);
    }
    o->flags[0] = b.flags[i];
    if (stats) o->stats[0] = b.stats ? b.stats[i] : rr_query_stats{};
    return RR_OK;
}

void worker_loop(rr_server *S, Worker *W) {
    DeviceGuard dg(S->ix->device);
    const rr_serve_cfg &C = S->cfg;
    const bool stats = C.params.collect_stats != 0;
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
            // admission: each request reserves reserve_per_request bytes of the budget
            batch.clear();
            while (!S->queue.empty() && (int64_t)batch.size() < C.max_batch) {
                bool fits = S->bytes_held + reserved + C.reserve_per_request <= C.result_budget_bytes;
                // always admit one when nothing is held; a stopping server drains its queue regardless
                bool progress = S->bytes_held + reserved == 0 || S->stop;
                if (!fits && !progress) break;
                batch.push_back(S->queue.front());
                S->queue.pop_front();
                reserved += C.reserve_per_request;
            }
            if (batch.empty()) {
                S->admission_waits++;
                // wait for a poll to free budget (or stop); re-check from the top
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
        rr_result res;
        memset(&res, 0, sizeof res);
        rr_status s = W->qpin ? rr_range_search(W->view, W->qpin, k, radii.data(), 0.0, C.variant, &P, W->st, 0, &res)
                              : RR_ENOMEM;
        if (s == RR_EOVERFLOW) s = RR_OK;  // truncated results are flagged per query
        std::string err = s == RR_OK ? std::string() : std::string(rr_last_error());
        std::vector<Done> out(k);
        for (int64_t j = 0; j < k; j++) {
            memset(&out[j].res, 0, sizeof out[j].res);
            out[j].status = s;
            out[j].err = err;
            out[j].bytes = 0;
            if (s == RR_OK) {
                rr_status t = split_one(res, j, stats, &out[j].res);
                if (t != RR_OK) { out[j].status = t; out[j].err = "result allocation failed"; }
                else out[j].bytes = result_bytes(out[j].res.total, stats);
            }
        }
        rr_result_free(&res);
        const Clock::time_point t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->bytes_held -= reserved;
            S->in_flight -= k;
            for (int64_t j = 0; j < k; j++) {
                S->bytes_held += out[j].bytes;
                S->lat_us.push_back(
                    (float)std::chrono::duration<double, std::micro>(t1 - batch[j].t0).count());
                S->done.emplace(batch[j].ticket, std::move(out[j]));
            }
            S->completed += k;
            S->batches += 1;
            S->batched += k;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // budget may have shrunk or grown
    }
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
    c->reserve_per_request = 0;  // 0: 8 bytes per beam slot
}

rr_status rr_serve_create(rr_index *ix, const rr_serve_cfg *cfg, rr_server **out) {
    if (!ix || !out) { set_error("rr_serve_create: NULL argument"); return RR_EINVAL; }
    *out = nullptr;
    rr_serve_cfg C;
    if (cfg) C = *cfg; else rr_serve_cfg_init(&C);
    if (C.workers < 1 || C.workers > 64 || C.max_batch < 1 || C.batch_wait_us < 0 || C.result_budget_bytes <= 0 ||
        C.reserve_per_request < 0 || C.variant < RR_BEAM || C.variant > RR_GREEDY_ES || C.params.beam < 1) {
        set_error("rr_serve_create: invalid configuration");
        return RR_EINVAL;
    }
    if (C.reserve_per_request == 0) C.reserve_per_request = 8 * (int64_t)C.params.beam + 32;
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
    S->row_bytes = (size_t)ix->d * elem_size(ix->dtype);
    S->t_reset = Clock::now();
    S->workers.resize(C.workers);
    for (auto &W : S->workers) {
        W.view = index_worker_view(ix);
        cudaError_t e = cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking);
        if (!W.view || e != cudaSuccess) {
            cudaGetLastError();
            for (auto &V : S->workers) {
                if (V.view) rr_free_index(V.view);
                if (V.st) cudaStreamDestroy(V.st);
            }
            delete S;
            set_error("rr_serve_create: worker set-up failed");
            return RR_ENOMEM;
        }
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
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->live.count(ticket)) { set_error("rr_serve_poll: unknown or retired ticket %llu", (unsigned long long)ticket); return RR_EINVAL; }
    auto ready = [&] { return S->done.count(ticket) != 0; };
    if (!ready()) {
        if (timeout_ms <= 0) return RR_EBUSY;
        if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return RR_EBUSY;
    }
    auto it = S->done.find(ticket);
    Done d = std::move(it->second);
    S->done.erase(it);
    S->live.erase(ticket);
    S->bytes_held -= d.bytes;
    S->polled++;
    lk.unlock();
    S->cv_work.notify_all();
    if (d.status != RR_OK) {
        set_error("%s", d.err.c_str());
        return d.status;
    }
    *out = d.res;
    return RR_OK;
}

rr_status rr_serve_collect(rr_server *S, uint64_t first, int64_t n, int32_t timeout_ms, rr_result *out) {
    if (!S || !out || n < 0) { set_error("rr_serve_collect: bad argument"); return RR_EINVAL; }
    memset(out, 0, sizeof *out);
    std::unique_lock<std::mutex> lk(S->mu);
    for (int64_t i = 0; i < n; i++)
        if (!S->live.count(first + (uint64_t)i)) {
            set_error("rr_serve_collect: unknown or retired ticket %llu", (unsigned long long)(first + i));
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
    std::vector<Done> got((size_t)n);
    int64_t total = 0, freed = 0;
    for (int64_t i = 0; i < n; i++) {
        auto it = S->done.find(first + (uint64_t)i);
        got[(size_t)i] = std::move(it->second);
        S->done.erase(it);
        S->live.erase(first + (uint64_t)i);
        freed += got[(size_t)i].bytes;
        total += got[(size_t)i].status == RR_OK ? got[(size_t)i].res.total : 0;
    }
    S->bytes_held -= freed;
    S->polled += n;
    lk.unlock();
    S->cv_work.notify_all();
    rr_status bad = RR_OK;
    std::string err;
    for (auto &g : got)
        if (g.status != RR_OK && bad == RR_OK) { bad = g.status; err = g.err; }
    const bool stats = S->cfg.params.collect_stats != 0;
    out->nq = n;
    out->total = total;
    out->dist_dtype = S->ix->dtype == RR_F32 ? 1 : 0;
    out->offsets = (int64_t *)malloc((size_t)(n + 1) * 8);
    out->ids = (uint32_t *)malloc((size_t)std::max<int64_t>(total, 1) * 4);
    out->dists = malloc((size_t)std::max<int64_t>(total, 1) * 4);
    out->flags = (uint8_t *)malloc((size_t)std::max<int64_t>(n, 1));
    if (stats) out->stats = (rr_query_stats *)calloc((size_t)std::max<int64_t>(n, 1), sizeof(rr_query_stats));
    const bool ok = out->offsets && out->ids && out->dists && out->flags && (!stats || out->stats);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; i++) {
        rr_result &r = got[(size_t)i].res;
        if (ok) {
            out->offsets[i] = pos;
            out->flags[i] = got[(size_t)i].status == RR_OK ? r.flags[0] : 0;
            if (got[(size_t)i].status == RR_OK && r.total) {
                memcpy(out->ids + pos, r.ids, (size_t)r.total * 4);
                memcpy((uint8_t *)out->dists + pos * 4, r.dists, (size_t)r.total * 4);
                pos += r.total;
            }
            if (stats && r.stats) out->stats[i] = r.stats[0];
        }
        rr_result_free(&r);
    }
    if (!ok) {
        rr_result_free(out);
        set_error("rr_serve_collect: result allocation failed");
        return RR_ENOMEM;
    }
    out->offsets[n] = pos;
    if (bad != RR_OK) {  // the requests are retired either way; report the first failure
        set_error("%s", err.c_str());
        return bad;
    }
    return RR_OK;
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
        S->submitted = S->completed = S->polled = S->batches = S->batched = S->admission_waits = 0;
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
    for (auto &W : S->workers) {
        if (W.st) cudaStreamSynchronize(W.st);
        if (W.view) rr_free_index(W.view);
        if (W.st) cudaStreamDestroy(W.st);
        if (W.qpin) cudaFreeHost(W.qpin);
    }
    for (auto &kv : S->done) rr_result_free(&kv.second.res);
    delete S;
    return RR_OK;
}

}  // extern "C"
