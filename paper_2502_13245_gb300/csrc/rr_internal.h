// rr_internal.h -- host-side internals shared by the librr translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rr.h"

namespace rr {

void set_error(const char *fmt, ...);
// kernels launched by this thread (a search counts its own launches)
void note_launch(int k = 1);
int64_t launches_so_far();
rr_status cuda_fail(cudaError_t e, const char *what);
// failure-path hooks set by rr_debug_set: true if this device allocation is to fail;
// the beam and doubling kernels' per-query iteration guard (default n + 1)
bool inject_alloc_failure();
int64_t beam_iteration_limit(int64_t n);

#define RR_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

// Grow-only device scratch arena owned by an index (one search at a time).
struct Arena {
    uint8_t *base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    rr_status reserve(size_t bytes);
    void reset() { used = 0; }
    // 256-byte aligned sub-allocation; nullptr if the reservation was too small
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

// Pinned host staging for small device->host reads.
struct Pinned {
    uint8_t *p = nullptr;
    size_t cap = 0;
};

// Grow-only device buffer.  grow() keeps the first `keep` bytes.
struct Grow {
    void *p = nullptr;
    size_t bytes = 0;
};
rr_status grow(Grow &g, size_t need, size_t keep, cudaStream_t st);
void grow_free(Grow &g);

}  // namespace rr

struct rr_index {
    int64_t n = 0;
    int32_t d = 0;
    int32_t dtype = 0;
    int32_t metric = 0;
    int32_t R = 0;
    int64_t start = 0;
    int32_t device = 0;
    int32_t row_stride = 0;  // bytes per stored vector, 16-byte aligned, zero padded
    uint8_t *vec = nullptr;  // n x row_stride
    uint32_t *adj = nullptr; // n x R
    int64_t device_bytes = 0;
    rr::Arena arena;        // per-call scratch sized before the beam phase
    rr::Pinned pinned;
    rr::Grow phase2;        // greedy / doubling per-query scratch
    rr::Grow item_key;      // greedy item list (keys)
    rr::Grow item_slot;     // greedy item list (slots)
    rr::Grow outbuf;        // output staging (sort keys, host-result staging)
    rr::Grow dbl_s[2];      // doubling: S of the active queries (double buffered)
    rr::Grow dbl_tmp;       // doubling: sort scratch of S u V
    rr::Grow cand;          // greedy candidate list of a level chunk (8-bit indexes)
    rr::Grow dbl_seen;      // warm-restart doubling: per-query bitmaps of every id evaluated
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // profile: start, beam, phase2, end
    rr_profile prof = {};
    // low-precision traversal copies of an fp32 index (built on first use)
    uint8_t *lp_bf16 = nullptr;
    int32_t lp_bf16_stride = 0;
    uint8_t *lp_fp8 = nullptr;
    int32_t lp_fp8_stride = 0;
    float2 *lp_fp8_info = nullptr;  // per row {scale, ||dequantised row||^2}
    float *lp_stats = nullptr;      // device scratch for max ||x|| and max |x_i|
    float max_norm = 0.f, max_abs = 0.f;
    // a worker view of another index: shares the vectors, adjacency and traversal copies
    // (not freed with it) and owns its own scratch, so views can search concurrently
    bool shared_data = false;
    // relabeled index: ext[internal id] = the caller's id (n entries), the caller's start point and the
    // order used; the parent of a worker view, and how many views of this index are alive
    uint32_t *ext = nullptr;
    int64_t start_ext = 0;
    int32_t order = 0;
    int32_t live_views = 0;
    rr_index *parent = nullptr;
};

namespace rr {
rr_index *index_worker_view(rr_index *parent);
// host arrays of a result: one pinned block from a small reuse pool (offsets at its base), else mallocs
bool host_result_arrays(rr_result *out, int64_t nq, int64_t total, bool stats);
void *host_pool_take(size_t bytes);
bool host_pool_give(void *p);
}  // namespace rr

namespace rr {

// Everything a search kernel reads about the index and the batch.
struct SearchArgs {
    const uint8_t *vec;       // n x row_stride
    const uint32_t *adj;      // n x R
    int64_t n;
    int32_t R;
    int32_t row_stride;       // bytes
    int32_t row_chunks;       // row_stride / 16
    int32_t lpv;              // lanes per vector (power of two)
    int32_t metric;
    uint32_t start;
    const uint8_t *queries;   // nq x row_stride (padded copy on the device)
    int64_t nq;
    const uint32_t *rkey;     // per query: dkey(radius)
    const uint32_t *eskey;    // per query: dkey(esr)
    int32_t beam;             // b
    int32_t use_es;
    int32_t es_vl;
    int32_t es_metric;        // rr_es_metric (the beam kernel; the doubling kernel takes RR_ES_VISITED)
    int32_t expand;           // parents per beam-kernel iteration (1 = Alg. 1; the doubling kernel takes 1)
    double es_ratio;          // threshold t of RR_ES_TOP10_RATIO
    int32_t phase2;           // 0 none, 1 greedy, 2 doubling: queries with |N| = b are queued
    // outputs of the beam phase
    uint64_t *res_keys;       // nq x beam: N (sorted keys, visited bit cleared)
    int32_t *res_count;       // nq
    uint8_t *flags;           // nq
    int32_t *p2_list;         // queries queued for phase 2
    int32_t *p2_count;        // device counter
    rr_query_stats *stats;    // nq or nullptr
    uint32_t *count_bits;     // exact distinct-id bitmaps (stats mode), nq x words_per_q, or nullptr
    int64_t words_per_q;
    int32_t *error;           // device status word (0 = fine)
    int32_t hash_lg;          // log2 of the beam kernel's seen-table slots (0 = library default)
    int32_t persistent;       // 1: resident grid, queries taken from *next_q (must start at 0)
    int32_t *next_q;
    // low-precision traversal (fp32 indexes): vec/row_* above describe the exact fp32 rows
    int32_t prec;             // RR_PREC_EXACT / BF16 / FP8
    int32_t d;                // elements per vector
    const uint8_t *lp_vec;    // traversal rows
    int32_t lp_stride, lp_chunks, lp_lpv;
    const float2 *lp_info;    // fp8: {scale, ||x||^2} per row
    float slackA, slackB, slackC;  // |d - d~| <= A ||q|| + B ||q||^2 + C
    float rel_eps;            // > 0: slack = rel_eps * |r| instead
    int64_t iter_limit;       // per-query iteration guard of the beam / doubling kernels (n + 1 by default)
    // graph construction (launch_build_search): query i is the stored row qids[i]; the first vis_cap
    // visits of query i are written, in visit order, to vis_out[i * vis_cap ..] and their number to
    // vis_count[i]
    const uint32_t *qids;
    uint32_t *adj_w;          // the adjacency, writable (construction only)
    uint64_t *vis_out;
    int32_t vis_cap;
    int32_t *vis_count;
    const uint32_t *ext;      // exhaustive scan of a relabeled index: internal id -> caller's id
};

rr_status ensure_lowp(rr_index *ix, int prec, cudaStream_t st);
void slack_coefficients(const rr_index *ix, int prec, float *A, float *Bq, float *C);

rr_status launch_beam(const SearchArgs &a, int warps_per_cta, cudaStream_t s, int dtype_code);
// Alg. 1 without early stop or range filter for graph construction: the queries are stored rows
// (a.qids), the visits are recorded (a.vis_out); 8-bit indexes only
rr_status launch_build_search(const SearchArgs &a, int warps_per_cta, cudaStream_t s, int dtype_code);
int beam_hash_lg(int beam);

struct GreedyArgs {
    SearchArgs s;
    int32_t ng;                // greedy queries
    const int32_t *qlist;      // slot -> query index
    uint32_t *seen;            // ng x words_per_q exact bitmaps
    int64_t seen_words;
    uint64_t *item_key;        // appended in-range results (keys)
    int32_t *item_slot;
    unsigned long long *tail;  // device append cursor
    int64_t cap;               // item capacity
    int32_t *slot_count;       // results per slot
    int32_t *slot_trunc;       // 1 if a result of the slot was dropped (capacity)
    int64_t begin, end;        // current level [begin, end)
    // 8-bit indexes: a level runs as an expand pass and an evaluate pass over a candidate list
    uint64_t *cand;            // {id, slot, query, 0} (16 bytes each) of the neighbours first seen in this
                               // chunk of the level
    unsigned long long *ccount;  // device: candidates appended (zeroed before each chunk)
    int64_t ccap;              // candidate capacity (items per chunk x R)
};

rr_status launch_greedy_init(const GreedyArgs &g, cudaStream_t s, int dtype_code);
rr_status launch_greedy_level(const GreedyArgs &g, cudaStream_t s, int dtype_code);
// true when launch_greedy_level runs the two-pass form (expand, then evaluate) for this element type;
// it then needs g.cand / g.ccount sized for the level's chunk, and processes items [begin, end) of g
bool greedy_two_pass(int dtype_code);

// One round of Alg. 3 (a BeamSearch with beam b from B = top-b(S)) for the
// active doubling slots; i indexes the active list, slot = act[i].
struct DoublingRound {
    SearchArgs s;             // s.beam = b of this round
    int32_t na;               // active slots
    const int32_t *act;       // i -> slot
    const int32_t *qlist;     // slot -> query
    int32_t first;            // round 1: S = {start}
    int32_t last;             // 2b > b_max: a full N ends the search (truncated)
    const uint64_t *s_old;    // i x s_cap: S (sorted keys, distinct ids)
    const int32_t *s_cnt;
    int64_t s_cap;
    uint64_t *bA, *bB;        // i x b: the beam (double buffered)
    uint64_t *v;              // i x v_cap: V of this round (keys)
    int64_t v_cap;
    int32_t *nv;              // |V| per i
    uint32_t *seen;           // i x seen_words: ids evaluated this round (exact)
    int64_t seen_words;
    int32_t *status;          // out per i: 1 continue (|N| = b), 0 finished
    uint64_t *item_key;       // results of finished slots are appended here
    int32_t *item_slot;
    unsigned long long *tail;
    int64_t cap;
    int32_t *slot_count;      // per slot: final |N|
    int32_t *slot_trunc;      // per slot: 1 if b_max or a capacity cut the search
    // warm restart (a variant of Alg. 3): s_old holds E, the closest keys evaluated so far with their
    // visited bits (kept as they are); seen is indexed by slot and kept across rounds (every id ever
    // evaluated); the round appends every key it evaluates to ev (ev_cap per i, counts in nev)
    int32_t warm;
    uint64_t *ev;
    int64_t ev_cap;
    int32_t *nev;
};

// S <- S u V for the continuing slots, truncated to the b_max smallest keys
// (later rounds never start from more than b_max of them); j indexes the
// continuing list, cont[j] its round index i.
struct DoublingSUpdate {
    int32_t nc;
    const int32_t *cont;
    const uint64_t *s_old;
    const int32_t *s_cnt_old;
    int64_t s_cap_old;
    const uint64_t *v;
    const int32_t *nv;
    int64_t v_cap;
    uint64_t *s_new;
    int32_t *s_cnt_new;
    int64_t s_cap_new;
    uint64_t *tmp;            // j x (s_cap_old + v_cap): sort scratch for long lists
    int32_t first;            // S_old = {start} (its key is V[0] of round 1)
    // warm restart: E_new <- the s_cap_new closest of E_old u ev, with the visited bit of every key of V set
    // (tmp then holds j x (s_cap_old + ev_cap + v_cap))
    int32_t warm;
    const uint64_t *ev;
    const int32_t *nev;
    int64_t ev_cap;
};

rr_status launch_doubling_round(const DoublingRound &d, cudaStream_t s, int dtype_code);
rr_status launch_doubling_supdate(const DoublingSUpdate &u, cudaStream_t s);
rr_status launch_zero_words(uint32_t *p, int64_t nwords, cudaStream_t s);

// Output assembly.
rr_status launch_scan(const int32_t *counts, int64_t n, int64_t *offsets, cudaStream_t s);
struct OutArgs {
    int64_t nq;
    const int64_t *offsets;
    int32_t dist_is_float;
    uint32_t *ids;
    void *dists;
    uint8_t *flags;
    int64_t total;            // entries in ids / dists (and in the sort keys); writes beyond are refused
    int32_t *error;           // device status word: set to 4 if a write would leave the arrays
    const uint32_t *ext;      // relabeled index: internal id -> caller's id (nullptr: ids pass through)
};
// copy sorted per-query key slots (stride per query) into the CSR
rr_status launch_copy_slots(const OutArgs &o, const uint64_t *keys, int64_t stride, const int32_t *count,
                            const int32_t *qlist, int32_t nlist, cudaStream_t s);
// scatter items (slot, key) to CSR positions of their queries, then sort each listed segment
rr_status launch_scatter_items(const OutArgs &o, const uint64_t *item_key, const int32_t *item_slot,
                               int64_t nitems, const int32_t *qlist, int32_t *cursor, uint64_t *tmp_keys,
                               cudaStream_t s);
rr_status launch_sort_segments(const OutArgs &o, uint64_t *tmp_keys, const int32_t *qlist, int32_t nlist,
                               int64_t max_seg, cudaStream_t s);

// Brute force (Def. 2.1): count pass and fill pass over all (query, point) pairs.
rr_status launch_brute(const SearchArgs &a, int32_t *counts, const int64_t *offsets, int32_t *cursor,
                       uint64_t *keys, int fill, cudaStream_t s, int dtype_code);
// after the greedy levels: slot_count[s] += the items of slot s among items [0, n)
rr_status launch_count_items(const int32_t *item_slot, int64_t n, int32_t *slot_count, cudaStream_t s);
// after phase 2: res_count[qlist[s]] = slot_count[s]; truncated slots flag their query
rr_status launch_set_counts(int32_t *res_count, uint8_t *flags, const int32_t *qlist, const int32_t *slot_count,
                            const int32_t *slot_trunc, int32_t n, cudaStream_t s);

}  // namespace rr

namespace rr {
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};
bool is_device_ptr(const void *p);
int elem_size(int dtype);
bool radius_key(double r, int dtype, uint32_t *key);
}  // namespace rr
