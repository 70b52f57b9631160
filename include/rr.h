/*
 * rr.h -- C ABI of librr.so: batched range retrieval on a proximity graph, on
 * one NVIDIA GB300 (sm_103a).
 *
 * The method is "Range Retrieval with Graph-Based Indices" (arXiv 2502.13245):
 *   Def. 2.1  range search: every point p with d(p, q) <= r;
 *   Alg. 1    BeamSearch, Alg. 5 early stopping on d_visited,
 *   Alg. 2    GreedySearch (in-radius expansion), Alg. 3 DoublingSearch,
 *   Alg. 6    GreedyRangeSearch, the per-query driver (a parallel for over
 *             queries; here one launch over the whole batch).
 * Distances are squared L2 or negative inner product (Sec. 2): exact int32 for
 * 8-bit vectors, fp32 for float vectors.  Ties are broken by (distance, id)
 * everywhere, so on 8-bit data the results are bit-exact against a plain CPU
 * transcription of the algorithms.
 *
 * Conventions for every entry point:
 *   - the return value is an rr_status; on failure rr_last_error() returns a
 *     message for the calling thread (valid until that thread's next call);
 *   - no C++ exception and no device trap crosses this boundary; device-side
 *     problems (iteration guard, result overflow) come back as statuses;
 *   - pointers may be host or device memory where stated ("host or device":
 *     the library asks the driver which it is);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); all device work of a call is ordered on it.
 * Thread safety: calls on different rr_index handles may run concurrently;
 * calls on the same handle must be serialised by the caller (the handle owns
 * one scratch arena).
 */
#ifndef RR_H
#define RR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RR_OK = 0,
    RR_EINVAL = 1,     /* bad argument */
    RR_ENOMEM = 2,     /* host or device allocation failed */
    RR_ECUDA = 3,      /* a CUDA runtime call failed */
    RR_EFORMAT = 4,    /* index file malformed or checksum mismatch */
    RR_EOVERFLOW = 5,  /* phase-2 results exceeded max_results_total, or doubling hit b_max
                          (a valid, truncated result is kept; RR_FLAG_TRUNCATED marks the queries) */
    RR_ETIMEOUT = 6,   /* a device wait or host poll ran out of time */
    RR_EBUSY = 7,      /* serving: request not finished yet, or queue full */
    RR_EINTERNAL = 8   /* a device-side guard tripped (should not happen) */
} rr_status;

/* Search variants (Sec. 4):
 *   RR_BEAM          Alg. 1, returns {n in B : d(n,q) <= r} (at most b results)
 *   RR_BEAM_ES       the same with Alg. 5 early stopping
 *   RR_DOUBLING(_ES) Alg. 3 from the start point: repeat Alg. 1 with S <- S u V,
 *                    b <- 2b while |N| = b (lambda = 1), beam capped at b_max
 *   RR_GREEDY(_ES)   Alg. 6: Alg. 1, then Alg. 2 seeded with N when |N| = b   */
typedef enum {
    RR_BEAM = 0,
    RR_BEAM_ES = 1,
    RR_DOUBLING = 2,
    RR_DOUBLING_ES = 3,
    RR_GREEDY = 4,
    RR_GREEDY_ES = 5,
    /* warm-restart doubling, a variant of Alg. 3 that is not in the paper: each round continues the
     * last instead of restarting from B = S with V = {}.  E (every point evaluated, with its distance)
     * and V are kept across rounds; a round with beam b starts from the b closest points of E and runs
     * Alg. 1's loop without visiting a point of V again; it stops when |N| < b, else b doubles (capped
     * by b_max as in Alg. 3).  The first round is Alg. 1 from the start point, as in Alg. 3. */
    RR_DOUBLING_WARM = 6,
    RR_DOUBLING_WARM_ES = 7
} rr_variant;

typedef enum { RR_U8 = 0, RR_I8 = 1, RR_F32 = 2 } rr_dtype;
typedef enum { RR_L2 = 0, RR_IP = 1 } rr_metric;

/* Traversal precision for fp32 indexes (Sec. 5 traverses floats in 8 bits and
 * re-ranks; here BF16 or FP8-e4m3 with a per-vector scale and FP32
 * accumulation).  Membership is always decided by an exact fp32 recheck. */
typedef enum { RR_PREC_EXACT = 0, RR_PREC_BF16 = 1, RR_PREC_FP8 = 2 } rr_precision;

/* Per-query result flags (rr_result.flags). */
enum {
    RR_FLAG_TRUNCATED = 1,     /* doubling hit b_max, or results hit max_results_total */
    RR_FLAG_EARLY_STOPPED = 2, /* Alg. 5 ended the first beam search */
    RR_FLAG_PHASE2 = 4,        /* the greedy or doubling phase ran */
    RR_FLAG_CANCELED = 8       /* serving: dropped by rr_serve_cancel before it was searched */
};

typedef struct rr_index rr_index;

typedef struct {
    int32_t beam;              /* b, the (starting) beam width, >= 1 */
    int32_t b_max;             /* doubling cap on b (default 32768) */
    int32_t es_visit_limit;    /* Alg. 5 vl (default 20) */
    int32_t es_radius_mode;    /* 0: esr = the query's radius; 1: esr = es_radius */
    double es_radius;          /* Alg. 5 esr when es_radius_mode = 1 */
    int32_t precision;         /* rr_precision (fp32 indexes only) */
    float recheck_eps;         /* low-precision slack: recheck when approx <= r + eps*|r| (0 = derive) */
    int32_t persistent;        /* 1: one persistent launch with a device work queue */
    int32_t collect_stats;     /* 1: fill rr_result.stats (exact visit / distinct-id counts) */
    int64_t max_results_total; /* cap on the summed results of the greedy / doubling phase (0 = default
                                  1<<28); each query's first beam (at most b results) is always kept */
    int32_t tile_hint;         /* warps per CTA for the beam kernel (0 = library choice) */
    int32_t profile;           /* 1: record per-phase device times, see rr_last_profile */
    int32_t seen_log2;         /* log2 slots of the beam kernel's seen table, 5..14 (0 = library choice) */
    int32_t es_metric;         /* the M of Alg. 4 (Sec. 3.2), see rr_es_metric; RR_ES_VISITED is Alg. 5 */
    int32_t expand;            /* parents per BeamSearch iteration, 1..4 (0 or 1 = Alg. 1 itself; beam and
                                  greedy variants only).  expand = E > 1 is a variant of Alg. 1 that is not
                                  in the paper: each iteration visits the E closest unvisited points of B
                                  at once (Alg. 5 tests the first), adds the out-neighbours of all of them
                                  that are not in V or B, then trims B to b once */
    int32_t reserved[3];
} rr_params;

/* Early-stopping metrics (Sec. 3.2; Alg. 4 with this M replacing Alg. 5's last
 * test).  The search stops when the closest point of B is outside r, |V| >= vl,
 * and M exceeds its threshold:
 *   RR_ES_VISITED      d(p*, q) > esr                      (Alg. 5, the default)
 *   RR_ES_TOP1         d of the closest point of B > esr
 *   RR_ES_TOP10        d of the 10th closest point of B (the farthest while
 *                      |B| < 10) > esr
 *   RR_ES_TOP10_RATIO  d_top10 > t * d(start, q), t = es_radius (es_radius_mode
 *                      must be 1; squared L2 only)
 * Beam and greedy variants take every metric (rr_beam_search_noalloc too);
 * the doubling variants take RR_ES_VISITED only (RR_EINVAL otherwise). */
typedef enum { RR_ES_VISITED = 0, RR_ES_TOP1 = 1, RR_ES_TOP10 = 2, RR_ES_TOP10_RATIO = 3 } rr_es_metric;

/* Exact per-query counters (collect_stats = 1).  visits_* count |V| of the
 * algorithms; distinct counts the distinct ids whose distance was evaluated. */
typedef struct {
    int32_t visits_beam;   /* summed over every BeamSearch round */
    int32_t visits_phase2; /* GreedySearch visits (= result count when it ran) */
    int32_t distinct;      /* distinct ids evaluated (start point included) */
    int32_t rounds;        /* BeamSearch calls */
    int32_t final_beam;    /* b of the last BeamSearch */
    int32_t evals;         /* distance evaluations actually performed by the GPU */
} rr_query_stats;

/* Results as CSR: query i owns ids[offsets[i] .. offsets[i+1]) sorted by
 * (distance, id).  dists holds int32 (integer indexes) or float32 (fp32
 * indexes), see dist_dtype.  Allocated by the library, freed by rr_result_free. */
typedef struct {
    int64_t nq;
    int64_t total;
    int64_t *offsets;        /* nq + 1 entries */
    uint32_t *ids;
    void *dists;
    int32_t dist_dtype;      /* 0 = int32, 1 = float32 */
    int32_t on_device;       /* 1: all arrays are device memory */
    uint8_t *flags;          /* nq entries of RR_FLAG_* */
    rr_query_stats *stats;   /* nq entries, or NULL unless collect_stats */
    void *_stream;           /* internal: stream the device arrays are ordered on */
    int32_t _device;
    int32_t _pad;
} rr_result;

/* Fill *p with the defaults: beam 64, b_max 32768, vl 20, esr = r, exact
 * precision, no persistent kernel, no stats, max_results_total 1<<28. */
void rr_params_init(rr_params *p);

/* Build an index from arrays in host or device memory; the library copies
 * them into device memory it owns on `device`.
 *   vectors    n x d row-major, element type dtype
 *   adjacency  n x R uint32 row-major; 0xFFFFFFFF pads rows of degree < R
 *   start      entry point of every search (the medoid), 0 <= start < n
 * Requirements: 1 <= n < 2^31, 1 <= d <= 512 (any element type; the BF16
 * traversal of the precision form takes d <= 256), 1 <= R <= 128, every
 * non-padding adjacency entry < n.  Adjacency entries are not validated on the device;
 * invalid ids give RR_EINVAL when validate != 0 (a host-side scan). */
rr_status rr_create_index(const void *vectors, int64_t n, int32_t d, int32_t dtype, int32_t metric,
                          const uint32_t *adjacency, int32_t R, int64_t start, int32_t device,
                          int32_t validate, rr_index **out);

/* Build a proximity graph on the GPU: a deterministic Vamana-style graph (the
 * paper searches a DiskANN / Vamana graph with parameters R, L and alpha,
 * Sec. 4.1, and leaves its construction to that system; this is the
 * construction step of the index, not the range search).
 *   vectors    n x d row-major uint8 or int8 (dtype), host or device memory
 *   metric     RR_L2 or RR_IP (alpha applies to the metric value: squared L2)
 *   R, L       out-degree bound (2..128) and construction beam (1..512)
 *   alpha      RobustPrune's alpha (>= 1); with passes >= 2 the first pass
 *              uses alpha = 1
 *   seed       insertion order (a seeded permutation with `start` first)
 *   start      the entry point (the medoid); every point ends up reachable
 *              from it (a final repair attaches unreached points)
 *   adjacency  out: n x R uint32 in HOST memory, 0xFFFFFFFF pads each row
 *   info       optional: batches run, points attached by the repair, time
 * Batches of 1, 2, 4, ... points (capped at n/50) each search the graph as it
 * stood before the batch (Alg. 1 with beam L from start), RobustPrune their
 * first 4L + 16 visits plus their current neighbours into a row of at most
 * R - max(1, R/16) entries, then merge reverse edges per target in batch
 * order (appended, or the target re-pruned when its row would overflow).
 * Every order is by (distance, id) and every step reads a snapshot, so the
 * result does not depend on the GPU's scheduling: for the same arguments it
 * equals the project's CPU builder (rrsynth) array for array.  Device memory:
 * about n*(row + 4R + 12) bytes plus n/50 * (8*(4L+16) + 28R) bytes of batch
 * scratch.  fp32 vectors: RR_EINVAL.  Errors: RR_EINVAL, RR_ENOMEM, RR_ECUDA,
 * RR_EINTERNAL (a device guard). */
typedef struct {
    int64_t batches;        /* insertion batches over all passes */
    int64_t repaired;       /* points attached by the reachability repair */
    double gpu_seconds;     /* wall time of the passes (device work + copies) */
    double repair_seconds;  /* wall time of the host-side repair */
} rr_build_info;

rr_status rr_build_graph(const void *vectors, int64_t n, int32_t d, int32_t dtype, int32_t metric, int32_t R,
                         int32_t L, double alpha, int32_t passes, uint64_t seed, int64_t start, int32_t device,
                         uint32_t *adjacency, rr_build_info *info);

/* Load an index file (.rrx, little endian): a 64-byte header
 *   'RRX1', u32 version 1, i64 n, i32 d, i32 dtype, i32 metric, i32 R,
 *   i64 start, u64 checksum, 16 zero bytes
 * then the vectors (n*d elements) and the adjacency (n*R uint32).  The
 * checksum is XOR over the payload's little-endian u64 words w_i (zero padded)
 * of (w_i * 0x100000001B3 + i).  Errors: RR_EFORMAT (bad header, size or
 * checksum), RR_EINVAL (bad values), RR_ENOMEM, RR_ECUDA. */
rr_status rr_load_index(const char *path, int32_t device, rr_index **out);

rr_status rr_free_index(rr_index *index);

typedef struct {
    int64_t n;
    int32_t d;
    int32_t dtype;
    int32_t metric;
    int32_t R;
    int64_t start;
    int64_t device_bytes;  /* HBM held by the index (vectors, low-precision copies, adjacency) */
    int32_t row_stride;    /* bytes per stored vector (16-byte aligned) */
    int32_t device;
    int64_t scratch_bytes; /* search scratch the index holds (device arenas + pinned staging); grow-only */
    int32_t order;         /* 0, or the rr_order the index was relabeled in (rr_index_relabel) */
    int32_t reserved;
} rr_index_info;

rr_status rr_index_info_get(const rr_index *index, rr_index_info *info);

/* Point orders for rr_index_relabel. */
typedef enum { RR_ORDER_BFS = 1 } rr_order;

/* Relabel an index's points so that points close in the graph are close in
 * device memory (a layout step of this library; the paper searches the graph
 * in the id order it was built in).  Internal id i is the i-th point of the
 * order; the vectors, the adjacency (entries renamed, slot order kept) and the
 * start point move with it, and every id the library hands back -- search,
 * server, no-alloc call, brute force -- is translated to the caller's id.  The
 * greedy expansion's per-query visited bitmaps (Alg. 2) and the vector and
 * adjacency gathers of every variant then touch fewer distinct sectors.
 *   RR_ORDER_BFS  a queue-based breadth-first traversal from the start point
 *                 that scans each row in slot order (padding skipped) and
 *                 numbers a point when it is first reached; points it never
 *                 reaches follow in ascending id order.
 * What changes for results: a search on the relabeled index is the search on
 * the relabeled arrays, so the beam phase's tie-breaks between equal keys
 * (Alg. 1, by (distance, id)) use internal ids, and the results of a query
 * come sorted by (distance, internal id) -- by distance, but equal distances
 * in internal order.  rr_brute_force stays in (distance, id) order.
 * Call it once, after rr_create_index / rr_load_index and before a server is
 * created on the index; low-precision traversal copies are rebuilt on their
 * next use.  Host memory: the adjacency (4nR bytes) and 13n bytes, freed on
 * return; device memory: a second copy of the vectors and the adjacency while
 * it runs, then 4n bytes for the id map.  Synchronous.  Errors: RR_EINVAL
 * (unknown order, an index already relabeled, a worker view, an index with a
 * live server, or an adjacency entry that is neither padding nor < n),
 * RR_ENOMEM, RR_ECUDA. */
rr_status rr_index_relabel(rr_index *index, int32_t order);

/* Batched range search (Alg. 6 / Alg. 3 / plain beam search over a batch).
 *   queries    nq x d, the index's element type, host or device memory
 *   radii      nq radii (host memory), or NULL to use `radius` for every query;
 *              in the metric's own units (squared L2, or negative inner product)
 *   variant    rr_variant; params may be NULL (defaults)
 *   result_on_device  1: result arrays in device memory (ordered on stream),
 *              0: host memory: one pinned block from a library-owned pool
 *              (at most 4 blocks, each reused once its result is freed, held
 *              until the process exits), or malloc'd arrays when none is free
 * Returns once the result sizes are known (one host synchronisation per
 * phase); the CSR is complete when the call returns for host results, and
 * when `stream` reaches this point for device results.  RR_EOVERFLOW keeps a
 * valid, truncated result with RR_FLAG_TRUNCATED set on the affected queries. */
rr_status rr_range_search(rr_index *index, const void *queries, int64_t nq, const double *radii, double radius,
                          int32_t variant, const rr_params *params, void *stream, int32_t result_on_device,
                          rr_result *out);

/* Exact range search by exhaustive scan (Def. 2.1), the ground truth for
 * average precision (Def. 2.2).  Same argument conventions as
 * rr_range_search; 8-bit indexes use exact integer arithmetic. */
rr_status rr_brute_force(rr_index *index, const void *queries, int64_t nq, const double *radii, double radius,
                         void *stream, int32_t result_on_device, rr_result *out);

/* Per-phase device times of the last rr_range_search on an index that ran
 * with params.profile = 1 (CUDA events on the call's stream), and the number
 * of kernels the call launched.  Waits for the call's last event. */
typedef struct {
    float beam_ms;        /* beam phase: Alg. 1 (+ Alg. 5), range filter, phase-2 queue */
    float phase2_ms;      /* Alg. 2 levels or Alg. 3 rounds (0 if none ran) */
    float output_ms;      /* scan, copy / scatter, per-query sort */
    float total_ms;       /* first to last event of the call */
    int32_t launches;     /* kernels launched by the call */
    int32_t phase2_steps; /* greedy levels or doubling rounds */
    int32_t phase2_queries;
    int32_t valid;        /* 1 if the last call on this index was profiled */
} rr_profile;

rr_status rr_last_profile(rr_index *index, rr_profile *out);

/* Beam search without any memory allocation (the paper has no counterpart:
 * this is a deployment variant of RR_BEAM / RR_BEAM_ES, Alg. 1 + Alg. 5 plus
 * the range filter).  For callers that may not allocate -- e.g. code running
 * under a memory budget reserved up front, inside a host callback, or after
 * start-up under a no-allocation policy.  rr_range_search allocates its
 * result and grows per-index scratch; this call allocates nothing.
 *   queries     nq x d device array of the index's element type
 *   radius      one radius for every query (metric units)
 *   variant     RR_BEAM or RR_BEAM_ES; params may be NULL (defaults; b <= 512).
 *               The beam, the early-stop settings (every rr_es_metric) and the
 *               launch shape (tile_hint, seen_log2, persistent) are honoured as
 *               in rr_range_search; precision must be RR_PREC_EXACT (the
 *               low-precision copies are allocated on first use): RR_EINVAL
 *               otherwise
 *   out_counts  nq int32 (device): |N| of each query
 *   out_ids     nq x b uint32 (device): N of query i in out_ids[i*b ..], sorted
 *               by (distance, id); slots past out_counts[i] hold 0xFFFFFFFF
 *   out_dists   nq x b int32 (8-bit indexes) or float32 (fp32 indexes), device
 * Intermediate data live in one static device array of 32 MiB per GPU that
 * loads the library, held until the process exits; a batch that needs more
 * (about nq*(b*8 + 16) bytes, plus nq*row for unaligned queries) is rejected
 * with RR_EINVAL -- split it.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress); make it before any stream capture.
 * Calls share the array: calls whose work overlaps on the GPU race, so
 * serialise them.  The call synchronises `stream`: it returns after the stream
 * has finished the call's work.  Results equal rr_range_search's for the same
 * variant and params. */
rr_status rr_beam_search_noalloc(rr_index *index, const void *queries, int64_t nq, double radius, int32_t variant,
                                 const rr_params *params, void *stream, int32_t *out_counts, uint32_t *out_ids,
                                 void *out_dists);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of range queries that arrive one by one (the
 * batched search of Alg. 6 / Alg. 3 run as a service).  `workers` host threads
 * each own a CUDA stream and a scratch view of the index; each repeatedly
 * forms a batch from everything queued (up to max_batch, waiting at most
 * batch_wait_us for it to fill), searches it, and publishes the requests'
 * results, so requests that arrive while other batches are on the GPU are
 * admitted into the next free worker and their work overlaps on the device.
 * A batch's CSR stays in host memory, or in device memory when
 * result_on_device = 1, until its requests are collected; each request's row
 * is copied out once, by rr_serve_poll / rr_serve_collect (device results: by
 * the copy engines, on a stream of the highest priority).
 * Admission is by result memory, because match counts are heavy-tailed: a
 * request is admitted only while the bytes of results held (finished but not
 * yet collected, plus a reservation for each request in flight) stay within
 * result_budget_bytes; one request is always admitted when nothing is held,
 * so the server makes progress.  The reservation is reserve_per_request, or
 * (0, the default) a running mean of the bytes requests have turned out to
 * hold, never below 8 * beam + 32.  A batch's results are capped at what
 * the budget has left (at least its reservation; each request's first beam of
 * up to b results is always kept); a request whose results were cut carries
 * RR_FLAG_TRUNCATED and holds a subset of its answer.
 * Each request's result is the same as in any other batch (every query is
 * searched independently).
 * ------------------------------------------------------------------------- */
typedef struct rr_server rr_server;

typedef struct {
    int32_t workers;             /* concurrent batches (default 2) */
    int32_t max_batch;           /* requests per batch (default 4096) */
    int32_t batch_wait_us;       /* wait for a batch to fill (default 200 us) */
    int32_t variant;             /* rr_variant of every request (default RR_GREEDY_ES) */
    rr_params params;            /* search parameters (rr_params_init defaults) */
    int64_t result_budget_bytes; /* admission budget (default 4 GiB) */
    int64_t reserve_per_request; /* bytes reserved per request in flight (0 = running mean, see above) */
    int32_t result_on_device;    /* 1: results in device memory (on the device the index lives on) */
    int32_t reserved_cfg[3];
} rr_serve_cfg;

typedef struct {
    int64_t submitted, completed, polled, queued, in_flight;
    int64_t batches;
    double mean_batch;           /* requests per batch */
    double p50_us, p99_us, mean_us, max_us;  /* submit -> result ready, since the last reset */
    double qps;                  /* completions per second since the last reset */
    int64_t bytes_held;          /* result bytes held + reserved */
    int64_t admission_waits;     /* times a worker stopped filling a batch for lack of budget */
    int64_t canceled;            /* requests dropped by rr_serve_cancel */
    int64_t reserve_per_request; /* the current reservation per admitted request (bytes) */
} rr_serve_stats_t;

void rr_serve_cfg_init(rr_serve_cfg *cfg);
/* Start a server on an index (the index must outlive it). */
rr_status rr_serve_create(rr_index *index, const rr_serve_cfg *cfg, rr_server **out);
/* Queue n requests: queries n x d in host memory (the index's element type),
 * radii (n, host) or NULL for `radius`.  Tickets first_ticket .. first_ticket+n-1. */
rr_status rr_serve_submit(rr_server *srv, const void *queries, int64_t n, const double *radii, double radius,
                          uint64_t *first_ticket);
/* Wait up to timeout_ms (0 = do not wait) for a ticket.  RR_OK: *out is that
 * request's result (nq = 1, host memory -- device memory with
 * result_on_device -- free with rr_result_free) and the ticket is retired;
 * RR_EBUSY: still pending (nothing allocated); RR_EINVAL: unknown or retired.
 * A request whose search failed is retired with an empty row: *out is
 * allocated all the same and the call returns the search's status. */
rr_status rr_serve_poll(rr_server *srv, uint64_t ticket, int32_t timeout_ms, rr_result *out);
/* Wait up to timeout_ms for the n consecutive tickets first .. first+n-1 (as
 * returned by one rr_serve_submit) and return their results as one CSR (nq =
 * n, in ticket order; host memory, or device memory with result_on_device,
 * complete when the call returns), retiring them.  RR_EBUSY: not all done yet
 * (nothing retired, nothing allocated).  A request that failed is retired with
 * an empty row; *out is allocated all the same and the call returns the first
 * failure's status. */
rr_status rr_serve_collect(rr_server *srv, uint64_t first, int64_t n, int32_t timeout_ms, rr_result *out);
/* Drop every request still queued (those in flight finish): each is retired
 * as done with an empty row flagged RR_FLAG_CANCELED, to be collected as
 * usual.  Returns how many were dropped.  For shedding load, and for ending a
 * measurement window under overload. */
int64_t rr_serve_cancel(rr_server *srv);
/* Counters and latency percentiles; reset = 1 starts a new measurement window. */
rr_status rr_serve_stats(rr_server *srv, rr_serve_stats_t *out, int32_t reset);
/* Stop the workers (queued requests are finished first) and free the server. */
rr_status rr_serve_destroy(rr_server *srv);

/* Copy a result into host memory: *host becomes a host result with the same
 * content (free with rr_result_free); a host result is copied as it is.
 * Waits for the stream a device result is ordered on. */
rr_status rr_result_to_host(const rr_result *result, rr_result *host);

/* sizeof of the public structs, for bindings to check their layouts against:
 * out[0..7] = rr_params, rr_query_stats, rr_result, rr_index_info, rr_profile,
 * rr_serve_cfg, rr_serve_stats_t, rr_build_info.  Needs no GPU. */
void rr_abi_sizes(int64_t out[8]);

/* Free the arrays of a result (host or device) and zero the struct; a pooled
 * host block goes back to the pool.  The arrays must not be freed any other way. */
rr_status rr_result_free(rr_result *result);

/* Message of the calling thread's last failure ("" if none). */
const char *rr_last_error(void);

/* Failure-path hooks for tests (the paper has no counterpart).  Process-wide,
 * off by default; each takes effect for calls that start after it is set.
 *   "fail_alloc_after"      value N >= 0: the library's (N+1)-th device
 *                           scratch or result allocation from now on fails as
 *                           if the device were out of memory (the call
 *                           returns RR_ENOMEM and frees what it took); -1 = off
 *   "beam_iteration_limit"  value L > 0: the beam and doubling kernels give up
 *                           a query after L iterations of Alg. 1's loop and
 *                           the call returns RR_EINTERNAL (the guard that
 *                           normally sits at n + 1 iterations); 0 = default
 * Returns RR_EINVAL for an unknown key. */
rr_status rr_debug_set(const char *key, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* RR_H */
