/*
 * rrsynth/vamana.c -- deterministic batch-parallel Vamana-style graph builder.
 *
 * This is INPUT GENERATION, not the range-search method.  The paper runs its
 * range searches on an in-memory DiskANN/Vamana graph built with ParlayANN
 * (Sec. 4.1; build parameters R, L, alpha in the appendix table of DiskANN
 * parameters) and does not describe the construction itself.  This file builds
 * such a graph from seeded inputs so that the oracle and the GPU library read
 * the very same adjacency.
 *
 * Construction (our own design, written from the published Vamana idea):
 *   - start point: the point nearest (L2, fp64) to the coordinate-wise mean,
 *     ties to the smaller id;
 *   - insertion order: a seeded permutation (splitmix64 Fisher-Yates) with the
 *     start point moved to the front;
 *   - batches of growing size (1, 2, 4, ... capped at max(1, n/50)): every
 *     point of a batch searches the graph as it stood before the batch (top-L
 *     beam from the start point), its visited list is pruned with RobustPrune
 *     (alpha applied to the stored metric value, i.e. squared for L2), then
 *     reverse edges are merged per target (appended while the degree stays
 *     <= R, else the target is re-pruned over old+new neighbours);
 *   - `passes` passes; with two passes the first uses alpha = 1;
 *   - construction fills at most R - max(1, R/16) slots per row; the reserved
 *     slots serve the reachability repair below, so the final out-degree is
 *     still <= R.
 * Every parallel step reads a snapshot and writes disjoint rows, and every
 * ordering uses (distance, id), so the graph does not depend on the number of
 * threads.  Integer data use exact integer distances; fp32 data accumulate in
 * double in index order, so x86 and Arm hosts build the same graph.
 *
 * Layout: adj is n x R uint32 row-major; unused slots hold 0xFFFFFFFF.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SENT 0xFFFFFFFFu

typedef struct {
    const char *X;
    int64_t n;
    int d;
    int dtype;  /* 0 = uint8, 1 = int8, 2 = float32 */
    int metric; /* 0 = squared L2, 1 = negative inner product */
    size_t row; /* bytes per vector */
} ds_t;

static inline const void *vec(const ds_t *D, uint32_t i) { return D->X + (size_t)i * D->row; }

static double dist_q(const ds_t *D, const void *qa, const void *pb) {
    int d = D->d;
    if (D->dtype == 0) {
        const uint8_t *a = (const uint8_t *)qa, *b = (const uint8_t *)pb;
        int32_t s = 0;
        if (D->metric == 0) {
            for (int i = 0; i < d; i++) { int32_t t = (int32_t)a[i] - (int32_t)b[i]; s += t * t; }
            return (double)s;
        }
        for (int i = 0; i < d; i++) s += (int32_t)a[i] * (int32_t)b[i];
        return -(double)s;
    } else if (D->dtype == 1) {
        const int8_t *a = (const int8_t *)qa, *b = (const int8_t *)pb;
        int32_t s = 0;
        if (D->metric == 0) {
            for (int i = 0; i < d; i++) { int32_t t = (int32_t)a[i] - (int32_t)b[i]; s += t * t; }
            return (double)s;
        }
        for (int i = 0; i < d; i++) s += (int32_t)a[i] * (int32_t)b[i];
        return -(double)s;
    } else {
        const float *a = (const float *)qa, *b = (const float *)pb;
        double s = 0.0;
        if (D->metric == 0) {
            for (int i = 0; i < d; i++) { double t = (double)a[i] - (double)b[i]; s += t * t; }
            return s;
        }
        for (int i = 0; i < d; i++) s += (double)a[i] * (double)b[i];
        return -s;
    }
}

static inline double dist_ij(const ds_t *D, uint32_t i, uint32_t j) { return dist_q(D, vec(D, i), vec(D, j)); }

typedef struct { double d; uint32_t id; uint32_t vis; } bent;

static inline int key_lt(double da, uint32_t ia, double db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

static int cmp_bent(const void *pa, const void *pb) {
    const bent *a = (const bent *)pa, *b = (const bent *)pb;
    if (key_lt(a->d, a->id, b->d, b->id)) return -1;
    if (key_lt(b->d, b->id, a->d, a->id)) return 1;
    return 0;
}

/* Top-L beam search from `start` towards query vector q.  Returns the number of
 * visited points written to vis/vd (at most maxv). */
static int build_search(const ds_t *D, const uint32_t *adj, const int32_t *deg, int R, uint32_t start,
                        const void *q, int L, uint32_t *stamp, uint32_t tag, bent *beam,
                        uint32_t *vis, double *vd, int maxv) {
    int nb = 1, nv = 0, cur = 0;
    beam[0].d = dist_q(D, q, vec(D, start));
    beam[0].id = start;
    beam[0].vis = 0;
    stamp[start] = tag;
    for (;;) {
        int i = cur;
        while (i < nb && beam[i].vis) i++;
        if (i >= nb) break;
        beam[i].vis = 1;
        uint32_t p = beam[i].id;
        if (nv < maxv) { vis[nv] = p; vd[nv] = beam[i].d; nv++; }
        cur = i + 1;
        const uint32_t *row = adj + (size_t)p * R;
        /* ask for the unseen neighbours' vectors first: their cache misses then overlap instead of
         * arriving one distance at a time (a hint only; the search is unchanged) */
        for (int k = 0; k < deg[p]; k++) {
            uint32_t j = row[k];
            if (stamp[j] == tag) continue;
            const char *v = (const char *)vec(D, j);
            for (size_t o = 0; o < D->row; o += 64) __builtin_prefetch(v + o, 0, 1);
        }
        for (int k = 0; k < deg[p]; k++) {
            uint32_t j = row[k];
            if (stamp[j] == tag) continue;
            stamp[j] = tag;
            double dj = dist_q(D, q, vec(D, j));
            if (nb == L && !key_lt(dj, j, beam[L - 1].d, beam[L - 1].id)) continue;
            int pos = (nb < L) ? nb : L - 1;
            while (pos > 0 && key_lt(dj, j, beam[pos - 1].d, beam[pos - 1].id)) {
                beam[pos] = beam[pos - 1];
                pos--;
            }
            beam[pos].d = dj;
            beam[pos].id = j;
            beam[pos].vis = 0;
            if (nb < L) nb++;
            if (pos < cur) cur = pos;
        }
    }
    return nv;
}

/* RobustPrune: cand[0..nc) with distances to p (any order, may hold
 * duplicates and p itself).  Writes at most R ids to out, returns the count. */
static int robust_prune(const ds_t *D, uint32_t p, bent *cand, int nc, double alpha, int R, uint32_t *out) {
    qsort(cand, (size_t)nc, sizeof(bent), cmp_bent);
    int m = 0;
    for (int i = 0; i < nc; i++) {
        if (cand[i].id == p) continue;
        if (m > 0 && cand[m - 1].id == cand[i].id) continue;
        cand[m] = cand[i];
        cand[m].vis = 0; /* reused as "removed" flag */
        m++;
    }
    int no = 0;
    for (int i = 0; i < m && no < R; i++) {
        if (cand[i].vis) continue;
        uint32_t c = cand[i].id;
        out[no++] = c;
        const void *pc = vec(D, c);
        for (int k = i + 1; k < m; k++) {
            if (cand[k].vis) continue;
            double dck = dist_q(D, pc, vec(D, cand[k].id));
            if (alpha * dck <= cand[k].d) cand[k].vis = 1;
        }
    }
    return no;
}

static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Start point: nearest point (fp64 squared L2) to the coordinate-wise mean,
 * ties to the smaller id.  Fixed-size chunks keep the sums deterministic. */
int64_t rrs_start_point(const void *X, int64_t n, int d, int dtype) {
    ds_t D = {(const char *)X, n, d, dtype, 0, (size_t)d * (dtype == 2 ? 4 : 1)};
    const int64_t CH = 65536;
    int64_t nch = (n + CH - 1) / CH;
    double *part = (double *)calloc((size_t)nch * d, sizeof(double));
    double *mean = (double *)calloc((size_t)d, sizeof(double));
    if (!part || !mean) { free(part); free(mean); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nch; c++) {
        double *ps = part + (size_t)c * d;
        int64_t e = (c + 1) * CH < n ? (c + 1) * CH : n;
        for (int64_t i = c * CH; i < e; i++) {
            const void *v = vec(&D, (uint32_t)i);
            for (int k = 0; k < d; k++) {
                double x = dtype == 0 ? ((const uint8_t *)v)[k] : dtype == 1 ? ((const int8_t *)v)[k] : ((const float *)v)[k];
                ps[k] += x;
            }
        }
    }
    for (int64_t c = 0; c < nch; c++)
        for (int k = 0; k < d; k++) mean[k] += part[(size_t)c * d + k];
    for (int k = 0; k < d; k++) mean[k] /= (double)n;
    double *bestd = part; /* reuse: one slot per chunk */
    int64_t *besti = (int64_t *)calloc((size_t)nch, sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nch; c++) {
        int64_t e = (c + 1) * CH < n ? (c + 1) * CH : n;
        double bd = 0; int64_t bi = -1;
        for (int64_t i = c * CH; i < e; i++) {
            const void *v = vec(&D, (uint32_t)i);
            double s = 0;
            for (int k = 0; k < d; k++) {
                double x = dtype == 0 ? ((const uint8_t *)v)[k] : dtype == 1 ? ((const int8_t *)v)[k] : ((const float *)v)[k];
                double t = x - mean[k];
                s += t * t;
            }
            if (bi < 0 || s < bd) { bd = s; bi = i; }
        }
        bestd[c] = bd; besti[c] = bi;
    }
    int64_t best = besti[0]; double bd = bestd[0];
    for (int64_t c = 1; c < nch; c++) if (bestd[c] < bd) { bd = bestd[c]; best = besti[c]; }
    free(part); free(mean); free(besti);
    return best;
}

/* Reachability repair (our addition): tight near-duplicate families are close
 * to equidistant, RobustPrune keeps no edge into some of their members, and
 * those points could never be returned by any search.  Until every point is
 * reachable from the start point: BFS from the start; visit unreached points in
 * id order; attach each one from its nearest reached out-neighbour v (else
 * from the nearest reached point found by a search from the start), appending
 * to v's row or, when the row is full, replacing the edge of v whose target has
 * the largest in-degree; then mark what the new edge makes reachable. */
static void bfs_mark(const uint32_t *adj, const int32_t *deg, int R, uint32_t src, uint8_t *seen, uint32_t *queue) {
    int64_t h = 0, t = 0;
    if (seen[src]) return;
    seen[src] = 1;
    queue[t++] = src;
    while (h < t) {
        uint32_t u = queue[h++];
        for (int k = 0; k < deg[u]; k++) {
            uint32_t v = adj[(size_t)u * R + k];
            if (!seen[v]) { seen[v] = 1; queue[t++] = v; }
        }
    }
}

static int repair_reachability(const ds_t *D, uint32_t *adj, int32_t *deg, int R, int L, uint32_t start) {
    int64_t n = D->n;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int32_t *indeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    uint32_t *stamp = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    int maxv = 4 * L + 16;
    bent *beam = (bent *)malloc((size_t)L * sizeof(bent));
    uint32_t *vis = (uint32_t *)malloc((size_t)maxv * sizeof(uint32_t));
    double *vd = (double *)malloc((size_t)maxv * sizeof(double));
    if (!seen || !queue || !indeg || !stamp || !beam || !vis || !vd) {
        free(seen); free(queue); free(indeg); free(stamp); free(beam); free(vis); free(vd);
        return -2;
    }
    for (int64_t u = 0; u < n; u++)
        for (int k = 0; k < deg[u]; k++) indeg[adj[(size_t)u * R + k]]++;
    bfs_mark(adj, deg, R, start, seen, queue);
    uint32_t tag = 0;
    for (int64_t u = 0; u < n; u++) {
        if (seen[u]) continue;
        /* nearest reached out-neighbour with a free slot, else nearest reached
         * point with a free slot on a search path, else nearest reached one */
        uint32_t v = SENT, vf = SENT;
        double bd = 0, bdf = 0;
        for (int k = 0; k < deg[u]; k++) {
            uint32_t w = adj[(size_t)u * R + k];
            if (!seen[w]) continue;
            double dw = dist_ij(D, (uint32_t)u, w);
            if (v == SENT || key_lt(dw, w, bd, v)) { v = w; bd = dw; }
            if (deg[w] < R && (vf == SENT || key_lt(dw, w, bdf, vf))) { vf = w; bdf = dw; }
        }
        if (vf == SENT) {
            int nv = build_search(D, adj, deg, R, start, vec(D, (uint32_t)u), L, stamp, ++tag, beam, vis, vd, maxv);
            for (int k = 0; k < nv; k++) {
                uint32_t w = vis[k];
                if (w == (uint32_t)u || !seen[w]) continue;
                if (v == SENT || key_lt(vd[k], w, bd, v)) { v = w; bd = vd[k]; }
                if (deg[w] < R && (vf == SENT || key_lt(vd[k], w, bdf, vf))) { vf = w; bdf = vd[k]; }
            }
        }
        if (vf != SENT) v = vf;
        if (v == SENT) v = start;
        uint32_t *row = adj + (size_t)v * R;
        if (deg[v] < R) {
            row[deg[v]++] = (uint32_t)u;
        } else {
            int kk = 0;
            for (int k = 1; k < R; k++)
                if (indeg[row[k]] > indeg[row[kk]] || (indeg[row[k]] == indeg[row[kk]] && row[k] > row[kk])) kk = k;
            indeg[row[kk]]--;
            row[kk] = (uint32_t)u;
        }
        indeg[u]++;
        bfs_mark(adj, deg, R, (uint32_t)u, seen, queue);
    }
    free(seen); free(queue); free(indeg); free(stamp); free(beam); free(vis); free(vd);
    return 0;
}

/* Build the graph.  Returns 0 on success, negative on allocation failure or
 * bad arguments.  adj must hold n*R uint32. */
int rrs_build_vamana(const void *X, int64_t n, int d, int dtype, int metric, int R, int L, double alpha,
                     int passes, uint64_t seed, int nthreads, uint32_t *adj, int64_t start) {
    if (n <= 0 || d <= 0 || R <= 0 || L <= 0 || passes <= 0 || start < 0 || start >= n || n >= (int64_t)SENT)
        return -1;
    ds_t D = {(const char *)X, n, d, dtype, metric, (size_t)d * (dtype == 2 ? 4 : 1)};
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int32_t *deg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int64_t maxb = n / 50 > 1 ? n / 50 : 1;
    int maxv = 4 * L + 16;
    int ccap = maxv + R + 8;
    uint32_t *stage = (uint32_t *)malloc((size_t)maxb * R * sizeof(uint32_t));
    int32_t *sdeg = (int32_t *)malloc((size_t)maxb * sizeof(int32_t));
    int64_t *bucket = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    uint32_t *rsrc = (uint32_t *)malloc((size_t)maxb * R * sizeof(uint32_t));
    uint32_t *tgts = (uint32_t *)malloc((size_t)maxb * R * sizeof(uint32_t));
    uint32_t *stamps = (uint32_t *)calloc((size_t)nthreads * n, sizeof(uint32_t));
    bent *tb = (bent *)malloc((size_t)nthreads * (L + ccap) * sizeof(bent));
    uint32_t *tv = (uint32_t *)malloc((size_t)nthreads * maxv * sizeof(uint32_t));
    double *tvd = (double *)malloc((size_t)nthreads * maxv * sizeof(double));
    if (!deg || !perm || !stage || !sdeg || !bucket || !rsrc || !tgts || !stamps || !tb || !tv || !tvd) {
        free(deg); free(perm); free(stage); free(sdeg); free(bucket); free(rsrc); free(tgts);
        free(stamps); free(tb); free(tv); free(tvd);
        return -2;
    }
    for (int64_t i = 0; i < n * (int64_t)R; i++) adj[i] = SENT;
    for (int64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
    uint64_t s = seed;
    for (int64_t i = n - 1; i > 0; i--) {
        int64_t j = (int64_t)(splitmix64(&s) % (uint64_t)(i + 1));
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int64_t i = 0; i < n; i++)
        if (perm[i] == (uint32_t)start) { perm[i] = perm[0]; perm[0] = (uint32_t)start; break; }

    int Rb = R - (R / 16 > 1 ? R / 16 : 1);
    if (Rb < 1) Rb = 1;
    uint32_t tagbase = 0;
    for (int pass = 0; pass < passes; pass++) {
        double a = (passes > 1 && pass == 0) ? 1.0 : alpha;
        int64_t pos = (pass == 0) ? 1 : 0;
        int64_t bs = 1;
        while (pos < n) {
            int64_t nbatch = bs < n - pos ? bs : n - pos;
            /* 1. search + prune every batch point against the current snapshot */
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
            for (int64_t i = 0; i < nbatch; i++) {
                int t = 0;
#ifdef _OPENMP
                t = omp_get_thread_num();
#endif
                uint32_t *stamp = stamps + (size_t)t * n;
                bent *beam = tb + (size_t)t * (L + ccap);
                bent *cand = beam + L;
                uint32_t *vis = tv + (size_t)t * maxv;
                double *vd = tvd + (size_t)t * maxv;
                uint32_t p = perm[pos + i];
                uint32_t tag = tagbase + (uint32_t)(i + 1);
                int nv = build_search(&D, adj, deg, R, (uint32_t)start, vec(&D, p), L, stamp, tag, beam, vis, vd, maxv);
                int nc = 0;
                for (int k = 0; k < nv; k++) { cand[nc].d = vd[k]; cand[nc].id = vis[k]; nc++; }
                for (int k = 0; k < deg[p]; k++) {
                    uint32_t j = adj[(size_t)p * R + k];
                    cand[nc].d = dist_ij(&D, p, j); cand[nc].id = j; nc++;
                }
                sdeg[i] = robust_prune(&D, p, cand, nc, a, Rb, stage + (size_t)i * R);
            }
            tagbase += (uint32_t)nbatch + 1;
            if (tagbase > 0xF0000000u) { /* stamp wrap: reset */
                memset(stamps, 0, (size_t)nthreads * n * sizeof(uint32_t));
                tagbase = 0;
            }
            /* 2. publish the new rows */
            for (int64_t i = 0; i < nbatch; i++) {
                uint32_t p = perm[pos + i];
                uint32_t *row = adj + (size_t)p * R;
                for (int k = 0; k < R; k++) row[k] = k < sdeg[i] ? stage[(size_t)i * R + k] : SENT;
                deg[p] = sdeg[i];
            }
            /* 3. reverse edges, grouped by target in batch order (counting sort) */
            int64_t ne = 0;
            for (int64_t i = 0; i < nbatch; i++)
                for (int k = 0; k < sdeg[i]; k++) bucket[stage[(size_t)i * R + k] + 1]++;
            int64_t nt = 0;
            for (int64_t i = 0; i < nbatch; i++)
                for (int k = 0; k < sdeg[i]; k++) {
                    uint32_t j = stage[(size_t)i * R + k];
                    if (bucket[j + 1] > 0) { tgts[nt++] = j; bucket[j + 1] = -bucket[j + 1]; }
                }
            /* tgts holds each distinct target once; give each a slice of rsrc */
            {
                int64_t off = 0;
                for (int64_t t = 0; t < nt; t++) {
                    uint32_t j = tgts[t];
                    int64_t c = -bucket[j + 1];
                    bucket[j + 1] = off; /* start offset; becomes write cursor */
                    off += c;
                }
                ne = off;
            }
            for (int64_t i = 0; i < nbatch; i++) {
                uint32_t p = perm[pos + i];
                for (int k = 0; k < sdeg[i]; k++) {
                    uint32_t j = stage[(size_t)i * R + k];
                    rsrc[bucket[j + 1]++] = p;
                }
            }
            /* after the scatter, bucket[j+1] is the end of j's slice */
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
            for (int64_t t = 0; t < nt; t++) {
                int th = 0;
#ifdef _OPENMP
                th = omp_get_thread_num();
#endif
                uint32_t j = tgts[t];
                int64_t e = bucket[j + 1];
                /* slice start = end of previous target's slice in tgts order */
                int64_t b0 = (t == 0) ? 0 : bucket[tgts[t - 1] + 1];
                uint32_t *row = adj + (size_t)j * R;
                int dj = deg[j];
                int nnew = 0;
                uint32_t *newv = tv + (size_t)th * maxv; /* scratch: new sources not yet present */
                for (int64_t x = b0; x < e; x++) {
                    uint32_t p = rsrc[x];
                    int dup = 0;
                    for (int k = 0; k < dj && !dup; k++) dup = (row[k] == p);
                    for (int k = 0; k < nnew && !dup; k++) dup = (newv[k] == p);
                    if (!dup && p != j && nnew < maxv) newv[nnew++] = p;
                }
                if (dj + nnew <= Rb) {
                    for (int k = 0; k < nnew; k++) row[dj + k] = newv[k];
                    deg[j] = dj + nnew;
                } else {
                    bent *cand = tb + (size_t)th * (L + ccap);
                    int nc = 0;
                    for (int k = 0; k < dj; k++) { cand[nc].d = dist_ij(&D, j, row[k]); cand[nc].id = row[k]; nc++; }
                    for (int k = 0; k < nnew && nc < L + ccap; k++) { cand[nc].d = dist_ij(&D, j, newv[k]); cand[nc].id = newv[k]; nc++; }
                    uint32_t outb[1024];
                    int no = robust_prune(&D, j, cand, nc, a, Rb < 1024 ? Rb : 1024, outb);
                    for (int k = 0; k < R; k++) row[k] = k < no ? outb[k] : SENT;
                    deg[j] = no;
                }
            }
            for (int64_t t = 0; t < nt; t++) bucket[tgts[t] + 1] = 0;
            (void)ne;
            pos += nbatch;
            bs = bs * 2 < maxb ? bs * 2 : maxb;
        }
    }
    /* an edge replaced by the repair can cut off another point: repeat until none is */
    int rc = 0;
    for (int it = 0; it < 8 && rc == 0; it++) {
        uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
        if (!seen) { rc = -2; break; }
        bfs_mark(adj, deg, R, (uint32_t)start, seen, (uint32_t *)stamps);
        int64_t miss = 0;
        for (int64_t u = 0; u < n; u++) miss += !seen[u];
        free(seen);
        if (miss == 0) break;
        rc = repair_reachability(&D, adj, deg, R, L, (uint32_t)start);
    }
    free(deg); free(perm); free(stage); free(sdeg); free(bucket); free(rsrc); free(tgts);
    free(stamps); free(tb); free(tv); free(tvd);
    return rc;
}
