/*
 * oracle/oracle.c -- CPU ORACLE for range retrieval on a proximity graph.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct reference
 * that the CUDA library is compared against.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the library never
 * does.  It shares no code with the CUDA path.
 *
 * It follows "Range Retrieval with Graph-Based Indices" (arXiv 2502.13245):
 *   Def. 2.1 (range search), Def. 2.2 (average precision),
 *   Alg. 1 BeamSearch, Alg. 2 GreedySearch, Alg. 3 DoublingSearch,
 *   Alg. 4/5 EarlyStopping with the d_visited metric, and with the other
 *            metrics of Sec. 3.2 (d_top1, d_top10, d_top10 / d_start),
 *   Alg. 6 GreedyRangeSearch (the per-query driver).
 * Readings where the paper is silent or garbled:
 *   - every argmin / "closest" / trim orders by the pair (distance, id);
 *   - B is a set: an id already in B is not added twice;
 *   - Alg. 5 stops iff  min_{p in B} d(p,q) > r  and  |V| >= vl  and
 *     d(p*,q) > esr, tested for the candidate p* before it joins V; on a stop
 *     BeamSearch returns the current (B, V);
 *   - the other metrics replace the last test of Alg. 5 (Alg. 4 with that M):
 *     d_top1 = d of the closest point of B, d_top10 = d of the 10th closest
 *     (the farthest one while |B| < 10), both against esr; d_top10 / d_start
 *     against a ratio t, written d_top10 > t * d_start with d_start the
 *     distance to the graph's start point (squared L2: distances >= 0);
 *   - Alg. 3 restarts every round from B = S, V = {} and continues iff
 *     |N| = b (lambda = 1); the beam never exceeds b_max: when doubling would
 *     pass b_max the last round's N is returned and flagged truncated;
 *   - Alg. 6 calls GreedySearch with the lower-case query q;
 *   - distances: squared L2 or negative inner product, exact int64 for 8-bit
 *     data and fp64 for fp32 data; a point is in range iff d <= r.
 *
 * Data structures are deliberately naive: B is a sorted array, V / F / "in B"
 * are byte markers of size n, argmin over F\V is a linear scan.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_SENT 0xFFFFFFFFu

enum { OR_U8 = 0, OR_I8 = 1, OR_F32 = 2 };
enum { OR_L2 = 0, OR_IP = 1 };
enum { OR_BEAM = 0, OR_BEAM_ES = 1, OR_DOUBLING = 2, OR_DOUBLING_ES = 3, OR_GREEDY = 4, OR_GREEDY_ES = 5,
       OR_DOUBLING_WARM = 6, OR_DOUBLING_WARM_ES = 7 };

typedef struct {
    const void *X;       /* n x d row-major */
    int64_t n;
    int32_t d;
    int32_t dtype;       /* OR_U8 / OR_I8 / OR_F32 */
    int32_t metric;      /* OR_L2 / OR_IP */
    int32_t R;
    const uint32_t *adj; /* n x R, OR_SENT pads rows */
    int64_t start;       /* entry point (medoid) */
} or_index;

typedef struct {
    int32_t variant;
    int32_t beam;        /* b (starting beam for doubling) */
    int32_t b_max;       /* doubling cap */
    int32_t es_vl;       /* Alg. 5 visit limit vl */
    double es_radius;    /* Alg. 5 esr (the ratio t for the d_top10 / d_start metric) */
    int32_t es_metric;   /* 0 d_visited, 1 d_top1, 2 d_top10, 3 d_top10 / d_start */
    int32_t expand;      /* parents expanded per BeamSearch iteration (0 or 1: Alg. 1 itself) */
} or_params;

typedef struct {
    int64_t visits_beam;   /* |V| summed over every BeamSearch call */
    int64_t visits_greedy; /* |V| of GreedySearch */
    int64_t evals;         /* distance evaluations as the algorithms are written */
    int64_t distinct;      /* distinct ids whose distance was evaluated */
    int32_t rounds;        /* BeamSearch calls (doubling rounds) */
    int32_t phase;         /* 0 = beam only, 1 = greedy, 2 = doubling */
    int32_t early_stopped; /* the first BeamSearch stopped through Alg. 5 */
    int32_t truncated;     /* doubling hit b_max */
    int32_t final_beam;    /* b of the last BeamSearch */
    int32_t pad;
} or_stats;

typedef struct { double d; uint32_t id; } ent;

/* ---------------------------------------------------------------- distance (Sec. 2) */
static double or_dist(const or_index *I, const void *q, uint32_t id) {
    int d = I->d;
    if (I->dtype == OR_F32) {
        const float *a = (const float *)q;
        const float *b = (const float *)I->X + (size_t)id * d;
        double s = 0.0;
        for (int k = 0; k < d; k++) {
            if (I->metric == OR_L2) { double t = (double)a[k] - (double)b[k]; s += t * t; }
            else s += (double)a[k] * (double)b[k];
        }
        return I->metric == OR_L2 ? s : -s;
    }
    int64_t s = 0;
    for (int k = 0; k < d; k++) {
        int64_t x, y;
        if (I->dtype == OR_U8) { x = ((const uint8_t *)q)[k]; y = ((const uint8_t *)I->X)[(size_t)id * d + k]; }
        else { x = ((const int8_t *)q)[k]; y = ((const int8_t *)I->X)[(size_t)id * d + k]; }
        if (I->metric == OR_L2) s += (x - y) * (x - y);
        else s += x * y;
    }
    return (double)(I->metric == OR_L2 ? s : -s);
}

static int key_less(ent a, ent b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

static int cmp_ent(const void *pa, const void *pb) {
    ent a = *(const ent *)pa, b = *(const ent *)pb;
    return key_less(a, b) ? -1 : (key_less(b, a) ? 1 : 0);
}

/* scratch markers of size n, owned by one search */
typedef struct {
    uint8_t *inB, *inV, *inE, *inF;
} marks;

static int marks_init(marks *m, int64_t n) {
    m->inB = (uint8_t *)calloc((size_t)n, 1);
    m->inV = (uint8_t *)calloc((size_t)n, 1);
    m->inE = (uint8_t *)calloc((size_t)n, 1);
    m->inF = (uint8_t *)calloc((size_t)n, 1);
    return m->inB && m->inV && m->inE && m->inF;
}
static void marks_free(marks *m) { free(m->inB); free(m->inV); free(m->inE); free(m->inF); }

static double eval(const or_index *I, const void *q, uint32_t id, marks *m, or_stats *st) {
    st->evals++;
    if (!m->inE[id]) { m->inE[id] = 1; st->distinct++; }
    return or_dist(I, q, id);
}

/* ---------------------------------------------------------------- early-stopping metrics (Sec. 3.2)
 * The metric M of Alg. 4, evaluated when p* (distance d_visit) is about to be
 * visited; B is sorted and holds nb >= 1 points. */
static int es_metric_exceeds(int metric, double d_visit, const ent *B, int64_t nb, double t, double d_start) {
    const double d_top10 = B[(nb < 10 ? nb : 10) - 1].d;
    switch (metric) {
    case 1: return B[0].d > t;            /* d_top1 */
    case 2: return d_top10 > t;           /* d_top10 */
    case 3: return d_top10 > t * d_start; /* d_top10 / d_start > t */
    default: return d_visit > t;          /* d_visited (Alg. 5) */
    }
}

/* ---------------------------------------------------------------- Alg. 1 + Alg. 5
 * BeamSearch(q, G, P, S, r, b, M).  S is given with its distances (S_d).
 * On return B[0..*nB) is sorted by (dist, id) and V[0..*nV) lists the visited
 * points in visit order.  B must hold |S| + R entries, V must hold n.
 * use_es selects M = Alg. 5 with the given metric (else M is never true);
 * d_start is q's distance to the graph's start point.  Returns 1 if M fired.
 *
 * expand > 1 (at most 64) is a variant of Alg. 1 that is not in the paper, a
 * multi-parent beam search: each iteration visits the `expand` closest
 * unvisited points of B at once (p* first; M is tested on p*), adds the
 * out-neighbours of all of them not in V or B, in parent order, then trims to
 * b once.  It trades a few extra visits for fewer, wider iterations (more
 * independent gathers per step on a GPU).  expand = 1 is Alg. 1 exactly. */
static int beam_search(const or_index *I, const void *q, const ent *S, int64_t nS, double r, int64_t b,
                       int use_es, int32_t vl, double esr, int es_metric, double d_start, int expand, ent *B,
                       int64_t *nB, uint32_t *V, int64_t *nV, marks *m, or_stats *st) {
    if (expand < 1) expand = 1;
    int64_t nb = 0, nv = 0;
    int stopped = 0;
    /* B <- S, V <- {} */
    for (int64_t i = 0; i < nS; i++) {
        if (m->inB[S[i].id]) continue;
        m->inB[S[i].id] = 1;
        B[nb++] = S[i];
    }
    qsort(B, (size_t)nb, sizeof(ent), cmp_ent);
    for (;;) {
        /* p* <- argmin over B \ V  (B is sorted, so the first unvisited entry) */
        int64_t ip = -1;
        for (int64_t i = 0; i < nb; i++)
            if (!m->inV[B[i].id]) { ip = i; break; }
        if (ip < 0) break; /* B \ V is empty */
        ent ps = B[ip];
        /* early stopping, Alg. 5: closest point of B outside r, enough visits, M above its threshold */
        if (use_es && B[0].d > r && nv >= vl && es_metric_exceeds(es_metric, ps.d, B, nb, esr, d_start)) {
            stopped = 1;
            break;
        }
        /* the parents of this iteration: p* and the next expand - 1 unvisited points of B */
        uint32_t par[64];
        int np = 0;
        for (int64_t i = ip; i < nb && np < expand && np < 64; i++)
            if (!m->inV[B[i].id]) par[np++] = B[i].id;
        for (int e = 0; e < np; e++) {
            /* V <- V u {p} */
            m->inV[par[e]] = 1;
            V[nv++] = par[e];
        }
        for (int e = 0; e < np; e++) {
            /* B <- B u (N_out(p) \ V) */
            const uint32_t *row = I->adj + (size_t)par[e] * I->R;
            for (int k = 0; k < I->R; k++) {
                uint32_t j = row[k];
                if (j == OR_SENT) continue;
                if (m->inV[j] || m->inB[j]) continue;
                B[nb].id = j;
                B[nb].d = eval(I, q, j, m, st);
                m->inB[j] = 1;
                nb++;
            }
        }
        qsort(B, (size_t)nb, sizeof(ent), cmp_ent);
        /* if |B| > b, keep the b closest */
        if (nb > b) {
            for (int64_t i = b; i < nb; i++) m->inB[B[i].id] = 0;
            nb = b;
        }
    }
    /* leave the markers clean for the caller (V is reported, not kept) */
    for (int64_t i = 0; i < nb; i++) m->inB[B[i].id] = 0;
    for (int64_t i = 0; i < nv; i++) m->inV[V[i]] = 0;
    st->visits_beam += nv;
    st->rounds++;
    *nB = nb;
    *nV = nv;
    return stopped;
}

/* ---------------------------------------------------------------- Alg. 2
 * GreedySearch(q, G, P, S, r): returns V (visit order) with distances.  out
 * must hold n entries.  S entries carry their distances. */
static int64_t greedy_search(const or_index *I, const void *q, const ent *S, int64_t nS, double r, ent *out,
                             marks *m, or_stats *st) {
    /* F <- S, V <- {} ; F is kept as a list with a membership marker */
    ent *F = (ent *)malloc((size_t)I->n * sizeof(ent));
    if (!F) return -1;
    int64_t nf = 0, nv = 0;
    for (int64_t i = 0; i < nS; i++) {
        if (m->inF[S[i].id]) continue;
        m->inF[S[i].id] = 1;
        F[nf++] = S[i];
    }
    for (;;) {
        /* p* <- argmin over F \ V (linear scan) */
        int64_t ip = -1;
        for (int64_t i = 0; i < nf; i++) {
            if (m->inV[F[i].id]) continue;
            if (ip < 0 || key_less(F[i], F[ip])) ip = i;
        }
        if (ip < 0) break;
        ent ps = F[ip];
        m->inV[ps.id] = 1;
        out[nv++] = ps;
        const uint32_t *row = I->adj + (size_t)ps.id * I->R;
        for (int k = 0; k < I->R; k++) {
            uint32_t f = row[k];
            if (f == OR_SENT || m->inV[f]) continue;
            double df = eval(I, q, f, m, st);
            if (df <= r && !m->inF[f]) {
                m->inF[f] = 1;
                F[nf].id = f;
                F[nf].d = df;
                nf++;
            }
        }
    }
    for (int64_t i = 0; i < nf; i++) m->inF[F[i].id] = 0;
    for (int64_t i = 0; i < nv; i++) m->inV[out[i].id] = 0;
    free(F);
    st->visits_greedy += nv;
    return nv;
}

/* ---------------------------------------------------------------- warm-restart doubling
 * A variant of Alg. 3 that is not in the paper: instead of restarting every
 * round from B = S with V = {} (which re-visits and re-evaluates), a round
 * continues the previous one.  E is every point whose distance has been
 * evaluated (with that distance) and V the visited points, both kept across
 * rounds.  A round with beam b starts from B = the b closest points of E and
 * runs Alg. 1's loop without visiting any point of V again (a neighbour
 * already in E re-enters B with its stored distance, no new evaluation);
 * N = {n in B : d <= r}; the search stops when |N| < b, else b doubles (capped
 * by b_max as in Alg. 3, the last N flagged truncated).  The first round is
 * Alg. 1 from the start point, as in Alg. 3.  Alg. 5 applies in every round.
 * Writes N (sorted) to res; returns |N|, or -1 on allocation failure. */
static int64_t warm_doubling(const or_index *I, const void *q, double r, const or_params *P, int use_es,
                             ent *res, marks *m, or_stats *st) {
    const int64_t n = I->n;
    ent *E = (ent *)malloc((size_t)n * sizeof(ent));
    ent *B = (ent *)malloc((size_t)(n + I->R + 1) * sizeof(ent));
    double *ed = (double *)malloc((size_t)n * sizeof(double));
    if (!E || !B || !ed) { free(E); free(B); free(ed); return -1; }
    int64_t nE = 0, nv = 0, nres = 0;
    ed[I->start] = eval(I, q, (uint32_t)I->start, m, st);
    E[nE].id = (uint32_t)I->start;
    E[nE++].d = ed[I->start];
    const double d_start = ed[I->start];
    int64_t b = P->beam;
    const int64_t bmax = P->b_max > 0 ? P->b_max : b;
    int first = 1;
    for (;;) {
        st->rounds++;
        st->final_beam = (int32_t)b;
        /* B <- the b closest points of E */
        memcpy(B, E, (size_t)nE * sizeof(ent));
        qsort(B, (size_t)nE, sizeof(ent), cmp_ent);
        int64_t nb = nE < b ? nE : b;
        for (int64_t i = 0; i < nb; i++) m->inB[B[i].id] = 1;
        int stopped = 0;
        int64_t round_visits = 0;
        for (;;) {
            int64_t ip = -1;
            for (int64_t i = 0; i < nb; i++)
                if (!m->inV[B[i].id]) { ip = i; break; }
            if (ip < 0) break;
            ent ps = B[ip];
            if (use_es && B[0].d > r && round_visits >= P->es_vl &&
                es_metric_exceeds(P->es_metric, ps.d, B, nb, P->es_radius, d_start)) {
                stopped = 1;
                break;
            }
            m->inV[ps.id] = 1;
            nv++;
            round_visits++;
            const uint32_t *row = I->adj + (size_t)ps.id * I->R;
            for (int k = 0; k < I->R; k++) {
                uint32_t j = row[k];
                if (j == OR_SENT || m->inV[j] || m->inB[j]) continue;
                if (!m->inE[j]) {
                    ed[j] = eval(I, q, j, m, st);
                    E[nE].id = j;
                    E[nE++].d = ed[j];
                }
                B[nb].id = j;
                B[nb].d = ed[j];
                m->inB[j] = 1;
                nb++;
            }
            qsort(B, (size_t)nb, sizeof(ent), cmp_ent);
            if (nb > b) {
                for (int64_t i = b; i < nb; i++) m->inB[B[i].id] = 0;
                nb = b;
            }
        }
        if (first) st->early_stopped = stopped;
        first = 0;
        nres = 0;
        for (int64_t i = 0; i < nb; i++) {
            m->inB[B[i].id] = 0;
            if (B[i].d <= r) res[nres++] = B[i];
        }
        if (nres < b) break;
        st->phase = 2;
        if (2 * b > bmax) { st->truncated = 1; break; }
        b = 2 * b;
    }
    st->visits_beam = nv;
    free(E); free(B); free(ed);
    return nres;
}

/* ---------------------------------------------------------------- per-query driver
 * Alg. 6 for the greedy variants, Alg. 3 for the doubling variants, and the
 * plain beam-search baseline (return {n in B : d <= r}).  Results are written
 * sorted by (dist, id).  Returns the number of results, or -1 on allocation
 * failure.  If the count exceeds cap, nothing is written past cap and the
 * caller should retry with a larger buffer. */
int64_t or_range_search_one(const or_index *I, const void *q, double r, const or_params *P, uint32_t *ids,
                            double *dists, int64_t cap, or_stats *st) {
    memset(st, 0, sizeof(*st));
    marks m;
    if (!marks_init(&m, I->n)) { marks_free(&m); return -1; }
    int use_es = (P->variant == OR_BEAM_ES || P->variant == OR_DOUBLING_ES || P->variant == OR_GREEDY_ES ||
                  P->variant == OR_DOUBLING_WARM_ES);
    if (P->variant == OR_DOUBLING_WARM || P->variant == OR_DOUBLING_WARM_ES) {
        ent *wres = (ent *)malloc((size_t)I->n * sizeof(ent));
        int64_t nw = wres ? warm_doubling(I, q, r, P, use_es, wres, &m, st) : -1;
        for (int64_t i = 0; i < nw && i < cap; i++) {
            ids[i] = wres[i].id;
            dists[i] = wres[i].d;
        }
        free(wres);
        marks_free(&m);
        return nw;
    }
    int doubling = (P->variant == OR_DOUBLING || P->variant == OR_DOUBLING_ES);
    int greedy = (P->variant == OR_GREEDY || P->variant == OR_GREEDY_ES);
    int64_t b = P->beam;
    int64_t bmax = P->b_max > 0 ? P->b_max : b;
    /* S <- {start} */
    int64_t scap = 1 + I->n;
    ent *S = (ent *)malloc((size_t)scap * sizeof(ent));
    ent *B = (ent *)malloc((size_t)(scap + I->R + 1) * sizeof(ent));
    uint32_t *V = (uint32_t *)malloc((size_t)I->n * sizeof(uint32_t));
    ent *res = (ent *)malloc((size_t)I->n * sizeof(ent));
    uint8_t *inS = (uint8_t *)calloc((size_t)I->n, 1);
    if (!S || !B || !V || !res || !inS) {
        free(S); free(B); free(V); free(res); free(inS); marks_free(&m);
        return -1;
    }
    int64_t nS = 1, nres = 0;
    S[0].id = (uint32_t)I->start;
    S[0].d = eval(I, q, (uint32_t)I->start, &m, st);
    const double d_start = S[0].d;
    inS[I->start] = 1;
    int first = 1;
    for (;;) {
        int64_t nB = 0, nV = 0;
        int stopped = beam_search(I, q, S, nS, r, b, use_es, P->es_vl, P->es_radius, P->es_metric, d_start,
                                  P->expand, B, &nB, V, &nV, &m, st);
        if (first) st->early_stopped = stopped;
        first = 0;
        st->final_beam = (int32_t)b;
        /* N <- {n in B : d(n,q) <= r}  (B is sorted, so N keeps that order) */
        nres = 0;
        for (int64_t i = 0; i < nB; i++)
            if (B[i].d <= r) res[nres++] = B[i];
        if (!doubling) break;
        /* Alg. 3: S <- S u V.  V's distances are known from B or recomputed */
        for (int64_t i = 0; i < nV; i++) {
            uint32_t v = V[i];
            if (inS[v]) continue;
            inS[v] = 1;
            S[nS].id = v;
            S[nS].d = or_dist(I, q, v); /* a repeat of an already-evaluated distance */
            nS++;
        }
        if (nres < b) break;
        st->phase = 2;
        if (2 * b > bmax) { st->truncated = 1; break; }
        b = 2 * b;
    }
    if (greedy && nres >= P->beam) {
        /* Alg. 6: |N| >= b -> V[q] <- GreedySearch(q, G, P, N, r) */
        st->phase = 1;
        ent *Sg = (ent *)malloc((size_t)(nres > 0 ? nres : 1) * sizeof(ent));
        if (!Sg) { free(S); free(B); free(V); free(res); free(inS); marks_free(&m); return -1; }
        memcpy(Sg, res, (size_t)nres * sizeof(ent));
        nres = greedy_search(I, q, Sg, nres, r, res, &m, st);
        free(Sg);
        if (nres < 0) { free(S); free(B); free(V); free(res); free(inS); marks_free(&m); return -1; }
        qsort(res, (size_t)nres, sizeof(ent), cmp_ent);
    }
    for (int64_t i = 0; i < nres && i < cap; i++) {
        ids[i] = res[i].id;
        dists[i] = res[i].d;
    }
    free(S); free(B); free(V); free(res); free(inS);
    marks_free(&m);
    return nres;
}

/* Alg. 1 alone, for tests: BeamSearch from S (ids) with ES optional.
 * Writes B (sorted) to b_ids/b_d (cap >= nS + R*n bound is the caller's job:
 * give n + R) and V in visit order.  Returns 1 if Alg. 5 fired, -1 on error. */
int or_beam_search(const or_index *I, const void *q, const uint32_t *S_ids, int64_t nS, double r, int64_t b,
                   int use_es, int32_t vl, double esr, int32_t es_metric, uint32_t *b_ids, double *b_d, int64_t *nB,
                   uint32_t *v_ids, int64_t *nV, or_stats *st) {
    memset(st, 0, sizeof(*st));
    marks m;
    if (!marks_init(&m, I->n)) { marks_free(&m); return -1; }
    ent *S = (ent *)malloc((size_t)(nS > 0 ? nS : 1) * sizeof(ent));
    ent *B = (ent *)malloc((size_t)(nS + I->n + I->R + 1) * sizeof(ent));
    if (!S || !B) { free(S); free(B); marks_free(&m); return -1; }
    for (int64_t i = 0; i < nS; i++) { S[i].id = S_ids[i]; S[i].d = eval(I, q, S_ids[i], &m, st); }
    /* d_start: distance to the graph's start point (not an evaluation of the search) */
    int stopped = beam_search(I, q, S, nS, r, b, use_es, vl, esr, es_metric, or_dist(I, q, (uint32_t)I->start), 1,
                              B, nB, v_ids, nV, &m, st);
    for (int64_t i = 0; i < *nB; i++) { b_ids[i] = B[i].id; b_d[i] = B[i].d; }
    free(S); free(B); marks_free(&m);
    return stopped;
}

/* Alg. 2 alone, for tests.  out must hold n entries; returned in visit order. */
int64_t or_greedy_search(const or_index *I, const void *q, const uint32_t *S_ids, int64_t nS, double r,
                         uint32_t *out_ids, double *out_d, or_stats *st) {
    memset(st, 0, sizeof(*st));
    marks m;
    if (!marks_init(&m, I->n)) { marks_free(&m); return -1; }
    ent *S = (ent *)malloc((size_t)(nS > 0 ? nS : 1) * sizeof(ent));
    ent *out = (ent *)malloc((size_t)I->n * sizeof(ent));
    if (!S || !out) { free(S); free(out); marks_free(&m); return -1; }
    for (int64_t i = 0; i < nS; i++) { S[i].id = S_ids[i]; S[i].d = eval(I, q, S_ids[i], &m, st); }
    int64_t nv = greedy_search(I, q, S, nS, r, out, &m, st);
    for (int64_t i = 0; i < nv; i++) { out_ids[i] = out[i].id; out_d[i] = out[i].d; }
    free(S); free(out); marks_free(&m);
    return nv;
}

/* Def. 2.1 by brute force: every point with d(p,q) <= r, sorted by (dist, id). */
int64_t or_brute_force(const or_index *I, const void *q, double r, uint32_t *ids, double *dists, int64_t cap) {
    int64_t c = 0;
    ent *all = (ent *)malloc((size_t)I->n * sizeof(ent));
    if (!all) return -1;
    for (int64_t i = 0; i < I->n; i++) {
        double di = or_dist(I, q, (uint32_t)i);
        if (di <= r) { all[c].id = (uint32_t)i; all[c].d = di; c++; }
    }
    qsort(all, (size_t)c, sizeof(ent), cmp_ent);
    for (int64_t i = 0; i < c && i < cap; i++) { ids[i] = all[i].id; dists[i] = all[i].d; }
    free(all);
    return c;
}

/* Distance of q to each listed id (fp64 / exact integer), for tests. */
void or_distances(const or_index *I, const void *q, const uint32_t *ids, int64_t m, double *out) {
    for (int64_t i = 0; i < m; i++) out[i] = or_dist(I, q, ids[i]);
}

/* Alg. 6's "parallel for q in Q": runs or_range_search_one over a batch with
 * nthreads OpenMP threads (1 = the single-threaded reference).  Results land in
 * per-query malloc'd buffers handed back through out_ids/out_d (free with
 * or_free).  Returns 0, or -1 if any query failed. */
int or_range_search_batch(const or_index *I, const void *Q, int64_t nq, const double *radii, const or_params *P,
                          int nthreads, int64_t *counts, uint32_t **out_ids, double **out_d, or_stats *stats) {
    size_t qbytes = (size_t)I->d * (I->dtype == OR_F32 ? 4 : 1);
    int fail = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : fail)
#endif
    for (int64_t i = 0; i < nq; i++) {
        const void *q = (const char *)Q + (size_t)i * qbytes;
        int64_t cap = 256;
        uint32_t *ids = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
        double *ds = (double *)malloc((size_t)cap * sizeof(double));
        int64_t c = ids && ds ? or_range_search_one(I, q, radii[i], P, ids, ds, cap, &stats[i]) : -1;
        if (c > cap) {
            free(ids); free(ds);
            cap = c;
            ids = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
            ds = (double *)malloc((size_t)cap * sizeof(double));
            c = ids && ds ? or_range_search_one(I, q, radii[i], P, ids, ds, cap, &stats[i]) : -1;
        }
        if (c < 0) { fail = 1; c = 0; }
        counts[i] = c;
        out_ids[i] = ids;
        out_d[i] = ds;
    }
    return fail ? -1 : 0;
}

void or_free(void *p) { free(p); }
