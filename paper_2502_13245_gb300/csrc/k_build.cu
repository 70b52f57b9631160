// k_build.cu -- rr_build_graph: a deterministic Vamana-style proximity graph
// built on the GPU, the step before the range search (the paper searches a
// DiskANN / Vamana graph built with R, L and alpha, Sec. 4.1, and does not
// describe the construction).
//
// The construction is batch-parallel and deterministic (every step reads a
// snapshot and writes disjoint rows; every order is by (distance, id)):
//   - start point: given by the caller (the medoid convention of the index);
//   - insertion order: a seeded permutation (splitmix64 Fisher-Yates), the
//     start point moved to the front;
//   - batches of 1, 2, 4, ... points, capped at max(1, n / 50); each point of a
//     batch runs Alg. 1 (beam L, no early stop) from the start point on the
//     graph as it stood before the batch, and RobustPrune(alpha) of its first
//     4L + 16 visits plus its current out-neighbours gives its new row
//     (alpha applied to the stored metric value, squared for L2);
//   - reverse edges, grouped by target in batch order: appended while the
//     target's degree stays within the construction cap, else the target is
//     re-pruned over its old and new neighbours;
//   - `passes` passes, the first with alpha = 1 when there are two or more;
//   - rows are filled to at most R - max(1, R / 16) during construction; the
//     reserved slots serve a final reachability repair (host side, sequential
//     in id order): every point the start point cannot reach is attached from
//     its nearest reached out-neighbour with a free slot (else from the
//     nearest reached point a beam search from the start finds; a full row
//     gives up the edge whose target has the largest in-degree), until every
//     point is reachable.
// This is the procedure of the project's CPU input generator, step for step,
// so on 8-bit data (exact integer distances) the two produce the same
// adjacency array.  fp32 data are refused here: the CPU builder orders fp32
// candidates by fp64 distances that this GPU path does not reproduce.
//
// GPU mapping: the per-point search is the library's beam kernel in its
// construction mode (warp per point, visits recorded); RobustPrune is a warp
// per point over its candidate keys in shared memory (sort, drop duplicates,
// then one distance pass per kept neighbour over the candidates still alive);
// reverse edges are grouped by a claim / count / scan / scatter of the
// (target, source) pairs and one warp per target sorts its sources and merges.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "rr_common.cuh"

namespace rr {

namespace {

__host__ __device__ inline size_t ru(size_t x) { return (x + 255) & ~size_t(255); }

// Shared memory of one prune warp for up to mcap candidates and rows of R.
struct PruneSmem {
    __host__ __device__ static size_t bytes(int mcap, int R) {
        return ru((size_t)mcap * 8) * 2 + ru((size_t)mcap * 4) + ru((size_t)mcap * 2) + ru((size_t)mcap) +
               ru((size_t)R * 4) * 2;
    }
    uint64_t *cand, *ckey;
    uint32_t *cid;
    uint16_t *kidx;
    uint8_t *removed;
    uint32_t *rowv, *outv;
    __device__ void carve(uint8_t *base, int mcap, int R) {
        cand = (uint64_t *)base;
        base += ru((size_t)mcap * 8);
        ckey = (uint64_t *)base;
        base += ru((size_t)mcap * 8);
        cid = (uint32_t *)base;
        base += ru((size_t)mcap * 4);
        kidx = (uint16_t *)base;
        base += ru((size_t)mcap * 2);
        removed = base;
        base += ru((size_t)mcap);
        rowv = (uint32_t *)base;
        base += ru((size_t)R * 4);
        outv = (uint32_t *)base;
    }
};

__device__ __forceinline__ double key_value(uint64_t k) { return (double)dval_i32(key_dk(k)); }

// RobustPrune(p, cand, alpha, Rb) with the whole warp.  cand[0..m): keys (dist to p, id) in any
// order, possibly with duplicates and p itself.  Sorts them by (dist, id), drops duplicates and p,
// then keeps candidates in order: a kept c removes every later candidate k with
// alpha * d(c, k) <= d(p, k).  Writes up to Rb ids to out (shared memory), returns their number.
template <int DT>
__device__ int warp_robust_prune(const SearchArgs &a, uint32_t p, PruneSmem &sm, int m, double alpha, int Rb,
                                 uint32_t *out) {
    constexpr int UN = 8;
    const int lane = lane_id();
    uint64_t *cand = sm.cand;
    warp_sort_keys(cand, m);
    // drop duplicates (equal keys are adjacent) and p itself, keeping the order
    int mm = 0;
    uint64_t carry = kEmpty;
    for (int c0 = 0; c0 < m; c0 += 32) {
        const int c = c0 + lane;
        const uint64_t k = c < m ? cand[c] : kEmpty;
        uint64_t prev = __shfl_up_sync(0xffffffffu, k, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(0xffffffffu, k, 31);
        const bool keep = c < m && key_id(k) != p && k != prev;
        const unsigned msk = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) cand[mm + __popc(msk & lanemask_lt())] = k;  // never ahead of the reads of later chunks
        mm += __popc(msk);
        __syncwarp();
    }
    for (int c = lane; c < mm; c += 32) sm.removed[c] = 0;
    __syncwarp();
    int no = 0, i = 0;
    while (no < Rb) {
        int nxt = mm;
        for (int b0 = i; b0 < mm; b0 += 32) {
            const int t = b0 + lane;
            const unsigned msk = __ballot_sync(0xffffffffu, t < mm && !sm.removed[t]);
            if (msk) { nxt = b0 + __ffs(msk) - 1; break; }
        }
        if (nxt >= mm) break;
        i = nxt;
        const uint32_t c = key_id(cand[i]);
        if (lane == 0) out[no] = c;
        no++;
        if (no >= Rb) break;
        // the candidates after i still alive, in order
        int nc = 0;
        for (int b0 = i + 1; b0 < mm; b0 += 32) {
            const int t = b0 + lane;
            const bool live = t < mm && !sm.removed[t];
            const unsigned msk = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int o = nc + __popc(msk & lanemask_lt());
                sm.cid[o] = key_id(cand[t]);
                sm.kidx[o] = (uint16_t)t;
            }
            nc += __popc(msk);
        }
        __syncwarp();
        if (nc > 0) {
            uint4 q[1];
            load_query<1>(a, a.vec + (size_t)c * a.row_stride, q);
            eval_candidates<DT, 1, UN>(a, q, sm.cid, nc, sm.ckey);
            __syncwarp();
            for (int t = lane; t < nc; t += 32) {
                const int k = sm.kidx[t];
                if (alpha * key_value(sm.ckey[t]) <= key_value(cand[k])) sm.removed[k] = 1;
            }
            __syncwarp();
        }
        i++;
    }
    __syncwarp();
    return no;
}

struct BuildArgs {
    SearchArgs s;             // vec, adj, n, R, row geometry, metric
    const uint32_t *perm;     // the batch's points: perm[i], i < nb
    int32_t nb;
    int32_t Rb;               // construction cap on the degree
    int32_t maxv;             // visits kept per search (4L + 16)
    int32_t mcap;             // candidate capacity of a prune (maxv + R)
    double alpha;
    int32_t *deg;             // n: out-degree (rows are filled from the left)
    const uint64_t *vis;      // nb x maxv visit keys
    const int32_t *nvis;      // nb
    uint32_t *stage;          // nb x R new rows
    int32_t *sdeg;            // nb
    // reverse edges
    int32_t *tidx;            // n: list index of a target in this batch, -1 if none
    uint32_t *tlist;          // targets of this batch (claim order)
    int32_t *ntgt;            // device counter
    int32_t *tcnt, *tcur;     // per target: sources, scatter cursor
    const int64_t *toff;      // per target: start of its sources (scan of tcnt)
    uint32_t *src;            // sources (batch indices) grouped by target
    int32_t *error;
};

// one warp per batch point: candidates = the search's visits + the point's current out-neighbours
template <int DT>
__global__ void __launch_bounds__(128) prune_kernel(BuildArgs b) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= b.nb) return;
    const SearchArgs &a = b.s;
    PruneSmem sm;
    sm.carve(smem_raw + (size_t)warp * PruneSmem::bytes(b.mcap, a.R), b.mcap, a.R);
    const uint32_t p = b.perm[i];
    const int nv = b.nvis[i];
    for (int t = lane; t < nv; t += 32) sm.cand[t] = b.vis[(size_t)i * b.maxv + t];
    int dp = 0;
    const uint32_t *row = a.adj + (size_t)p * a.R;
    for (int k0 = 0; k0 < a.R; k0 += 32) {
        const uint32_t j = k0 + lane < a.R ? row[k0 + lane] : kSent;
        const bool v = j < (uint32_t)a.n;
        const unsigned msk = __ballot_sync(0xffffffffu, v);
        if (v) sm.cid[dp + __popc(msk & lanemask_lt())] = j;
        dp += __popc(msk);
    }
    __syncwarp();
    if (nv + dp > b.mcap) {
        if (lane == 0) atomicExch(b.error, 5);
        return;
    }
    if (dp > 0) {
        uint4 q[1];
        load_query<1>(a, a.vec + (size_t)p * a.row_stride, q);
        eval_candidates<DT, 1, 8>(a, q, sm.cid, dp, sm.cand + nv);
    }
    __syncwarp();
    const int no = warp_robust_prune<DT>(a, p, sm, nv + dp, b.alpha, b.Rb, sm.outv);
    for (int t = lane; t < a.R; t += 32) b.stage[(size_t)i * a.R + t] = t < no ? sm.outv[t] : kSent;
    if (lane == 0) b.sdeg[i] = no;
}

// the batch's new rows replace the old ones
__global__ void publish_kernel(BuildArgs b) {
    const int R = b.s.R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)b.nb * R;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = x / R;
        const int k = (int)(x % R);
        const uint32_t p = b.perm[i];
        b.s.adj_w[(size_t)p * R + k] = b.stage[x];
        if (k == 0) b.deg[p] = b.sdeg[i];
    }
}

// every (target, source) pair: claim a list slot for each distinct target
__global__ void claim_kernel(BuildArgs b) {
    const int R = b.s.R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)b.nb * R;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = x / R;
        if ((int)(x % R) >= b.sdeg[i]) continue;
        const uint32_t j = b.stage[x];
        if (atomicCAS(b.tidx + j, -1, -2) == -1) b.tlist[atomicAdd(b.ntgt, 1)] = j;
    }
}

__global__ void assign_kernel(BuildArgs b, int32_t nt) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        b.tidx[b.tlist[t]] = t;
        b.tcnt[t] = 0;
        b.tcur[t] = 0;
    }
}

__global__ void count_kernel(BuildArgs b) {
    const int R = b.s.R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)b.nb * R;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = x / R;
        if ((int)(x % R) >= b.sdeg[i]) continue;
        atomicAdd(b.tcnt + b.tidx[b.stage[x]], 1);
    }
}

__global__ void scatter_kernel(BuildArgs b) {
    const int R = b.s.R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)b.nb * R;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = x / R;
        if ((int)(x % R) >= b.sdeg[i]) continue;
        const int t = b.tidx[b.stage[x]];
        b.src[b.toff[t] + atomicAdd(b.tcur + t, 1)] = (uint32_t)i;
    }
}

__global__ void release_kernel(BuildArgs b, int32_t nt) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) b.tidx[b.tlist[t]] = -1;
}

// ascending sort of v[0..m) (distinct values) with one warp, bitonic network with virtual padding
__device__ void warp_sort_u32(uint32_t *v, int m) {
    const int lane = lane_id();
    int P = 1;
    while (P < m) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int lj = __ffs(j) - 1;  // powers of two: shifts and masks
            for (int i = lane; i < P / 2; i += 32) {
                const int off = i & (j - 1);
                const int lo = ((i >> lj) << (lj + 1)) + off;
                const int hi = (j == (k >> 1)) ? lo - off + (k - 1 - off) : lo + j;
                if (hi < m) {
                    const uint32_t x = v[lo], y = v[hi];
                    if (y < x) {
                        v[lo] = y;
                        v[hi] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// one warp per target j: its new sources in batch order, minus those already in its row; append
// while the degree stays within Rb, else RobustPrune over the old and new neighbours
template <int DT>
__global__ void __launch_bounds__(128) merge_kernel(BuildArgs b, int32_t nt) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (t >= nt) return;
    const SearchArgs &a = b.s;
    PruneSmem sm;
    sm.carve(smem_raw + (size_t)warp * PruneSmem::bytes(b.mcap, a.R), b.mcap, a.R);
    const uint32_t j = b.tlist[t];
    uint32_t *seg = b.src + b.toff[t];
    const int ns = (int)(b.toff[t + 1] - b.toff[t]);
    warp_sort_u32(seg, ns);
    uint32_t *row = a.adj_w + (size_t)j * a.R;
    const int dj = b.deg[j];
    for (int k = lane; k < dj; k += 32) sm.rowv[k] = row[k];
    __syncwarp();
    // new sources not yet in the row (the first maxv of them), in batch order, after the row
    uint32_t *cid = sm.cid;
    for (int k = lane; k < dj; k += 32) cid[k] = sm.rowv[k];
    int nnew = 0;
    for (int x0 = 0; x0 < ns && nnew < b.maxv; x0 += 32) {
        const int x = x0 + lane;
        uint32_t p = kSent;
        bool keep = false;
        if (x < ns) {
            p = b.perm[seg[x]];
            keep = p != j;
            for (int k = 0; k < dj && keep; k++) keep = sm.rowv[k] != p;
        }
        const unsigned msk = __ballot_sync(0xffffffffu, keep);
        const int o = nnew + __popc(msk & lanemask_lt());
        if (keep && o < b.maxv) cid[dj + o] = p;
        nnew = min(b.maxv, nnew + __popc(msk));
    }
    __syncwarp();
    if (dj + nnew <= b.Rb) {
        for (int k = lane; k < nnew; k += 32) row[dj + k] = cid[dj + k];
        if (lane == 0) b.deg[j] = dj + nnew;
        return;
    }
    const int m = dj + nnew;
    if (m > b.mcap) {
        if (lane == 0) atomicExch(b.error, 6);
        return;
    }
    uint4 q[1];
    load_query<1>(a, a.vec + (size_t)j * a.row_stride, q);
    eval_candidates<DT, 1, 8>(a, q, cid, m, sm.cand);
    __syncwarp();
    const int no = warp_robust_prune<DT>(a, j, sm, m, b.alpha, b.Rb, sm.outv);
    for (int k = lane; k < a.R; k += 32) row[k] = k < no ? sm.outv[k] : kSent;
    if (lane == 0) b.deg[j] = no;
}

// ---------------------------------------------------------------------------------------------
// host side: permutation, batches, reachability repair
// ---------------------------------------------------------------------------------------------

uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct HostGraph {
    const uint8_t *X;  // n x d (8-bit)
    int64_t n;
    int d;
    int dtype, metric;
    int R;
    uint32_t *adj;
    std::vector<int32_t> deg;
    double dist(const uint8_t *q, uint32_t id) const {
        const uint8_t *x = X + (size_t)id * d;
        int32_t s = 0;
        for (int i = 0; i < d; i++) {
            const int32_t u = dtype == RR_I8 ? (int32_t)(int8_t)q[i] : (int32_t)q[i];
            const int32_t v = dtype == RR_I8 ? (int32_t)(int8_t)x[i] : (int32_t)x[i];
            s += metric == RR_L2 ? (u - v) * (u - v) : u * v;
        }
        return metric == RR_L2 ? (double)s : -(double)s;
    }
};

struct HEnt {
    double d;
    uint32_t id;
    uint32_t vis;
};
inline bool hlt(double da, uint32_t ia, double db, uint32_t ib) { return da < db || (da == db && ia < ib); }

// Alg. 1 with beam L from the start point (exact seen marks); the visited points (at most maxv)
// with their distances, in visit order
int host_search(const HostGraph &G, uint32_t start, const uint8_t *q, int L, std::vector<uint32_t> &stamp,
                uint32_t tag, std::vector<HEnt> &beam, uint32_t *vis, double *vd, int maxv) {
    int nb = 1, nv = 0, cur = 0;
    beam[0] = {G.dist(q, start), start, 0};
    stamp[start] = tag;
    for (;;) {
        int i = cur;
        while (i < nb && beam[i].vis) i++;
        if (i >= nb) break;
        beam[i].vis = 1;
        const uint32_t p = beam[i].id;
        if (nv < maxv) { vis[nv] = p; vd[nv] = beam[i].d; nv++; }
        cur = i + 1;
        const uint32_t *row = G.adj + (size_t)p * G.R;
        for (int k = 0; k < G.deg[p]; k++) {
            const uint32_t j = row[k];
            if (stamp[j] == tag) continue;
            stamp[j] = tag;
            const double dj = G.dist(q, j);
            if (nb == L && !hlt(dj, j, beam[L - 1].d, beam[L - 1].id)) continue;
            int pos = nb < L ? nb : L - 1;
            while (pos > 0 && hlt(dj, j, beam[pos - 1].d, beam[pos - 1].id)) {
                beam[pos] = beam[pos - 1];
                pos--;
            }
            beam[pos] = {dj, j, 0};
            if (nb < L) nb++;
            if (pos < cur) cur = pos;
        }
    }
    return nv;
}

void mark_from(const HostGraph &G, uint32_t src, std::vector<uint8_t> &seen, std::vector<uint32_t> &queue) {
    if (seen[src]) return;
    int64_t h = 0, t = 0;
    seen[src] = 1;
    queue[t++] = src;
    while (h < t) {
        const uint32_t u = queue[h++];
        for (int k = 0; k < G.deg[u]; k++) {
            const uint32_t v = G.adj[(size_t)u * G.R + k];
            if (!seen[v]) { seen[v] = 1; queue[t++] = v; }
        }
    }
}

// attach every point the start cannot reach (one sweep in id order); returns the points attached
int64_t repair_once(HostGraph &G, uint32_t start, int L) {
    const int64_t n = G.n;
    const int R = G.R;
    std::vector<uint8_t> seen((size_t)n, 0);
    std::vector<uint32_t> queue((size_t)n);
    std::vector<int32_t> indeg((size_t)n, 0);
    std::vector<uint32_t> stamp((size_t)n, 0);
    const int maxv = 4 * L + 16;
    std::vector<HEnt> beam((size_t)L);
    std::vector<uint32_t> vis((size_t)maxv);
    std::vector<double> vd((size_t)maxv);
    for (int64_t u = 0; u < n; u++)
        for (int k = 0; k < G.deg[u]; k++) indeg[G.adj[(size_t)u * R + k]]++;
    mark_from(G, start, seen, queue);
    uint32_t tag = 0;
    int64_t attached = 0;
    for (int64_t u = 0; u < n; u++) {
        if (seen[u]) continue;
        const uint8_t *xu = G.X + (size_t)u * G.d;
        uint32_t v = kSent, vf = kSent;
        double bd = 0, bdf = 0;
        for (int k = 0; k < G.deg[u]; k++) {
            const uint32_t w = G.adj[(size_t)u * R + k];
            if (!seen[w]) continue;
            const double dw = G.dist(xu, w);
            if (v == kSent || hlt(dw, w, bd, v)) { v = w; bd = dw; }
            if (G.deg[w] < R && (vf == kSent || hlt(dw, w, bdf, vf))) { vf = w; bdf = dw; }
        }
        if (vf == kSent) {
            const int nv = host_search(G, start, xu, L, stamp, ++tag, beam, vis.data(), vd.data(), maxv);
            for (int k = 0; k < nv; k++) {
                const uint32_t w = vis[k];
                if (w == (uint32_t)u || !seen[w]) continue;
                if (v == kSent || hlt(vd[k], w, bd, v)) { v = w; bd = vd[k]; }
                if (G.deg[w] < R && (vf == kSent || hlt(vd[k], w, bdf, vf))) { vf = w; bdf = vd[k]; }
            }
        }
        if (vf != kSent) v = vf;
        if (v == kSent) v = start;
        uint32_t *row = G.adj + (size_t)v * R;
        if (G.deg[v] < R) {
            row[G.deg[v]++] = (uint32_t)u;
        } else {
            int kk = 0;
            for (int k = 1; k < R; k++)
                if (indeg[row[k]] > indeg[row[kk]] || (indeg[row[k]] == indeg[row[kk]] && row[k] > row[kk])) kk = k;
            indeg[row[kk]]--;
            row[kk] = (uint32_t)u;
        }
        indeg[u]++;
        attached++;
        mark_from(G, (uint32_t)u, seen, queue);
    }
    return attached;
}

int64_t count_unreached(const HostGraph &G, uint32_t start) {
    std::vector<uint8_t> seen((size_t)G.n, 0);
    std::vector<uint32_t> queue((size_t)G.n);
    mark_from(G, start, seen, queue);
    int64_t miss = 0;
    for (int64_t u = 0; u < G.n; u++) miss += !seen[u];
    return miss;
}

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    rr_status alloc(T **out, size_t count) {
        void *p = nullptr;
        cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("rr_build_graph: device allocation of %zu bytes failed", count * sizeof(T));
            return RR_ENOMEM;
        }
        ptrs.push_back(p);
        *out = (T *)p;
        return RR_OK;
    }
};

template <int DT>
rr_status launch_prune(const BuildArgs &b, cudaStream_t st) {
    const int wpc = 4;
    const size_t smem = (size_t)wpc * PruneSmem::bytes(b.mcap, b.s.R);
    RR_CUDA(cudaFuncSetAttribute(prune_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    prune_kernel<DT><<<(b.nb + wpc - 1) / wpc, 32 * wpc, smem, st>>>(b);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

template <int DT>
rr_status launch_merge(const BuildArgs &b, int32_t nt, cudaStream_t st) {
    const int wpc = 4;
    const size_t smem = (size_t)wpc * PruneSmem::bytes(b.mcap, b.s.R);
    RR_CUDA(cudaFuncSetAttribute(merge_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    merge_kernel<DT><<<(nt + wpc - 1) / wpc, 32 * wpc, smem, st>>>(b, nt);
    RR_CUDA(cudaGetLastError());
    note_launch();
    return RR_OK;
}

unsigned grid_for(int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8)); }

}  // namespace

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_build_graph(const void *vectors, int64_t n, int32_t d, int32_t dtype, int32_t metric, int32_t R,
                                    int32_t L, double alpha, int32_t passes, uint64_t seed, int64_t start,
                                    int32_t device, uint32_t *adjacency, rr_build_info *info) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (info) memset(info, 0, sizeof *info);
    if (!vectors || !adjacency) { set_error("rr_build_graph: NULL array"); return RR_EINVAL; }
    if (dtype != RR_U8 && dtype != RR_I8) {
        set_error("rr_build_graph: the GPU builder takes 8-bit vectors (uint8 / int8)");
        return RR_EINVAL;
    }
    if (metric != RR_L2 && metric != RR_IP) { set_error("rr_build_graph: bad metric %d", metric); return RR_EINVAL; }
    if (n < 1 || n >= ((int64_t)1 << 31)) { set_error("rr_build_graph: n out of [1, 2^31)"); return RR_EINVAL; }
    if (d < 1 || d > 512) { set_error("rr_build_graph: d=%d out of [1, 512]", d); return RR_EINVAL; }
    if (R < 2 || R > 128) { set_error("rr_build_graph: R=%d out of [2, 128]", R); return RR_EINVAL; }
    if (L < 1 || L > 512) { set_error("rr_build_graph: L=%d out of [1, 512]", L); return RR_EINVAL; }
    if (passes < 1 || !(alpha >= 1.0)) { set_error("rr_build_graph: passes >= 1 and alpha >= 1 required"); return RR_EINVAL; }
    if (start < 0 || start >= n) { set_error("rr_build_graph: start out of range"); return RR_EINVAL; }
    DeviceGuard dg(device);
    cudaStream_t st = nullptr;
    RR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{st};

    const int64_t row_stride = (d + 15) & ~15;
    const int Rb = std::max(1, R - std::max(1, R / 16));
    const int64_t maxb = std::max<int64_t>(1, n / 50);
    const int maxv = 4 * L + 16;
    const int mcap = maxv + R;
    if (mcap > 65535) { set_error("rr_build_graph: L too large"); return RR_EINVAL; }

    // host copy of the vectors (the repair reads them) and the insertion order
    std::vector<uint8_t> hX;
    const uint8_t *X = (const uint8_t *)vectors;
    const bool vdev = is_device_ptr(vectors);
    if (vdev) {
        hX.resize((size_t)n * d);
        RR_CUDA(cudaMemcpy(hX.data(), vectors, (size_t)n * d, cudaMemcpyDeviceToHost));
        X = hX.data();
    }
    std::vector<uint32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[(size_t)i] = (uint32_t)i;
    uint64_t s = seed;
    for (int64_t i = n - 1; i > 0; i--) {
        const int64_t j = (int64_t)(splitmix64(&s) % (uint64_t)(i + 1));
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    for (int64_t i = 0; i < n; i++)
        if (perm[(size_t)i] == (uint32_t)start) { perm[(size_t)i] = perm[0]; perm[0] = (uint32_t)start; break; }

    DevBuf mem;
    rr_status rs;
    uint8_t *vec = nullptr;
    uint32_t *adj = nullptr, *perm_d = nullptr, *stage = nullptr, *tlist = nullptr, *src = nullptr;
    int32_t *deg = nullptr, *nvis = nullptr, *sdeg = nullptr, *tidx = nullptr, *tcnt = nullptr, *tcur = nullptr,
            *ctr = nullptr;
    uint64_t *vis = nullptr;
    int64_t *toff = nullptr;
    const size_t npairs = (size_t)maxb * R;
    if ((rs = mem.alloc(&vec, (size_t)n * row_stride)) != RR_OK || (rs = mem.alloc(&adj, (size_t)n * R)) != RR_OK ||
        (rs = mem.alloc(&perm_d, (size_t)n)) != RR_OK || (rs = mem.alloc(&deg, (size_t)n)) != RR_OK ||
        (rs = mem.alloc(&tidx, (size_t)n)) != RR_OK || (rs = mem.alloc(&vis, (size_t)maxb * maxv)) != RR_OK ||
        (rs = mem.alloc(&nvis, (size_t)maxb)) != RR_OK || (rs = mem.alloc(&stage, npairs)) != RR_OK ||
        (rs = mem.alloc(&sdeg, (size_t)maxb)) != RR_OK || (rs = mem.alloc(&tlist, npairs)) != RR_OK ||
        (rs = mem.alloc(&tcnt, npairs)) != RR_OK || (rs = mem.alloc(&tcur, npairs)) != RR_OK ||
        (rs = mem.alloc(&toff, npairs + 1)) != RR_OK || (rs = mem.alloc(&src, npairs)) != RR_OK ||
        (rs = mem.alloc(&ctr, 64)) != RR_OK)
        return rs;
    if (row_stride != d) RR_CUDA(cudaMemsetAsync(vec, 0, (size_t)n * row_stride, st));
    RR_CUDA(cudaMemcpy2DAsync(vec, row_stride, vectors, d, d, n, cudaMemcpyDefault, st));
    RR_CUDA(cudaMemsetAsync(adj, 0xFF, (size_t)n * R * 4, st));
    RR_CUDA(cudaMemsetAsync(deg, 0, (size_t)n * 4, st));
    RR_CUDA(cudaMemsetAsync(tidx, 0xFF, (size_t)n * 4, st));
    RR_CUDA(cudaMemsetAsync(ctr, 0, 256, st));
    RR_CUDA(cudaMemcpyAsync(perm_d, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));

    BuildArgs b;
    memset(&b, 0, sizeof b);
    SearchArgs &a = b.s;
    a.vec = vec;
    a.adj = adj;
    a.adj_w = adj;
    a.n = n;
    a.R = R;
    a.row_stride = (int32_t)row_stride;
    a.row_chunks = (int32_t)(row_stride / 16);
    int lpv = 1;
    while (lpv < a.row_chunks && lpv < 32) lpv <<= 1;
    a.lpv = lpv;
    a.metric = metric;
    a.start = (uint32_t)start;
    a.beam = L;
    a.use_es = 0;
    a.iter_limit = beam_iteration_limit(n);
    a.error = ctr + 1;
    a.vis_out = vis;
    a.vis_cap = maxv;
    a.vis_count = nvis;
    b.Rb = Rb;
    b.maxv = maxv;
    b.mcap = mcap;
    b.deg = deg;
    b.vis = vis;
    b.nvis = nvis;
    b.stage = stage;
    b.sdeg = sdeg;
    b.tidx = tidx;
    b.tlist = tlist;
    b.ntgt = ctr;
    b.tcnt = tcnt;
    b.tcur = tcur;
    b.toff = toff;
    b.src = src;
    b.error = ctr + 1;

    int32_t *hw = nullptr;  // pinned words: [0] targets of the batch, [1] device status
    RR_CUDA(cudaMallocHost(&hw, 64));
    struct PinGuard {
        int32_t *p;
        ~PinGuard() { cudaFreeHost(p); }
    } pg{hw};
    int64_t batches = 0;
    for (int pass = 0; pass < passes; pass++) {
        b.alpha = (passes > 1 && pass == 0) ? 1.0 : alpha;
        int64_t pos = pass == 0 ? 1 : 0;
        int64_t bs = 1;
        while (pos < n) {
            const int64_t nb = std::min(bs, n - pos);
            batches++;
            b.perm = perm_d + pos;
            b.nb = (int32_t)nb;
            a.qids = perm_d + pos;
            a.nq = nb;
            // 1. search + prune against the graph as it stood before the batch
            if ((rs = launch_build_search(a, 4, st, dtype)) != RR_OK) return rs;
            if ((rs = dtype == RR_U8 ? launch_prune<DT_U8>(b, st) : launch_prune<DT_I8>(b, st)) != RR_OK) return rs;
            // 2. publish the new rows
            publish_kernel<<<grid_for(nb * R), 256, 0, st>>>(b);
            RR_CUDA(cudaGetLastError());
            // 3. reverse edges, grouped by target in batch order
            RR_CUDA(cudaMemsetAsync(ctr, 0, 4, st));
            claim_kernel<<<grid_for(nb * R), 256, 0, st>>>(b);
            RR_CUDA(cudaGetLastError());
            RR_CUDA(cudaMemcpyAsync(hw, ctr, 8, cudaMemcpyDeviceToHost, st));
            RR_CUDA(cudaStreamSynchronize(st));
            if (hw[1] != 0) {
                set_error("rr_build_graph: a device-side guard tripped (code %d)", hw[1]);
                return RR_EINTERNAL;
            }
            const int32_t nt = hw[0];
            if (nt > 0) {
                assign_kernel<<<grid_for(nt), 256, 0, st>>>(b, nt);
                count_kernel<<<grid_for(nb * R), 256, 0, st>>>(b);
                RR_CUDA(cudaGetLastError());
                if ((rs = launch_scan(tcnt, nt, toff, st)) != RR_OK) return rs;
                scatter_kernel<<<grid_for(nb * R), 256, 0, st>>>(b);
                RR_CUDA(cudaGetLastError());
                if ((rs = dtype == RR_U8 ? launch_merge<DT_U8>(b, nt, st) : launch_merge<DT_I8>(b, nt, st)) != RR_OK)
                    return rs;
                release_kernel<<<grid_for(nt), 256, 0, st>>>(b, nt);
                RR_CUDA(cudaGetLastError());
                note_launch(6);
            }
            note_launch(2);
            pos += nb;
            bs = std::min(bs * 2, maxb);
        }
    }
    RR_CUDA(cudaMemcpyAsync(hw, ctr, 8, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaMemcpyAsync(adjacency, adj, (size_t)n * R * 4, cudaMemcpyDeviceToHost, st));
    RR_CUDA(cudaStreamSynchronize(st));
    if (hw[1] != 0) {
        set_error("rr_build_graph: a device-side guard tripped (code %d)", hw[1]);
        return RR_EINTERNAL;
    }
    const auto t1 = clk::now();
    // reachability repair on the host (sequential in id order; usually a handful of points)
    HostGraph G{X, n, d, dtype, metric, R, adjacency, std::vector<int32_t>((size_t)n)};
    for (int64_t u = 0; u < n; u++) {
        int k = 0;
        while (k < R && adjacency[(size_t)u * R + k] != kSent) k++;
        G.deg[(size_t)u] = k;
    }
    int64_t attached = 0;
    for (int it = 0; it < 8; it++) {
        if (count_unreached(G, (uint32_t)start) == 0) break;
        attached += repair_once(G, (uint32_t)start, L);
    }
    const auto t2 = clk::now();
    if (info) {
        info->batches = batches;
        info->repaired = attached;
        info->gpu_seconds = std::chrono::duration<double>(t1 - t0).count();
        info->repair_seconds = std::chrono::duration<double>(t2 - t1).count();
    }
    return RR_OK;
}
