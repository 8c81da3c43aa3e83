// batched.cu -- many personalised PageRank vectors and multi-source BFS runs
// over several graphs in one persistent launch (replayed from a CUDA graph).
//
// Personalised PageRank (Section 3.1 formula with a one-hot teleport vector
// s = e_seed per vector): for each graph the K iterates are one row-major
// matrix X[n][K], so the pull sweep (Algorithm 1, pulling) gathers neighbour
// rows -- one coalesced read per in-edge instead of K scattered 4-byte reads:
//     Y[v][j] = (1-d) [v == seed_j] + d * sum_{u in in(v)} w_uv inv_deg[u] X[u][j]
// The work is cut into jobs: one graph and a slice of KS consecutive columns,
// KS the widest of 128, 64 or 32 (at most K) for which the slice of both
// iterates fits the L2 budget, so every gathered row segment (KS * 4 bytes, a whole number of
// 128-byte lines) comes from L2 for the job's whole run.  Jobs run one after
// another over the whole grid; each sweeps its slice to convergence.  Every
// vector (column) starts at its seed's one-hot vector (or at 1/n), has its own
// L1 residual, reduced in FP64, and stops at its first sweep below tol; its
// column is then carried forward unchanged.
//
// Multi-source BFS (Section 3.3 / Algorithm 3 with ready = 1, up to 64 sources
// at once): F[v], V[v] and N[v] are 64-bit masks (bit j = search j).  Each
// graph chooses per level between top-down (frontier vertices OR their masks
// into their out-neighbours' N with 64-bit atomics) and bottom-up (every vertex
// not yet reached by all searches ORs the frontier masks of its in-neighbours,
// stopping once every missing search is covered), by the rule of the single
// search: bottom-up when the frontier's out-edges times alpha exceed the
// in-edges of vertices still missing a search, back to top-down when the
// frontier shrinks below n / beta.  An owner-only update then advances V, F and
// the levels.
//
// Both kernels are cooperative launches whose phases are separated by a grid
// barrier with a bounded spin-wait (on expiry an error flag is set, every
// block returns and the host reports GP_ERR_TIMEOUT).
#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "gp_internal.cuh"

namespace gp {

constexpr int BT_THREADS = 512;  // threads per block of the persistent kernels
constexpr int BT_SEG = 8;        // vertices per warp work unit (light rows)
constexpr int BT_MAX_KS = 128;   // widest column slice of one PageRank job (a float4 per lane)

struct BGraph {  // per-graph device descriptor
    int64_t n;
    const int64_t *csc_off;
    const int32_t *csc_idx;
    const float *csc_w;
    const int64_t *csr_off;
    const int32_t *csr_idx;
    const float *inv_deg;
    float *X0, *X1;          // PPR iterates [n][K]; X0 doubles as the output
    uint64_t *F, *V, *N;     // MS-BFS masks
    int32_t *levels;         // MS-BFS output [n][64]
    int64_t big0, nbig;      // big in-degree vertices of this graph in the big list
    int64_t chunk0, nchunk;  // their in-edge chunks in the chunk list
};

struct BChunk {  // warp work item: a piece of a big vertex's in-edge list
    int64_t beg;
    int32_t len;
    int32_t graph;
};

struct BJob {  // one graph and the column slice [c0, c0 + 32 * kpl)
    int32_t graph;
    int32_t c0;
    int32_t kpl;
    int32_t pad;
};

struct BPend {  // a PageRank column a job left iterating, for a packed job
    int32_t graph;
    int32_t col;    // its column in the graph's iterates
    int32_t kdone;  // sweeps it has had
    int32_t pad;
};

struct BatchDev {
    int ngraphs, K, nsrc;
    float d, one_minus_d;
    double tol;
    int iters;
    int64_t big_min;        // in-degree above which a vertex's in-edges are split into chunks
    int32_t one_hot_start;  // PPR iterates start at e_seed (else 1/n)
    float alpha, beta;      // MS-BFS direction rule
    const BGraph *graphs;
    const BJob *jobs;
    int njobs;
    const int32_t *big;     // [nbig_total] vertex ids, grouped by graph
    const int64_t *bcstart; // [nbig_total + 1] chunk range of each big vertex
    const BChunk *chunks;
    float *part;            // [max chunks of one graph][K] chunk partial rows
    double *res_acc;        // [3][K] per-sweep column residuals (a ring)
    const int32_t *seeds;   // [ngraphs][K]
    int32_t *iters_done;    // [ngraphs][K]
    const int32_t *sources; // [ngraphs][64] (MS-BFS)
    int32_t *counters;      // [0] most PPR sweeps of any column, [1] BFS levels, [2] packed columns
    int32_t pack_max;       // a job stops once at most this many of its columns iterate (0: never)
    BPend *pend;            // [ngraphs * K] the columns left iterating, in job order
    float *XP0, *XP1;       // [max n][32] iterates of a packed job
    unsigned long long *mcount;  // MS-BFS [2][ngraphs][4]: frontier vertices, their out-edges, open in-edges, new bits
    GridSync *sync;
};

// ------------------------------------------------------------------ batched PPR

// Compensated (Kahan) accumulation: a column sums up to thousands of terms one
// after another, so the running rounding error is carried in `comp`.
__device__ __forceinline__ void kahan_add(float &acc, float &comp, float x) {
    const float y = x - comp;
    const float t = acc + y;
    comp = (t - acc) - y;
    acc = t;
}

// A job of KS columns maps a warp onto NG = 32 / (KS / 4) edge groups of
// KS / 4 lanes; lane c4 of a group holds columns 4*c4 .. 4*c4+3 of a row (one
// float4), so one warp-wide load fetches NG row segments.  Light vertices take
// one group each; the edges of a chunk or of a big vertex are split over the
// groups, whose sums are then added with shuffles.
template <int KS>
struct Lanes {
    static constexpr int LPR = KS / 4;   // lanes per row segment
    static constexpr int NG = 32 / LPR;  // edge groups per warp
};

#ifndef GP_BT_INFLIGHT
#define GP_BT_INFLIGHT 8
#endif
constexpr int BT_INFLIGHT = GP_BT_INFLIGHT;  // row segments in flight per lane

// Row segments are read through L2 (ld.global.cg): the iterates are rewritten
// by the kernel itself between sweeps, so the non-coherent read-only path may
// not be used for them.
__device__ __forceinline__ float4 ld_seg(const float *X, int K, int32_t u, int c4) {
    return __ldcg(reinterpret_cast<const float4 *>(X + (int64_t)u * K) + c4);
}

// Compensated partial sums of a lane's four columns: the value is hi - lo.
struct Sum4 {
    float hi[4], lo[4];
};

// Sum over in-edges beg, beg + step, beg + 2 step, ... < end of the rows' four
// columns at c4 (X points at column c0 of row 0; rows are K floats apart), each
// product folded into a compensated (Kahan) sum: a column sums up to
// thousands of terms, and a hub's FP32 rounding feeds back into every sweep.
__device__ __forceinline__ Sum4 gather_seg(const BGraph &G, const float *X, int K, int64_t beg, int64_t end, int step,
                                           int c4) {
    Sum4 a;
#pragma unroll
    for (int i = 0; i < 4; ++i) a.hi[i] = a.lo[i] = 0.f;
    int64_t e = beg;
    for (; e + (BT_INFLIGHT - 1) * step < end; e += BT_INFLIGHT * step) {
        int32_t u[BT_INFLIGHT];
        float f[BT_INFLIGHT];
#pragma unroll
        for (int q = 0; q < BT_INFLIGHT; ++q) u[q] = __ldg(G.csc_idx + e + q * step);
        float4 r[BT_INFLIGHT];
#pragma unroll
        for (int q = 0; q < BT_INFLIGHT; ++q) r[q] = ld_seg(X, K, u[q], c4);
#pragma unroll
        for (int q = 0; q < BT_INFLIGHT; ++q) {
            f[q] = __ldg(G.inv_deg + u[q]);
            if (G.csc_w) f[q] *= __ldg(G.csc_w + e + q * step);
        }
#pragma unroll
        for (int q = 0; q < BT_INFLIGHT; ++q) {
            kahan_add(a.hi[0], a.lo[0], f[q] * r[q].x);
            kahan_add(a.hi[1], a.lo[1], f[q] * r[q].y);
            kahan_add(a.hi[2], a.lo[2], f[q] * r[q].z);
            kahan_add(a.hi[3], a.lo[3], f[q] * r[q].w);
        }
    }
    for (; e < end; e += step) {
        const int32_t u = __ldg(G.csc_idx + e);
        float f = __ldg(G.inv_deg + u);
        if (G.csc_w) f *= __ldg(G.csc_w + e);
        const float4 r = ld_seg(X, K, u, c4);
        kahan_add(a.hi[0], a.lo[0], f * r.x);
        kahan_add(a.hi[1], a.lo[1], f * r.y);
        kahan_add(a.hi[2], a.lo[2], f * r.z);
        kahan_add(a.hi[3], a.lo[3], f * r.w);
    }
    return a;
}

__device__ __forceinline__ float4 value4(const Sum4 &a) {
    return make_float4(a.hi[0] - a.lo[0], a.hi[1] - a.lo[1], a.hi[2] - a.lo[2], a.hi[3] - a.lo[3]);
}

// Adds the groups' compensated sums of a warp (every group then holds the
// total): error-free two-sums of the leading parts, corrections added.
template <int KS>
__device__ __forceinline__ float4 groups_total(Sum4 a) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.lo[i] = -a.lo[i];  // value = hi + lo from here on
#pragma unroll
    for (int o = Lanes<KS>::LPR; o < 32; o <<= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float ohi = __shfl_xor_sync(FULL, a.hi[i], o), olo = __shfl_xor_sync(FULL, a.lo[i], o);
            const float t = a.hi[i] + ohi;
            const float bp = t - a.hi[i];
            const float err = (a.hi[i] - (t - bp)) + (ohi - bp);
            a.hi[i] = t;
            a.lo[i] = a.lo[i] + olo + err;
        }
    }
    return make_float4(a.hi[0] + a.lo[0], a.hi[1] + a.lo[1], a.hi[2] + a.lo[2], a.hi[3] + a.lo[3]);
}

// The columns one PageRank job iterates: a slice of a graph's own iterates
// (pend == nullptr: columns c0 .. c0 + KS - 1 of X0/X1, rows K apart), or a
// packed job over the batch's packed iterates (rows 32 apart), whose column j
// continues the graph's column pend[j].col after pend[j].kdone sweeps.
struct PView {
    int graph;
    float *X0, *X1;     // the start and the result are in X0
    int ld;             // row stride of X0 and X1 (floats)
    int c0;
    const BPend *pend;  // packed job, or nullptr
    int cnt;            // packed job: columns in use (the rest idle)
    __device__ int col(int c) const { return pend ? pend[c].col : c0 + c; }
    __device__ int kbase(int c) const { return pend ? pend[c].kdone : 0; }
};

// Writes the lane's four columns of row v of the slice of Y from the gathered
// sum, carrying stopped columns forward; adds |y - x| of the columns still
// iterating to the lane's residual slots (shared memory, one owner each).
__device__ __forceinline__ void finish_seg(const BatchDev &B, const PView &V, const float *Xc, float *Y, int64_t v,
                                           int c4, float4 sum, float *my_res, const int *s_active) {
    const int64_t o = v * V.ld + V.c0 + 4 * c4;
    const float4 x = __ldcg(reinterpret_cast<const float4 *>(Xc + o));
    const float xs[4] = {x.x, x.y, x.z, x.w}, ss[4] = {sum.x, sum.y, sum.z, sum.w};
    float ys[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = 4 * c4 + q;
        ys[q] = xs[q];
        if (s_active[c]) {
            const float base = (B.seeds[V.graph * B.K + V.col(c)] == (int32_t)v) ? B.one_minus_d : 0.f;
            ys[q] = base + B.d * ss[q];
            my_res[q] += fabsf(ys[q] - xs[q]);
        }
    }
    *reinterpret_cast<float4 *>(Y + o) = make_float4(ys[0], ys[1], ys[2], ys[3]);
}

// One job: the slice's sweeps from the start vector to convergence, or, for a
// slice of the graph's own iterates, until at most B.pack_max of its columns
// still iterate (those are then left, at their latest iterate, to a packed job).
// Returns false when a grid barrier gave up.
template <int KS>
__device__ bool ppr_job(const BatchDev &B, const PView &J, float (*s_res)[32][4], int *s_active) {
    constexpr int LPR = Lanes<KS>::LPR, NG = Lanes<KS>::NG;
    const int K = B.K;
    const int ld = J.ld;
    const BGraph &G = B.graphs[J.graph];
    const int64_t n = G.n;
    const int lane = lane_id(), grp = lane / LPR, c4 = lane % LPR;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gthread >> 5, nwarps = nthreads >> 5;
    if (!J.pend) {
        // start: every column at 1/n, or at its seed's one-hot vector
        const float x0 = 1.0f / (float)n;
        for (int64_t i = gthread; i < n * KS; i += nthreads) {
            const int64_t v = i / KS;
            const int c = (int)(i % KS);
            J.X0[v * ld + J.c0 + c] =
                B.one_hot_start ? (B.seeds[J.graph * K + J.c0 + c] == (int32_t)v ? 1.0f : 0.0f) : x0;
        }
    } else {
        // start: the packed columns' latest iterates (idle columns at zero)
        for (int64_t i = gthread; i < n * KS; i += nthreads) {
            const int64_t v = i / KS;
            const int c = (int)(i % KS);
            J.X0[v * ld + c] = c < J.cnt ? __ldcg(G.X0 + v * K + J.pend[c].col) : 0.f;
        }
    }
    for (int c = threadIdx.x; c < KS; c += blockDim.x) s_active[c] = !J.pend || (c < J.cnt && J.kbase(c) < B.iters);
    if (gthread < 3 * KS) B.res_acc[(gthread / KS) * K + (gthread % KS)] = 0.0;
    if (!grid_sync(B.sync, gridDim.x)) return false;
    const int64_t nseg = (n + BT_SEG - 1) / BT_SEG;
    const float *Xj0 = J.X0 + J.c0, *Xj1 = J.X1 + J.c0;
    int k = 1, last = 0;
    for (; k <= B.iters; ++k) {
        const float *Xc = (k & 1) ? J.X0 : J.X1;
        const float *Xs = (k & 1) ? Xj0 : Xj1;  // column c0 of the current iterate
        float *Y = (k & 1) ? J.X1 : J.X0;
        double *racc = B.res_acc + (k % 3) * K;
        if (blockIdx.x == 0)  // the ring slot of sweep k + 1 (last read two sweeps ago)
            for (int c = threadIdx.x; c < KS; c += blockDim.x) B.res_acc[((k + 1) % 3) * K + c] = 0.0;
        float *my_res = s_res[wib][lane];
#pragma unroll
        for (int q = 0; q < 4; ++q) my_res[q] = 0.f;
        // phase A: light rows (BT_SEG vertices per warp unit, a vertex per group)
        // and chunks of big vertices (split over the groups)
        for (int64_t u = gwarp; u < nseg + G.nchunk; u += nwarps) {
            if (u < nseg) {
                const int64_t v1 = min(n, (u + 1) * BT_SEG);
                for (int64_t v = u * BT_SEG + grp; v < v1; v += NG) {
                    const int64_t b = G.csc_off[v], e = G.csc_off[v + 1];
                    if (e - b > B.big_min) continue;  // big vertex: finished in phase B
                    const float4 sum = value4(gather_seg(G, Xs, ld, b, e, 1, c4));
                    finish_seg(B, J, Xc, Y, v, c4, sum, my_res, s_active);
                }
            } else {
                const int64_t c = u - nseg;
                const BChunk ch = B.chunks[G.chunk0 + c];
                const float4 sum = groups_total<KS>(gather_seg(G, Xs, ld, ch.beg + grp, ch.beg + ch.len, NG, c4));
                if (grp == 0) *reinterpret_cast<float4 *>(B.part + c * KS + 4 * c4) = sum;
            }
        }
        if (!grid_sync(B.sync, gridDim.x)) return false;
        // phase B: big vertices add their chunks' partial rows (chunks split over the groups)
        for (int64_t r = gwarp; r < G.nbig; r += nwarps) {
            const int64_t v = B.big[G.big0 + r];
            Sum4 a;
#pragma unroll
            for (int i = 0; i < 4; ++i) a.hi[i] = a.lo[i] = 0.f;
            for (int64_t c = B.bcstart[G.big0 + r] - G.chunk0 + grp; c < B.bcstart[G.big0 + r + 1] - G.chunk0; c += NG) {
                const float4 p = __ldcg(reinterpret_cast<const float4 *>(B.part + c * KS + 4 * c4));
                kahan_add(a.hi[0], a.lo[0], p.x);
                kahan_add(a.hi[1], a.lo[1], p.y);
                kahan_add(a.hi[2], a.lo[2], p.z);
                kahan_add(a.hi[3], a.lo[3], p.w);
            }
            const float4 sum = groups_total<KS>(a);
            if (grp == 0) finish_seg(B, J, Xc, Y, v, c4, sum, my_res, s_active);
        }
        // the block's column residuals: the slots of every warp and group added
        // in a fixed order, then one FP64 atomic per column into the sweep's ring slot
        __syncthreads();
        for (int c = threadIdx.x; c < KS; c += blockDim.x) {
            if (!s_active[c]) continue;
            ResSum t;
            for (int i = 0; i < wpb; ++i)
                for (int g = 0; g < NG; ++g) t.push(s_res[i][g * LPR + c / 4][c % 4]);
            const double r = t.get();
            if (r != 0.0) atomicAdd(racc + c, r);
        }
        if (!grid_sync(B.sync, gridDim.x)) return false;
        // every block takes the same decision from the same totals
        int any = 0;
        for (int c = threadIdx.x; c < KS; c += blockDim.x) {
            if (!s_active[c]) continue;
            const double r = __ldcg(racc + c);
            const int kc = J.kbase(c) + k;  // the column's sweeps
            if (blockIdx.x == 0) B.iters_done[J.graph * K + J.col(c)] = kc;
            if (r < B.tol || kc >= B.iters)
                s_active[c] = 0;
            else
                any = 1;
        }
        const int nact = __syncthreads_count(any);  // one column per thread (KS <= blockDim)
        last = k;
        if (!nact) break;
        if (!J.pend && nact <= B.pack_max) {
            // the few columns left go to a packed job; block 0 lists them in column order
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                int at = atomicAdd(B.counters + 2, nact);
                for (int c = 0; c < KS; ++c)
                    if (s_active[c]) B.pend[at++] = BPend{J.graph, J.c0 + c, k, 0};
            }
            break;
        }
    }
    // the slice's last iterate was written by sweep `last`: into X1 when odd
    if (last & 1)
        for (int64_t i = gthread; i < n * KS; i += nthreads) {
            const int64_t o = (i / KS) * ld + J.c0 + (i % KS);
            J.X0[o] = __ldcg(J.X1 + o);
        }
    if (J.pend) {
        if (!grid_sync(B.sync, gridDim.x)) return false;
        // the packed columns' results back into the graph's iterates
        for (int64_t i = gthread; i < n * KS; i += nthreads) {
            const int64_t v = i / KS;
            const int c = (int)(i % KS);
            if (c < J.cnt) G.X0[v * K + J.pend[c].col] = __ldcg(J.X0 + v * ld + c);
        }
    }
    if (gthread == 0) {
        // packed columns: their own counts (written by this block's threads before the last block barrier)
        int most = J.pend ? 0 : last;
        for (int c = 0; J.pend && c < J.cnt; ++c) most = max(most, B.iters_done[J.graph * K + J.pend[c].col]);
        B.counters[0] = max(B.counters[0], most);
    }
    return grid_sync(B.sync, gridDim.x);  // the next job reuses part and res_acc
}

#ifndef GP_BT_MINB
#define GP_BT_MINB 2
#endif
__global__ void __launch_bounds__(BT_THREADS, GP_BT_MINB) k_ppr_persistent(BatchDev B) {
    __shared__ float s_res[BT_THREADS / 32][32][4];  // per lane: |y - x| of its four columns
    __shared__ int s_active[BT_MAX_KS];
    for (int ji = 0; ji < B.njobs; ++ji) {
        const BJob Jb = B.jobs[ji];
        const BGraph &G = B.graphs[Jb.graph];
        const PView J = {Jb.graph, G.X0, G.X1, B.K, Jb.c0, nullptr, 0};
        bool ok;
        switch (Jb.kpl) {
            case 1: ok = ppr_job<32>(B, J, s_res, s_active); break;
            case 2: ok = ppr_job<64>(B, J, s_res, s_active); break;
            default: ok = ppr_job<128>(B, J, s_res, s_active); break;
        }
        if (!ok) return;
    }
    // the columns the jobs left: packed 32 at a time, a packed job never
    // mixing graphs (the list is in job order, so a graph's columns are adjacent)
    const int np = *(volatile int32_t *)(B.counters + 2);
    for (int i = 0; i < np;) {
        const int g = B.pend[i].graph;
        int j = i + 1;
        while (j < np && j - i < 32 && B.pend[j].graph == g) ++j;
        const PView J = {g, B.XP0, B.XP1, 32, 0, B.pend + i, j - i};
        if (!ppr_job<32>(B, J, s_res, s_active)) return;
        i = j;
    }
}

// ------------------------------------------------------------------ batched multi-source BFS

__global__ void __launch_bounds__(BT_THREADS) k_msbfs_persistent(BatchDev B) {
    __shared__ int s_dir[256];  // per graph: 0 top-down, 1 bottom-up for the current level
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gthread >> 5, nwarps = nthreads >> 5;
    const int lane = lane_id();
    const int nsrc = B.nsrc;
    const uint64_t full = nsrc == 64 ? ~0ull : ((1ull << nsrc) - 1ull);
    const int ng = B.ngraphs;
    for (int gi = 0; gi < ng; ++gi) {
        const BGraph &G = B.graphs[gi];
        for (int64_t v = gthread; v < G.n; v += nthreads) {
            G.F[v] = 0;
            G.V[v] = 0;
            G.N[v] = 0;
        }
        for (int64_t i = gthread; i < G.n * 64; i += nthreads) G.levels[i] = -1;
    }
    if (gthread < 8 * (int64_t)ng) B.mcount[gthread] = 0;
    if (!grid_sync(B.sync, gridDim.x)) return;
    if (gthread < (int64_t)ng) {  // one thread per graph seeds its searches
        const BGraph &G = B.graphs[gthread];
        for (int j = 0; j < nsrc; ++j) {
            const int32_t s = B.sources[gthread * 64 + j];
            G.F[s] |= 1ull << j;
            G.V[s] |= 1ull << j;
            G.levels[(int64_t)s * 64 + j] = 0;
        }
    }
    for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) s_dir[gi] = 0;  // a few sources: top-down
    if (!grid_sync(B.sync, gridDim.x)) return;
    int L = 0;
    for (;; ++L) {
        for (int gi = 0; gi < ng; ++gi) {
            const BGraph &G = B.graphs[gi];
            if (s_dir[gi] == 0) {
                // top-down: a lane per frontier vertex of light out-degree scans its
                // out-edges; heavy frontier vertices are scanned by the whole warp
                for (int64_t v0 = gwarp * 32; v0 < G.n; v0 += nwarps * 32) {
                    const int64_t v = v0 + lane;
                    uint64_t f = 0;
                    int64_t b = 0, e = 0;
                    if (v < G.n) {
                        f = G.F[v];
                        if (f) {
                            b = G.csr_off[v];
                            e = G.csr_off[v + 1];
                        }
                    }
                    const bool heavy = f && e - b > 32;
                    if (f && !heavy)
                        for (int64_t j = b; j < e; ++j) {
                            const int32_t w = __ldg(G.csr_idx + j);
                            const uint64_t nb = f & ~G.V[w];
                            if (nb) atomicOr((unsigned long long *)G.N + w, (unsigned long long)nb);
                        }
                    for (unsigned hm = __ballot_sync(FULL, heavy); hm; hm &= hm - 1) {
                        const int hl = __ffs(hm) - 1;
                        const uint64_t hf = __shfl_sync(FULL, f, hl);
                        const int64_t hb = __shfl_sync(FULL, b, hl), he = __shfl_sync(FULL, e, hl);
                        for (int64_t j = hb + lane; j < he; j += 32) {
                            const int32_t w = __ldg(G.csr_idx + j);
                            const uint64_t nb = hf & ~G.V[w];
                            if (nb) atomicOr((unsigned long long *)G.N + w, (unsigned long long)nb);
                        }
                    }
                }
            } else {
                // bottom-up: pull the frontier masks of in-neighbours (early exit once
                // covered); high in-degree vertices are scanned by a whole warp
                for (int64_t v = gthread; v < G.n; v += nthreads) {
                    const uint64_t vis = G.V[v];
                    if (vis == full) continue;
                    const int64_t b = G.csc_off[v], e = G.csc_off[v + 1];
                    if (e - b > B.big_min) continue;
                    uint64_t acc = 0;
                    for (int64_t j = b; j < e; ++j) {
                        acc |= G.F[__ldg(G.csc_idx + j)];
                        if ((acc | vis) == full) break;
                    }
                    G.N[v] = acc & ~vis;
                }
                for (int64_t r = gwarp; r < G.nbig; r += nwarps) {
                    const int64_t v = B.big[G.big0 + r];
                    const uint64_t vis = G.V[v];
                    if (vis == full) continue;
                    const int64_t b = G.csc_off[v], e = G.csc_off[v + 1];
                    uint64_t acc = 0;
                    for (int64_t j0 = b; j0 < e; j0 += 32) {
                        const int64_t j = j0 + lane;
                        uint64_t f = j < e ? G.F[__ldg(G.csc_idx + j)] : 0ull;
                        const unsigned lo = __reduce_or_sync(FULL, (unsigned)f);
                        const unsigned hi = __reduce_or_sync(FULL, (unsigned)(f >> 32));
                        acc |= ((uint64_t)hi << 32) | lo;
                        if ((acc | vis) == full) break;
                    }
                    if (lane == 0) G.N[v] = acc & ~vis;
                }
            }
        }
        if (!grid_sync(B.sync, gridDim.x)) return;
        // update: owner-only writes of V, F and the levels of newly reached
        // searches, and the counters of the next level's direction rule
        unsigned long long *mc = B.mcount + (L & 1) * 4 * ng;
        for (int gi = 0; gi < ng; ++gi) {
            const BGraph &G = B.graphs[gi];
            unsigned long long nf = 0, mf = 0, mu = 0, bits = 0;
            for (int64_t v = gthread; v < G.n; v += nthreads) {
                const uint64_t vis = G.V[v];
                const uint64_t nw = G.N[v] & ~vis;
                G.F[v] = nw;
                if (nw) {
                    G.V[v] = vis | nw;
                    G.N[v] = 0;
                    bits += __popcll(nw);
                    nf += 1;
                    mf += (unsigned long long)(G.csr_off[v + 1] - G.csr_off[v]);
                    for (uint64_t bb = nw; bb; bb &= bb - 1) G.levels[v * 64 + (__ffsll((long long)bb) - 1)] = L + 1;
                } else if (G.N[v]) {
                    G.N[v] = 0;
                }
                if ((vis | nw) != full) mu += (unsigned long long)(G.csc_off[v + 1] - G.csc_off[v]);
            }
            nf = warp_sum(nf);
            mf = warp_sum(mf);
            mu = warp_sum(mu);
            bits = warp_sum(bits);
            if (lane == 0) {
                if (nf) atomicAdd(mc + 4 * gi + 0, nf);
                if (mf) atomicAdd(mc + 4 * gi + 1, mf);
                if (mu) atomicAdd(mc + 4 * gi + 2, mu);
                if (bits) atomicAdd(mc + 4 * gi + 3, bits);
            }
        }
        if (!grid_sync(B.sync, gridDim.x)) return;
        // every block reads the same counters: next directions, and whether any search moved
        unsigned long long total = 0;
        const volatile unsigned long long *vmc = mc;
        for (int gi = 0; gi < ng; ++gi) total += vmc[4 * gi + 3];
        for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
            const unsigned long long nf = vmc[4 * gi], mf = vmc[4 * gi + 1], mu = vmc[4 * gi + 2];
            const int64_t n = B.graphs[gi].n;
            if (s_dir[gi] == 0)
                s_dir[gi] = ((float)mf * B.alpha > (float)mu) ? 1 : 0;
            else
                s_dir[gi] = ((float)nf * B.beta < (float)n) ? 0 : 1;
        }
        __syncthreads();
        // the other parity's record, last read two barriers ago, is cleared for the next level
        if (gthread < 4 * (int64_t)ng) B.mcount[((L + 1) & 1) * 4 * ng + gthread] = 0;
        if (total == 0) break;
    }
    if (gthread == 0) B.counters[1] = L + 1;
}

}  // namespace gp

// ================================================================== host side

struct gp_batch {
    int device = 0, num_sms = 0;
    int64_t l2_bytes = 0;
    int ngraphs = 0, K = 0;
    gp_batch_options opt;
    std::vector<gp_graph *> graphs;
    std::vector<gp::BGraph> hg;
    std::vector<gp::BJob> jobs;
    gp::BatchDev dev;
    gp::Arena mem;     // iterates, masks, levels and per-batch records
    gp::Arena layout;  // work lists that depend on the options
    gp::BGraph *dgraphs = nullptr;
    int32_t *seeds = nullptr, *sources = nullptr;
    int32_t *counters = nullptr;
    int32_t *hcounters = nullptr;  // pinned
    cudaStream_t home = nullptr;
    cudaGraphExec_t ppr_exec = nullptr, bfs_exec = nullptr;
    bool ppr_stale = true, bfs_stale = true;
    int ppr_iters = -1, bfs_nsrc = -1;
    double ppr_tol = -1.0;
    float ppr_d = -1.f;
    int grid = 0;
};

namespace gp {

static int batch_grid(gp_batch *b, const void *kernel, int &grid) {
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BT_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    grid = per_sm * b->num_sms;
    return GP_OK;
}

// Launch (or capture into a CUDA graph and replay) the cooperative kernel.
static int coop_launch(gp_batch *b, const void *kernel, cudaGraphExec_t &exec, bool rebuild, cudaStream_t s) {
    if (rebuild && exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    if (!exec) {
        cudaStream_t cap;
        GP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->dev.sync, 0, sizeof(GridSync), cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->counters, 0, 4 * sizeof(int32_t), cap);
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3((unsigned)b->grid);
            cfg.blockDim = dim3(BT_THREADS);
            cfg.stream = cap;
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeCooperative;
            attr.val.cooperative = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            void *args[] = {&b->dev};
            e = cudaLaunchKernelExC(&cfg, kernel, args);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            exec = nullptr;
            return set_error(GP_ERR_CUDA, "capturing the batched launch: %s", cudaGetErrorString(e));
        }
    }
    GP_CUDA(cudaGraphLaunch(exec, s));
    return GP_OK;
}

// Work lists for the current options: big in-degree vertices and their chunks,
// big out-degree vertices, and the PPR jobs (column slices sized to the L2
// budget).  Reads the offsets once; synchronises the stream.
static int batch_layout(gp_batch *b, cudaStream_t s) {
    const int K = b->K;
    const int64_t big_min = b->opt.big_in_degree, C = b->opt.chunk_edges;
    std::vector<int32_t> big;
    std::vector<int64_t> bcstart(1, 0);
    std::vector<BChunk> chunks;
    int64_t max_chunks = 1;
    b->jobs.clear();
    const int64_t budget = (int64_t)b->opt.l2_budget_mb << 20;
    for (int gi = 0; gi < b->ngraphs; ++gi) {
        gp_graph *g = b->graphs[gi];
        std::vector<int64_t> off((size_t)g->n + 1);
        cudaError_t e = cudaMemcpyAsync(off.data(), g->csc_off, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "batch layout: %s", cudaGetErrorString(e));
        BGraph &G = b->hg[gi];
        G.big0 = (int64_t)big.size();
        G.chunk0 = (int64_t)chunks.size();
        for (int64_t v = 0; v < g->n; ++v) {
            const int64_t d = off[v + 1] - off[v];
            if (d <= big_min) continue;
            big.push_back((int32_t)v);
            for (int64_t p = off[v]; p < off[v + 1]; p += C)
                chunks.push_back(BChunk{p, (int32_t)std::min<int64_t>(C, off[v + 1] - p), gi});
            bcstart.push_back((int64_t)chunks.size());
        }
        G.nbig = (int64_t)big.size() - G.big0;
        G.nchunk = (int64_t)chunks.size() - G.chunk0;
        max_chunks = std::max(max_chunks, G.nchunk);
        // the widest slice whose two iterates fit the budget (at least 32 columns)
        int ks = std::min(K, BT_MAX_KS);
        while (ks > 32 && 2 * g->n * (int64_t)ks * 4 > budget) ks /= 2;
        for (int c0 = 0; c0 < K; c0 += ks) b->jobs.push_back(BJob{gi, c0, ks / 32, 0});
    }
    b->layout.release(s);
    BatchDev &D = b->dev;
    int32_t *dbig = nullptr;
    int64_t *dbc = nullptr;
    BChunk *dch = nullptr;
    BJob *djobs = nullptr;
    int st = GP_OK;
    if (st == GP_OK) st = b->layout.alloc(dbig, std::max<size_t>(big.size(), 1), s);
    if (st == GP_OK) st = b->layout.alloc(dbc, bcstart.size(), s);
    if (st == GP_OK) st = b->layout.alloc(dch, std::max<size_t>(chunks.size(), 1), s);
    if (st == GP_OK) st = b->layout.alloc(djobs, b->jobs.size(), s);
    if (st == GP_OK) st = b->layout.alloc(D.part, (size_t)max_chunks * K, s);
    if (st != GP_OK) return st;
    cudaError_t e = cudaMemcpyAsync(b->dgraphs, b->hg.data(), b->ngraphs * sizeof(BGraph), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !big.empty()) e = cudaMemcpyAsync(dbig, big.data(), big.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbc, bcstart.data(), bcstart.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !chunks.empty()) e = cudaMemcpyAsync(dch, chunks.data(), chunks.size() * sizeof(BChunk), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(djobs, b->jobs.data(), b->jobs.size() * sizeof(BJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "batch layout copy: %s", cudaGetErrorString(e));
    D.big_min = big_min;
    D.big = dbig;
    D.bcstart = dbc;
    D.chunks = dch;
    D.jobs = djobs;
    D.njobs = (int)b->jobs.size();
    D.alpha = b->opt.msbfs_alpha;
    D.beta = b->opt.msbfs_beta;
    D.one_hot_start = b->opt.ppr_start;
    D.pack_max = b->opt.ppr_pack;
    b->ppr_stale = b->bfs_stale = true;  // captured launches hold the old arguments
    return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" int gp_batch_options_default(gp_batch_options *opt) {
    clear_error();
    if (!opt) return set_error(GP_ERR_INVALID, "gp_batch_options_default: NULL");
    memset(opt, 0, sizeof(*opt));
    opt->big_in_degree = 32;
    opt->chunk_edges = 128;
    opt->l2_budget_mb = 128;
    opt->msbfs_alpha = 16.0f;
    opt->msbfs_beta = 24.0f;
    opt->ppr_start = 1;
    opt->ppr_pack = 16;
    return GP_OK;
}

extern "C" int gp_batch_create(gp_batch **out, gp_graph *const *graphs, int ngraphs, int k_ppr, void *stream) {
    clear_error();
    if (!out) return set_error(GP_ERR_INVALID, "gp_batch_create: out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1) return set_error(GP_ERR_INVALID, "gp_batch_create: need at least one graph");
    if (ngraphs > 256) return set_error(GP_ERR_INVALID, "gp_batch_create: at most 256 graphs");
    if (k_ppr != 32 && k_ppr != 64 && k_ppr != 128 && k_ppr != 256)
        return set_error(GP_ERR_INVALID, "gp_batch_create: k_ppr must be 32, 64, 128 or 256");
    for (int i = 0; i < ngraphs; ++i)
        if (!graphs[i] || graphs[i]->n < 1) return set_error(GP_ERR_INVALID, "gp_batch_create: graph %d empty or NULL", i);
    cudaStream_t s = (cudaStream_t)stream;
    gp_batch *b = new gp_batch();
    b->home = s;
    b->ngraphs = ngraphs;
    b->K = k_ppr;
    b->graphs.assign(graphs, graphs + ngraphs);
    gp_batch_options_default(&b->opt);
    auto fail = [&](int st) {
        b->layout.release(s);
        b->mem.release(s);
        pinned_free(b->hcounters, 8 * sizeof(int32_t));
        delete b;
        return st;
    };
    {
        cudaError_t e = cudaGetDevice(&b->device);
        int l2 = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
        if (e != cudaSuccess) return fail(set_error(GP_ERR_CUDA, "gp_batch_create: %s", cudaGetErrorString(e)));
        b->l2_bytes = l2;
    }
    b->hg.resize(ngraphs);
    const int K = k_ppr;
    BatchDev &D = b->dev;
    memset(&D, 0, sizeof(D));
    D.ngraphs = ngraphs;
    D.K = K;
    int st = GP_OK;
    int64_t nmax = 1;
    for (int gi = 0; gi < ngraphs && st == GP_OK; ++gi) {
        gp_graph *g = graphs[gi];
        nmax = std::max(nmax, g->n);
        BGraph &G = b->hg[gi];
        memset(&G, 0, sizeof(G));
        G.n = g->n;
        G.csc_off = g->csc_off;
        G.csc_idx = g->csc_idx;
        G.csc_w = g->csc_w;
        G.csr_off = g->csr_off;
        G.csr_idx = g->csr_idx;
        G.inv_deg = g->inv_deg;
        const size_t n = (size_t)G.n;
        if (st == GP_OK) st = b->mem.alloc(G.X0, n * K, s);
        if (st == GP_OK) st = b->mem.alloc(G.X1, n * K, s);
        if (st == GP_OK) st = b->mem.alloc(G.F, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.V, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.N, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.levels, n * 64, s);
    }
    if (st == GP_OK) st = b->mem.alloc(b->dgraphs, (size_t)ngraphs, s);
    if (st == GP_OK) st = b->mem.alloc(D.res_acc, (size_t)3 * K, s);
    if (st == GP_OK) st = b->mem.alloc(b->seeds, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(b->sources, (size_t)ngraphs * 64, s);
    if (st == GP_OK) st = b->mem.alloc(D.iters_done, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(b->counters, 8, s);
    if (st == GP_OK) st = b->mem.alloc(D.mcount, (size_t)ngraphs * 8, s);
    if (st == GP_OK) st = b->mem.alloc(D.pend, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(D.XP0, (size_t)nmax * 32, s);
    if (st == GP_OK) st = b->mem.alloc(D.XP1, (size_t)nmax * 32, s);
    GridSync *sync = nullptr;
    if (st == GP_OK) st = b->mem.alloc(sync, 1, s);
    if (st != GP_OK) return fail(st);
    {
        void *h = nullptr;
        st = pinned_alloc(&h, 8 * sizeof(int32_t));
        if (st != GP_OK) return fail(st);
        b->hcounters = (int32_t *)h;
    }
    D.graphs = b->dgraphs;
    D.seeds = b->seeds;
    D.sources = b->sources;
    D.counters = b->counters;
    D.sync = sync;
    st = batch_layout(b, s);
    if (st != GP_OK) return fail(st);
    *out = b;
    return GP_OK;
}

extern "C" int gp_batch_set_options(gp_batch *b, const gp_batch_options *opt, void *stream) {
    clear_error();
    if (!b || !opt) return set_error(GP_ERR_INVALID, "gp_batch_set_options: NULL argument");
    if (opt->big_in_degree < 0 || opt->chunk_edges < 32 || opt->chunk_edges > (1 << 20) || opt->l2_budget_mb < 1 ||
        opt->l2_budget_mb > (1 << 20) || !(opt->msbfs_alpha > 0.f) || !(opt->msbfs_beta > 0.f) ||
        (opt->ppr_start != 0 && opt->ppr_start != 1) || opt->ppr_pack < 0 || opt->ppr_pack > BT_MAX_KS)
        return set_error(GP_ERR_INVALID, "gp_batch_set_options: option out of range");
    const gp_batch_options old = b->opt;
    b->opt = *opt;
    if (old.big_in_degree != opt->big_in_degree || old.chunk_edges != opt->chunk_edges ||
        old.l2_budget_mb != opt->l2_budget_mb)
        return batch_layout(b, (cudaStream_t)stream);
    b->dev.alpha = opt->msbfs_alpha;
    b->dev.beta = opt->msbfs_beta;
    b->dev.one_hot_start = opt->ppr_start;
    b->dev.pack_max = opt->ppr_pack;
    b->bfs_stale = b->ppr_stale = true;
    return GP_OK;
}

extern "C" int gp_batch_get_options(const gp_batch *b, gp_batch_options *opt) {
    clear_error();
    if (!b || !opt) return set_error(GP_ERR_INVALID, "gp_batch_get_options: NULL argument");
    *opt = b->opt;
    return GP_OK;
}

extern "C" int gp_batch_free(gp_batch *b) {
    clear_error();
    if (!b) return GP_OK;
    cudaDeviceSynchronize();
    if (b->ppr_exec) cudaGraphExecDestroy(b->ppr_exec);
    if (b->bfs_exec) cudaGraphExecDestroy(b->bfs_exec);
    b->layout.release(b->home);
    b->mem.release(b->home);
    pinned_free(b->hcounters, 8 * sizeof(int32_t));
    cudaError_t e = cudaStreamSynchronize(b->home);
    delete b;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_batch_free: %s", cudaGetErrorString(e));
    return GP_OK;
}

extern "C" int gp_ppr_batched(gp_batch *b, const int32_t *seeds, float damping, int iters, double tol, float *const *out,
                              int32_t *iters_done, gp_batch_stats *stats, void *stream) {
    clear_error();
    if (!b || !seeds) return set_error(GP_ERR_INVALID, "gp_ppr_batched: NULL argument");
    if (!(damping > 0.f && damping < 1.f)) return set_error(GP_ERR_INVALID, "damping %g outside (0, 1)", (double)damping);
    if (iters < 1 || !(tol >= 0.0)) return set_error(GP_ERR_INVALID, "gp_ppr_batched: iters >= 1 and tol >= 0 required");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = b->K;
    for (int gi = 0; gi < b->ngraphs; ++gi)
        for (int j = 0; j < K; ++j) {
            const int32_t v = seeds[(size_t)gi * K + j];
            if (v < 0 || (int64_t)v >= b->hg[gi].n)
                return set_error(GP_ERR_INVALID, "seed %d of graph %d outside [0, n)", v, gi);
        }
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
    }
    GP_CUDA(cudaMemcpyAsync(b->seeds, seeds, (size_t)b->ngraphs * K * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const void *kernel = (const void *)k_ppr_persistent;
    const bool rebuild = b->ppr_stale || b->ppr_iters != iters || b->ppr_tol != tol || b->ppr_d != damping;
    if (rebuild) {
        GP_TRY(batch_grid(b, kernel, b->grid));
        b->dev.d = damping;
        b->dev.one_minus_d = 1.0f - damping;
        b->dev.tol = tol;
        b->dev.iters = iters;
        b->ppr_iters = iters;
        b->ppr_tol = tol;
        b->ppr_d = damping;
        b->ppr_stale = false;
    }
    if (stats) GP_CUDA(cudaEventRecord(ev0, s));
    GP_TRY(coop_launch(b, kernel, b->ppr_exec, rebuild, s));
    if (stats) GP_CUDA(cudaEventRecord(ev1, s));
    for (int gi = 0; gi < b->ngraphs; ++gi)
        if (out && out[gi])
            GP_CUDA(cudaMemcpyAsync(out[gi], b->hg[gi].X0, (size_t)b->hg[gi].n * K * sizeof(float), cudaMemcpyDefault, s));
    if (iters_done)
        GP_CUDA(cudaMemcpyAsync(iters_done, b->dev.iters_done, (size_t)b->ngraphs * K * sizeof(int32_t), cudaMemcpyDefault, s));
    GP_CUDA(cudaMemcpyAsync(b->hcounters, b->counters, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GridSync hs;
    GP_CUDA(cudaMemcpyAsync(&hs, b->dev.sync, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->sweeps = b->hcounters[0];
        stats->ms = ms;
        stats->blocks = b->grid;
        stats->jobs = (int32_t)b->jobs.size();
        stats->packed = b->hcounters[2];
    }
    if (hs.err) return set_error(GP_ERR_TIMEOUT, "batched PageRank: a grid barrier wait ran out");
    return GP_OK;
}

extern "C" int gp_msbfs_batched(gp_batch *b, const int32_t *sources, int nsrc, int32_t *const *levels_out,
                                gp_batch_stats *stats, void *stream) {
    clear_error();
    if (!b || !sources) return set_error(GP_ERR_INVALID, "gp_msbfs_batched: NULL argument");
    if (nsrc < 1 || nsrc > 64) return set_error(GP_ERR_INVALID, "gp_msbfs_batched: nsrc %d outside [1, 64]", nsrc);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> src((size_t)b->ngraphs * 64, 0);
    for (int gi = 0; gi < b->ngraphs; ++gi)
        for (int j = 0; j < nsrc; ++j) {
            const int32_t v = sources[(size_t)gi * nsrc + j];
            if (v < 0 || (int64_t)v >= b->hg[gi].n)
                return set_error(GP_ERR_INVALID, "source %d of graph %d outside [0, n)", v, gi);
            src[(size_t)gi * 64 + j] = v;
        }
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
    }
    GP_CUDA(cudaMemcpyAsync(b->sources, src.data(), src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const bool rebuild = b->bfs_stale || b->bfs_nsrc != nsrc;
    int grid = 0;
    GP_TRY(batch_grid(b, (const void *)k_msbfs_persistent, grid));
    const int saved = b->grid;
    b->grid = grid;
    b->dev.nsrc = nsrc;
    b->bfs_nsrc = nsrc;
    b->bfs_stale = false;
    if (stats) GP_CUDA(cudaEventRecord(ev0, s));
    int st = coop_launch(b, (const void *)k_msbfs_persistent, b->bfs_exec, rebuild, s);
    b->grid = saved;
    GP_TRY(st);
    if (stats) GP_CUDA(cudaEventRecord(ev1, s));
    for (int gi = 0; gi < b->ngraphs; ++gi)
        if (levels_out && levels_out[gi])
            GP_CUDA(cudaMemcpyAsync(levels_out[gi], b->hg[gi].levels, (size_t)b->hg[gi].n * 64 * sizeof(int32_t),
                                    cudaMemcpyDefault, s));
    GP_CUDA(cudaMemcpyAsync(b->hcounters, b->counters, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GridSync hs;
    GP_CUDA(cudaMemcpyAsync(&hs, b->dev.sync, sizeof(hs), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->levels = b->hcounters[1];
        stats->ms = ms;
        stats->blocks = grid;
        stats->jobs = (int32_t)b->jobs.size();
    }
    if (hs.err) return set_error(GP_ERR_TIMEOUT, "batched BFS: a grid barrier wait ran out");
    return GP_OK;
}

// ------------------------------------------------------------------ tuning

namespace gp {

// Device time of one batched call (a warm-up call first: a changed option
// re-captures the launch).
static int time_ppr(gp_batch *b, const int32_t *seeds, int sweeps, cudaStream_t s, float &ms) {
    gp_batch_stats st;
    GP_TRY(gp_ppr_batched(b, seeds, 0.85f, sweeps, 0.0, nullptr, nullptr, &st, s));
    GP_TRY(gp_ppr_batched(b, seeds, 0.85f, sweeps, 0.0, nullptr, nullptr, &st, s));
    ms = st.ms;
    return GP_OK;
}

static int time_msbfs(gp_batch *b, const int32_t *sources, int nsrc, cudaStream_t s, float &ms) {
    gp_batch_stats st;
    GP_TRY(gp_msbfs_batched(b, sources, nsrc, nullptr, &st, s));
    GP_TRY(gp_msbfs_batched(b, sources, nsrc, nullptr, &st, s));
    ms = st.ms;
    return GP_OK;
}

}  // namespace gp

extern "C" int gp_batch_autotune(gp_batch *b, const int32_t *seeds, const int32_t *sources, int nsrc, int ppr_sweeps,
                                 gp_batch_tune_result *res, void *stream) {
    clear_error();
    if (!b || !res) return set_error(GP_ERR_INVALID, "gp_batch_autotune: NULL argument");
    if (ppr_sweeps < 1) return set_error(GP_ERR_INVALID, "gp_batch_autotune: ppr_sweeps must be >= 1");
    if (sources && (nsrc < 1 || nsrc > 64)) return set_error(GP_ERR_INVALID, "gp_batch_autotune: nsrc outside [1, 64]");
    cudaStream_t s = (cudaStream_t)stream;
    memset(res, 0, sizeof(*res));
    gp_batch_options best = b->opt;
    int trials = 0;
    // coordinate descent, each axis over its candidates with the others fixed
    auto axis_i32 = [&](int32_t gp_batch_options::*field, std::initializer_list<int32_t> cands, bool ppr,
                        float &best_ms) -> int {
        for (int32_t c : cands) {
            gp_batch_options o = best;
            o.*field = c;
            GP_TRY(gp_batch_set_options(b, &o, stream));
            float ms = 0.f;
            if (ppr)
                GP_TRY(time_ppr(b, seeds, ppr_sweeps, s, ms));
            else
                GP_TRY(time_msbfs(b, sources, nsrc, s, ms));
            ++trials;
            if (best_ms <= 0.f || ms < best_ms) {
                best_ms = ms;
                best = o;
            }
        }
        return gp_batch_set_options(b, &best, stream);
    };
    auto axis_f32 = [&](float gp_batch_options::*field, std::initializer_list<float> cands, float &best_ms) -> int {
        for (float c : cands) {
            gp_batch_options o = best;
            o.*field = c;
            GP_TRY(gp_batch_set_options(b, &o, stream));
            float ms = 0.f;
            GP_TRY(time_msbfs(b, sources, nsrc, s, ms));
            ++trials;
            if (best_ms <= 0.f || ms < best_ms) {
                best_ms = ms;
                best = o;
            }
        }
        return gp_batch_set_options(b, &best, stream);
    };
    float ppr_ms = 0.f, bfs_ms = 0.f;
    if (seeds) {
        GP_TRY(axis_i32(&gp_batch_options::big_in_degree, {8, 16, 32, 64, 128}, true, ppr_ms));
        GP_TRY(axis_i32(&gp_batch_options::chunk_edges, {64, 128, 256}, true, ppr_ms));
        GP_TRY(axis_i32(&gp_batch_options::l2_budget_mb, {48, 64, 96, 128, 192}, true, ppr_ms));
    }
    if (sources) {
        GP_TRY(axis_f32(&gp_batch_options::msbfs_alpha, {2.f, 4.f, 8.f, 16.f, 32.f, 64.f}, bfs_ms));
        GP_TRY(axis_f32(&gp_batch_options::msbfs_beta, {8.f, 24.f, 64.f}, bfs_ms));
    }
    res->options = best;
    res->ppr_ms = ppr_ms;
    res->msbfs_ms = bfs_ms;
    res->trials = trials;
    return GP_OK;
}
