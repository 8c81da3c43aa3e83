// batched.cu -- many personalised PageRank vectors and multi-source BFS runs
// over several graphs in one persistent launch (replayed from a CUDA graph).
//
// Personalised PageRank (Section 3.1 formula with a one-hot teleport vector
// s = e_seed per vector): for each graph the K iterates are one row-major
// matrix X[n][K], so the pull sweep (Algorithm 1, pulling) gathers whole
// neighbour rows -- one coalesced K*4-byte read per in-edge instead of K
// scattered 4-byte reads:
//     Y[v][j] = (1-d) [v == seed_j] + d * sum_{u in in(v)} w_uv inv_deg[u] X[u][j]
// Every vector j has its own L1 residual (reduced in FP64 from per-tile partial
// rows, in a fixed order) and stops at its first sweep below tol; its column is
// then carried forward unchanged.
//
// Multi-source BFS (Section 3.3 / Algorithm 3 with ready = 1, up to 64 sources
// at once): F[v], V[v] and N[v] are 64-bit masks (bit j = search j).  Each level
// is a pull step -- every vertex not yet reached by all searches ORs the
// frontier masks of its in-neighbours, stopping once every missing search is
// covered -- followed by an owner-only update of V, F and the levels.
//
// Both run as one cooperative kernel: phases are separated by a grid barrier
// whose spin-wait has an iteration limit (then an error flag is set and every
// block returns; the host reports GP_ERR_TIMEOUT).  Work is laid out at batch
// creation: per graph, tiles of consecutive vertices and warp chunks of the
// in-edge lists of high in-degree vertices.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gp_internal.cuh"

namespace gp {

constexpr int BT_TILE = 1024;       // vertices per block tile
constexpr int BT_THREADS = 512;     // threads per block of the persistent kernels
constexpr int BT_BIG = 256;         // in-degree above which a vertex is split into chunks
constexpr int BT_CHUNK = 256;       // edges per chunk

struct BGraph {  // per-graph device descriptor
    int64_t n;
    const int64_t *csc_off;
    const int32_t *csc_idx;
    const float *csc_w;
    const float *inv_deg;
    float *X0, *X1;        // PPR iterates [n][K]; X0 doubles as the output
    uint64_t *F, *V, *N;   // MS-BFS masks
    int32_t *levels;       // MS-BFS output [n][64]
    int64_t tile0, ntiles; // light tiles of this graph in the tile list
    int64_t big0, nbig;    // big vertices of this graph in the big list
};

struct BChunk {  // warp work item: a piece of a big vertex's in-edge list
    int64_t beg;
    int32_t len;
    int32_t graph;
};

struct BTile {  // block work item: vertices [v0, v0 + cnt) of a graph (or big list entries)
    int32_t graph;
    int32_t cnt;
    int64_t v0;
};

struct BatchDev {
    int ngraphs, K, nsrc;
    float d, one_minus_d;
    double tol;
    int iters;
    const BGraph *graphs;
    const BTile *tiles;     // light tiles, grouped by graph
    int64_t ntiles;
    const BTile *btiles;    // big-vertex tiles (entries of `big`), grouped by graph
    int64_t nbtiles;
    const int32_t *big;     // [nbig_total] vertex ids
    const int64_t *bcstart; // [nbig_total + 1] chunk range of each big vertex
    const BChunk *chunks;
    int64_t nchunks;
    float *part;            // [nchunks][K] chunk partial rows
    double *res_part;       // [(ntiles + nbtiles)][K] residual partial rows
    const int32_t *seeds;   // [ngraphs][K]
    int32_t *active;        // [ngraphs][K] 1 while vector j still iterates
    int32_t *iters_done;    // [ngraphs][K]
    int32_t *gdone;         // [ngraphs] sweep after which every vector of the graph had stopped (0: not yet)
    const int32_t *sources; // [ngraphs][64] (MS-BFS)
    int32_t *counters;      // [2]: sweeps done / levels done
    unsigned long long *mcount;  // [ngraphs] MS-BFS newly visited per level
    GridSync *sync;
};

// ------------------------------------------------------------------ batched PPR

// Compensated (Kahan) accumulation: each column sums up to hundreds of terms
// one after another, so the running rounding error is carried in `comp`.
__device__ __forceinline__ void kahan_add(float &acc, float &comp, float x) {
    const float y = x - comp;
    const float t = acc + y;
    comp = (t - acc) - y;
    acc = t;
}

template <int KPL>  // floats per lane: K = 32 * KPL
__device__ __forceinline__ void row_fma(float (&acc)[KPL], float (&comp)[KPL], const float *row, float f) {
    if (KPL % 4 == 0) {
#pragma unroll
        for (int q = 0; q < KPL / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(row) + q);
            kahan_add(acc[4 * q], comp[4 * q], f * t.x);
            kahan_add(acc[4 * q + 1], comp[4 * q + 1], f * t.y);
            kahan_add(acc[4 * q + 2], comp[4 * q + 2], f * t.z);
            kahan_add(acc[4 * q + 3], comp[4 * q + 3], f * t.w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < KPL; ++q) kahan_add(acc[q], comp[q], f * __ldg(row + q));
    }
}

// Gathered sum over in-edges [beg, end) of vertex rows of X (lane's columns).
template <int KPL>
__device__ __forceinline__ void gather_rows(const BatchDev &B, const BGraph &G, const float *X, int64_t beg,
                                            int64_t end, float (&acc)[KPL]) {
    const int lane = lane_id();
    const int K = 32 * KPL;
    float comp[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) comp[q] = 0.f;
    int64_t e = beg;
    // four rows in flight per warp: indices and scale factors first, then the rows
    for (; e + 4 <= end; e += 4) {
        int32_t u[4];
        float f[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q] = __ldg(G.csc_idx + e + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            f[q] = __ldg(G.inv_deg + u[q]);
            if (G.csc_w) f[q] *= __ldg(G.csc_w + e + q);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) row_fma<KPL>(acc, comp, X + (int64_t)u[q] * K + lane * KPL, f[q]);
    }
    for (; e < end; ++e) {
        const int32_t u = __ldg(G.csc_idx + e);
        float f = __ldg(G.inv_deg + u);
        if (G.csc_w) f *= __ldg(G.csc_w + e);
        row_fma<KPL>(acc, comp, X + (int64_t)u * K + lane * KPL, f);
    }
}

// Writes row v of Y from the gathered sum, carrying frozen columns forward;
// accumulates |y - x| of active columns.
template <int KPL>
__device__ __forceinline__ void finish_row(const BatchDev &B, int gi, const BGraph &G, const float *Xc, float *Y,
                                           int64_t v, const float (&acc)[KPL], ResSum (&res)[KPL]) {
    const int lane = lane_id();
    const int K = 32 * KPL;
    const int64_t o = v * K + lane * KPL;
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int j = lane * KPL + q;
        const float x = Xc[o + q];
        float y = x;
        if (B.active[gi * K + j]) {
            const float base = (B.seeds[gi * K + j] == (int32_t)v) ? B.one_minus_d : 0.f;
            y = base + B.d * acc[q];
            res[q].add(y, x);
        }
        Y[o + q] = y;
    }
}

// Block-level reduction of per-lane column residuals into res_part[row][K]:
// every warp leaves its column partials in shared memory, then one thread per
// column adds the warps' partials in warp order (deterministic), compensated.
template <int KPL>
__device__ void flush_res(const BatchDev &B, int64_t row, ResSum (&res)[KPL], float *sm /* [warps][K] */) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int K = 32 * KPL;
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        sm[w * K + lane * KPL + q] = res[q].getf();
        res[q] = ResSum();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        ResSum t;
        for (int i = 0; i < nw; ++i) t.push(sm[i * K + j]);
        B.res_part[row * K + j] = t.get();
    }
    __syncthreads();
}

template <int KPL>
__global__ void __launch_bounds__(BT_THREADS) k_ppr_persistent(BatchDev B) {
    __shared__ float sm[(BT_THREADS / 32) * 32 * KPL];
    const int K = 32 * KPL;
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // initial iterate 1/n per column, every vector active
    for (int gi = 0; gi < B.ngraphs; ++gi) {
        const BGraph &G = B.graphs[gi];
        const float x0 = 1.0f / (float)G.n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.n * K; i += (int64_t)gridDim.x * blockDim.x)
            G.X0[i] = x0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B.ngraphs * K;
         i += (int64_t)gridDim.x * blockDim.x) {
        B.active[i] = 1;
        B.iters_done[i] = 0;
        if (i < B.ngraphs) B.gdone[i] = 0;
    }
    if (!grid_sync(B.sync, gridDim.x)) return;
    int k = 1;
    for (; k <= B.iters; ++k) {
        // phase 1a: chunks of big vertices -> partial rows
        for (int64_t c = gwarp; c < B.nchunks; c += nwarps) {
            const BChunk ch = B.chunks[c];
            if (B.gdone[ch.graph]) continue;  // every vector of this graph has stopped
            const BGraph &G = B.graphs[ch.graph];
            const float *Xc = (k & 1) ? G.X0 : G.X1;
            float acc[KPL];
#pragma unroll
            for (int q = 0; q < KPL; ++q) acc[q] = 0.f;
            gather_rows<KPL>(B, G, Xc, ch.beg, ch.beg + ch.len, acc);
#pragma unroll
            for (int q = 0; q < KPL; ++q) B.part[c * K + lane * KPL + q] = acc[q];
        }
        // phase 1b: light tiles, one vertex per warp at a time
        for (int64_t t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
            const BTile tl = B.tiles[t];
            if (B.gdone[tl.graph]) continue;
            const BGraph &G = B.graphs[tl.graph];
            const float *Xc = (k & 1) ? G.X0 : G.X1;
            float *Y = (k & 1) ? G.X1 : G.X0;
            ResSum res[KPL];
            for (int i = wib; i < tl.cnt; i += wpb) {
                const int64_t v = tl.v0 + i;
                const int64_t b = G.csc_off[v], e = G.csc_off[v + 1];
                if (e - b > BT_BIG) continue;  // big vertex: finished in phase 2
                float acc[KPL];
#pragma unroll
                for (int q = 0; q < KPL; ++q) acc[q] = 0.f;
                gather_rows<KPL>(B, G, Xc, b, e, acc);
                finish_row<KPL>(B, tl.graph, G, Xc, Y, v, acc, res);
            }
            flush_res<KPL>(B, t, res, sm);
        }
        if (!grid_sync(B.sync, gridDim.x)) return;
        // phase 2: big vertices combine their chunk rows
        for (int64_t t = blockIdx.x; t < B.nbtiles; t += gridDim.x) {
            const BTile tl = B.btiles[t];
            if (B.gdone[tl.graph]) continue;
            const BGraph &G = B.graphs[tl.graph];
            const float *Xc = (k & 1) ? G.X0 : G.X1;
            float *Y = (k & 1) ? G.X1 : G.X0;
            ResSum res[KPL];
            for (int i = wib; i < tl.cnt; i += wpb) {
                const int64_t r = tl.v0 + i;
                const int64_t v = B.big[r];
                float acc[KPL], comp[KPL];
#pragma unroll
                for (int q = 0; q < KPL; ++q) acc[q] = comp[q] = 0.f;
                for (int64_t c = B.bcstart[r]; c < B.bcstart[r + 1]; ++c)
#pragma unroll
                    for (int q = 0; q < KPL; ++q) kahan_add(acc[q], comp[q], B.part[c * K + lane * KPL + q]);
                finish_row<KPL>(B, tl.graph, G, Xc, Y, v, acc, res);
            }
            flush_res<KPL>(B, B.ntiles + t, res, sm);
        }
        if (!grid_sync(B.sync, gridDim.x)) return;
        // phase 3: per-vector residuals (fixed order) and convergence masks
        int still = 0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B.ngraphs * K;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int gi = (int)(i / K), j = (int)(i % K);
            const BGraph &G = B.graphs[gi];
            if (!B.active[i]) continue;
            double r = 0.0;
            for (int64_t t = G.tile0; t < G.tile0 + G.ntiles; ++t) r += B.res_part[t * K + j];
            for (int64_t t = 0; t < B.nbtiles; ++t)
                if (B.btiles[t].graph == gi) r += B.res_part[(B.ntiles + t) * K + j];
            B.iters_done[i] = k;
            if (r < B.tol)
                B.active[i] = 0;
            else
                still = 1;
        }
        still = __syncthreads_or(still);
        if (threadIdx.x == 0 && still) atomicAdd(B.counters + 2 + (k & 1), 1);
        if (!grid_sync(B.sync, gridDim.x)) return;
        const int any = ((volatile int *)B.counters)[2 + (k & 1)];
        if (threadIdx.x == 0 && blockIdx.x == 0) B.counters[2 + ((k + 1) & 1)] = 0;  // reset the other slot
        // a graph whose vectors have all stopped is skipped from now on (one writer per graph)
        for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < B.ngraphs;
             gi += (int64_t)gridDim.x * blockDim.x) {
            if (B.gdone[gi]) continue;
            int act = 0;
            for (int j = 0; j < K; ++j) act |= B.active[gi * K + j];
            if (!act) B.gdone[gi] = k;
        }
        if (!any) break;
        if (!grid_sync(B.sync, gridDim.x)) return;
    }
    // graph gi's last iterate was written by its last sweep (gdone, or the final
    // sweep if it never finished): X1 after an odd sweep, X0 after an even one
    const int last = std::min(k, B.iters);
    if (!grid_sync(B.sync, gridDim.x)) return;
    for (int gi = 0; gi < B.ngraphs; ++gi) {
        const int lg = B.gdone[gi] ? B.gdone[gi] : last;
        if (!(lg & 1)) continue;
        const BGraph &G = B.graphs[gi];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.n * K; i += (int64_t)gridDim.x * blockDim.x)
            G.X0[i] = G.X1[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) B.counters[0] = last;
}

// ------------------------------------------------------------------ batched multi-source BFS

__global__ void __launch_bounds__(BT_THREADS) k_msbfs_persistent(BatchDev B) {
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gthread >> 5, nwarps = nthreads >> 5;
    const int lane = lane_id();
    const int nsrc = B.nsrc;
    const uint64_t full = nsrc == 64 ? ~0ull : ((1ull << nsrc) - 1ull);
    for (int gi = 0; gi < B.ngraphs; ++gi) {
        const BGraph &G = B.graphs[gi];
        for (int64_t v = gthread; v < G.n; v += nthreads) {
            G.F[v] = 0;
            G.V[v] = 0;
            G.N[v] = 0;
        }
        for (int64_t i = gthread; i < G.n * 64; i += nthreads) G.levels[i] = -1;
    }
    if (gthread < 2 * (int64_t)B.ngraphs) B.mcount[gthread] = 0;
    if (!grid_sync(B.sync, gridDim.x)) return;
    if (gthread < (int64_t)B.ngraphs) {  // one thread per graph seeds its searches
        const BGraph &G = B.graphs[gthread];
        for (int j = 0; j < nsrc; ++j) {
            const int32_t s = B.sources[gthread * 64 + j];
            G.F[s] |= 1ull << j;
            G.V[s] |= 1ull << j;
            G.levels[(int64_t)s * 64 + j] = 0;
        }
    }
    if (!grid_sync(B.sync, gridDim.x)) return;
    int L = 0;
    for (;; ++L) {
        // expand: pull the frontier masks of in-neighbours (early exit once covered);
        // high in-degree vertices are scanned by a whole warp
        for (int gi = 0; gi < B.ngraphs; ++gi) {
            const BGraph &G = B.graphs[gi];
            for (int64_t v = gthread; v < G.n; v += nthreads) {
                const uint64_t vis = G.V[v];
                if (vis == full) continue;
                const int64_t b = G.csc_off[v], e = G.csc_off[v + 1];
                if (e - b > BT_BIG) continue;
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
        if (!grid_sync(B.sync, gridDim.x)) return;
        // update: owner-only writes of V, F and the levels of newly reached searches
        for (int gi = 0; gi < B.ngraphs; ++gi) {
            const BGraph &G = B.graphs[gi];
            unsigned long long cnt = 0;
            for (int64_t v = gthread; v < G.n; v += nthreads) {
                const uint64_t nw = G.N[v];
                G.F[v] = nw;
                if (nw) {
                    G.V[v] |= nw;
                    G.N[v] = 0;
                    cnt += __popcll(nw);
                    for (uint64_t bits = nw; bits; bits &= bits - 1)
                        G.levels[v * 64 + (__ffsll((long long)bits) - 1)] = L + 1;
                }
            }
            cnt = warp_sum(cnt);
            if (lane == 0 && cnt) atomicAdd(B.mcount + (L & 1) * B.ngraphs + gi, cnt);
        }
        if (!grid_sync(B.sync, gridDim.x)) return;
        unsigned long long total = 0;
        for (int gi = 0; gi < B.ngraphs; ++gi) total += ((volatile unsigned long long *)B.mcount)[(L & 1) * B.ngraphs + gi];
        if (gthread < (int64_t)B.ngraphs) B.mcount[((L + 1) & 1) * B.ngraphs + gthread] = 0;
        if (!grid_sync(B.sync, gridDim.x)) return;
        if (total == 0) break;
    }
    if (gthread == 0) B.counters[1] = L + 1;
}

}  // namespace gp

// ================================================================== host side

struct gp_batch {
    int device = 0, num_sms = 0;
    int ngraphs = 0, K = 0;
    std::vector<gp_graph *> graphs;
    std::vector<gp::BGraph> hg;
    gp::BatchDev dev;
    gp::Arena mem;
    gp::BGraph *dgraphs = nullptr;
    int32_t *seeds = nullptr, *sources = nullptr;
    int32_t *counters = nullptr;
    int32_t *hcounters = nullptr;  // pinned
    cudaStream_t home = nullptr;
    cudaGraphExec_t ppr_exec = nullptr, bfs_exec = nullptr;
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

}  // namespace gp

using namespace gp;

extern "C" int gp_batch_create(gp_batch **out, gp_graph *const *graphs, int ngraphs, int k_ppr, void *stream) {
    clear_error();
    if (!out) return set_error(GP_ERR_INVALID, "gp_batch_create: out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1) return set_error(GP_ERR_INVALID, "gp_batch_create: need at least one graph");
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
    GP_CUDA(cudaGetDevice(&b->device));
    GP_CUDA(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
    auto fail = [&](int st) {
        b->mem.release(s);
        if (b->hcounters) cudaFreeHost(b->hcounters);
        delete b;
        return st;
    };
    // work lists: read the in-degrees on the host once (batch set-up, not the sweep)
    std::vector<BTile> tiles, btiles;
    std::vector<int32_t> big;
    std::vector<int64_t> bcstart(1, 0);
    std::vector<BChunk> chunks;
    b->hg.resize(ngraphs);
    const int K = k_ppr;
    for (int gi = 0; gi < ngraphs; ++gi) {
        gp_graph *g = graphs[gi];
        std::vector<int64_t> off((size_t)g->n + 1);
        cudaError_t e = cudaMemcpyAsync(off.data(), g->csc_off, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(set_error(GP_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e)));
        BGraph &G = b->hg[gi];
        memset(&G, 0, sizeof(G));
        G.n = g->n;
        G.csc_off = g->csc_off;
        G.csc_idx = g->csc_idx;
        G.csc_w = g->csc_w;
        G.inv_deg = g->inv_deg;
        G.tile0 = (int64_t)tiles.size();
        for (int64_t v0 = 0; v0 < g->n; v0 += BT_TILE)
            tiles.push_back(BTile{gi, (int32_t)std::min<int64_t>(BT_TILE, g->n - v0), v0});
        G.ntiles = (int64_t)tiles.size() - G.tile0;
        G.big0 = (int64_t)big.size();
        for (int64_t v = 0; v < g->n; ++v) {
            const int64_t d = off[v + 1] - off[v];
            if (d <= BT_BIG) continue;
            big.push_back((int32_t)v);
            for (int64_t p = off[v]; p < off[v + 1]; p += BT_CHUNK)
                chunks.push_back(BChunk{p, (int32_t)std::min<int64_t>(BT_CHUNK, off[v + 1] - p), gi});
            bcstart.push_back((int64_t)chunks.size());
        }
        G.nbig = (int64_t)big.size() - G.big0;
        for (int64_t r = 0; r < G.nbig; r += BT_TILE)
            btiles.push_back(BTile{gi, (int32_t)std::min<int64_t>(BT_TILE, G.nbig - r), G.big0 + r});
    }
    BatchDev &D = b->dev;
    memset(&D, 0, sizeof(D));
    D.ngraphs = ngraphs;
    D.K = K;
    int st = GP_OK;
    BTile *dt = nullptr, *dbt = nullptr;
    int32_t *dbig = nullptr;
    int64_t *dbc = nullptr;
    BChunk *dch = nullptr;
    for (int gi = 0; gi < ngraphs && st == GP_OK; ++gi) {
        BGraph &G = b->hg[gi];
        const size_t n = (size_t)G.n;
        if (st == GP_OK) st = b->mem.alloc(G.X0, n * K, s);
        if (st == GP_OK) st = b->mem.alloc(G.X1, n * K, s);
        if (st == GP_OK) st = b->mem.alloc(G.F, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.V, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.N, n, s);
        if (st == GP_OK) st = b->mem.alloc(G.levels, n * 64, s);
    }
    if (st == GP_OK) st = b->mem.alloc(b->dgraphs, (size_t)ngraphs, s);
    if (st == GP_OK) st = b->mem.alloc(dt, std::max<size_t>(tiles.size(), 1), s);
    if (st == GP_OK) st = b->mem.alloc(dbt, std::max<size_t>(btiles.size(), 1), s);
    if (st == GP_OK) st = b->mem.alloc(dbig, std::max<size_t>(big.size(), 1), s);
    if (st == GP_OK) st = b->mem.alloc(dbc, bcstart.size(), s);
    if (st == GP_OK) st = b->mem.alloc(dch, std::max<size_t>(chunks.size(), 1), s);
    if (st == GP_OK) st = b->mem.alloc(D.part, std::max<size_t>(chunks.size(), 1) * K, s);
    if (st == GP_OK) st = b->mem.alloc(D.res_part, (tiles.size() + btiles.size() + 1) * K, s);
    if (st == GP_OK) st = b->mem.alloc(b->seeds, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(b->sources, (size_t)ngraphs * 64, s);
    if (st == GP_OK) st = b->mem.alloc(D.active, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(D.iters_done, (size_t)ngraphs * K, s);
    if (st == GP_OK) st = b->mem.alloc(D.gdone, (size_t)ngraphs, s);
    if (st == GP_OK) st = b->mem.alloc(b->counters, 8, s);
    if (st == GP_OK) st = b->mem.alloc(D.mcount, (size_t)ngraphs * 2, s);
    GridSync *sync = nullptr;
    if (st == GP_OK) st = b->mem.alloc(sync, 1, s);
    if (st != GP_OK) return fail(st);
    {
        cudaError_t e = cudaMallocHost(&b->hcounters, 8 * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->dgraphs, b->hg.data(), ngraphs * sizeof(BGraph), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !tiles.empty()) e = cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !btiles.empty()) e = cudaMemcpyAsync(dbt, btiles.data(), btiles.size() * sizeof(BTile), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !big.empty()) e = cudaMemcpyAsync(dbig, big.data(), big.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dbc, bcstart.data(), bcstart.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !chunks.empty()) e = cudaMemcpyAsync(dch, chunks.data(), chunks.size() * sizeof(BChunk), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(D.mcount, 0, (size_t)ngraphs * 2 * sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(set_error(GP_ERR_CUDA, "batch set-up copy: %s", cudaGetErrorString(e)));
    }
    D.graphs = b->dgraphs;
    D.tiles = dt;
    D.ntiles = (int64_t)tiles.size();
    D.btiles = dbt;
    D.nbtiles = (int64_t)btiles.size();
    D.big = dbig;
    D.bcstart = dbc;
    D.chunks = dch;
    D.nchunks = (int64_t)chunks.size();
    D.seeds = b->seeds;
    D.sources = b->sources;
    D.counters = b->counters;
    D.sync = sync;
    *out = b;
    return GP_OK;
}

extern "C" int gp_batch_free(gp_batch *b) {
    clear_error();
    if (!b) return GP_OK;
    cudaDeviceSynchronize();
    if (b->ppr_exec) cudaGraphExecDestroy(b->ppr_exec);
    if (b->bfs_exec) cudaGraphExecDestroy(b->bfs_exec);
    b->mem.release(b->home);
    if (b->hcounters) cudaFreeHost(b->hcounters);
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
    const void *kernel = K == 32 ? (const void *)k_ppr_persistent<1>
                       : K == 64 ? (const void *)k_ppr_persistent<2>
                       : K == 128 ? (const void *)k_ppr_persistent<4> : (const void *)k_ppr_persistent<8>;
    const bool rebuild = b->ppr_iters != iters || b->ppr_tol != tol || b->ppr_d != damping;
    if (rebuild) {
        GP_TRY(batch_grid(b, kernel, b->grid));
        b->dev.d = damping;
        b->dev.one_minus_d = 1.0f - damping;
        b->dev.tol = tol;
        b->dev.iters = iters;
        b->ppr_iters = iters;
        b->ppr_tol = tol;
        b->ppr_d = damping;
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
    const bool rebuild = b->bfs_nsrc != nsrc;
    int grid = 0;
    GP_TRY(batch_grid(b, (const void *)k_msbfs_persistent, grid));
    const int saved = b->grid;
    b->grid = grid;
    b->dev.nsrc = nsrc;
    b->bfs_nsrc = nsrc;
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
    }
    if (hs.err) return set_error(GP_ERR_TIMEOUT, "batched BFS: a grid barrier wait ran out");
    return GP_OK;
}
