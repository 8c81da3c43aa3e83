// pagerank.cu -- push and pull PageRank sweeps and the gp_pagerank driver.
//
// One sweep computes (Section 3.1 formula; Algorithm 1, push- and pull-based PR)
//     y[v] = (1-d) s[v] + d * sum_{(u->v)} P_vu x[u]
// from the contribution vector c[u] = x[u] * inv_deg[u] (so the gather never
// fetches a neighbour's degree, the extra cost of pulling named in Section 7.3)
// and edge factor w_uv (1 when unweighted).
//
// Pull (owner-only writes, no atomics; Section 4.1 "Atomics/Locks"):
//   k_pull_big    -- vertices whose in-degree exceeds pull_light_max: their
//                    in-edge lists are cut into chunks of <= chunk_edges edges,
//                    one warp per chunk, coalesced index loads, warp tree sum
//                    (Section 4's CREW binary merge-tree) into a per-chunk slot.
//   k_pull_light  -- blocks [0, light_blocks): one warp per tile of 32
//                    consecutive vertices; the tile's light in-edges are one
//                    contiguous stream walked 32 edges at a time, each lane
//                    finds the vertex owning its edge, and a segmented warp
//                    scan forms per-vertex sums.  Blocks after that: one thread
//                    per big vertex adds its chunk slots.  Every vertex's
//                    y, c' = y*inv_deg and |y - x| are written by its owner.
// Push (scatter with atomics; Section 4.1: O(Lm) write conflicts):
//   k_push_scatter   -- each source adds d*c[u]*w_uv into y[v] for its
//                       out-edges with FP32 atomicAdd (RED), big sources in
//                       warp chunks, light sources in 32-vertex tiles.
//   k_push_epilogue  -- per vertex: residual, c' and the (1-d)s reset of the
//                       buffer the next sweep accumulates into.
// Convergence (not in the paper, which runs a fixed L): the L1 residual is
// reduced in FP64 per block; the first kernel of the next sweep reduces the
// block partials (every block, same order, so all agree) and stops the
// iteration on the device, so the host only polls every few sweeps.
#include <algorithm>
#include <cmath>

#include "gp_internal.cuh"

namespace gp {

struct PrStatus {
    int32_t done;
    int32_t iters_done;
    double residual;
    int32_t converged;
    int32_t pad;
};

struct PrArgs {
    int64_t n;
    const int64_t *off;  // CSC (pull) or CSR (push) offsets
    const int32_t *idx;
    const float *w;      // edge factors in the same order, or nullptr
    const float *inv_deg;
    // big-vertex chunks
    const int32_t *big;
    const int64_t *cstart;
    const Chunk *chunks;
    int64_t nbig, nchunks;
    int32_t light_max;
    // vectors
    const float *x;  // previous iterate
    float *y;        // new iterate
    const float *c;  // contributions of x
    float *c_next;   // contributions of y (pull)
    const float *s;  // personalization or nullptr
    float base_uniform;  // (1-d)/n
    float one_minus_d, d;
    double tol;
    int32_t k;  // sweep number, 1-based
    int32_t nprev;
    double *partials;
    float *chunk_part;
    double *acc64;  // FP64 push accumulator (or nullptr)
    const float *c_hot;  // hot contributions (pull, HOT kernels)
    int64_t nhot;
    PrStatus *status;
    int32_t split_blocks;  // pull: light-tile blocks; push: big-chunk blocks
};

__device__ __forceinline__ float base_term(const PrArgs &a, int64_t v) {
    return a.s ? a.one_minus_d * a.s[v] : a.base_uniform;
}

// Convergence gate at the start of sweep k: every block reduces the residual
// partials of sweep k-1 in the same order, so all blocks take the same
// decision; block 0 records it.  Returns true when the iteration has stopped.
__device__ bool pr_gate(const PrArgs &a, int k) {
    __shared__ double sm[32];
    __shared__ int stop;
    volatile PrStatus *st = a.status;
    if (threadIdx.x == 0) stop = st->done;
    __syncthreads();
    if (stop) return true;
    if (k > 1) {
        double r = 0.0;
        for (int i = threadIdx.x; i < a.nprev; i += blockDim.x) r += a.partials[i];
        r = block_sum(r, sm);
        if (threadIdx.x == 0) {
            const int conv = r < a.tol;
            if (blockIdx.x == 0) {
                st->residual = r;
                st->iters_done = k - 1;
                if (conv) {
                    st->converged = 1;
                    st->done = 1;
                }
            }
            stop = conv;
        }
        __syncthreads();
    }
    return stop != 0;
}

__global__ void k_pr_init(int64_t n, const float *x0, const float *inv_deg, float *r0, float *c, float *r_push,
                          double *acc64, const float *s, float one_minus_d, float base_uniform, PrStatus *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float x_uniform = 1.0f / (float)n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const float x = x0 ? x0[v] : x_uniform;
        r0[v] = x;
        c[v] = x * inv_deg[v];
        if (r_push) r_push[v] = s ? one_minus_d * s[v] : base_uniform;
        if (acc64) acc64[v] = (double)(s ? one_minus_d * s[v] : base_uniform);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status->done = 0;
        status->iters_done = 0;
        status->residual = 0.0;
        status->converged = 0;
    }
}

// Records the decision for the last sweep enqueued (sweep k-1) without doing a sweep.
__global__ void k_pr_finish(PrArgs a) { pr_gate(a, a.k); }

// ------------------------------------------------------------------ pull

// Shared-memory copy of the hot contributions (see HotSet): loaded once per
// block, then every gather of a hot vertex is a shared-memory read.
template <bool HOT>
__device__ __forceinline__ void load_hot(const PrArgs &a, float *sh) {
    if (!HOT) return;
    const int64_t nh = a.nhot;
    const float4 *src = reinterpret_cast<const float4 *>(a.c_hot);
    float4 *dst = reinterpret_cast<float4 *>(sh);
    for (int64_t i = threadIdx.x; i < nh / 4; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int64_t i = (nh & ~int64_t(3)) + threadIdx.x; i < nh; i += blockDim.x) sh[i] = __ldg(a.c_hot + i);
    __syncthreads();
}

template <bool HOT>
__device__ __forceinline__ float gather_c(const float *__restrict__ c, const float *sh, int32_t u) {
    if (HOT && u < 0) return sh[u & 0x7fffffff];
    return __ldg(c + u);
}

constexpr int BIG_UNROLL = 8;

// Index arrays are streamed once per sweep: loaded with the evict-first hint so
// they do not push the gathered contribution vector out of L2.
#ifndef GP_IDX_STREAMING
#define GP_IDX_STREAMING 1
#endif
__device__ __forceinline__ int32_t ld_idx(const int32_t *p) {
#if GP_IDX_STREAMING
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

template <bool W, bool HOT>
__global__ void __launch_bounds__(1024) k_pull_big(PrArgs a) {
    extern __shared__ float sh_hot[];
    if (pr_gate(a, a.k)) return;
    load_hot<HOT>(a, sh_hot);
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t *__restrict__ idx = a.idx;
    const float *__restrict__ c = a.c;
    const float *__restrict__ w = a.w;
    for (int64_t j = warp; j < a.nchunks; j += nwarps) {
        const Chunk ch = a.chunks[j];
        const int32_t *ip = idx + ch.beg;
        const float *wp = W ? w + ch.beg : nullptr;
        float acc = 0.f;
        for (int i0 = 0; i0 < ch.len; i0 += 32 * BIG_UNROLL) {
            // all index loads of the window first, then all gathers: BIG_UNROLL in flight per lane
            int32_t u[BIG_UNROLL];
#pragma unroll
            for (int q = 0; q < BIG_UNROLL; ++q) {
                const int i = i0 + q * 32 + lane;
                u[q] = i < ch.len ? ld_idx(ip + i) : 0;
            }
            float f[BIG_UNROLL];
#pragma unroll
            for (int q = 0; q < BIG_UNROLL; ++q) {
                const int i = i0 + q * 32 + lane;
                f[q] = 0.f;
                if (i < ch.len) {
                    f[q] = gather_c<HOT>(c, sh_hot, u[q]);
                    if (W) f[q] *= __ldg(wp + i);
                }
            }
#pragma unroll
            for (int q = 0; q < BIG_UNROLL; ++q) acc += f[q];
        }
        acc = warp_sum(acc);
        if (lane == 0) a.chunk_part[j] = acc;
    }
}

// Owner lane of virtual edge `eid` in a tile: the last lane k with excl[k] <= eid
// (zero-degree lanes share their successor's excl, so the last one is non-empty).
__device__ __forceinline__ int tile_owner(int excl, int eid) {
    int k = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int ex = __shfl_sync(FULL, excl, k + s);
        if (ex <= eid) k += s;
    }
    return k;
}

// Sum of the lanes of `val` that belong to the same vertex in this 32-edge
// window, delivered to that vertex's own lane (segmented warp scan).
__device__ __forceinline__ float window_segment_sum(float val, int kex, int base, int deg, int excl, int incl) {
    const int lane = lane_id();
    const int head = max(kex, base) - base;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float tv = __shfl_up_sync(FULL, val, s);
        if (lane - s >= head) val += tv;
    }
    const bool has = deg > 0 && excl < base + 32 && incl > base;
    const int tail = has ? min(incl, base + 32) - base - 1 : 0;
    const float seg = __shfl_sync(FULL, val, tail);
    return has ? seg : 0.f;
}

#ifndef GP_LIGHT_WINDOWS
#define GP_LIGHT_WINDOWS 4
#endif
#ifndef GP_LIGHT_MIN_BLOCKS
#define GP_LIGHT_MIN_BLOCKS 3
#endif
constexpr int LW = GP_LIGHT_WINDOWS;  // 32-edge windows in flight per step of the light tiles

template <bool W, bool HOT>
__global__ void __launch_bounds__(512, GP_LIGHT_MIN_BLOCKS) k_pull_light(PrArgs a) {
    extern __shared__ float sh_hot[];
    __shared__ double sm[32];
    if (((volatile PrStatus *)a.status)->done) return;
    const int lane = lane_id();
    double res = 0.0;
    const int64_t n = a.n;
    if ((int)blockIdx.x < a.split_blocks) {
        load_hot<HOT>(a, sh_hot);
        const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)a.split_blocks * blockDim.x) >> 5;
        const int64_t ntiles = (n + 31) >> 5;
        const int32_t *__restrict__ idx = a.idx;
        const float *__restrict__ c = a.c;
        const float *__restrict__ wv = a.w;
        // offsets of the first tile; inside the loop the next tile's are fetched early
        int64_t t = warp;
        int64_t nb = 0, ne = 0;
        if (t < ntiles && t * 32 + lane < n) {
            nb = a.off[t * 32 + lane];
            ne = a.off[t * 32 + lane + 1];
        }
        for (; t < ntiles; t += nwarps) {
            const int64_t v = t * 32 + lane;
            const int64_t b = nb, e = ne;
            // per-vertex operands, independent of the edges: issued now
            float xv = 0.f, inv = 0.f, base_v = 0.f;
            if (v < n) {
                xv = a.x[v];
                inv = a.inv_deg[v];
                base_v = base_term(a, v);
            }
            const int64_t tn = t + nwarps, vn = tn * 32 + lane;
            nb = ne = 0;
            if (tn < ntiles && vn < n) {
                nb = a.off[vn];
                ne = a.off[vn + 1];
            }
            const int64_t dd = e - b;
            const bool big = dd > a.light_max;
            const int deg = big ? 0 : (int)dd;
            const int incl = warp_incl_scan(deg);
            const int excl = incl - deg;
            const int E = __shfl_sync(FULL, incl, 31);
            float acc = 0.f;
            for (int base = 0; base < E; base += 32 * LW) {
                // LW 32-edge windows per step: all index loads, then all gathers, then the sums
                int kx[LW];
                int64_t p[LW];
                int32_t u[LW];
#pragma unroll
                for (int q = 0; q < LW; ++q) {
                    const int eq = base + 32 * q + lane;
                    const int k = tile_owner(excl, eq);
                    kx[q] = __shfl_sync(FULL, excl, k);
                    p[q] = __shfl_sync(FULL, b, k) + (eq - kx[q]);
                }
#pragma unroll
                for (int q = 0; q < LW; ++q) u[q] = base + 32 * q + lane < E ? ld_idx(idx + p[q]) : 0;
                float f[LW];
#pragma unroll
                for (int q = 0; q < LW; ++q) {
                    f[q] = 0.f;
                    if (base + 32 * q + lane < E) {
                        f[q] = gather_c<HOT>(c, sh_hot, u[q]);
                        if (W) f[q] *= __ldg(wv + p[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < LW; ++q)
                    if (base + 32 * q < E) acc += window_segment_sum(f[q], kx[q], base + 32 * q, deg, excl, incl);
            }
            if (v < n && !big) {
                const float y = base_v + a.d * acc;
                res += fabs((double)y - (double)xv);
                a.y[v] = y;
                a.c_next[v] = y * inv;
            }
        }
    } else {
        const int64_t nth = (int64_t)(gridDim.x - a.split_blocks) * blockDim.x;
        for (int64_t r = (int64_t)(blockIdx.x - a.split_blocks) * blockDim.x + threadIdx.x; r < a.nbig; r += nth) {
            const int32_t v = a.big[r];
            float acc = 0.f;
            for (int64_t j = a.cstart[r]; j < a.cstart[r + 1]; ++j) acc += a.chunk_part[j];
            const float y = base_term(a, v) + a.d * acc;
            res += fabs((double)y - (double)a.x[v]);
            a.y[v] = y;
            a.c_next[v] = y * a.inv_deg[v];
        }
    }
    res = block_sum(res, sm);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = res;
}

// c_hot[slot] = c[hot_id[slot]] for the sweep that reads c next.
__global__ void k_hot_gather(const int32_t *hot_id, int64_t nhot, const float *c, float *c_hot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nhot; i += stride) c_hot[i] = c[hot_id[i]];
}

// ------------------------------------------------------------------ push

// Accumulator of the scattered updates: FP32 (the paper's float atomics) or
// FP64 (same atomic count; the order-dependent rounding of FP32 atomics at hubs
// otherwise leaves an L1 residual floor above 1e-7 on graphs with 4M vertices).
template <bool W, class T>
__global__ void __launch_bounds__(256) k_push_scatter(PrArgs a) {
    if (pr_gate(a, a.k)) return;
    const int lane = lane_id();
    const int32_t *__restrict__ idx = a.idx;
    const float *__restrict__ wv = a.w;
    T *y = sizeof(T) == 8 ? (T *)a.acc64 : (T *)a.y;
    if ((int)blockIdx.x < a.split_blocks) {
        const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)a.split_blocks * blockDim.x) >> 5;
        for (int64_t j = warp; j < a.nchunks; j += nwarps) {
            const Chunk ch = a.chunks[j];
            const float cu = a.d * __ldg(a.c + ch.v);
            const int32_t *ip = idx + ch.beg;
            const float *wp = W ? wv + ch.beg : nullptr;
            int i = lane;
            for (; i + 96 < ch.len; i += 128) {
                const int v0 = __ldg(ip + i), v1 = __ldg(ip + i + 32), v2 = __ldg(ip + i + 64), v3 = __ldg(ip + i + 96);
                atomicAdd(y + v0, (T)(W ? cu * __ldg(wp + i) : cu));
                atomicAdd(y + v1, (T)(W ? cu * __ldg(wp + i + 32) : cu));
                atomicAdd(y + v2, (T)(W ? cu * __ldg(wp + i + 64) : cu));
                atomicAdd(y + v3, (T)(W ? cu * __ldg(wp + i + 96) : cu));
            }
            for (; i < ch.len; i += 32) atomicAdd(y + __ldg(ip + i), (T)(W ? cu * __ldg(wp + i) : cu));
        }
    } else {
        __shared__ T agg[256];
        const int64_t n = a.n;
        const int64_t warp = ((int64_t)(blockIdx.x - a.split_blocks) * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)(gridDim.x - a.split_blocks) * blockDim.x) >> 5;
        const int64_t ntiles = (n + 31) >> 5;
        for (int64_t t = warp; t < ntiles; t += nwarps) {
            const int64_t u = t * 32 + lane;
            int64_t b = 0, e = 0;
            float cu = 0.f;
            if (u < n) {
                b = a.off[u];
                e = a.off[u + 1];
            }
            const int64_t dd = e - b;
            const bool big = dd > a.light_max;
            const int deg = big ? 0 : (int)dd;
            if (deg > 0) cu = a.d * __ldg(a.c + u);
            const int incl = warp_incl_scan(deg);
            const int excl = incl - deg;
            const int E = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < E; base += 32) {
                const int eid = base + lane;
                int k = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const int ex = __shfl_sync(FULL, excl, k + s);
                    if (ex <= eid) k += s;
                }
                const int64_t kb = __shfl_sync(FULL, b, k);
                const int kex = __shfl_sync(FULL, excl, k);
                const float ck = __shfl_sync(FULL, cu, k);
                int32_t dst = -1 - lane;  // distinct dummy keys for idle lanes
                T val = 0;
                if (eid < E) {
                    const int64_t pos = kb + (eid - kex);
                    dst = __ldg(idx + pos);
                    val = (T)(W ? ck * __ldg(wv + pos) : ck);
                }
                // Updates from different sources of the tile that hit the same vertex
                // (typically a hub) are summed in the warp first, so the vertex takes one
                // atomic per window instead of one per edge.
                const unsigned peers = __match_any_sync(FULL, dst);
                if (__all_sync(FULL, peers == (1u << lane))) {
                    if (eid < E) atomicAdd(y + dst, val);
                } else {
                    agg[threadIdx.x] = val;
                    __syncwarp();
                    if (eid < E && (peers & ((1u << lane) - 1u)) == 0) {  // lowest lane of its group
                        T sum = val;
                        for (unsigned rest = peers & ~(1u << lane); rest; rest &= rest - 1)
                            sum += agg[(threadIdx.x & ~31u) + (__ffs(rest) - 1)];
                        atomicAdd(y + dst, sum);
                    }
                    __syncwarp();
                }
            }
        }
    }
}

// Per vertex: the finished sum (rounded to the FP32 rank), the residual, the
// next contribution, and the reset of the buffer the next sweep accumulates into.
template <class T>
__global__ void __launch_bounds__(256) k_push_epilogue(PrArgs a) {
    __shared__ double sm[32];
    if (((volatile PrStatus *)a.status)->done) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double res = 0.0;
    float *x_reset = const_cast<float *>(a.x);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        if (sizeof(T) == 8) {
            const float y = (float)a.acc64[v];
            res += fabs((double)y - (double)a.x[v]);
            a.y[v] = y;
            a.c_next[v] = y * a.inv_deg[v];
            a.acc64[v] = (double)base_term(a, v);
        } else {
            const float y = a.y[v];
            res += fabs((double)y - (double)a.x[v]);
            a.c_next[v] = y * a.inv_deg[v];
            x_reset[v] = base_term(a, v);  // the next sweep accumulates into this buffer
        }
    }
    res = block_sum(res, sm);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = res;
}

// ------------------------------------------------------------------ driver

struct PrGrids {
    int big, light, epi_big, total2;
};

void release_pr_work(gp_graph *g, cudaStream_t s) {
    if (g->pr.status_host) cudaFreeHost(g->pr.status_host);
    g->pr.status_host = nullptr;
    g->pr.mem.release(s);
    g->pr = PrWork();
}

// Resident blocks per SM of `kernel` (raising its dynamic shared-memory limit first).
static int occupancy(const void *kernel, int threads, size_t smem, int &blocks) {
    // the opt-in is needed whenever dynamic + static shared memory exceeds 48 KiB; set it for any size
    if (smem > 0) GP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem));
    if (blocks < 1) return set_error(GP_ERR_UNSUPPORTED, "kernel does not fit on an SM (%zu B shared memory)", smem);
    return GP_OK;
}

static int ensure_pr_work(gp_graph *g, cudaStream_t s) {
    PrWork &w = g->pr;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const int64_t epi = (g->pull_bins.nbig + 255) / 256;
    // covers any grid: at most 32 resident blocks per SM, plus the epilogue blocks
    w.max_blocks = (int)(std::max(g->num_sms * 32, grid_blocks(g, 256)) + epi + 64);
    GP_TRY(w.mem.alloc(w.r1, n, s));
    GP_TRY(w.mem.alloc(w.c0, n, s));
    GP_TRY(w.mem.alloc(w.c1, n, s));
    GP_TRY(w.mem.alloc(w.partials, (size_t)w.max_blocks, s));
    GP_TRY(w.mem.alloc(w.chunk_part, (size_t)std::max<int64_t>(g->pull_bins.nchunks, 1), s));
    PrStatus *st = nullptr;
    GP_TRY(w.mem.alloc(st, 1, s));
    w.status = st;
    GP_CUDA(cudaMallocHost(&w.status_host, 4 * sizeof(PrStatus)));
    w.ready = true;
    return GP_OK;
}

static int ensure_vec(gp_graph *g, float *&slot, cudaStream_t s) {
    if (slot) return GP_OK;
    return g->pr.mem.alloc(slot, (size_t)std::max<int64_t>(g->n, 1), s);
}

}  // namespace gp

using namespace gp;

extern "C" int gp_pagerank(const gp_graph *gc, int mode, float damping, int iters, double tol,
                           const float *personalization, const float *x0, float *ranks_out, gp_pr_stats *stats,
                           void *stream) {
    clear_error();
    gp_graph *g = const_cast<gp_graph *>(gc);
    if (!g) return set_error(GP_ERR_INVALID, "gp_pagerank: graph is NULL");
    if (!ranks_out) return set_error(GP_ERR_INVALID, "gp_pagerank: ranks_out is NULL");
    if (!(damping > 0.f && damping < 1.f)) return set_error(GP_ERR_INVALID, "damping %g outside (0, 1)", (double)damping);
    if (iters < 1) return set_error(GP_ERR_INVALID, "iters = %d < 1", iters);
    if (!(tol >= 0.0)) return set_error(GP_ERR_INVALID, "tol must be >= 0");
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "bad mode %d", mode);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == GP_AUTO) mode = g->opt.pr_auto_mode >= 0 ? g->opt.pr_auto_mode : GP_PULL;
    const int64_t n = g->n;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0) {
        if (stats) {
            stats->mode_used = mode;
            stats->converged = 1;
        }
        return GP_OK;
    }
    GP_TRY(ensure_pr_work(g, s));
    PrWork &w = g->pr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    // inputs and outputs that live in host memory go through library buffers
    const bool out_dev = is_device_ptr(ranks_out);
    float *R0 = ranks_out;
    if (!out_dev) {
        GP_TRY(ensure_vec(g, w.out_dev, s));
        R0 = w.out_dev;
    }
    const float *S = personalization;
    if (S && !is_device_ptr(S)) {
        GP_TRY(ensure_vec(g, w.s_dev, s));
        GP_CUDA(cudaMemcpyAsync(w.s_dev, S, n * sizeof(float), cudaMemcpyHostToDevice, s));
        S = w.s_dev;
    }
    const float *X0 = x0;
    if (X0 && !is_device_ptr(X0)) {
        GP_TRY(ensure_vec(g, w.x0_dev, s));
        GP_CUDA(cudaMemcpyAsync(w.x0_dev, X0, n * sizeof(float), cudaMemcpyHostToDevice, s));
        X0 = w.x0_dev;
    }
    float *R[2] = {R0, w.r1};
    float *C[2] = {w.c0, w.c1};
    PrStatus *status = (PrStatus *)w.status;
    const bool push = mode == GP_PUSH;
    const bool W = g->weighted;

    PrArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.off = push ? g->csr_off : g->csc_off;
    a.idx = push ? g->csr_idx : g->csc_idx;
    a.w = W ? (push ? g->csr_w : g->csc_w) : nullptr;
    a.inv_deg = g->inv_deg;
    const BigBins &bins = push ? g->push_bins : g->pull_bins;
    a.big = bins.big;
    a.cstart = bins.cstart;
    a.chunks = bins.chunks;
    a.nbig = bins.nbig;
    a.nchunks = bins.nchunks;
    a.light_max = bins.light_max;
    a.s = S;
    a.one_minus_d = 1.0f - damping;
    a.d = damping;
    a.base_uniform = (float)((1.0 - (double)damping) / (double)n);
    a.tol = tol;
    a.partials = w.partials;
    a.chunk_part = w.chunk_part;
    a.status = status;

    const int gb = grid_blocks(g, 256);
    const int64_t ntiles = (n + 31) / 32;
    // pull: hot-contribution cache in shared memory (built once per graph)
    bool hot = false;
    int tbp = 256, tbl = 256;  // threads per block of pull_big / pull_light
    size_t smem = 0;
    if (!push) {
        if (g->pull_hot.slots != g->opt.pull_hot_slots) GP_TRY(build_pull_hot(g, g->opt.pull_hot_slots, s));
        hot = g->pull_hot.nhot > 0;
        if (hot) {
            tbp = 1024;
            tbl = 512;
            smem = (size_t)((g->pull_hot.nhot + 3) & ~int64_t(3)) * sizeof(float);
            a.c_hot = g->pull_hot.c_hot;
            a.nhot = g->pull_hot.nhot;
            a.idx = g->pull_hot.enc_idx;
        }
    }
    // grids
    int g1, g2, split;
    if (!push) {
        int ob = 0, ol = 0;
        if (W) {
            GP_TRY(occupancy(hot ? (const void *)k_pull_big<true, true> : (const void *)k_pull_big<true, false>, tbp, smem, ob));
            GP_TRY(occupancy(hot ? (const void *)k_pull_light<true, true> : (const void *)k_pull_light<true, false>, tbl, smem, ol));
        } else {
            GP_TRY(occupancy(hot ? (const void *)k_pull_big<false, true> : (const void *)k_pull_big<false, false>, tbp, smem, ob));
            GP_TRY(occupancy(hot ? (const void *)k_pull_light<false, true> : (const void *)k_pull_light<false, false>, tbl, smem, ol));
        }
        const int wpb = tbp / 32, wpl = tbl / 32;
        g1 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ob * g->num_sms, (bins.nchunks + wpb - 1) / wpb));
        split = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ol * g->num_sms, (ntiles + wpl - 1) / wpl));
        g2 = split + (int)((bins.nbig + tbl - 1) / tbl);
    } else {
        split = (int)std::min<int64_t>(gb, (bins.nchunks + 7) / 8);
        g1 = split + (int)std::max<int64_t>(1, std::min<int64_t>(gb, (ntiles + 7) / 8));
        g2 = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
    }
    if (g2 > w.max_blocks) return set_error(GP_ERR_INVALID, "internal: partials too small");
    a.nprev = g2;
    a.split_blocks = split;

    const int ib = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
    const bool fp64 = push && g->opt.push_fp64_accum;
    if (fp64 && !w.acc64) GP_TRY(w.mem.alloc(w.acc64, (size_t)n, s));
    a.acc64 = fp64 ? w.acc64 : nullptr;
    GP_LAUNCH("pr_init", s, (k_pr_init<<<ib, 256, 0, s>>>(n, X0, g->inv_deg, R[0], C[0], (push && !fp64) ? R[1] : nullptr,
                                                          a.acc64, S,
                                                          a.one_minus_d, a.base_uniform, status)));
    GP_TRY(check_launch("pr_init"));
    auto enqueue_hot_gather = [&](const float *c_src) -> int {
        const int hb = (int)std::max<int64_t>(1, std::min<int64_t>((g->pull_hot.nhot + 255) / 256, 4096));
        GP_LAUNCH("hot_gather", s, (k_hot_gather<<<hb, 256, 0, s>>>(g->pull_hot.hot_id, g->pull_hot.nhot, c_src,
                                                                    g->pull_hot.c_hot)));
        return check_launch("hot_gather");
    };
    if (hot) GP_TRY(enqueue_hot_gather(C[0]));

    auto enqueue_sweep = [&](int k) -> int {
        PrArgs b = a;
        b.k = k;
        b.x = R[(k - 1) & 1];
        b.y = R[k & 1];
        if (!push) {
            b.c = C[(k - 1) & 1];
            b.c_next = C[k & 1];
            if (W && hot) {
                GP_LAUNCH("pull_big", s, (k_pull_big<true, true><<<g1, tbp, smem, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<true, true><<<g2, tbl, smem, s>>>(b)));
            } else if (W) {
                GP_LAUNCH("pull_big", s, (k_pull_big<true, false><<<g1, tbp, 0, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<true, false><<<g2, tbl, 0, s>>>(b)));
            } else if (hot) {
                GP_LAUNCH("pull_big", s, (k_pull_big<false, true><<<g1, tbp, smem, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<false, true><<<g2, tbl, smem, s>>>(b)));
            } else {
                GP_LAUNCH("pull_big", s, (k_pull_big<false, false><<<g1, tbp, 0, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<false, false><<<g2, tbl, 0, s>>>(b)));
            }
            if (hot) GP_TRY(enqueue_hot_gather(b.c_next));
        } else {
            b.c = C[0];
            b.c_next = C[0];
            if (fp64) {
                if (W)
                    GP_LAUNCH("push_scatter", s, (k_push_scatter<true, double><<<g1, 256, 0, s>>>(b)));
                else
                    GP_LAUNCH("push_scatter", s, (k_push_scatter<false, double><<<g1, 256, 0, s>>>(b)));
                GP_LAUNCH("push_epilogue", s, (k_push_epilogue<double><<<g2, 256, 0, s>>>(b)));
            } else {
                if (W)
                    GP_LAUNCH("push_scatter", s, (k_push_scatter<true, float><<<g1, 256, 0, s>>>(b)));
                else
                    GP_LAUNCH("push_scatter", s, (k_push_scatter<false, float><<<g1, 256, 0, s>>>(b)));
                GP_LAUNCH("push_epilogue", s, (k_push_epilogue<float><<<g2, 256, 0, s>>>(b)));
            }
        }
        return check_launch("pagerank sweep");
    };
    auto enqueue_finish = [&](int k_next, int slot) -> int {
        PrArgs b = a;
        b.k = k_next;
        GP_LAUNCH("pr_finish", s, (k_pr_finish<<<1, 256, 0, s>>>(b)));
        GP_TRY(check_launch("pr_finish"));
        GP_CUDA(cudaMemcpyAsync((PrStatus *)w.status_host + slot, status, sizeof(PrStatus), cudaMemcpyDeviceToHost, s));
        return GP_OK;
    };

    const int poll = std::max(1, g->opt.poll_interval);
    int issued = 0;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    GP_CUDA(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
    GP_CUDA(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
    int pending[2] = {-1, -1};  // batch ids waiting on each slot
    int batch = 0, oldest = 0;
    bool stop = false;
    int st = GP_OK;
    if (tol <= 0.0) {
        for (int k = 1; k <= iters && st == GP_OK; ++k) st = enqueue_sweep(k);
        if (st == GP_OK) st = enqueue_finish(iters + 1, 0);
        issued = iters;
    } else {
        while (st == GP_OK) {
            const int slot = batch & 1;
            if (!stop && issued < iters && pending[slot] < 0) {
                const int kb = std::min(poll, iters - issued);
                for (int i = 0; i < kb && st == GP_OK; ++i) st = enqueue_sweep(++issued);
                if (st == GP_OK) st = enqueue_finish(issued + 1, slot);
                if (st == GP_OK) {
                    cudaError_t e = cudaEventRecord(evs[slot], s);
                    if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "event: %s", cudaGetErrorString(e));
                }
                pending[slot] = batch++;
                continue;
            }
            const int os = oldest & 1;
            if (pending[os] < 0) break;  // nothing outstanding
            cudaError_t e = cudaEventSynchronize(evs[os]);
            if (e != cudaSuccess) {
                st = set_error(GP_ERR_CUDA, "pagerank poll: %s", cudaGetErrorString(e));
                break;
            }
            pending[os] = -1;
            ++oldest;
            if (((PrStatus *)w.status_host)[os].done) stop = true;
            if (stop && pending[oldest & 1] < 0) break;
            if (!stop && issued >= iters && pending[oldest & 1] < 0) break;
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaEventDestroy(evs[0]);
    cudaEventDestroy(evs[1]);
    if (st != GP_OK) return st;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_pagerank: %s", cudaGetErrorString(e));
    // authoritative final status
    PrStatus fin;
    GP_CUDA(cudaMemcpy(&fin, status, sizeof(PrStatus), cudaMemcpyDeviceToHost));
    const int kdone = fin.iters_done;
    if ((kdone & 1) && kdone > 0)
        GP_CUDA(cudaMemcpyAsync(R0, R[1], n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (!out_dev) GP_CUDA(cudaMemcpyAsync(ranks_out, R0, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (stats) {
        GP_CUDA(cudaEventRecord(ev1, s));
        GP_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->iters_done = kdone;
        stats->mode_used = mode;
        stats->residual = fin.residual;
        stats->ms = ms;
        stats->converged = (tol <= 0.0) ? 1 : fin.converged;
    } else if (!out_dev) {
        GP_CUDA(cudaStreamSynchronize(s));
    }
    if (tol > 0.0 && !fin.converged)
        return set_error(GP_ERR_NOT_CONVERGED, "residual %.3e >= tol %.3e after %d sweeps", fin.residual, tol, kdone);
    return GP_OK;
}
