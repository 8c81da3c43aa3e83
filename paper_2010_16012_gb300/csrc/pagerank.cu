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
//                    consecutive vertices; each lane sums its own light
//                    vertex's in-list with 8 loads in flight (no shuffles: the
//                    kernel is issue-bound, and light lists are short).  Blocks
//                    after that: one thread per big vertex adds its chunk
//                    slots.  Every vertex's y, c' = y*inv_deg and |y - x| are
//                    written by its owner.
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
    // push scatter, summed over the sweeps of a call: updates sent to L2 as
    // atomics, added into a block's shared-memory accumulators, and folded into
    // another lane's update inside a warp; plus the flushes of the shared ones
    unsigned long long upd_l2, upd_shared, upd_merged, flush_l2;
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
    const float *s;  // teleport vector (forward) or dL/dx (adjoint), or nullptr
    float s_scale;       // factor of s in the base term: 1-d (forward), 1 (adjoint)
    float base_uniform;  // base term when s is nullptr: (1-d)/n
    const float *post_scale;  // factor of the gathered sum per owner (adjoint: inv_deg), or nullptr
    const float *cmul;        // c_next = y * cmul (forward: inv_deg), or nullptr (c_next = y)
    float one_minus_d, d;
    double tol;
    int32_t k;  // sweep number, 1-based
    int32_t nprev;
    double *partials;
    float *chunk_part;
    double *acc64;  // FP64 push accumulator (or nullptr)
    const float *c_hot;  // hot contributions (pull, HOT kernels)
    const int32_t *hot_id;  // hot vertices (push HOT kernels)
    int64_t nhot;
    PrStatus *status;
    int32_t split_blocks;  // pull: light-tile blocks; push: big-chunk blocks
};

__device__ __forceinline__ float base_term(const PrArgs &a, int64_t v) {
    return a.s ? a.s_scale * a.s[v] : a.base_uniform;
}
__device__ __forceinline__ float post_factor(const PrArgs &a, int64_t v) { return a.post_scale ? a.post_scale[v] : 1.f; }
__device__ __forceinline__ float c_factor(const PrArgs &a, int64_t v) { return a.cmul ? a.cmul[v] : 1.f; }

// Whether the iteration has stopped, read by one thread per block: every warp
// loading the flag itself would queue thousands of requests on the one L2 line
// that holds it at each launch.  Called by all threads of the block.
__device__ __forceinline__ bool pr_stopped(const PrStatus *status) {
    __shared__ int stop;
    if (threadIdx.x == 0) stop = ((volatile const PrStatus *)status)->done;
    __syncthreads();
    return stop != 0;
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

// x = x0 (or 1/n), c = x * cmul, and the push accumulators zeroed.
__global__ void k_pr_init(int64_t n, const float *x0, const float *cmul, float *r0, float *c, float *r_push,
                          double *acc64, PrStatus *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float x_uniform = 1.0f / (float)n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const float x = x0 ? x0[v] : x_uniform;
        r0[v] = x;
        c[v] = cmul ? x * cmul[v] : x;
        if (r_push) r_push[v] = 0.f;
        if (acc64) acc64[v] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status->done = 0;
        status->iters_done = 0;
        status->residual = 0.0;
        status->converged = 0;
        status->upd_l2 = status->upd_shared = status->upd_merged = status->flush_l2 = 0;
    }
}

// Records the decision for the last sweep enqueued (sweep k-1) without doing a
// sweep, and writes the status into the host's mapped mirror slot: the host
// polls it with no copy, so polling never waits behind other transfers.
__global__ void k_pr_finish(PrArgs a, PrStatus *mirror) {
    pr_gate(a, a.k);
    if (threadIdx.x == 0) {
        *mirror = *a.status;  // the gate ended with a block barrier
        __threadfence_system();
    }
}

// dst = src over n floats (the result's move into the caller's buffer, kept
// off the copy engines for the same reason).
__global__ void k_copy_f32(int64_t n, const float *__restrict__ src, float *__restrict__ dst) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

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

// The same gather with the hot contributions read from their compact global
// copy (pull_light: its few hot gathers do not pay for a shared-memory copy,
// whose size would also cut the light kernel's resident blocks).
template <bool HOT>
__device__ __forceinline__ float gather_c_glob(const float *__restrict__ c, const float *__restrict__ c_hot, int32_t u) {
    if (HOT && u < 0) return __ldg(c_hot + (u & 0x7fffffff));
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

#ifndef GP_LIGHT_MIN_BLOCKS
#define GP_LIGHT_MIN_BLOCKS 3
#endif
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

constexpr int LIGHT_UNROLL = 8;  // in-edges of a light vertex in flight per lane

template <bool W, bool HOT>
__global__ void __launch_bounds__(512, GP_LIGHT_MIN_BLOCKS) k_pull_light(PrArgs a) {
    __shared__ double sm[32];
    if (pr_stopped(a.status)) return;
    const int lane = lane_id();
    ResSum res;
    const int64_t n = a.n;
    if ((int)blockIdx.x < a.split_blocks) {
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
            float xv = 0.f, cm = 0.f, ps = 0.f, base_v = 0.f;
            if (v < n) {
                xv = a.x[v];
                cm = c_factor(a, v);
                ps = post_factor(a, v);
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
            // a light vertex's own lane sums its in-list, LIGHT_UNROLL loads in flight
            const int64_t e1 = big ? b : e;
            float acc = 0.f;
            for (int64_t p0 = b; p0 < e1; p0 += LIGHT_UNROLL) {
                int32_t u[LIGHT_UNROLL];
                float f[LIGHT_UNROLL];
#pragma unroll
                for (int q = 0; q < LIGHT_UNROLL; ++q) u[q] = p0 + q < e1 ? ld_idx(idx + p0 + q) : 0;
#pragma unroll
                for (int q = 0; q < LIGHT_UNROLL; ++q) {
                    f[q] = 0.f;
                    if (p0 + q < e1) {
                        f[q] = gather_c_glob<HOT>(c, a.c_hot, u[q]);
                        if (W) f[q] *= __ldg(wv + p0 + q);
                    }
                }
#pragma unroll
                for (int q = 0; q < LIGHT_UNROLL; ++q) acc += f[q];
            }
            if (v < n && !big) {
                const float y = base_v + a.d * (ps * acc);
                res.add(y, xv);
                a.y[v] = y;
                a.c_next[v] = y * cm;
            }
        }
    } else {
        const int64_t nth = (int64_t)(gridDim.x - a.split_blocks) * blockDim.x;
        for (int64_t r = (int64_t)(blockIdx.x - a.split_blocks) * blockDim.x + threadIdx.x; r < a.nbig; r += nth) {
            const int32_t v = a.big[r];
            float acc = 0.f;
            for (int64_t j = a.cstart[r]; j < a.cstart[r + 1]; ++j) acc += a.chunk_part[j];
            const float y = base_term(a, v) + a.d * (post_factor(a, v) * acc);
            res.add(y, a.x[v]);
            a.y[v] = y;
            a.c_next[v] = y * c_factor(a, v);
        }
    }
    const double r = block_residual(res, sm);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = r;
}

// c_hot[slot] = c[hot_id[slot]] for the sweep that reads c next (none once
// the iteration has stopped: the launches enqueued past that point return).
__global__ void k_hot_gather(const int32_t *hot_id, int64_t nhot, const float *c, float *c_hot, const PrStatus *status) {
    if (status && pr_stopped(status)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nhot; i += stride) c_hot[i] = c[hot_id[i]];
}

// ------------------------------------------------------------------ push

// Accumulator of the scattered updates: FP32 (the paper's float atomics) or
// FP64 (same atomic count; the order-dependent rounding of FP32 atomics at hubs
// otherwise leaves an L1 residual floor above 1e-7 on graphs with 4M vertices).
// HOT: the partition-awareness of the paper's Section 5 recast for a GPU block --
// updates to the H most updated vertices (encoded in the index array) are
// summed in the block's shared memory with shared-memory atomics and flushed
// once per block; only the other updates use global atomics.
struct PushCount {
    unsigned l2 = 0, shared = 0, merged = 0, flush = 0;
};

template <class T, bool HOT>
__device__ __forceinline__ void scatter_add(T *y, float *sh, int32_t dst, float val, PushCount &cnt) {
    if (HOT && dst < 0) {
        atomicAdd(sh + (dst & 0x7fffffff), val);
        ++cnt.shared;
    } else {
        atomicAdd(y + dst, (T)val);
        ++cnt.l2;
    }
}

template <bool W, class T, bool HOT>
__global__ void __launch_bounds__(1024) k_push_scatter(PrArgs a) {
    extern __shared__ float sh_acc[];
    if (pr_gate(a, a.k)) return;
    if (HOT) {
        for (int64_t i = threadIdx.x; i < a.nhot; i += blockDim.x) sh_acc[i] = 0.f;
        __syncthreads();
    }
    const int lane = lane_id();
    const int32_t *__restrict__ idx = a.idx;
    const float *__restrict__ wv = a.w;
    T *y = sizeof(T) == 8 ? (T *)a.acc64 : (T *)a.y;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    PushCount cnt;
    // big sources: one warp per chunk of out-edges
    for (int64_t j = warp; j < a.nchunks; j += nwarps) {
        const Chunk ch = a.chunks[j];
        const float cu = a.d * __ldg(a.c + ch.v);
        const int32_t *ip = idx + ch.beg;
        const float *wp = W ? wv + ch.beg : nullptr;
        int i = lane;
        for (; i + 96 < ch.len; i += 128) {
            const int v0 = __ldg(ip + i), v1 = __ldg(ip + i + 32), v2 = __ldg(ip + i + 64), v3 = __ldg(ip + i + 96);
            scatter_add<T, HOT>(y, sh_acc, v0, W ? cu * __ldg(wp + i) : cu, cnt);
            scatter_add<T, HOT>(y, sh_acc, v1, W ? cu * __ldg(wp + i + 32) : cu, cnt);
            scatter_add<T, HOT>(y, sh_acc, v2, W ? cu * __ldg(wp + i + 64) : cu, cnt);
            scatter_add<T, HOT>(y, sh_acc, v3, W ? cu * __ldg(wp + i + 96) : cu, cnt);
        }
        for (; i < ch.len; i += 32) scatter_add<T, HOT>(y, sh_acc, __ldg(ip + i), W ? cu * __ldg(wp + i) : cu, cnt);
    }
    // light sources: 32 consecutive sources per warp, one merged edge stream
    __shared__ float agg[1024];
    const int64_t n = a.n;
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
            // idle lanes get keys no real edge has: positive and >= n is impossible for
            // plain vertices, and HOT keys are negative
            int32_t dst = (int32_t)(0x7fffffff - lane);
            float val = 0.f;
            if (eid < E) {
                const int64_t pos = kb + (eid - kex);
                dst = __ldg(idx + pos);
                val = W ? ck * __ldg(wv + pos) : ck;
            }
            // Updates from different sources of the tile that hit the same vertex
            // (typically a hub) are summed in the warp first, so the vertex takes one
            // atomic per window instead of one per edge.
            const unsigned peers = __match_any_sync(FULL, dst);
            if (__all_sync(FULL, peers == (1u << lane))) {
                if (eid < E) scatter_add<T, HOT>(y, sh_acc, dst, val, cnt);
            } else {
                agg[threadIdx.x] = val;
                __syncwarp();
                if (eid < E && (peers & ((1u << lane) - 1u)) == 0) {  // lowest lane of its group
                    float sum = val;
                    for (unsigned rest = peers & ~(1u << lane); rest; rest &= rest - 1)
                        sum += agg[(threadIdx.x & ~31u) + (__ffs(rest) - 1)];
                    scatter_add<T, HOT>(y, sh_acc, dst, sum, cnt);
                    cnt.merged += __popc(peers) - 1;
                }
                __syncwarp();
            }
        }
    }
    if (HOT) {  // flush: one global atomic per touched hot vertex per block
        __syncthreads();
        for (int64_t i = threadIdx.x; i < a.nhot; i += blockDim.x) {
            const float v = sh_acc[i];
            if (v != 0.f) {
                atomicAdd(y + a.hot_id[i], (T)v);
                ++cnt.flush;
            }
        }
    }
    // the block's update counts, one reduction and four atomics per block
    __shared__ unsigned long long csum[4][32];
    unsigned long long c4[4] = {cnt.l2, cnt.shared, cnt.merged, cnt.flush};
#pragma unroll
    for (int i = 0; i < 4; ++i) c4[i] = warp_sum(c4[i]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) csum[i][threadIdx.x >> 5] = c4[i];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i) c4[i] = warp_sum(threadIdx.x < (blockDim.x >> 5) ? csum[i][threadIdx.x] : 0ull);
        if (threadIdx.x == 0) {
            if (c4[0]) atomicAdd(&a.status->upd_l2, c4[0]);
            if (c4[1]) atomicAdd(&a.status->upd_shared, c4[1]);
            if (c4[2]) atomicAdd(&a.status->upd_merged, c4[2]);
            if (c4[3]) atomicAdd(&a.status->flush_l2, c4[3]);
        }
    }
}

// Per vertex: y = base + post_scale * (scattered sum), rounded to the FP32 rank;
// the residual, the next contribution, and the zeroing of the buffer the next
// sweep accumulates into.
template <class T>
__global__ void __launch_bounds__(256) k_push_epilogue(PrArgs a) {
    __shared__ double sm[32];
    if (pr_stopped(a.status)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    ResSum res;
    float *x_reset = const_cast<float *>(a.x);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += stride) {
        const float base = base_term(a, v), ps = post_factor(a, v);
        float y;
        if (sizeof(T) == 8) {
            // the FP64 sum rounded once to FP32, then the FP32 epilogue
            y = fmaf(ps, f64_to_f32_rn(a.acc64[v]), base);
            a.acc64[v] = 0.0;
        } else {
            y = base + ps * a.y[v];
        }
        res.add(y, a.x[v]);
        a.y[v] = y;
        a.c_next[v] = y * c_factor(a, v);
        if (sizeof(T) != 8) x_reset[v] = 0.f;  // the next sweep accumulates into this buffer
    }
    const double r = block_residual(res, sm);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = r;
}

// ------------------------------------------------------------------ adjoint gradients

// grad_s[v] = (1-d) lambda_v
__global__ void k_grad_s(int64_t n, float one_minus_d, const float *lam, float *grad_s) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) grad_s[v] = one_minus_d * lam[v];
}

struct GradArgs {
    int64_t n;
    const int64_t *off;  // CSR
    const int32_t *idx;
    const float *x, *lam, *g, *inv_deg;
    const Chunk *chunks;
    int64_t nchunks;
    int32_t light_max;
    float d;
    int normalized;
    float *grad_w;
    int32_t split_blocks;
};

// dL/dP_vu = d lambda_v x_u for the CSR edge e = (u -> v); with per-source
// normalisation P_vu = w_uv / S_u the raw-weight gradient is
// (x_u / S_u) (d lambda_v - lambda_u + g_u), using lambda_u = g_u + d (P^T lambda)_u.
__device__ __forceinline__ float edge_grad(const GradArgs &a, int32_t u, int32_t v, float xu_or_coef, float lam_u_term) {
    return a.normalized ? xu_or_coef * (a.d * a.lam[v] - lam_u_term) : a.d * a.lam[v] * xu_or_coef;
}

__global__ void __launch_bounds__(256) k_grad_w(GradArgs a) {
    const int lane = lane_id();
    if ((int)blockIdx.x < a.split_blocks) {
        const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)a.split_blocks * blockDim.x) >> 5;
        for (int64_t j = warp; j < a.nchunks; j += nwarps) {
            const Chunk ch = a.chunks[j];
            const int32_t u = ch.v;
            const float coef = a.normalized ? a.x[u] * a.inv_deg[u] : a.x[u];
            const float lt = a.normalized ? a.lam[u] - a.g[u] : 0.f;
            for (int i = lane; i < ch.len; i += 32) {
                const int64_t pos = ch.beg + i;
                a.grad_w[pos] = edge_grad(a, u, a.idx[pos], coef, lt);
            }
        }
    } else {
        const int64_t warp = ((int64_t)(blockIdx.x - a.split_blocks) * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)(gridDim.x - a.split_blocks) * blockDim.x) >> 5;
        const int64_t ntiles = (a.n + 31) >> 5;
        for (int64_t t = warp; t < ntiles; t += nwarps) {
            const int64_t u = t * 32 + lane;
            int64_t b = 0, e = 0;
            float coef = 0.f, lt = 0.f;
            if (u < a.n) {
                b = a.off[u];
                e = a.off[u + 1];
                coef = a.normalized ? a.x[u] * a.inv_deg[u] : a.x[u];
                lt = a.normalized ? a.lam[u] - a.g[u] : 0.f;
            }
            const int64_t dd = e - b;
            const int deg = dd > a.light_max ? 0 : (int)dd;
            const int incl = warp_incl_scan(deg);
            const int excl = incl - deg;
            const int E = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < E; base += 32) {
                const int eid = base + lane;
                const int k = tile_owner(excl, eid);
                const int64_t kb = __shfl_sync(FULL, b, k);
                const int kex = __shfl_sync(FULL, excl, k);
                const float kc = __shfl_sync(FULL, coef, k);
                const float kl = __shfl_sync(FULL, lt, k);
                const int32_t ku = (int32_t)(t * 32 + k);
                if (eid < E) {
                    const int64_t pos = kb + (eid - kex);
                    a.grad_w[pos] = edge_grad(a, ku, a.idx[pos], kc, kl);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ driver

void release_pr_work(gp_graph *g, cudaStream_t s) {
    pinned_free(g->pr.status_host, 4 * sizeof(PrStatus));
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
    const int64_t nbig = std::max(g->pull_bins.nbig, g->push_bins.nbig);
    const int64_t epi = (nbig + 255) / 256;
    // covers any grid: at most 32 resident blocks per SM, plus the epilogue blocks
    w.max_blocks = (int)(std::max(g->num_sms * 32, grid_blocks(g, 256)) + epi + 64);
    GP_TRY(w.mem.alloc(w.r1, n, s));
    GP_TRY(w.mem.alloc(w.c0, n, s));
    GP_TRY(w.mem.alloc(w.c1, n, s));
    GP_TRY(w.mem.alloc(w.partials, (size_t)w.max_blocks, s));
    GP_TRY(w.mem.alloc(w.chunk_part, (size_t)std::max<int64_t>(std::max(g->pull_bins.nchunks, g->push_bins.nchunks), 1), s));
    PrStatus *st = nullptr;
    GP_TRY(w.mem.alloc(st, 1, s));
    w.status = st;
    GP_TRY(pinned_alloc(&w.status_host, 4 * sizeof(PrStatus)));
    GP_TRY(pinned_device_ptr(w.status_host, &w.status_mirror));
    w.ready = true;
    return GP_OK;
}

static int ensure_vec(gp_graph *g, float *&slot, cudaStream_t s) {
    if (slot) return GP_OK;
    return g->pr.mem.alloc(slot, (size_t)std::max<int64_t>(g->n, 1), s);
}

static const void *push_kernel(bool W, bool fp64, bool hot) {
    if (fp64) {
        if (W) return hot ? (const void *)k_push_scatter<true, double, true> : (const void *)k_push_scatter<true, double, false>;
        return hot ? (const void *)k_push_scatter<false, double, true> : (const void *)k_push_scatter<false, double, false>;
    }
    if (W) return hot ? (const void *)k_push_scatter<true, float, true> : (const void *)k_push_scatter<true, float, false>;
    return hot ? (const void *)k_push_scatter<false, float, true> : (const void *)k_push_scatter<false, float, false>;
}

// Width of the push accumulator.  FP64 sums make the scattered result independent
// of the atomic order up to one final rounding, and cost no throughput while the
// 8n-byte accumulator stays in L2; above half the L2 its reductions reach DRAM
// (Erdos-Renyi 2^24: 4.7 ms per scatter against 2.5 ms in FP32), so the default
// (-1) switches to FP32 there unless some vertex takes more than
// PUSH_FP32_MAX_UPDATES updates per sweep (FP32 order noise at such hubs sets a
// residual floor near 1e-7).
constexpr int64_t PUSH_FP32_MAX_UPDATES = 4096;
static bool push_fp64(const gp_graph *g, int64_t max_updates) {
    if (g->opt.push_fp64_accum >= 0) return g->opt.push_fp64_accum != 0;
    const bool fits = 8 * g->n <= g->l2_bytes / 2;
    return fits || max_updates > PUSH_FP32_MAX_UPDATES;
}

// One power iteration y = base + d * post_scale * (gather or scatter over the
// given adjacency) of a PageRank-type linear system, with on-device
// convergence; used for the forward pass and for the adjoint.
struct IterSpec {
    bool push;        // scatter with atomics (else gather, owner-only writes)
    bool hot;         // use the pull hot-contribution cache (forward pull only)
    const int64_t *off;
    const int32_t *idx;
    const float *w;
    const BigBins *bins;
    const float *s;   // base vector (nullable: uniform base_uniform)
    float s_scale, base_uniform, d;
    const float *x0;  // start vector (nullable: 1/n)
    const float *post_scale, *cmul;
    int iters;
    double tol;
    int64_t max_updates;  // push: most updates any vertex takes per sweep (its max in-degree)
};

static int pr_iterate(gp_graph *g, const IterSpec &sp, float *out, PrStatus &fin, cudaStream_t s) {
    const int64_t n = g->n;
    PrWork &w = g->pr;
    float *R[2] = {out, w.r1};
    float *C[2] = {w.c0, w.c1};
    PrStatus *status = (PrStatus *)w.status;
    const bool push = sp.push;
    const bool W = sp.w != nullptr;
    const BigBins &bins = *sp.bins;

    PrArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.off = sp.off;
    a.idx = sp.idx;
    a.w = sp.w;
    a.big = bins.big;
    a.cstart = bins.cstart;
    a.chunks = bins.chunks;
    a.nbig = bins.nbig;
    a.nchunks = bins.nchunks;
    a.light_max = bins.light_max;
    a.s = sp.s;
    a.s_scale = sp.s_scale;
    a.base_uniform = sp.base_uniform;
    a.post_scale = sp.post_scale;
    a.cmul = sp.cmul;
    a.one_minus_d = 1.0f - sp.d;
    a.d = sp.d;
    a.tol = sp.tol;
    a.partials = w.partials;
    a.chunk_part = w.chunk_part;
    a.status = status;

    const int gb = grid_blocks(g, 256);
    const int64_t ntiles = (n + 31) / 32;
    bool hot = false;
    int tbp = 256, tbl = 256;  // threads per block of pull_big / pull_light
    size_t smem = 0;
    if (!push && sp.hot) {
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
    if (!push && !hot) {
        tbp = 1024;
        tbl = 512;
    }
    if (push && sp.hot) {
        if (g->push_hot.slots != g->opt.push_hot_slots) GP_TRY(build_push_hot(g, g->opt.push_hot_slots, s));
        hot = g->push_hot.nhot > 0;
        if (hot) {
            smem = (size_t)g->push_hot.nhot * sizeof(float);
            a.hot_id = g->push_hot.hot_id;
            a.nhot = g->push_hot.nhot;
            a.idx = g->push_hot.enc_idx;
        }
    }
    int g1, g2, split;
    if (!push) {
        int ob = 0, ol = 0;
        const void *kb_ = W ? (hot ? (const void *)k_pull_big<true, true> : (const void *)k_pull_big<true, false>)
                            : (hot ? (const void *)k_pull_big<false, true> : (const void *)k_pull_big<false, false>);
        const void *kl_ = W ? (hot ? (const void *)k_pull_light<true, true> : (const void *)k_pull_light<true, false>)
                            : (hot ? (const void *)k_pull_light<false, true> : (const void *)k_pull_light<false, false>);
        GP_TRY(occupancy(kb_, tbp, smem, ob));
        GP_TRY(occupancy(kl_, tbl, 0, ol));
        const int wpb = tbp / 32, wpl = tbl / 32;
        g1 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ob * g->num_sms, (bins.nchunks + wpb - 1) / wpb));
        split = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ol * g->num_sms, (ntiles + wpl - 1) / wpl));
        g2 = split + (int)((bins.nbig + tbl - 1) / tbl);
    } else {
        // one grid for big chunks and light tiles; as many resident blocks as fit,
        // capped by blocks_per_sm (256-thread units)
        const void *ks = push_kernel(W, push_fp64(g, sp.max_updates), hot);
        int os = 0;
        GP_TRY(occupancy(ks, 1024, smem, os));
        const int cap = std::max(1, g->opt.blocks_per_sm / 4) * g->num_sms;
        const int64_t work = std::max<int64_t>((bins.nchunks + 31) / 32, (ntiles + 31) / 32);
        split = 0;
        g1 = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>((int64_t)os * g->num_sms, cap), work));
        g2 = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
    }
    if (g2 > w.max_blocks) return set_error(GP_ERR_INVALID, "internal: partials too small");
    a.nprev = g2;
    a.split_blocks = split;

    const int ib = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
    const bool fp64 = push && push_fp64(g, sp.max_updates);
    if (fp64 && !w.acc64) GP_TRY(w.mem.alloc(w.acc64, (size_t)n, s));
    a.acc64 = fp64 ? w.acc64 : nullptr;
    GP_LAUNCH("pr_init", s, (k_pr_init<<<ib, 256, 0, s>>>(n, sp.x0, sp.cmul, R[0], C[0], (push && !fp64) ? R[1] : nullptr,
                                                          a.acc64, status)));
    GP_TRY(check_launch("pr_init"));
    auto enqueue_hot_gather = [&](const float *c_src) -> int {
        const int hb = (int)std::max<int64_t>(1, std::min<int64_t>((g->pull_hot.nhot + 255) / 256, 4096));
        GP_LAUNCH("hot_gather", s, (k_hot_gather<<<hb, 256, 0, s>>>(g->pull_hot.hot_id, g->pull_hot.nhot, c_src,
                                                                    g->pull_hot.c_hot, status)));
        return check_launch("hot_gather");
    };
    if (hot && !push) GP_TRY(enqueue_hot_gather(C[0]));

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
                GP_LAUNCH("pull_light", s, (k_pull_light<true, true><<<g2, tbl, 0, s>>>(b)));
            } else if (W) {
                GP_LAUNCH("pull_big", s, (k_pull_big<true, false><<<g1, tbp, 0, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<true, false><<<g2, tbl, 0, s>>>(b)));
            } else if (hot) {
                GP_LAUNCH("pull_big", s, (k_pull_big<false, true><<<g1, tbp, smem, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<false, true><<<g2, tbl, 0, s>>>(b)));
            } else {
                GP_LAUNCH("pull_big", s, (k_pull_big<false, false><<<g1, tbp, 0, s>>>(b)));
                GP_LAUNCH("pull_light", s, (k_pull_light<false, false><<<g2, tbl, 0, s>>>(b)));
            }
            if (hot) GP_TRY(enqueue_hot_gather(b.c_next));
        } else {
            b.c = C[0];
            b.c_next = C[0];
            const void *ks = push_kernel(W, fp64, hot);
            {
                ProfScope ps("push_scatter", s);
                void *args[] = {&b};
                GP_CUDA(cudaLaunchKernel(ks, dim3((unsigned)g1), dim3(1024), args, smem, s));
            }
            if (fp64)
                GP_LAUNCH("push_epilogue", s, (k_push_epilogue<double><<<g2, 256, 0, s>>>(b)));
            else
                GP_LAUNCH("push_epilogue", s, (k_push_epilogue<float><<<g2, 256, 0, s>>>(b)));
        }
        return check_launch("pagerank sweep");
    };
    auto enqueue_finish = [&](int k_next, int slot) -> int {
        PrArgs b = a;
        b.k = k_next;
        GP_LAUNCH("pr_finish", s, (k_pr_finish<<<1, 256, 0, s>>>(b, (PrStatus *)w.status_mirror + slot)));
        return check_launch("pr_finish");
    };

    const int poll = std::max(1, g->opt.poll_interval);
    const int iters = sp.iters;
    int issued = 0;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    GP_CUDA(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
    GP_CUDA(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
    int pending[2] = {-1, -1};  // batch ids waiting on each slot
    int batch = 0, oldest = 0;
    bool stop = false;
    int st = GP_OK;
    if (sp.tol <= 0.0) {
        for (int k = 1; k <= iters && st == GP_OK; ++k) st = enqueue_sweep(k);
        if (st == GP_OK) st = enqueue_finish(iters + 1, 0);
        issued = iters;
    } else {
        // Sweeps worth enqueuing: the cap, lowered once two polls give the
        // residual's rate of decrease to the predicted stopping sweep plus one
        // (sweeps enqueued past the stop only return at once, but each still costs
        // a few microseconds of launches per kernel); raised again a batch at a
        // time if the iteration outlives the prediction.
        int limit = iters;
        int k_last = 0;
        double r_last = 0.0;
        while (st == GP_OK) {
            const int slot = batch & 1;
            if (!stop && issued < limit && pending[slot] < 0) {
                const int kb = std::min(poll, limit - issued);
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
            if (pending[os] < 0) {  // nothing outstanding
                if (!stop && issued < iters) {
                    limit = std::min(iters, issued + poll);
                    continue;
                }
                break;
            }
            cudaError_t e = cudaEventSynchronize(evs[os]);
            if (e != cudaSuccess) {
                st = set_error(GP_ERR_CUDA, "pagerank poll: %s", cudaGetErrorString(e));
                break;
            }
            pending[os] = -1;
            ++oldest;
            const PrStatus ps = ((const PrStatus *)w.status_host)[os];
            if (ps.done) {
                stop = true;
            } else {
                if (k_last > 0 && ps.iters_done > k_last && ps.residual > 0.0 && ps.residual < r_last) {
                    const double rate = std::pow(ps.residual / r_last, 1.0 / (ps.iters_done - k_last));
                    const double more = std::ceil(std::log(sp.tol / ps.residual) / std::log(rate));
                    if (more >= 0.0 && more < (double)iters)
                        limit = std::max<int64_t>(issued, std::min<int64_t>(iters, (int64_t)ps.iters_done + (int64_t)more + 1));
                }
                k_last = ps.iters_done;
                r_last = ps.residual;
            }
            if (stop && pending[oldest & 1] < 0) break;
            if (!stop && issued >= iters && pending[oldest & 1] < 0) break;
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaEventDestroy(evs[0]);
    cudaEventDestroy(evs[1]);
    if (st != GP_OK) return st;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "pagerank iteration: %s", cudaGetErrorString(e));
    // the final status: one more gate-only launch (the iteration has stopped,
    // so it changes nothing) writes it into mirror slot 2
    {
        PrArgs b = a;
        b.k = issued + 1;
        GP_LAUNCH("pr_finish", s, (k_pr_finish<<<1, 256, 0, s>>>(b, (PrStatus *)w.status_mirror + 2)));
        GP_TRY(check_launch("pr_finish"));
    }
    GP_CUDA(cudaStreamSynchronize(s));
    memcpy(&fin, (const PrStatus *)w.status_host + 2, sizeof(fin));  // written by the kernel, complete after the sync
    if ((fin.iters_done & 1) && fin.iters_done > 0) {
        const int cb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * (int64_t)g->num_sms));
        GP_LAUNCH("copy_result", s, (k_copy_f32<<<cb, 256, 0, s>>>(n, R[1], out)));
        GP_TRY(check_launch("copy_result"));
    }
    return GP_OK;
}

// Device pointer for a caller array of n floats that may live in host memory.
static int device_input(gp_graph *g, const float *p, float *&slot, const float *&dev, cudaStream_t s) {
    dev = p;
    if (p && !is_device_ptr(p)) {
        GP_TRY(ensure_vec(g, slot, s));
        GP_CUDA(cudaMemcpyAsync(slot, p, g->n * sizeof(float), cudaMemcpyHostToDevice, s));
        dev = slot;
    }
    return GP_OK;
}

static int pr_validate(const gp_graph *g, int mode, float damping, int iters, double tol) {
    if (!g) return set_error(GP_ERR_INVALID, "graph is NULL");
    if (!(damping > 0.f && damping < 1.f)) return set_error(GP_ERR_INVALID, "damping %g outside (0, 1)", (double)damping);
    if (iters < 1) return set_error(GP_ERR_INVALID, "iters = %d < 1", iters);
    if (!(tol >= 0.0)) return set_error(GP_ERR_INVALID, "tol must be >= 0");
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "bad mode %d", mode);
    return GP_OK;
}

__global__ void k_recompute_inv(const int64_t *csr_off, const float *csr_w, int64_t n, int normalize, float *inv_deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t b = csr_off[u], e = csr_off[u + 1];
        float inv = 0.f;
        if (e > b) {
            if (normalize) {
                double sw = 0.0;
                for (int64_t j = b; j < e; ++j) sw += (double)csr_w[j];
                inv = sw > 0.0 ? (float)(1.0 / sw) : 0.f;
            } else {
                inv = 1.f;
            }
        }
        inv_deg[u] = inv;
    }
}

}  // namespace gp

using namespace gp;

extern "C" int gp_pagerank(const gp_graph *gc, int mode, float damping, int iters, double tol,
                           const float *personalization, const float *x0, float *ranks_out, gp_pr_stats *stats,
                           void *stream) {
    clear_error();
    gp_graph *g = const_cast<gp_graph *>(gc);
    GP_TRY(pr_validate(g, mode, damping, iters, tol));
    if (!ranks_out) return set_error(GP_ERR_INVALID, "gp_pagerank: ranks_out is NULL");
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
    const bool out_dev = is_device_ptr(ranks_out);
    float *R0 = ranks_out;
    if (!out_dev) {
        GP_TRY(ensure_vec(g, w.out_dev, s));
        R0 = w.out_dev;
    }
    const float *S = nullptr, *X0 = nullptr;
    GP_TRY(device_input(g, personalization, w.s_dev, S, s));
    GP_TRY(device_input(g, x0, w.x0_dev, X0, s));
    const bool push = mode == GP_PUSH;
    IterSpec sp;
    sp.push = push;
    sp.hot = true;
    sp.off = push ? g->csr_off : g->csc_off;
    sp.idx = push ? g->csr_idx : g->csc_idx;
    sp.w = g->weighted ? (push ? g->csr_w : g->csc_w) : nullptr;
    sp.bins = push ? &g->push_bins : &g->pull_bins;
    sp.s = S;
    sp.s_scale = 1.0f - damping;
    sp.base_uniform = (float)((1.0 - (double)damping) / (double)n);
    sp.d = damping;
    sp.x0 = X0;
    sp.post_scale = nullptr;
    sp.cmul = g->inv_deg;
    sp.iters = iters;
    sp.tol = tol;
    sp.max_updates = g->max_in;
    PrStatus fin;
    GP_TRY(pr_iterate(g, sp, R0, fin, s));
    if (!out_dev) GP_CUDA(cudaMemcpyAsync(ranks_out, R0, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (stats) {
        GP_CUDA(cudaEventRecord(ev1, s));
        GP_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->iters_done = fin.iters_done;
        stats->mode_used = mode;
        stats->residual = fin.residual;
        stats->ms = ms;
        stats->converged = (tol <= 0.0) ? 1 : fin.converged;
        stats->push_updates_l2 = (int64_t)fin.upd_l2;
        stats->push_updates_shared = (int64_t)fin.upd_shared;
        stats->push_updates_merged = (int64_t)fin.upd_merged;
        stats->push_flush_l2 = (int64_t)fin.flush_l2;
    } else if (!out_dev) {
        GP_CUDA(cudaStreamSynchronize(s));
    }
    if (tol > 0.0 && !fin.converged)
        return set_error(GP_ERR_NOT_CONVERGED, "residual %.3e >= tol %.3e after %d sweeps", fin.residual, tol,
                         fin.iters_done);
    return GP_OK;
}

extern "C" int gp_pagerank_backward(const gp_graph *gc, int mode, float damping, const float *ranks,
                                    const float *grad_ranks, float *grad_weights, float *grad_personalization,
                                    int iters, double tol, gp_pr_stats *stats, void *stream) {
    clear_error();
    gp_graph *g = const_cast<gp_graph *>(gc);
    GP_TRY(pr_validate(g, mode, damping, iters, tol));
    if (!ranks || !grad_ranks) return set_error(GP_ERR_INVALID, "gp_pagerank_backward: ranks and grad_ranks are required");
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == GP_AUTO) mode = GP_PULL;
    const int64_t n = g->n, m = g->m;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0) return GP_OK;
    GP_TRY(ensure_pr_work(g, s));
    PrWork &w = g->pr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    const float *X = nullptr, *G = nullptr;
    GP_TRY(device_input(g, ranks, w.x0_dev, X, s));
    GP_TRY(device_input(g, grad_ranks, w.s_dev, G, s));
    GP_TRY(ensure_vec(g, w.lam, s));
    // (I - d P^T) lambda = g: the transposed sweep.  Pull gathers lambda over the
    // out-edges (CSR) of every vertex; push scatters lambda_v over the in-edges (CSC).
    const bool push = mode == GP_PUSH;
    IterSpec sp;
    sp.push = push;
    sp.hot = false;
    sp.off = push ? g->csc_off : g->csr_off;
    sp.idx = push ? g->csc_idx : g->csr_idx;
    sp.w = g->weighted ? (push ? g->csc_w : g->csr_w) : nullptr;
    sp.bins = push ? &g->pull_bins : &g->push_bins;
    sp.s = G;
    sp.s_scale = 1.0f;
    sp.base_uniform = 0.f;
    sp.d = damping;
    sp.x0 = G;
    sp.post_scale = g->inv_deg;
    sp.cmul = nullptr;
    sp.iters = iters;
    sp.tol = tol;
    sp.max_updates = g->max_out;  // the transposed scatter lands on sources
    PrStatus fin;
    GP_TRY(pr_iterate(g, sp, w.lam, fin, s));
    const int gb = grid_blocks(g, 256);
    if (grad_personalization) {
        const bool dev = is_device_ptr(grad_personalization);
        float *dst = grad_personalization;
        if (!dev) {
            GP_TRY(ensure_vec(g, w.out_dev, s));
            dst = w.out_dev;
        }
        const int b = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
        GP_LAUNCH("grad_s", s, (k_grad_s<<<b, 256, 0, s>>>(n, 1.0f - damping, w.lam, dst)));
        GP_TRY(check_launch("grad_s"));
        if (!dev) GP_CUDA(cudaMemcpyAsync(grad_personalization, dst, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (grad_weights && m > 0) {
        const bool dev = is_device_ptr(grad_weights);
        float *dst = grad_weights;
        if (!dev) {
            if (!w.gw_dev) GP_TRY(w.mem.alloc(w.gw_dev, (size_t)m, s));
            dst = w.gw_dev;
        }
        GradArgs ga;
        ga.n = n;
        ga.off = g->csr_off;
        ga.idx = g->csr_idx;
        ga.x = X;
        ga.lam = w.lam;
        ga.g = G;
        ga.inv_deg = g->inv_deg;
        ga.chunks = g->push_bins.chunks;
        ga.nchunks = g->push_bins.nchunks;
        ga.light_max = g->push_bins.light_max;
        ga.d = damping;
        ga.normalized = g->normalized ? 1 : 0;
        ga.grad_w = dst;
        const int64_t ntiles = (n + 31) / 32;
        ga.split_blocks = (int)std::min<int64_t>(gb, (ga.nchunks + 7) / 8);
        const int b = ga.split_blocks + (int)std::max<int64_t>(1, std::min<int64_t>(gb, (ntiles + 7) / 8));
        GP_LAUNCH("grad_w", s, (k_grad_w<<<b, 256, 0, s>>>(ga)));
        GP_TRY(check_launch("grad_w"));
        if (!dev) GP_CUDA(cudaMemcpyAsync(grad_weights, dst, m * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (stats) {
        GP_CUDA(cudaEventRecord(ev1, s));
        GP_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->iters_done = fin.iters_done;
        stats->mode_used = mode;
        stats->residual = fin.residual;
        stats->ms = ms;
        stats->converged = (tol <= 0.0) ? 1 : fin.converged;
    }
    GP_CUDA(cudaStreamSynchronize(s));
    if (tol > 0.0 && !fin.converged)
        return set_error(GP_ERR_NOT_CONVERGED, "adjoint residual %.3e >= tol %.3e after %d sweeps", fin.residual, tol,
                         fin.iters_done);
    return GP_OK;
}

extern "C" int gp_graph_set_weights(gp_graph *g, const float *csr_w, const float *csc_w, void *stream) {
    clear_error();
    if (!g) return set_error(GP_ERR_INVALID, "gp_graph_set_weights: graph is NULL");
    if (!g->weighted) return set_error(GP_ERR_UNSUPPORTED, "gp_graph_set_weights: the graph was uploaded without weights");
    if (!csr_w || !is_device_ptr(csr_w)) return set_error(GP_ERR_INVALID, "gp_graph_set_weights: csr_w must be device memory");
    const bool shared = g->csc_idx == g->csr_idx;
    if (!shared && (!csc_w || !is_device_ptr(csc_w)))
        return set_error(GP_ERR_INVALID, "gp_graph_set_weights: csc_w must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    g->csr_w = csr_w;
    g->csc_w = shared ? csr_w : csc_w;
    const int64_t n = g->n;
    if (n > 0) {
        const int b = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->num_sms * 8));
        GP_LAUNCH("recompute_inv", s, (k_recompute_inv<<<b, 256, 0, s>>>(g->csr_off, g->csr_w, n, g->normalized, g->inv_deg)));
        GP_TRY(check_launch("recompute_inv"));
    }
    return GP_OK;
}
