// bfs.cu -- top-down (push) and bottom-up (pull) BFS levels, frontier
// conversion, and the gp_bfs driver with its per-level direction switch.
//
// Section 3.3 and Algorithm 3 (push- and pull-based BFS, every ready counter
// equal to one):
//   top-down  (push): every frontier vertex v scans its out-edges (v->w) and
//             claims each unvisited w with a compare-and-swap on level[w]
//             (Section 4.3: O(m) CAS in total); the winner records the parent
//             and appends w to the next frontier (the k-filter of Section 4,
//             here a warp-aggregated queue append).
//   bottom-up (pull): every unvisited vertex v scans its in-edges (u->v) and
//             stops at the first u in the frontier bitmap; only v's owner
//             writes v's level, parent and bitmap bit (a warp owns one 32-bit
//             bitmap word), so vertex state needs no atomics.
// The frontier is a sparse queue after a top-down level and a bitmap after a
// bottom-up level; k_queue_to_bits / k_bits_to_queue convert when the
// direction changes.  Frontier vertices whose out-degree exceeds
// push_light_max are kept as chunk ids of the push chunk table, so one warp
// handles at most chunk_edges of a hub's edges.
// The direction heuristic (not given in the paper, which cites direction-
// optimising BFS in Section 1 and describes switching thresholds as
// Generic-Switch in Section 5): top-down -> bottom-up when the frontier's
// out-edge count m_f exceeds m_u/alpha (m_u = in-edges of unvisited vertices),
// bottom-up -> top-down when the frontier shrinks below n/beta.
#include <algorithm>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {

struct BfsCtr {
    unsigned long long q_len;     // light queue entries
    unsigned long long h_len;     // heavy chunk ids
    unsigned long long nf;        // frontier vertices
    unsigned long long mf;        // sum of out-degrees of the frontier
    unsigned long long mu_dec;    // sum of in-degrees of the newly visited vertices
    unsigned long long examined;  // edges scanned by the level
    unsigned long long pad[2];
};

struct BfsArgs {
    int64_t n;
    const int64_t *csr_off, *csc_off;
    const int32_t *csr_idx, *csc_idx;
    const int32_t *push_rank;   // [n] rank among big out-degree vertices, -1 if light
    const int64_t *push_cstart;
    const Chunk *push_chunks;
    int32_t *level, *parent;    // parent may be nullptr
    const int32_t *queue_cur;
    int32_t *queue_next;
    const int32_t *h_cur;
    int32_t *h_next;
    const uint32_t *bits_cur;
    uint32_t *bits_next;
    BfsCtr *cur, *nxt;
    int32_t L;  // level being expanded: new vertices get L + 1
};

// Append w (newly visited) to the next frontier: light vertices to the queue
// (warp-aggregated), heavy ones as their chunk ids.  Must be called by all 32
// lanes together; `take` marks the lanes that append.
__device__ __forceinline__ void frontier_append(const BfsArgs &a, bool take, int32_t w, unsigned long long &nf,
                                                unsigned long long &mf, unsigned long long &mu) {
    const int lane = lane_id();
    int32_t r = -1;
    if (take) {
        const int64_t dout = a.csr_off[w + 1] - a.csr_off[w];
        mf += (unsigned long long)dout;
        mu += (unsigned long long)(a.csc_off[w + 1] - a.csc_off[w]);
        nf += 1;
        r = a.push_rank[w];
    }
    const bool light = take && r < 0;
    const unsigned bal = __ballot_sync(FULL, light);
    if (bal) {
        unsigned long long base = 0;
        const int leader = __ffs(bal) - 1;
        if (lane == leader) base = atomicAdd(&a.nxt->q_len, (unsigned long long)__popc(bal));
        base = __shfl_sync(FULL, base, leader);
        if (light) a.queue_next[base + __popc(bal & ((1u << lane) - 1u))] = w;
    }
    if (take && r >= 0) {
        const int64_t c0 = a.push_cstart[r], c1 = a.push_cstart[r + 1];
        const unsigned long long pos = atomicAdd(&a.nxt->h_len, (unsigned long long)(c1 - c0));
        for (int64_t j = c0; j < c1; ++j) a.h_next[pos + (j - c0)] = (int32_t)j;
    }
}

// Claim w from u at level L+1; returns true for the winner.
__device__ __forceinline__ bool td_claim(const BfsArgs &a, int32_t w, int32_t u) {
    if (a.level[w] != -1) return false;
    if (atomicCAS(a.level + w, -1, a.L + 1) != -1) return false;
    if (a.parent) a.parent[w] = u;
    return true;
}

__device__ void flush_counters(const BfsArgs &a, unsigned long long nf, unsigned long long mf, unsigned long long mu,
                               unsigned long long ex) {
    __shared__ unsigned long long sm[32];
    nf = block_sum(nf, sm);
    mf = block_sum(mf, sm);
    mu = block_sum(mu, sm);
    ex = block_sum(ex, sm);
    if (threadIdx.x == 0) {
        if (nf) atomicAdd(&a.nxt->nf, nf);
        if (mf) atomicAdd(&a.nxt->mf, mf);
        if (mu) atomicAdd(&a.nxt->mu_dec, mu);
        if (ex) atomicAdd(&a.nxt->examined, ex);
    }
}

__global__ void __launch_bounds__(256) k_bfs_topdown(BfsArgs a) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t h_len = (int64_t)a.cur->h_len, q_len = (int64_t)a.cur->q_len;
    unsigned long long nf = 0, mf = 0, mu = 0, ex = 0;
    // heavy frontier vertices: one warp per chunk of out-edges
    for (int64_t j = warp; j < h_len; j += nwarps) {
        const Chunk ch = a.push_chunks[a.h_cur[j]];
        for (int i0 = 0; i0 < ch.len; i0 += 32) {
            const int i = i0 + lane;
            bool take = false;
            int32_t w = 0;
            if (i < ch.len) {
                w = __ldg(a.csr_idx + ch.beg + i);
                take = td_claim(a, w, ch.v);
                ++ex;
            }
            frontier_append(a, take, w, nf, mf, mu);
        }
    }
    // light frontier vertices: 32 queue entries per warp, one merged edge stream
    const int64_t ntiles = (q_len + 31) >> 5;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t qi = t * 32 + lane;
        int32_t u = -1;
        int64_t b = 0;
        int deg = 0;
        if (qi < q_len) {
            u = a.queue_cur[qi];
            b = a.csr_off[u];
            deg = (int)(a.csr_off[u + 1] - b);
        }
        const int incl = warp_incl_scan(deg);
        const int excl = incl - deg;
        const int E = __shfl_sync(FULL, incl, 31);
        for (int base = 0; base < E; base += 32) {
            const int eid = base + lane;
            int k = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const int exk = __shfl_sync(FULL, excl, k + s);
                if (exk <= eid) k += s;
            }
            const int64_t kb = __shfl_sync(FULL, b, k);
            const int kex = __shfl_sync(FULL, excl, k);
            const int32_t ku = __shfl_sync(FULL, u, k);
            bool take = false;
            int32_t w = 0;
            if (eid < E) {
                w = __ldg(a.csr_idx + kb + (eid - kex));
                take = td_claim(a, w, ku);
                ++ex;
            }
            frontier_append(a, take, w, nf, mf, mu);
        }
    }
    flush_counters(a, nf, mf, mu, ex);
}

__global__ void __launch_bounds__(256) k_bfs_bottomup(BfsArgs a) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwords = (a.n + 31) >> 5;
    unsigned long long nf = 0, mf = 0, mu = 0, ex = 0;
    for (int64_t wd = warp; wd < nwords; wd += nwarps) {
        const int64_t v = wd * 32 + lane;
        bool found = false;
        if (v < a.n && a.level[v] == -1) {
            const int64_t b = a.csc_off[v], e = a.csc_off[v + 1];
            for (int64_t j = b; j < e; ++j) {
                const int32_t u = __ldg(a.csc_idx + j);
                ++ex;
                if ((a.bits_cur[u >> 5] >> (u & 31)) & 1u) {
                    a.level[v] = a.L + 1;
                    if (a.parent) a.parent[v] = u;
                    found = true;
                    break;
                }
            }
            if (found) {
                nf += 1;
                mf += (unsigned long long)(a.csr_off[v + 1] - a.csr_off[v]);
                mu += (unsigned long long)(e - b);
            }
        }
        const unsigned word = __ballot_sync(FULL, found);
        if (lane == 0) a.bits_next[wd] = word;
    }
    flush_counters(a, nf, mf, mu, ex);
}

// Frontier queue (+ heavy chunk ids) -> bitmap (bits must be zeroed first).
__global__ void k_queue_to_bits(const BfsCtr *cur, const int32_t *queue, const int32_t *h, const Chunk *chunks,
                                uint32_t *bits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t q_len = (int64_t)cur->q_len, h_len = (int64_t)cur->h_len;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q_len + h_len; i += stride) {
        const int32_t v = i < q_len ? queue[i] : chunks[h[i - q_len]].v;
        atomicOr(bits + (v >> 5), 1u << (v & 31));
    }
}

// Bitmap -> queue + heavy chunk ids (the counters' q_len/h_len must be zero).
__global__ void k_bits_to_queue(BfsArgs a) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwords = (a.n + 31) >> 5;
    unsigned long long nf = 0, mf = 0, mu = 0;  // already known to the host: discarded
    for (int64_t wd = warp; wd < nwords; wd += nwarps) {
        const uint32_t word = a.bits_cur[wd];
        if (!word) continue;  // uniform across the warp
        const int32_t v = (int32_t)(wd * 32 + lane_id());
        const bool take = (word >> lane_id()) & 1u;
        frontier_append(a, take, v, nf, mf, mu);
    }
}

__global__ void k_bfs_init(int64_t n, int32_t *level, int32_t *parent) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        level[v] = -1;
        if (parent) parent[v] = -1;
    }
}

// Seeds the frontier {src} in queue form and its counters.
__global__ void k_bfs_seed(BfsArgs a, int32_t src) {
    unsigned long long nf = 0, mf = 0, mu = 0;
    const bool take = lane_id() == 0;
    if (take) {
        a.level[src] = 0;
        if (a.parent) a.parent[src] = src;
    }
    frontier_append(a, take, src, nf, mf, mu);
    if (take) {
        a.nxt->nf = nf;
        a.nxt->mf = mf;
        a.nxt->mu_dec = mu;
    }
}

// ------------------------------------------------------------------ driver

void release_bfs_work(gp_graph *g, cudaStream_t s) {
    if (g->bfs.ctr_host) cudaFreeHost(g->bfs.ctr_host);
    g->bfs.ctr_host = nullptr;
    g->bfs.mem.release(s);
    g->bfs = BfsWork();
}

static int ensure_bfs_work(gp_graph *g, cudaStream_t s) {
    BfsWork &w = g->bfs;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    const size_t hcap = (size_t)std::max<int64_t>(g->push_bins.nchunks, 1);
    for (int i = 0; i < 2; ++i) {
        GP_TRY(w.mem.alloc(w.queue[i], n, s));
        GP_TRY(w.mem.alloc(w.hchunk[i], hcap, s));
        GP_TRY(w.mem.alloc(w.bits[i], words, s));
    }
    BfsCtr *c = nullptr;
    GP_TRY(w.mem.alloc(c, 2, s));
    w.ctr = c;
    GP_CUDA(cudaMallocHost(&w.ctr_host, 2 * sizeof(BfsCtr)));
    w.ready = true;
    return GP_OK;
}

static int bfs_run(const gp_graph *gc, int32_t src, int mode, const int8_t *dirs, int ndirs, int32_t *level_out,
                   int32_t *parent_out, gp_bfs_stats *stats, cudaStream_t s) {
    gp_graph *g = const_cast<gp_graph *>(gc);
    const int64_t n = g->n;
    if (src < 0 || (int64_t)src >= n) return set_error(GP_ERR_INVALID, "source %d outside [0, %lld)", src, (long long)n);
    if (!level_out) return set_error(GP_ERR_INVALID, "gp_bfs: level_out is NULL");
    GP_TRY(ensure_bfs_work(g, s));
    BfsWork &w = g->bfs;
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    int32_t *level = level_out, *parent = parent_out;
    const bool lvl_dev = is_device_ptr(level_out);
    const bool par_dev = !parent_out || is_device_ptr(parent_out);
    if (!lvl_dev) {
        if (!w.level_dev) GP_TRY(w.mem.alloc(w.level_dev, (size_t)n, s));
        level = w.level_dev;
    }
    if (!par_dev) {
        if (!w.parent_dev) GP_TRY(w.mem.alloc(w.parent_dev, (size_t)n, s));
        parent = w.parent_dev;
    }
    BfsCtr *ctr = (BfsCtr *)w.ctr;
    BfsCtr *hctr = (BfsCtr *)w.ctr_host;
    const int gb = grid_blocks(g, 256);
    const int ib = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (n + 255) / 256));
    const int64_t nwords = (n + 31) / 32;
    const int wb = (int)std::max<int64_t>(1, std::min<int64_t>(gb, (nwords + 7) / 8));

    BfsArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.csr_off = g->csr_off;
    a.csc_off = g->csc_off;
    a.csr_idx = g->csr_idx;
    a.csc_idx = g->csc_idx;
    a.push_rank = g->push_bins.rank;
    a.push_cstart = g->push_bins.cstart;
    a.push_chunks = g->push_bins.chunks;
    a.level = level;
    a.parent = parent;

    GP_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(BfsCtr), s));
    GP_LAUNCH("bfs_init", s, (k_bfs_init<<<ib, 256, 0, s>>>(n, level, parent)));
    // frontier 0 = {src} in queue form, counters in ctr[0]
    int cur = 0;
    a.cur = ctr + 1;
    a.nxt = ctr + 0;
    a.queue_next = w.queue[0];
    a.h_next = w.hchunk[0];
    GP_LAUNCH("bfs_seed", s, (k_bfs_seed<<<1, 32, 0, s>>>(a, src)));
    GP_TRY(check_launch("bfs seed"));
    GP_CUDA(cudaMemcpyAsync(hctr, ctr, sizeof(BfsCtr), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    unsigned long long nf = hctr[0].nf, mf = hctr[0].mf;
    long long mu = (long long)g->m - (long long)hctr[0].mu_dec;
    bool in_queue = true;  // frontier form
    int prev_dir = GP_PUSH;
    unsigned long long prev_nf = 0;
    int L = 0;
    int64_t reached = 1, examined = 0, edges_reached = (int64_t)mf;
    int switches = 0;
    const float alpha = g->opt.bfs_alpha, beta = g->opt.bfs_beta;
    while (nf > 0) {
        int dir;
        if (dirs) {
            dir = dirs[std::min(L, ndirs - 1)];
        } else if (mode == GP_PUSH || mode == GP_PULL) {
            dir = mode;
        } else if (prev_dir == GP_PUSH) {
            dir = ((double)mf > (double)std::max(mu, 0LL) / alpha) ? GP_PULL : GP_PUSH;
        } else {
            dir = ((double)nf < (double)n / beta && nf < prev_nf) ? GP_PUSH : GP_PULL;
        }
        if (L > 0 && dir != prev_dir) ++switches;
        const int nxt = cur ^ 1;
        a.L = L;
        a.cur = ctr + cur;
        a.nxt = ctr + nxt;
        a.queue_cur = w.queue[cur];
        a.h_cur = w.hchunk[cur];
        a.bits_cur = w.bits[cur];
        a.queue_next = w.queue[nxt];
        a.h_next = w.hchunk[nxt];
        a.bits_next = w.bits[nxt];
        if (dir == GP_PUSH && !in_queue) {
            BfsArgs conv = a;  // the queue form is written in place of the bitmap's slot
            conv.nxt = a.cur;
            conv.queue_next = w.queue[cur];
            conv.h_next = w.hchunk[cur];
            GP_LAUNCH("bfs_bits_to_queue", s, (k_bits_to_queue<<<wb, 256, 0, s>>>(conv)));
            GP_TRY(check_launch("bits_to_queue"));
        } else if (dir == GP_PULL && in_queue) {
            GP_CUDA(cudaMemsetAsync(w.bits[cur], 0, (size_t)nwords * sizeof(uint32_t), s));
            GP_LAUNCH("bfs_queue_to_bits", s,
                      (k_queue_to_bits<<<ib, 256, 0, s>>>(ctr + cur, w.queue[cur], w.hchunk[cur], g->push_bins.chunks,
                                                          w.bits[cur])));
            GP_TRY(check_launch("queue_to_bits"));
        }
        GP_CUDA(cudaMemsetAsync(ctr + nxt, 0, sizeof(BfsCtr), s));
        if (dir == GP_PUSH) {
            GP_LAUNCH("bfs_topdown", s, (k_bfs_topdown<<<gb, 256, 0, s>>>(a)));
            in_queue = true;
        } else {
            GP_LAUNCH("bfs_bottomup", s, (k_bfs_bottomup<<<wb, 256, 0, s>>>(a)));
            in_queue = false;
        }
        GP_TRY(check_launch("bfs level"));
        GP_CUDA(cudaMemcpyAsync(hctr + nxt, ctr + nxt, sizeof(BfsCtr), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaStreamSynchronize(s));
        const BfsCtr &c = hctr[nxt];
        if (stats && L < GP_BFS_MAX_LEVELS) {
            stats->direction[L] = (int8_t)dir;
            stats->frontier[L] = (int64_t)nf;
            stats->examined[L] = (int64_t)c.examined;
        }
        examined += (int64_t)c.examined;
        reached += (int64_t)c.nf;
        edges_reached += (int64_t)c.mf;
        prev_nf = nf;
        nf = c.nf;
        mf = c.mf;
        mu -= (long long)c.mu_dec;
        prev_dir = dir;
        cur = nxt;
        ++L;
    }
    if (!lvl_dev) GP_CUDA(cudaMemcpyAsync(level_out, level, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (!par_dev) GP_CUDA(cudaMemcpyAsync(parent_out, parent, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (stats) {
        GP_CUDA(cudaEventRecord(ev1, s));
        GP_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->levels = L;
        stats->switches = switches;
        stats->reached = reached;
        stats->edges_examined = examined;
        stats->edges_reached = edges_reached;
        stats->ms = ms;
    }
    if (!lvl_dev || !par_dev) GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" int gp_bfs(const gp_graph *g, int32_t src, int mode, int32_t *level_out, int32_t *parent_out,
                      gp_bfs_stats *stats, void *stream) {
    clear_error();
    if (!g) return set_error(GP_ERR_INVALID, "gp_bfs: graph is NULL");
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "bad mode %d", mode);
    return bfs_run(g, src, mode, nullptr, 0, level_out, parent_out, stats, (cudaStream_t)stream);
}

extern "C" int gp_bfs_directed(const gp_graph *g, int32_t src, const int8_t *dirs, int ndirs, int32_t *level_out,
                               int32_t *parent_out, gp_bfs_stats *stats, void *stream) {
    clear_error();
    if (!g) return set_error(GP_ERR_INVALID, "gp_bfs_directed: graph is NULL");
    if (!dirs || ndirs < 1) return set_error(GP_ERR_INVALID, "gp_bfs_directed: need at least one direction");
    for (int i = 0; i < ndirs; ++i)
        if (dirs[i] != GP_PUSH && dirs[i] != GP_PULL)
            return set_error(GP_ERR_INVALID, "gp_bfs_directed: dirs[%d] = %d is not GP_PUSH or GP_PULL", i, dirs[i]);
    return bfs_run(g, src, GP_AUTO, dirs, ndirs, level_out, parent_out, stats, (cudaStream_t)stream);
}
