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
// A top-down level produces the next frontier both as a sparse queue and as a
// bitmap (the winner of each claim also sets the vertex's bit), so a switch to
// bottom-up needs no conversion; a bottom-up level produces only the bitmap,
// which is compacted into a queue when the search switches back.  Bottom-up
// levels visit only the 32-vertex words that still hold candidates: a bitmap
// of vertices with in-edges that may be unvisited, thinned by each bottom-up
// level (vertices claimed top-down are dropped when a bottom-up level meets
// them).  Frontier vertices whose out-degree exceeds
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
    unsigned long long deferred;  // bottom-up: hubs whose first in-edges held no frontier vertex
    unsigned long long pad;
};

struct BfsArgs {
    int64_t n;
    const int64_t *csr_off, *csc_off;
    const int32_t *csr_idx, *csc_idx;
    const int32_t *push_rank;   // [n] rank among big out-degree vertices, -1 if light
    const int64_t *push_cstart;
    const Chunk *push_chunks;
    const Chunk *pull_chunks;   // in-edge chunks of the vertices above the pull light limit
    int64_t pull_nchunks;
    int64_t bu_probe;           // bottom-up: in-edges a lane probes before deferring a hub
    int32_t *level, *parent;    // parent may be nullptr
    const int32_t *queue_cur;
    int32_t *queue_next;
    const int32_t *h_cur;
    int32_t *h_next;
    const uint32_t *bits_cur;
    uint32_t *bits_next;   // next frontier bitmap (zero on entry)
    uint32_t *unvis;       // bottom-up candidates; each word owned by one warp of a bottom-up level
    BfsCtr *cur, *nxt;
    int32_t L;           // level being expanded: new vertices get L + 1
    int32_t make_queue;  // top-down: also build the next frontier's queue
    int64_t q_len, h_len;  // top-down: lengths of the current frontier's queue and heavy list
    int32_t gblk, ngblk;   // this block's index among the blocks running the search, and their number
};

// Warp index and warp count within the blocks that run one search (the whole
// grid for gp_bfs, one group of blocks for gp_bfs_multi).
__device__ __forceinline__ int64_t search_warp(const BfsArgs &a) {
    return ((int64_t)a.gblk * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ int64_t search_nwarps(const BfsArgs &a) { return ((int64_t)a.ngblk * blockDim.x) >> 5; }

// Count w (newly visited) into the next frontier's statistics and, when the
// level builds a queue, append it: light vertices to the queue (warp-
// aggregated), heavy ones as their chunk ids.  Must be called by all 32 lanes
// together; `take` marks the lanes that append.
__device__ __forceinline__ void frontier_append(const BfsArgs &a, bool take, int32_t w, unsigned long long &nf,
                                                unsigned long long &mf, unsigned long long &mu) {
    const int lane = lane_id();
    int32_t r = -1;
    if (take) {
        const int64_t dout = a.csr_off[w + 1] - a.csr_off[w];
        mf += (unsigned long long)dout;
        mu += (unsigned long long)(a.csc_off[w + 1] - a.csc_off[w]);
        nf += 1;
        if (a.make_queue) r = a.push_rank[w];
    }
    if (!a.make_queue) return;  // uniform
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

// Claim w from u at level L+1; returns true for the winner, which also marks w
// in the next frontier's bitmap and removes it from the bottom-up candidates.
__device__ __forceinline__ bool td_claim(const BfsArgs &a, int32_t w, int32_t u) {
    if (a.level[w] != -1) return false;
    if (atomicCAS(a.level + w, -1, a.L + 1) != -1) return false;
    if (a.parent) a.parent[w] = u;
    const uint32_t bit = 1u << (w & 31);
    atomicOr(a.bits_next + (w >> 5), bit);
    atomicAnd(a.unvis + (w >> 5), ~bit);
    return true;
}

// The five counters of a block summed in one pass (one shared-memory round
// and two block barriers), then added to the next level's record.
__device__ void flush_counters(const BfsArgs &a, unsigned long long nf, unsigned long long mf, unsigned long long mu,
                               unsigned long long ex, unsigned long long deferred = 0) {
    constexpr int K = 5;
    __shared__ unsigned long long sm[K][32];
    unsigned long long v[K] = {nf, mf, mu, ex, deferred};
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane_id() == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) sm[i][w] = v[i];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = warp_sum(lane_id() < nw ? sm[i][lane_id()] : 0ull);
        if (lane_id() == 0) {
            if (v[0]) atomicAdd(&a.nxt->nf, v[0]);
            if (v[1]) atomicAdd(&a.nxt->mf, v[1]);
            if (v[2]) atomicAdd(&a.nxt->mu_dec, v[2]);
            if (v[3]) atomicAdd(&a.nxt->examined, v[3]);
            if (v[4]) atomicAdd(&a.nxt->deferred, v[4]);
        }
    }
}

// ------------------------------------------------------------------ level steps (device functions)

constexpr int TD_SPLIT = 4;
constexpr unsigned long long TD_QUEUE_EDGES = 1ull << 14;

// Top-down level: heavy frontier vertices (chunk ids) split over warps, light
// ones 32 queue entries per warp with a merged edge stream.
__device__ void bfs_topdown_step(const BfsArgs &a) {
    const int lane = lane_id();
    const int64_t warp = search_warp(a);
    const int64_t nwarps = search_nwarps(a);
    const int64_t h_len = a.h_len, q_len = a.q_len;
    unsigned long long nf = 0, mf = 0, mu = 0, ex = 0;
    // each heavy chunk is split TD_SPLIT ways so a frontier of a few hubs still spreads over many warps
    for (int64_t j = warp; j < h_len * TD_SPLIT; j += nwarps) {
        const Chunk ch = a.push_chunks[a.h_cur[j / TD_SPLIT]];
        const int part = (int)(j % TD_SPLIT);
        const int plen = (ch.len + TD_SPLIT - 1) / TD_SPLIT;
        const int lo = part * plen, hi = min(ch.len, lo + plen);
        for (int i0 = lo; i0 < hi; i0 += 32) {
            const int i = i0 + lane;
            bool take = false;
            int32_t w = 0;
            if (i < hi) {
                w = __ldg(a.csr_idx + ch.beg + i);
                take = td_claim(a, w, ch.v);
                ++ex;
            }
            frontier_append(a, take, w, nf, mf, mu);
        }
    }
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

// Bottom-up level.  A warp takes 32 consecutive words of the candidate bitmap
// (unvisited vertices with in-edges), ranks their candidates with a warp
// prefix sum, and gives them out 32 at a time, one per lane, so every lane works
// on a real candidate whatever the density; each scans its in-edges and stops
// at the first frontier vertex.  Found bits gather in the warp's shared words,
// then each lane writes its own word of the next frontier (zero on entry) and
// of the candidates: each word has one writer, so vertex state needs no atomics.
#ifndef GP_BFS_WARPS
#define GP_BFS_WARPS 16
#endif
#ifndef GP_BFS_MINB
#define GP_BFS_MINB 2
#endif
constexpr int BFS_WARPS = GP_BFS_WARPS;  // warps per block of the persistent kernel
#ifndef GP_BU_SCAN
#define GP_BU_SCAN 4
#endif
constexpr int BU_SCAN = GP_BU_SCAN;  // in-edges a bottom-up lane checks per step
// A candidate with more in-edges than this is a hub: its lane probes only that
// many, and a hub with no frontier vertex among them is finished by the chunk
// pass (one lane walking a hub's whole in-list would hold up its warp).
#ifndef GP_BU_PROBE
#define GP_BU_PROBE 64
#endif
constexpr int64_t BU_PROBE = GP_BU_PROBE;

__device__ void bfs_bottomup_step(const BfsArgs &a) {
    __shared__ uint32_t s_found[BFS_WARPS][32];
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const int64_t warp = search_warp(a);
    const int64_t nwarps = search_nwarps(a);
    const int64_t nwords = (a.n + 31) >> 5;
    unsigned long long nf = 0, mf = 0, mu = 0, ex = 0, deferred = 0;
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t cand = wd < nwords ? a.unvis[wd] : 0u;
        const int cnt = __popc(cand);
        const int incl = warp_incl_scan(cnt);
        const int excl = incl - cnt;
        const int total = __shfl_sync(FULL, incl, 31);
        if (total == 0) continue;  // uniform across the warp
        s_found[wib][lane] = 0u;
        __syncwarp();
        // Round r's candidate (vertex and in-edge range) is located and its
        // offsets loaded during round r - 1, so they arrive while that round scans.
        auto locate = [&](int id, int &k, int &bit, int64_t &b, int64_t &e) {
            k = 0;  // the lane (word) whose candidates [excl, incl) hold id
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ek = __shfl_sync(FULL, excl, k + st);
                if (ek <= id) k += st;
            }
            const uint32_t kc = __shfl_sync(FULL, cand, k);
            const int kex = __shfl_sync(FULL, excl, k);
            bit = 0;
            b = e = 0;
            if (id < total) {
                bit = nth_set_bit(kc, id - kex);
                const int64_t v = (base + k) * 32 + bit;
                b = a.csc_off[v];
                e = a.csc_off[v + 1];
            }
        };
        int k, bit;
        int64_t b, e;
        locate(lane, k, bit, b, e);
        for (int r = 0; r < total; r += 32) {
            int kn, bitn;
            int64_t bn, en;
            locate(r + 32 + lane, kn, bitn, bn, en);
            if (r + lane < total) {
                const int64_t v = (base + k) * 32 + bit;
                // a hub's lane probes only its first bu_probe in-edges; if none is in
                // the frontier the hub is deferred to the chunk pass (bfs_bottomup_hubs)
                const bool hub = e - b > a.bu_probe;
                const int64_t e1 = hub ? b + a.bu_probe : e;
                bool found = false;
                // BU_SCAN in-edges per step: their bitmap probes are independent
                for (int64_t j = b; j < e1; j += BU_SCAN) {
                    int32_t u[BU_SCAN];
                    bool hit[BU_SCAN];
#pragma unroll
                    for (int q = 0; q < BU_SCAN; ++q) u[q] = j + q < e1 ? __ldg(a.csc_idx + j + q) : 0;
#pragma unroll
                    for (int q = 0; q < BU_SCAN; ++q)
                        hit[q] = j + q < e1 && ((a.bits_cur[u[q] >> 5] >> (u[q] & 31)) & 1u);
                    int first = -1;
#pragma unroll
                    for (int q = BU_SCAN - 1; q >= 0; --q)
                        if (hit[q]) first = q;
                    if (first >= 0) {
                        int32_t p = u[0];
#pragma unroll
                        for (int q = 1; q < BU_SCAN; ++q)
                            if (q == first) p = u[q];
                        ex += (unsigned long long)(first + 1);
                        a.level[v] = a.L + 1;
                        if (a.parent) a.parent[v] = p;
                        atomicOr(&s_found[wib][k], 1u << bit);
                        nf += 1;
                        mf += (unsigned long long)(a.csr_off == a.csc_off ? e - b : a.csr_off[v + 1] - a.csr_off[v]);
                        mu += (unsigned long long)(e - b);
                        found = true;
                        break;
                    }
                    ex += (unsigned long long)(e1 - j < BU_SCAN ? e1 - j : BU_SCAN);
                }
                if (hub && !found) ++deferred;
            }
            k = kn;
            bit = bitn;
            b = bn;
            e = en;
        }
        __syncwarp();
        const uint32_t fw = s_found[wib][lane];
        if (fw) {
            a.bits_next[wd] = fw;
            a.unvis[wd] = cand & ~fw;
        }
        __syncwarp();
    }
    flush_counters(a, nf, mf, mu, ex, deferred);
}

// Second pass of a bottom-up level, run only when some hub was deferred: the
// in-edge chunks (chunk_edges each) of every hub still unvisited are scanned by
// warps across the whole grid, so a hub's in-list is spread over many warps.
// Each chunk stops at its first frontier vertex, or when another chunk has
// claimed the hub; chunks of one hub settle the claim with one compare-and-swap
// on its level (the owner-only rule applied to the hub's set of chunks).
constexpr int BU_WARP_UNROLL = 8;

__device__ void bfs_bottomup_hubs(const BfsArgs &a) {
    const int lane = lane_id();
    const int64_t warp = search_warp(a);
    const int64_t nwarps = search_nwarps(a);
    volatile int32_t *vlevel = a.level;
    unsigned long long nf = 0, mf = 0, mu = 0, ex = 0;
    for (int64_t base = warp * 32; base < a.pull_nchunks; base += nwarps * 32) {
        const int64_t j = base + lane;
        Chunk ch;
        ch.beg = 0;
        ch.len = 0;
        ch.v = 0;
        bool need = false;
        if (j < a.pull_nchunks) {
            ch = a.pull_chunks[j];
            if (vlevel[ch.v] == -1) need = a.csc_off[ch.v + 1] - a.csc_off[ch.v] > a.bu_probe;
        }
        for (unsigned nm = __ballot_sync(FULL, need); nm; nm &= nm - 1) {
            const int hl = __ffs(nm) - 1;
            const int64_t cb = __shfl_sync(FULL, ch.beg, hl);
            const int cl = __shfl_sync(FULL, ch.len, hl);
            const int32_t v = __shfl_sync(FULL, ch.v, hl);
            int64_t hit = -1;
            int32_t par = 0;
            int scanned = 0;
            for (int i0 = 0; i0 < cl && hit < 0; i0 += 32 * BU_WARP_UNROLL) {
                int claimed = 0;
                if (lane == 0 && i0 > 0) claimed = vlevel[v] != -1;
                if (__shfl_sync(FULL, claimed, 0)) break;  // uniform
                int32_t u[BU_WARP_UNROLL];
#pragma unroll
                for (int q = 0; q < BU_WARP_UNROLL; ++q) {
                    const int i = i0 + q * 32 + lane;
                    u[q] = i < cl ? __ldg(a.csc_idx + cb + i) : 0;
                }
                unsigned bm[BU_WARP_UNROLL];
#pragma unroll
                for (int q = 0; q < BU_WARP_UNROLL; ++q) {
                    const int i = i0 + q * 32 + lane;
                    bm[q] = __ballot_sync(FULL, i < cl && ((a.bits_cur[u[q] >> 5] >> (u[q] & 31)) & 1u));
                }
#pragma unroll
                for (int q = 0; q < BU_WARP_UNROLL; ++q) {
                    if (hit < 0 && bm[q]) {  // uniform: the ballots are the warp's
                        const int fl = __ffs(bm[q]) - 1;
                        hit = cb + i0 + q * 32 + fl;
                        par = __shfl_sync(FULL, u[q], fl);
                    }
                }
                scanned = min(cl, i0 + 32 * BU_WARP_UNROLL);
            }
            if (lane == 0) {
                ex += (unsigned long long)(hit >= 0 ? hit - cb + 1 : scanned);
                if (hit >= 0 && atomicCAS(a.level + v, -1, a.L + 1) == -1) {
                    if (a.parent) a.parent[v] = par;
                    const uint32_t bit = 1u << (v & 31);
                    atomicOr(a.bits_next + (v >> 5), bit);
                    atomicAnd(a.unvis + (v >> 5), ~bit);
                    const int64_t din = a.csc_off[v + 1] - a.csc_off[v];
                    nf += 1;
                    mf += (unsigned long long)(a.csr_off == a.csc_off ? din : a.csr_off[v + 1] - a.csr_off[v]);
                    mu += (unsigned long long)din;
                }
            }
        }
    }
    flush_counters(a, nf, mf, mu, ex);
}

// Bitmap -> queue + heavy chunk ids (the counters' q_len/h_len must be zero):
// a warp ranks the set bits of 32 words and appends them 32 at a time.
__device__ void bits_to_queue_step(const BfsArgs &a) {
    const int lane = lane_id();
    const int64_t warp = search_warp(a);
    const int64_t nwarps = search_nwarps(a);
    const int64_t nwords = (a.n + 31) >> 5;
    unsigned long long nf = 0, mf = 0, mu = 0;  // already counted by the level that made the bitmap
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t word = wd < nwords ? a.bits_cur[wd] : 0u;
        const int cnt = __popc(word);
        const int incl = warp_incl_scan(cnt);
        const int excl = incl - cnt;
        const int total = __shfl_sync(FULL, incl, 31);
        for (int r = 0; r < total; r += 32) {
            const int id = r + lane;
            int k = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ek = __shfl_sync(FULL, excl, k + st);
                if (ek <= id) k += st;
            }
            const uint32_t kw = __shfl_sync(FULL, word, k);
            const int kex = __shfl_sync(FULL, excl, k);
            const bool take = id < total;
            const int32_t v = take ? (int32_t)((base + k) * 32 + nth_set_bit(kw, id - kex)) : 0;
            frontier_append(a, take, v, nf, mf, mu);
        }
    }
}

// ------------------------------------------------------------------ the whole search in one launch

struct BfsLevelStat {
    int32_t direction;
    int32_t ns;  // device time of the level (global timer, block 0)
    int64_t frontier;
    int64_t examined;
};

struct BfsSummary {
    int64_t levels, reached, examined, edges_reached, switches, init_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct BfsRun {
    BfsArgs base;  // graph arrays, level/parent, chunk table
    int32_t *queue[2];
    int32_t *hchunk[2];
    uint32_t *bits[3];      // a ring: level k's frontier bitmap in bits[k % 3]
    const uint32_t *nzin;   // vertices with in-edges
    BfsCtr *ctr;  // [3], a ring
    const int8_t *dirs;  // forced directions (device) or nullptr
    int32_t ndirs;
    int32_t mode;
    float alpha, beta;
    int64_t m;
    int32_t src;
    BfsLevelStat *stats;  // [GP_BFS_MAX_LEVELS]
    BfsSummary *summary;
    GridSync *sync;
};

// 512-thread blocks, two per SM (R-MAT 22, 64 searches: 11.5 ms one launch
// per search and 5.8 ms in 16 groups, against 11.7 and 6.0 ms with one
// 1024-thread block per SM, whose barriers have half the arrivals).
constexpr int BFS_THREADS = BFS_WARPS * 32;

// The outputs and source of one search.
struct SearchIO {
    int32_t src;
    int32_t *level, *parent;  // parent may be nullptr
    BfsSummary *summary;
};

// One whole search, run by `ngblk` blocks (gblk = this block's index among
// them) that share R's workspace and barrier.  Every block keeps identical
// copies of the frontier statistics (read from the counters after each
// barrier), so all blocks take the same direction decision without a host
// round trip.  Returns false when a barrier wait ran out.
__device__ bool bfs_search(const BfsRun &R, const SearchIO &io, int gblk, int ngblk) {
    const unsigned long long t_start = global_ns();
    const int64_t n = R.base.n;
    const int64_t gthread = (int64_t)gblk * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)ngblk * blockDim.x;
    const int64_t nwords = (n + 31) >> 5;
    // level/parent, counters, bitmaps and candidates set for frontier 0 = {src}
    const int32_t src = io.src;
    const int32_t s_rank = R.base.push_rank[src];
    const int64_t s_c0 = s_rank >= 0 ? R.base.push_cstart[s_rank] : 0;
    const int64_t s_c1 = s_rank >= 0 ? R.base.push_cstart[s_rank + 1] : 0;
    for (int64_t v = gthread; v < n; v += nthreads) {
        io.level[v] = v == src ? 0 : -1;
        if (io.parent) io.parent[v] = v == src ? src : -1;
    }
    constexpr int CW = (int)(sizeof(BfsCtr) / sizeof(unsigned long long));
    if (gthread < 3 * CW) {
        unsigned long long val = 0;  // ctr[0] describes {src}; ctr[1], ctr[2] start at zero
        if (gthread == 0) val = s_rank < 0 ? 1 : 0;                                                 // q_len
        if (gthread == 1) val = (unsigned long long)(s_c1 - s_c0);                                  // h_len
        if (gthread == 2) val = 1;                                                                  // nf
        if (gthread == 3) val = (unsigned long long)(R.base.csr_off[src + 1] - R.base.csr_off[src]);  // mf
        if (gthread == 4) val = (unsigned long long)(R.base.csc_off[src + 1] - R.base.csc_off[src]);  // mu_dec
        ((unsigned long long *)R.ctr)[gthread] = val;
    }
    if (gthread == 0 && s_rank < 0) R.queue[0][0] = src;
    for (int64_t j = gthread; j < s_c1 - s_c0; j += nthreads) R.hchunk[0][j] = (int32_t)(s_c0 + j);
    const int64_t sw = src >> 5;
    const uint32_t sbit = 1u << (src & 31);
    for (int64_t i = gthread; i < nwords; i += nthreads) {
        R.bits[0][i] = i == sw ? sbit : 0u;
        R.bits[1][i] = 0u;
        R.base.unvis[i] = R.nzin[i] & (i == sw ? ~sbit : ~0u);
    }
    if (!grid_sync(R.sync, ngblk)) return false;
    unsigned long long t_level = global_ns();
    const unsigned long long t_init = t_level - t_start;
    BfsArgs a = R.base;
    a.level = io.level;
    a.parent = io.parent;
    a.gblk = gblk;
    a.ngblk = ngblk;
    // counter records are read by one thread per block and shared through
    // shared memory: every thread loading the same line would queue tens of
    // thousands of requests on one L2 slice per level
    volatile BfsCtr *vc = (volatile BfsCtr *)R.ctr;
    __shared__ unsigned long long s_ctr[7];
    auto read_ctr = [&](int slot) {
        if (threadIdx.x == 0) {
            s_ctr[0] = vc[slot].q_len;
            s_ctr[1] = vc[slot].h_len;
            s_ctr[2] = vc[slot].nf;
            s_ctr[3] = vc[slot].mf;
            s_ctr[4] = vc[slot].mu_dec;
            s_ctr[5] = vc[slot].examined;
            s_ctr[6] = vc[slot].deferred;
        }
        __syncthreads();
    };
    read_ctr(0);
    unsigned long long nf = s_ctr[2], mf = s_ctr[3];
    long long mu = (long long)R.m - (long long)s_ctr[4];
    int64_t q_len = (int64_t)s_ctr[0], h_len = (int64_t)s_ctr[1];
    unsigned long long prev_nf = 0;
    int cur = 0, prev_dir = GP_PUSH, L = 0, switches = 0;
    bool in_queue = true;
    long long reached = 1, examined = 0, edges_reached = (long long)mf;
    // Counters and bitmaps form rings of three: level L reads slot L%3 (its
    // frontier) and fills slot (L+1)%3; slot (L+2)%3, last used by level L-1, is
    // zeroed during level L's step for level L+1, so no barrier is spent on
    // clearing it.
    while (nf > 0) {
        int dir;
        if (R.dirs) {
            dir = R.dirs[L < R.ndirs ? L : R.ndirs - 1];
        } else if (R.mode == GP_PUSH || R.mode == GP_PULL) {
            dir = R.mode;
        } else if (prev_dir == GP_PUSH) {
            dir = ((float)mf * R.alpha > (float)(mu > 0 ? mu : 0)) ? GP_PULL : GP_PUSH;
        } else {
            dir = ((float)nf * R.beta < (float)n && nf < prev_nf) ? GP_PUSH : GP_PULL;
        }
        if (L > 0 && dir != prev_dir) ++switches;
        const int nxt = (cur + 1) % 3, spare = (cur + 2) % 3;
        a.L = L;
        a.cur = R.ctr + cur;
        a.nxt = R.ctr + nxt;
        a.queue_cur = R.queue[L & 1];
        a.h_cur = R.hchunk[L & 1];
        a.bits_cur = R.bits[cur];
        a.queue_next = R.queue[(L + 1) & 1];
        a.h_next = R.hchunk[(L + 1) & 1];
        a.bits_next = R.bits[nxt];
        if (dir == GP_PUSH && !in_queue) {
            BfsArgs c = a;  // the queue form of the current frontier goes to its own slot
            c.make_queue = 1;
            c.nxt = a.cur;
            c.queue_next = R.queue[L & 1];
            c.h_next = R.hchunk[L & 1];
            bits_to_queue_step(c);
            if (!grid_sync(R.sync, ngblk)) return false;
            read_ctr(cur);
            q_len = (int64_t)s_ctr[0];
            h_len = (int64_t)s_ctr[1];
        }
        if (gthread < CW) ((unsigned long long *)(R.ctr + spare))[gthread] = 0;
        for (int64_t i = gthread; i < nwords; i += nthreads) R.bits[spare][i] = 0u;
        if (dir == GP_PUSH) {
            // a queue of the next frontier only when this frontier is small (so
            // are the appends); otherwise the bitmap alone, compacted later if
            // another top-down level follows
            a.make_queue = mf < TD_QUEUE_EDGES;
            a.q_len = q_len;
            a.h_len = h_len;
            bfs_topdown_step(a);
            in_queue = a.make_queue != 0;
        } else {
            bfs_bottomup_step(a);
            in_queue = false;
        }
        if (!grid_sync(R.sync, ngblk)) return false;
        read_ctr(nxt);
        if (dir == GP_PULL && s_ctr[6] > 0) {  // hubs deferred by the lanes: the chunk pass
            bfs_bottomup_hubs(a);
            if (!grid_sync(R.sync, ngblk)) return false;
            read_ctr(nxt);
        }
        const unsigned long long nf2 = s_ctr[2], mf2 = s_ctr[3], mud = s_ctr[4], ex = s_ctr[5];
        q_len = (int64_t)s_ctr[0];
        h_len = (int64_t)s_ctr[1];
        if (gthread == 0 && R.stats && L < GP_BFS_MAX_LEVELS) {
            const unsigned long long t = global_ns();
            R.stats[L].ns = (int32_t)min(t - t_level, 0x7fffffffull);
            t_level = t;
            R.stats[L].direction = dir;
            R.stats[L].frontier = (int64_t)nf;
            R.stats[L].examined = (int64_t)ex;
        }
        examined += (long long)ex;
        reached += (long long)nf2;
        edges_reached += (long long)mf2;
        prev_nf = nf;
        nf = nf2;
        mf = mf2;
        mu -= (long long)mud;
        prev_dir = dir;
        cur = nxt;
        ++L;
    }
    if (gthread == 0) {
        io.summary->levels = L;
        io.summary->reached = reached;
        io.summary->examined = examined;
        io.summary->edges_reached = edges_reached;
        io.summary->switches = switches;
        io.summary->init_ns = (int64_t)t_init;
    }
    return true;
}

__global__ void __launch_bounds__(BFS_THREADS, GP_BFS_MINB) k_bfs_persistent(BfsRun R) {
    const SearchIO io = {R.src, R.base.level, R.base.parent, R.summary};
    bfs_search(R, io, blockIdx.x, gridDim.x);
}

// Several searches in one launch: the grid is cut into `groups` groups of
// `bpg` consecutive blocks, each with its own workspace and barrier (runs[g]).
// A group takes the next search from a shared counter whenever it finishes
// one, so groups that drew short searches take more of them.  The groups
// never wait on one another, so each search's fixed per-level cost (barrier
// and counter round trip) overlaps the other groups' work.
constexpr int BFS_MULTI_MAX_GROUPS = 32;
// Passed by value: the runs sit in the kernel's parameter space, which every
// thread reads at the cost of a constant load.
struct BfsMulti {
    BfsRun runs[BFS_MULTI_MAX_GROUPS];  // the groups' workspaces and barriers (kernel parameters)
    const int32_t *src;      // [nsrc]
    int32_t *const *level;   // [nsrc] device pointers
    int32_t *const *parent;  // [nsrc] device pointers, or nullptr
    BfsSummary *summary;     // [nsrc]
    int32_t *next;           // the next search to hand out (zero at launch)
    int32_t *slot;           // [2 * groups]: the search a group's leader drew, by draw parity
    int32_t nsrc, groups, bpg;
};

static_assert(sizeof(BfsMulti) <= 32764, "kernel parameters are limited to 32764 bytes");

__global__ void __launch_bounds__(BFS_THREADS, GP_BFS_MINB) k_bfs_multi(BfsMulti M) {
    const int grp = blockIdx.x / M.bpg;
    const int gblk = blockIdx.x - grp * M.bpg;
    if (grp >= M.groups) return;
    const BfsRun &R = M.runs[grp];
    for (int draw = 0;; ++draw) {
        // the leader draws a search and the group's barrier publishes it; the
        // same barrier also ends the previous search in every block before the
        // workspace is reset.  Draws alternate between two slots, so a slot is
        // rewritten only after every block has read it (two barriers later).
        int32_t *sl = M.slot + 2 * grp + (draw & 1);
        if (gblk == 0 && threadIdx.x == 0) *sl = atomicAdd(M.next, 1);
        if (!grid_sync(R.sync, M.bpg)) return;
        const int i = *(volatile int32_t *)sl;
        if (i >= M.nsrc) return;
        const SearchIO io = {M.src[i], M.level[i], M.parent ? M.parent[i] : nullptr, M.summary + i};
        if (!bfs_search(R, io, gblk, M.bpg)) return;
    }
}

// ------------------------------------------------------------------ driver

// Bit v of word v/32: vertex v has in-edges.
__global__ void k_nzin_bits(int64_t n, const int64_t *csc_off, uint32_t *bits) {
    const int64_t nwords = (n + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < nwords; wd += stride) {
        uint32_t word = 0;
        const int64_t v0 = wd * 32, v1 = min(n, v0 + 32);
        int64_t prev = csc_off[v0];
        for (int64_t v = v0; v < v1; ++v) {
            const int64_t next = csc_off[v + 1];
            if (next > prev) word |= 1u << (v - v0);
            prev = next;
        }
        bits[wd] = word;
    }
}

// host mirror: summary, per-level statistics, barrier status
constexpr size_t BFS_HOST_BYTES = sizeof(BfsSummary) + GP_BFS_MAX_LEVELS * sizeof(BfsLevelStat) + sizeof(GridSync);

void release_bfs_work(gp_graph *g, cudaStream_t s) {
    if (g->bfs.done_ev) {
        cudaEventSynchronize(g->bfs.done_ev);
        cudaEventDestroy(g->bfs.done_ev);
    }
    if (g->bfs.mdone_ev) {
        cudaEventSynchronize(g->bfs.mdone_ev);
        cudaEventDestroy(g->bfs.mdone_ev);
    }
    pinned_free(g->bfs.ctr_host, BFS_HOST_BYTES);
    pinned_free(g->bfs.mhost, g->bfs.mhost_bytes);
    g->bfs.ctr_host = nullptr;
    g->bfs.mem.release(s);
    g->bfs.mmem.release(s);
    g->bfs = BfsWork();
}

// The multi-search workspace alone (the group count changed); a pending
// asynchronous gp_bfs_multi is waited for first.
void release_bfs_multi(gp_graph *g, cudaStream_t s) {
    BfsWork &w = g->bfs;
    if (w.mdone_ev) cudaEventSynchronize(w.mdone_ev);
    w.mpending = false;
    pinned_free(w.mhost, w.mhost_bytes);
    w.mhost = nullptr;
    w.mhost_bytes = 0;
    w.mmem.release(s);
    w.mgrp.clear();
    w.msrc_cap = 0;
    w.mtab = nullptr;
    w.msummary = nullptr;
    w.msync = nullptr;
    w.mdraw = nullptr;
}

// The out-degree bins top-down levels expand the frontier with: vertices above
// bfs_light_max go by chunks.  The push sweep's bins when the two limits agree,
// else the graph's BFS bins, built on first use for the current options.
static int bfs_bins(gp_graph *g, const BigBins *&b, cudaStream_t s) {
    if (g->opt.bfs_light_max == g->opt.push_light_max) {
        b = &g->push_bins;
        return GP_OK;
    }
    BigBins &own = g->bfs_bins;
    if (own.light_max != g->opt.bfs_light_max || own.chunk_edges != g->opt.chunk_edges || !own.rank) {
        const int st = build_bins(g, own, g->csr_off, g->opt.bfs_light_max, g->opt.chunk_edges, s);
        if (st != GP_OK) {
            own.mem.release(s);
            own.rank = nullptr;  // rebuilt by the next call
            return st;
        }
    }
    b = &own;
    return GP_OK;
}

static int ensure_bfs_work(gp_graph *g, const BigBins &bins, cudaStream_t s) {
    BfsWork &w = g->bfs;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    const size_t hcap = (size_t)std::max<int64_t>(bins.nchunks, 1);
    for (int i = 0; i < 2; ++i) {
        GP_TRY(w.mem.alloc(w.queue[i], n, s));
        GP_TRY(w.mem.alloc(w.hchunk[i], hcap, s));
    }
    for (int i = 0; i < 3; ++i) GP_TRY(w.mem.alloc(w.bits[i], words, s));
    GP_TRY(w.mem.alloc(w.unvis, words, s));
    GP_TRY(w.mem.alloc(w.nzin, words, s));
    if (g->n > 0) {
        k_nzin_bits<<<(int)std::min<size_t>((words + 255) / 256, 4096), 256, 0, s>>>(g->n, g->csc_off, w.nzin);
        GP_CUDA(cudaGetLastError());
    }
    BfsCtr *c = nullptr;
    GP_TRY(w.mem.alloc(c, 3, s));
    w.ctr = c;
    BfsLevelStat *st = nullptr;
    GP_TRY(w.mem.alloc(st, GP_BFS_MAX_LEVELS, s));
    w.stats = st;
    BfsSummary *sum = nullptr;
    GP_TRY(w.mem.alloc(sum, 1, s));
    w.summary = sum;
    GridSync *sync = nullptr;
    GP_TRY(w.mem.alloc(sync, 1, s));
    w.sync = sync;
    int8_t *d = nullptr;
    GP_TRY(w.mem.alloc(d, GP_BFS_MAX_LEVELS, s));
    w.dirs = d;
    w.dirs_cap = GP_BFS_MAX_LEVELS;
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persistent, BFS_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "BFS kernel does not fit on an SM");
    w.grid = per_sm * g->num_sms;
    GP_TRY(pinned_alloc(&w.ctr_host, BFS_HOST_BYTES));
    GP_CUDA(cudaEventCreateWithFlags(&w.done_ev, cudaEventDisableTiming));
    w.ready = true;
    return GP_OK;
}

// The fields of a search that depend only on the graph, its options, the
// top-down bins and the mode.
static void run_common(const gp_graph *g, const BigBins &bins, int mode, BfsRun &R) {
    memset(&R, 0, sizeof(R));
    R.base.n = g->n;
    R.base.csr_off = g->csr_off;
    R.base.csc_off = g->csc_off;
    R.base.csr_idx = g->csr_idx;
    R.base.csc_idx = g->csc_idx;
    R.base.push_rank = bins.rank;
    R.base.push_cstart = bins.cstart;
    R.base.push_chunks = bins.chunks;
    R.base.pull_chunks = g->pull_bins.chunks;
    R.base.pull_nchunks = g->pull_bins.nchunks;
    // every hub a lane defers has in-edge chunks: the probe is at least the pull light limit
    R.base.bu_probe = std::max<int64_t>(BU_PROBE, g->pull_bins.light_max);
    R.nzin = g->bfs.nzin;
    R.mode = mode;
    R.alpha = g->opt.bfs_alpha;
    R.beta = g->opt.bfs_beta;
    R.m = g->m;
}

static int bfs_run(const gp_graph *gc, int32_t src, int mode, const int8_t *dirs, int ndirs, int32_t *level_out,
                   int32_t *parent_out, gp_bfs_stats *stats, cudaStream_t s) {
    gp_graph *g = const_cast<gp_graph *>(gc);
    const int64_t n = g->n;
    if (src < 0 || (int64_t)src >= n) return set_error(GP_ERR_INVALID, "source %d outside [0, %lld)", src, (long long)n);
    if (!level_out) return set_error(GP_ERR_INVALID, "gp_bfs: level_out is NULL");
    const BigBins *bins = nullptr;
    GP_TRY(bfs_bins(g, bins, s));
    GP_TRY(ensure_bfs_work(g, *bins, s));
    BfsWork &w = g->bfs;
    char *h = (char *)w.ctr_host;
    BfsSummary *hs = (BfsSummary *)h;
    BfsLevelStat *hl = (BfsLevelStat *)(h + sizeof(BfsSummary));
    GridSync *hsync = (GridSync *)(h + sizeof(BfsSummary) + GP_BFS_MAX_LEVELS * sizeof(BfsLevelStat));
    if (w.pending) {  // the barrier status of the previous, asynchronous search
        GP_CUDA(cudaEventSynchronize(w.done_ev));
        w.pending = false;
        if (hsync->err) {
            hsync->err = 0;
            return set_error(GP_ERR_TIMEOUT, "BFS: a grid barrier wait ran out in the previous asynchronous search");
        }
    }
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
    BfsRun R;
    run_common(g, *bins, mode, R);
    R.base.level = level;
    R.base.parent = parent;
    for (int i = 0; i < 2; ++i) {
        R.queue[i] = w.queue[i];
        R.hchunk[i] = w.hchunk[i];
    }
    for (int i = 0; i < 3; ++i) R.bits[i] = w.bits[i];
    R.base.unvis = w.unvis;
    R.ctr = (BfsCtr *)w.ctr;
    R.src = src;
    R.stats = (BfsLevelStat *)w.stats;
    R.summary = (BfsSummary *)w.summary;
    R.sync = (GridSync *)w.sync;
    if (dirs) {
        // every given direction is used (level i takes dirs[i]), however deep the search
        if (ndirs > w.dirs_cap) {
            int8_t *d = nullptr;
            GP_TRY(w.mem.alloc(d, (size_t)ndirs, s));
            w.dirs = d;
            w.dirs_cap = ndirs;
        }
        GP_CUDA(cudaMemcpyAsync(w.dirs, dirs, (size_t)ndirs, cudaMemcpyHostToDevice, s));
        R.dirs = (const int8_t *)w.dirs;
        R.ndirs = ndirs;
    }
    GP_CUDA(cudaMemsetAsync(w.sync, 0, sizeof(GridSync), s));
    {
        ProfScope ps("bfs_persistent", s);
        void *args[] = {&R};
        GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs_persistent, dim3((unsigned)w.grid), dim3(BFS_THREADS), args,
                                            0, s));
    }
    if (!lvl_dev) GP_CUDA(cudaMemcpyAsync(level_out, level, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (!par_dev) GP_CUDA(cudaMemcpyAsync(parent_out, parent, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hsync, w.sync, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    if (!stats && lvl_dev && par_dev) {
        // nothing for the host to read: return without waiting; the barrier
        // status is checked by the next search on this graph
        GP_CUDA(cudaEventRecord(w.done_ev, s));
        w.pending = true;
        return GP_OK;
    }
    if (stats) {
        GP_CUDA(cudaMemcpyAsync(hs, w.summary, sizeof(BfsSummary), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaMemcpyAsync(hl, w.stats, GP_BFS_MAX_LEVELS * sizeof(BfsLevelStat), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaEventRecord(ev1, s));
        GP_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->levels = (int32_t)hs->levels;
        stats->switches = (int32_t)hs->switches;
        stats->reached = hs->reached;
        stats->edges_examined = hs->examined;
        stats->edges_reached = hs->edges_reached;
        stats->ms = ms;
        stats->init_ns = (int32_t)std::min<int64_t>(hs->init_ns, INT32_MAX);
        const int L = (int)std::min<int64_t>(hs->levels, GP_BFS_MAX_LEVELS);
        for (int i = 0; i < L; ++i) {
            stats->direction[i] = (int8_t)hl[i].direction;
            stats->frontier[i] = hl[i].frontier;
            stats->examined[i] = hl[i].examined;
            stats->level_ns[i] = hl[i].ns;
        }
    }
    GP_CUDA(cudaStreamSynchronize(s));
    if (hsync->err) return set_error(GP_ERR_TIMEOUT, "BFS: a grid barrier wait ran out");
    return GP_OK;
}

// ------------------------------------------------------------------ several searches per launch

// Byte layout of the staged tables: src[cap], level[cap], parent[cap].
struct MultiLayout {
    size_t src, level, parent, tab_bytes, summary, sync, host_bytes;
    MultiLayout(int groups, int cap) {
        auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
        src = 0;
        level = up(src + cap * sizeof(int32_t));
        parent = up(level + cap * sizeof(int32_t *));
        tab_bytes = up(parent + cap * sizeof(int32_t *));
        summary = tab_bytes;  // in the pinned block, the summaries and barrier words follow the tables
        sync = up(summary + cap * sizeof(BfsSummary));
        host_bytes = sync + groups * sizeof(GridSync);
    }
};

static int ensure_bfs_multi(gp_graph *g, const BigBins &bins, int groups, int nsrc, cudaStream_t s) {
    BfsWork &w = g->bfs;
    if ((int)w.mgrp.size() >= groups && w.msrc_cap >= nsrc) return GP_OK;
    groups = std::max<int>(groups, (int)w.mgrp.size());
    nsrc = std::max(nsrc, w.msrc_cap);
    w.mmem.release(s);
    pinned_free(w.mhost, w.mhost_bytes);
    w.mhost = nullptr;
    w.mhost_bytes = 0;
    w.mgrp.clear();
    w.msrc_cap = 0;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    const size_t hcap = (size_t)std::max<int64_t>(bins.nchunks, 1);
    std::vector<BfsWork::Group> grp((size_t)groups);
    for (auto &q : grp) {
        for (int i = 0; i < 2; ++i) {
            GP_TRY(w.mmem.alloc(q.queue[i], n, s));
            GP_TRY(w.mmem.alloc(q.hchunk[i], hcap, s));
        }
        for (int i = 0; i < 3; ++i) GP_TRY(w.mmem.alloc(q.bits[i], words, s));
        GP_TRY(w.mmem.alloc(q.unvis, words, s));
        BfsCtr *c = nullptr;
        GP_TRY(w.mmem.alloc(c, 3, s));
        q.ctr = c;
    }
    const MultiLayout lay(groups, nsrc);
    char *tab = nullptr;
    GP_TRY(w.mmem.alloc(tab, lay.tab_bytes, s));
    w.mtab = tab;
    BfsSummary *sum = nullptr;
    GP_TRY(w.mmem.alloc(sum, (size_t)nsrc, s));
    w.msummary = sum;
    GridSync *sync = nullptr;
    GP_TRY(w.mmem.alloc(sync, (size_t)groups, s));
    w.msync = sync;
    int32_t *draw = nullptr;
    GP_TRY(w.mmem.alloc(draw, 1 + 2 * (size_t)groups, s));
    w.mdraw = draw;
    GP_TRY(pinned_alloc(&w.mhost, lay.host_bytes));
    w.mhost_bytes = lay.host_bytes;
    if (!w.mdone_ev) GP_CUDA(cudaEventCreateWithFlags(&w.mdone_ev, cudaEventDisableTiming));
    w.mgrp = std::move(grp);
    w.msrc_cap = nsrc;
    return GP_OK;
}

// Groups when neither the caller nor the graph's bfs_groups option chooses.
constexpr int BFS_MULTI_GROUPS = 16;

static int bfs_multi(const gp_graph *gc, const int32_t *sources, int nsrc, int mode, int32_t *const *level_out,
                     int32_t *const *parent_out, int groups, gp_bfs_summary *summary, cudaStream_t s) {
    gp_graph *g = const_cast<gp_graph *>(gc);
    const int64_t n = g->n;
    for (int i = 0; i < nsrc; ++i) {
        if (sources[i] < 0 || (int64_t)sources[i] >= n)
            return set_error(GP_ERR_INVALID, "gp_bfs_multi: sources[%d] = %d outside [0, %lld)", i, sources[i], (long long)n);
        if (!level_out[i] || !is_device_ptr(level_out[i]))
            return set_error(GP_ERR_INVALID, "gp_bfs_multi: level_out[%d] is not device memory", i);
        if (parent_out && (!parent_out[i] || !is_device_ptr(parent_out[i])))
            return set_error(GP_ERR_INVALID, "gp_bfs_multi: parent_out[%d] is not device memory", i);
    }
    if (summary) memset(summary, 0, (size_t)nsrc * sizeof(gp_bfs_summary));
    if (nsrc == 0) return GP_OK;
    const BigBins *bins = nullptr;
    GP_TRY(bfs_bins(g, bins, s));
    GP_TRY(ensure_bfs_work(g, *bins, s));
    BfsWork &w = g->bfs;
    if (w.mpending) {  // the previous asynchronous call: its barrier status, and its staged tables are free again
        GP_CUDA(cudaEventSynchronize(w.mdone_ev));
        w.mpending = false;
        const MultiLayout old((int)w.mgrp.size(), w.msrc_cap);
        const GridSync *hs = (const GridSync *)((char *)w.mhost + old.sync);
        int err = 0;
        for (size_t i = 0; i < w.mgrp.size(); ++i) err |= hs[i].err;
        if (err) return set_error(GP_ERR_TIMEOUT, "BFS: a grid barrier wait ran out in the previous asynchronous gp_bfs_multi");
    }
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_multi, BFS_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "BFS kernel does not fit on an SM");
    const int blocks = per_sm * g->num_sms;
    int G = groups > 0 ? groups : g->opt.bfs_groups > 0 ? g->opt.bfs_groups : BFS_MULTI_GROUPS;
    G = std::max(1, std::min(std::min(std::min(G, nsrc), blocks), BFS_MULTI_MAX_GROUPS));
    const int bpg = blocks / G;
    GP_TRY(ensure_bfs_multi(g, *bins, G, nsrc, s));
    const int gcap = (int)w.mgrp.size();
    const MultiLayout lay(gcap, w.msrc_cap);
    char *h = (char *)w.mhost;
    char *d = (char *)w.mtab;
    BfsMulti M;
    memset(&M, 0, sizeof(M));
    for (int q = 0; q < G; ++q) {
        BfsRun &R = M.runs[q];
        run_common(g, *bins, mode, R);
        const BfsWork::Group &b = w.mgrp[(size_t)q];
        for (int i = 0; i < 2; ++i) {
            R.queue[i] = b.queue[i];
            R.hchunk[i] = b.hchunk[i];
        }
        for (int i = 0; i < 3; ++i) R.bits[i] = b.bits[i];
        R.base.unvis = b.unvis;
        R.ctr = (BfsCtr *)b.ctr;
        R.sync = (GridSync *)w.msync + q;
        R.stats = nullptr;  // per-level statistics are gp_bfs's
    }
    memcpy(h + lay.src, sources, (size_t)nsrc * sizeof(int32_t));
    memcpy(h + lay.level, level_out, (size_t)nsrc * sizeof(int32_t *));
    if (parent_out) memcpy(h + lay.parent, parent_out, (size_t)nsrc * sizeof(int32_t *));
    GP_CUDA(cudaMemcpyAsync(d, h, lay.tab_bytes, cudaMemcpyHostToDevice, s));
    GP_CUDA(cudaMemsetAsync(w.msync, 0, (size_t)G * sizeof(GridSync), s));
    GP_CUDA(cudaMemsetAsync(w.mdraw, 0, sizeof(int32_t), s));
    M.src = (const int32_t *)(d + lay.src);
    M.level = (int32_t *const *)(d + lay.level);
    M.parent = parent_out ? (int32_t *const *)(d + lay.parent) : nullptr;
    M.summary = (BfsSummary *)w.msummary;
    M.next = w.mdraw;
    M.slot = w.mdraw + 1;
    M.nsrc = nsrc;
    M.groups = G;
    M.bpg = bpg;
    {
        ProfScope ps("bfs_multi", s);
        void *args[] = {&M};
        GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs_multi, dim3((unsigned)(G * bpg)), dim3(BFS_THREADS), args, 0,
                                            s));
    }
    GridSync *hsync = (GridSync *)(h + lay.sync);
    GP_CUDA(cudaMemcpyAsync(hsync, w.msync, (size_t)G * sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    for (int q = G; q < gcap; ++q) hsync[q].err = 0;  // groups this call left unused
    if (!summary) {
        GP_CUDA(cudaEventRecord(w.mdone_ev, s));
        w.mpending = true;
        return GP_OK;
    }
    BfsSummary *hs = (BfsSummary *)(h + lay.summary);
    GP_CUDA(cudaMemcpyAsync(hs, w.msummary, (size_t)nsrc * sizeof(BfsSummary), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaStreamSynchronize(s));
    int err = 0;
    for (int q = 0; q < G; ++q) err |= hsync[q].err;
    if (err) return set_error(GP_ERR_TIMEOUT, "BFS: a grid barrier wait ran out in gp_bfs_multi");
    for (int i = 0; i < nsrc; ++i) {
        summary[i].levels = (int32_t)hs[i].levels;
        summary[i].switches = (int32_t)hs[i].switches;
        summary[i].reached = hs[i].reached;
        summary[i].edges_examined = hs[i].examined;
        summary[i].edges_reached = hs[i].edges_reached;
    }
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

extern "C" int gp_bfs_multi(const gp_graph *g, const int32_t *sources, int nsources, int mode, int32_t *const *level_out,
                            int32_t *const *parent_out, int groups, gp_bfs_summary *summary, void *stream) {
    clear_error();
    if (!g) return set_error(GP_ERR_INVALID, "gp_bfs_multi: graph is NULL");
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "bad mode %d", mode);
    if (nsources < 0) return set_error(GP_ERR_INVALID, "gp_bfs_multi: nsources %d < 0", nsources);
    if (groups < 0) return set_error(GP_ERR_INVALID, "gp_bfs_multi: groups %d < 0", groups);
    if (nsources > 0 && (!sources || !level_out)) return set_error(GP_ERR_INVALID, "gp_bfs_multi: sources or level_out is NULL");
    return bfs_multi(g, sources, nsources, mode, level_out, parent_out, groups, summary, (cudaStream_t)stream);
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
