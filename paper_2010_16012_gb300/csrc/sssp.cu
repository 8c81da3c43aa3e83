// sssp.cu -- single-source shortest paths by push- and pull-based
// Delta-Stepping (the paper's Section 3 listing), the whole search in one
// persistent cooperative launch.
//
// Epoch b handles bucket b: the vertices whose tentative distance lies in
// [b*delta, (b+1)*delta).  Its relaxation iterations repeat until no vertex of
// bucket b improved; the next epoch is the smallest non-empty bucket above b.
// Active in an iteration: every vertex of bucket b at the epoch's start, then
// the vertices of bucket b whose distance decreased in the previous iteration.
//   push (atomics): each active u relaxes its out-edges u->w with a 64-bit
//        atomicMin on w's key (distance bits high, predecessor low), so the key
//        ends at (shortest distance, smallest shortest-path predecessor)
//        whatever the order of relaxations (the paper's O(m l) CAS atomics);
//   pull: each vertex not settled in an earlier bucket takes the minimum of
//        dist(u) + W over its in-edges from active u; light vertices are
//        written by their own lane (no atomics), the in-lists of heavy ones are
//        split into warp chunks whose minima are combined with atomicMin.
// The direction of each iteration: push while the active set's out-edges are
// few against the in-edges of the unsettled vertices (m_a * alpha <= m_u),
// else pull -- the BFS switch rule applied per relaxation iteration, or a
// caller-given sequence.
// Vertex sets are bitmaps: the active set (a ring of three: current, next, and
// a spare cleared one iteration ahead), the vertices improved into a later
// bucket (pending), the current bucket's members (settled at the epoch's end)
// and the unsettled vertices with in-edges (pull candidates).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {

constexpr int SS_WARPS = 32;
constexpr int SS_THREADS = SS_WARPS * 32;
constexpr unsigned long long SS_NONE = ~0ull;  // key of an unreached vertex: (+inf, 0xffffffff)

__device__ __forceinline__ unsigned long long ss_pack(float d, uint32_t pred) {
    return ((unsigned long long)__float_as_uint(d) << 32) | pred;
}
__device__ __forceinline__ float ss_dist(unsigned long long k) {
    return k == SS_NONE ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(k >> 32));
}

struct SsCtr {
    unsigned long long nact;   // vertices of the active set this record describes
    unsigned long long mact;   // their out-degree sum
    unsigned long long npend;  // vertices newly pending (improved into a later bucket)
    unsigned long long h_len;  // push: heavy chunk ids queued by the iteration using this record
    unsigned long long examined;
    unsigned long long settled_in;  // in-degree of the vertices settled at an epoch end
    unsigned long long nb_key;      // epoch end: max of (~0 - bucket) over pending vertices; 0 = none
    unsigned long long pad;
};

struct SsIterStat {
    int32_t direction;
    int32_t ns;
    int64_t bucket;
    int64_t active;
    int64_t examined;
};

struct SsSummary {
    int64_t iterations, epochs, reached, examined, pushes, pulls, init_ns;
};

struct SsRun {
    int64_t n, m;
    const int64_t *csr_off, *csc_off;
    const int32_t *csr_idx, *csc_idx;
    const float *csr_w, *csc_w;  // nullptr: unit weights
    const int32_t *push_rank;    // [n] rank among vertices with out-degree > push light limit, -1 if light
    const int64_t *push_cstart;
    const Chunk *push_chunks;
    const int32_t *pull_rank;    // [n] rank among vertices with in-degree > pull light limit, -1 if light
    const Chunk *pull_chunks;
    int64_t pull_nchunks;
    unsigned long long *key;
    uint32_t *act[3];
    uint32_t *pend, *members, *unset;
    const uint32_t *nzin;
    int32_t *hq;
    SsCtr *ctr;  // [3]
    float delta, alpha;
    int32_t mode, src;
    const int8_t *dirs;
    int32_t ndirs;
    int64_t max_iters;
    float *dist_out;
    int32_t *pred_out;
    SsIterStat *stats;  // [GP_SSSP_MAX_ITERS]
    SsSummary *summary;
    GridSync *sync;
};

__device__ __forceinline__ unsigned long long ss_bucket(float d, float delta) {
    const float q = floorf(d / delta);
    return q < 4.0e18f ? (unsigned long long)q : 4000000000000000000ull;
}

__device__ __forceinline__ unsigned long long ss_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Edge indices and weights are streamed with the evict-first hint (__ldcs) so
// that they do not push the 8-byte keys, gathered at random, out of L2.

struct SsLocal {  // per-thread counter contributions of an iteration
    unsigned long long nact = 0, mact = 0, npend = 0, examined = 0;
};

// Offer (nd, u) to w, whose key was read as `seen`; on a strict distance
// improvement mark w active (same bucket) or pending (later bucket), counting
// first marks only.  Keys only decrease, so a `seen` that is not above the
// offer (a plain, possibly stale, read is never below the current key) means
// the atomic could not change anything.
__device__ __forceinline__ void ss_offer_seen(const SsRun &R, uint32_t *act_next, unsigned long long b, float nd,
                                              int32_t u, int32_t w, unsigned long long seen, SsLocal &c) {
    if (w == R.src) return;  // (0, src) is final; a zero-weight edge into it must not change its predecessor
    const unsigned long long cand = ss_pack(nd, (uint32_t)u);
    if (cand >= seen) return;
    const unsigned long long old = atomicMin(R.key + w, cand);
    if (!(nd < ss_dist(old))) return;
    const uint32_t bit = 1u << (w & 31);
    if (ss_bucket(nd, R.delta) == b) {
        atomicOr(R.members + (w >> 5), bit);
        if (!(atomicOr(act_next + (w >> 5), bit) & bit)) {
            c.nact += 1;
            c.mact += (unsigned long long)(R.csr_off[w + 1] - R.csr_off[w]);
        }
    } else if (!(atomicOr(R.pend + (w >> 5), bit) & bit)) {
        c.npend += 1;
    }
}

__device__ __forceinline__ void ss_offer(const SsRun &R, uint32_t *act_next, unsigned long long b, float nd, int32_t u,
                                         int32_t w, SsLocal &c) {
    ss_offer_seen(R, act_next, b, nd, u, w, R.key[w], c);
}

__device__ void ss_flush(SsCtr *nx, const SsLocal &c) {
    __shared__ unsigned long long sm[32];
    const unsigned long long a = block_sum(c.nact, sm), b = block_sum(c.mact, sm), p = block_sum(c.npend, sm),
                             e = block_sum(c.examined, sm);
    if (threadIdx.x == 0) {
        if (a) atomicAdd(&nx->nact, a);
        if (b) atomicAdd(&nx->mact, b);
        if (p) atomicAdd(&nx->npend, p);
        if (e) atomicAdd(&nx->examined, e);
    }
}

// Push, phase A: a warp ranks the active vertices of 32 bitmap words; light
// ones relax their out-edges as one merged edge stream over the warp, heavy
// ones queue their chunk ids for phase B.
__device__ void ss_push_a(const SsRun &R, const uint32_t *act_cur, uint32_t *act_next, SsCtr *cur,
                          unsigned long long b, SsLocal &c) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwords = (R.n + 31) >> 5;
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t word = wd < nwords ? act_cur[wd] : 0u;
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
            int32_t u = -1;
            int deg = 0;
            int64_t eb = 0;
            float du = 0.f;
            if (id < total) {
                u = (int32_t)((base + k) * 32 + nth_set_bit(kw, id - kex));
                const int32_t rk = R.push_rank[u];
                if (rk >= 0) {  // heavy: its chunks go to phase B
                    const int64_t c0 = R.push_cstart[rk], c1 = R.push_cstart[rk + 1];
                    const unsigned long long pos = atomicAdd(&cur->h_len, (unsigned long long)(c1 - c0));
                    for (int64_t j = c0; j < c1; ++j) R.hq[pos + (j - c0)] = (int32_t)j;
                } else {
                    eb = R.csr_off[u];
                    deg = (int)(R.csr_off[u + 1] - eb);
                    du = ss_dist(R.key[u]);
                }
            }
            const int dincl = warp_incl_scan(deg);
            const int dexcl = dincl - deg;
            const int E = __shfl_sync(FULL, dincl, 31);
            for (int eb0 = 0; eb0 < E; eb0 += 32) {
                const int eid = eb0 + lane;
                int o = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int ek = __shfl_sync(FULL, dexcl, o + st);
                    if (ek <= eid) o += st;
                }
                const int64_t ob = __shfl_sync(FULL, eb, o);
                const int oex = __shfl_sync(FULL, dexcl, o);
                const int32_t ou = __shfl_sync(FULL, u, o);
                const float odu = __shfl_sync(FULL, du, o);
                if (eid < E) {
                    const int64_t pos = ob + (eid - oex);
                    const int32_t w = __ldcs(R.csr_idx + pos);
                    const float wt = R.csr_w ? __ldcs(R.csr_w + pos) : 1.f;
                    ++c.examined;
                    ss_offer(R, act_next, b, odu + wt, ou, w, c);
                }
            }
        }
    }
}

// Push, phase B: the queued chunks of heavy active vertices, one warp each.
__device__ void ss_push_b(const SsRun &R, uint32_t *act_next, int64_t h_len, unsigned long long b, SsLocal &c) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int U = 4;  // relaxations in flight per lane
    for (int64_t j = warp; j < h_len; j += nwarps) {
        const Chunk ch = R.push_chunks[R.hq[j]];
        const float du = ss_dist(R.key[ch.v]);
        for (int i0 = lane; i0 < ch.len; i0 += 32 * U) {
            int32_t w[U];
            float wt[U];
            unsigned long long seen[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int i = i0 + 32 * q;
                w[q] = i < ch.len ? __ldcs(R.csr_idx + ch.beg + i) : -1;
                wt[q] = i < ch.len && R.csr_w ? __ldcs(R.csr_w + ch.beg + i) : 1.f;
            }
#pragma unroll
            for (int q = 0; q < U; ++q) seen[q] = w[q] >= 0 ? R.key[w[q]] : 0ull;
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (w[q] >= 0) {
                    ++c.examined;
                    ss_offer_seen(R, act_next, b, du + wt[q], ch.v, w[q], seen[q], c);
                }
        }
    }
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULL, v, o);
        v = t < v ? t : v;
    }
    return v;
}

// Pull: heavy unsettled vertices by chunks (warp minimum, atomicMin into the
// key), then the light unsettled vertices, one lane each over all in-edges.
__device__ void ss_pull(const SsRun &R, const uint32_t *act_cur, uint32_t *act_next, unsigned long long b, SsLocal &c) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < R.pull_nchunks; j += nwarps) {
        const Chunk ch = R.pull_chunks[j];
        if (!((R.unset[ch.v >> 5] >> (ch.v & 31)) & 1u) || ch.v == R.src) continue;  // uniform: settled
        unsigned long long best = SS_NONE;
        for (int i = lane; i < ch.len; i += 32) {
            const int32_t u = __ldcs(R.csc_idx + ch.beg + i);
            ++c.examined;
            if ((act_cur[u >> 5] >> (u & 31)) & 1u) {
                const float wt = R.csc_w ? __ldcs(R.csc_w + ch.beg + i) : 1.f;
                const unsigned long long cand = ss_pack(ss_dist(R.key[u]) + wt, (uint32_t)u);
                best = cand < best ? cand : best;
            }
        }
        best = warp_min_u64(best);
        if (lane == 0 && best != SS_NONE) ss_offer(R, act_next, b, ss_dist(best), (int32_t)(uint32_t)best, ch.v, c);
    }
    const int64_t nwords = (R.n + 31) >> 5;
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t word = wd < nwords ? R.unset[wd] : 0u;
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
            if (id >= total) continue;
            const int32_t v = (int32_t)((base + k) * 32 + nth_set_bit(kw, id - kex));
            if (R.pull_rank[v] >= 0 || v == R.src) continue;  // heavy: done by chunks
            const unsigned long long own = R.key[v];
            unsigned long long best = own;
            const int64_t e = R.csc_off[v + 1];
            for (int64_t p = R.csc_off[v]; p < e; ++p) {
                const int32_t u = __ldcs(R.csc_idx + p);
                ++c.examined;
                if ((act_cur[u >> 5] >> (u & 31)) & 1u) {
                    const float wt = R.csc_w ? __ldcs(R.csc_w + p) : 1.f;
                    const unsigned long long cand = ss_pack(ss_dist(R.key[u]) + wt, (uint32_t)u);
                    best = cand < best ? cand : best;
                }
            }
            if (best < own) {
                R.key[v] = best;  // the vertex's own lane: no other writer this iteration
                const float nd = ss_dist(best);
                if (nd < ss_dist(own)) {
                    const uint32_t bit = 1u << (v & 31);
                    if (ss_bucket(nd, R.delta) == b) {
                        atomicOr(R.members + (v >> 5), bit);
                        if (!(atomicOr(act_next + (v >> 5), bit) & bit)) {
                            c.nact += 1;
                            c.mact += (unsigned long long)(R.csr_off[v + 1] - R.csr_off[v]);
                        }
                    } else if (!(atomicOr(R.pend + (v >> 5), bit) & bit)) {
                        c.npend += 1;
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(SS_THREADS) k_sssp_persistent(SsRun R) {
    const unsigned long long t_start = ss_now();
    const int64_t n = R.n;
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t nwords = (n + 31) >> 5;
    constexpr int CW = (int)(sizeof(SsCtr) / sizeof(unsigned long long));
    const int32_t src = R.src;
    const int64_t sw = src >> 5;
    const uint32_t sbit = 1u << (src & 31);
    // keys, bitmaps and counters for the first epoch: bucket 0 = {src}
    for (int64_t v = gthread; v < n; v += nthreads) R.key[v] = v == src ? ss_pack(0.f, (uint32_t)src) : SS_NONE;
    for (int64_t i = gthread; i < nwords; i += nthreads) {
        R.act[0][i] = i == sw ? sbit : 0u;
        R.act[1][i] = 0u;
        R.act[2][i] = 0u;
        R.pend[i] = 0u;
        R.members[i] = i == sw ? sbit : 0u;
        R.unset[i] = R.nzin[i];
    }
    if (gthread < 3 * CW) {
        unsigned long long val = 0;
        if (gthread == 0) val = 1;                                                              // nact
        if (gthread == 1) val = (unsigned long long)(R.csr_off[src + 1] - R.csr_off[src]);      // mact
        ((unsigned long long *)R.ctr)[gthread] = val;
    }
    if (!grid_sync(R.sync, gridDim.x)) return;
    unsigned long long t_iter = ss_now();
    const unsigned long long t_init = t_iter - t_start;
    volatile SsCtr *vc = (volatile SsCtr *)R.ctr;
    __shared__ unsigned long long s_c[CW];
    auto read_ctr = [&](int slot) {  // one thread per block reads, the block shares
        if (threadIdx.x < CW) s_c[threadIdx.x] = ((volatile unsigned long long *)(vc + slot))[threadIdx.x];
        __syncthreads();
    };
    unsigned long long b = 0;
    long long m_unset = (long long)R.m;
    int64_t it = 0, epochs = 1, examined = 0, pushes = 0, pulls = 0;
    read_ctr(0);
    unsigned long long nact = s_c[0], mact = s_c[1];
    while (true) {
        if (nact == 0) {
            // epoch end: settle bucket b, find the smallest pending bucket above b
            const int cur = (int)(it % 3), scratch = (int)((it + 1) % 3);  // scratch: zeroed one iteration ago
            unsigned long long best = 0, settled_in = 0;
            for (int64_t i = gthread; i < nwords; i += nthreads) {
                const uint32_t mw = R.members[i];
                if (mw) {
                    R.unset[i] &= ~mw;
                    R.members[i] = 0u;
                    for (uint32_t x = mw; x; x &= x - 1) {
                        const int64_t v = i * 32 + (__ffs(x) - 1);
                        settled_in += (unsigned long long)(R.csc_off[v + 1] - R.csc_off[v]);
                    }
                }
                for (uint32_t x = R.pend[i]; x; x &= x - 1) {
                    const int64_t v = i * 32 + (__ffs(x) - 1);
                    const unsigned long long bv = ss_bucket(ss_dist(R.key[v]), R.delta);
                    if (bv > b) {
                        const unsigned long long kb = ~0ull - bv;
                        best = kb > best ? kb : best;
                    }
                }
            }
            {
                __shared__ unsigned long long sm[32];
                settled_in = block_sum(settled_in, sm);
                unsigned long long wmax = best;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long t = __shfl_xor_sync(FULL, wmax, o);
                    wmax = t > wmax ? t : wmax;
                }
                __shared__ unsigned long long smax[32];
                if (lane_id() == 0) smax[threadIdx.x >> 5] = wmax;
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned long long mx = 0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = smax[w] > mx ? smax[w] : mx;
                    if (mx) atomicMax(&R.ctr[scratch].nb_key, mx);
                    if (settled_in) atomicAdd(&R.ctr[scratch].settled_in, settled_in);
                }
            }
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr(scratch);
            m_unset -= (long long)s_c[5];
            if (s_c[6] == 0) break;  // nothing pending: done
            const unsigned long long nb = ~0ull - s_c[6];
            // the pending vertices of bucket nb become the active set; stale ones
            // (improved into an earlier, now settled bucket) leave the pending set
            SsLocal c;
            for (int64_t i = gthread; i < nwords; i += nthreads) {
                const uint32_t pw = R.pend[i];
                if (!pw) continue;
                uint32_t moved = 0, stale = 0;
                for (uint32_t x = pw; x; x &= x - 1) {
                    const int bit = __ffs(x) - 1;
                    const int64_t v = i * 32 + bit;
                    const unsigned long long bv = ss_bucket(ss_dist(R.key[v]), R.delta);
                    if (bv == nb) {
                        moved |= 1u << bit;
                        c.nact += 1;
                        c.mact += (unsigned long long)(R.csr_off[v + 1] - R.csr_off[v]);
                    } else if (bv <= b) {
                        stale |= 1u << bit;
                    }
                }
                R.pend[i] = pw & ~(moved | stale);
                if (moved) {
                    R.act[cur][i] |= moved;
                    R.members[i] |= moved;
                }
            }
            ss_flush(R.ctr + cur, c);
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr(cur);
            nact = s_c[0];
            mact = s_c[1];
            b = nb;
            ++epochs;
            continue;
        }
        if (it >= R.max_iters) {  // cannot happen with non-negative weights; guards the loop
            if (gthread == 0) atomicExch(&R.sync->err, 2);
            return;
        }
        int dir;
        if (R.dirs) {
            dir = R.dirs[it < R.ndirs ? it : R.ndirs - 1];
        } else if (R.mode == GP_PUSH || R.mode == GP_PULL) {
            dir = R.mode;
        } else {
            dir = ((float)mact * R.alpha > (float)(m_unset > 0 ? m_unset : 0)) ? GP_PULL : GP_PUSH;
        }
        const int cur = (int)(it % 3), nxt = (int)((it + 1) % 3), spare = (int)((it + 2) % 3);
        const uint32_t *act_cur = R.act[cur];
        uint32_t *act_next = R.act[nxt];
        if (gthread < CW) ((unsigned long long *)(R.ctr + spare))[gthread] = 0;
        for (int64_t i = gthread; i < nwords; i += nthreads) R.act[spare][i] = 0u;
        SsLocal c;
        if (dir == GP_PUSH) {
            ss_push_a(R, act_cur, act_next, R.ctr + cur, b, c);
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr(cur);
            const int64_t h_len = (int64_t)s_c[3];
            if (h_len > 0) {
                ss_push_b(R, act_next, h_len, b, c);
            }
            ++pushes;
        } else {
            ss_pull(R, act_cur, act_next, b, c);
            ++pulls;
        }
        ss_flush(R.ctr + nxt, c);
        if (!grid_sync(R.sync, gridDim.x)) return;
        read_ctr(nxt);
        if (gthread == 0 && it < GP_SSSP_MAX_ITERS) {
            const unsigned long long t = ss_now();
            R.stats[it].direction = dir;
            R.stats[it].ns = (int32_t)min(t - t_iter, 0x7fffffffull);
            R.stats[it].bucket = (int64_t)b;
            R.stats[it].active = (int64_t)nact;
            R.stats[it].examined = (int64_t)s_c[4];
            t_iter = t;
        }
        examined += (int64_t)s_c[4];
        nact = s_c[0];
        mact = s_c[1];
        ++it;
    }
    // outputs
    unsigned long long reached = 0;
    for (int64_t v = gthread; v < n; v += nthreads) {
        const unsigned long long k = R.key[v];
        R.dist_out[v] = ss_dist(k);
        if (R.pred_out) R.pred_out[v] = k == SS_NONE ? -1 : (int32_t)(uint32_t)k;
        reached += k != SS_NONE;
    }
    __shared__ unsigned long long sm2[32];
    reached = block_sum(reached, sm2);
    if (threadIdx.x == 0 && reached) atomicAdd((unsigned long long *)&R.summary->reached, reached);
    if (gthread == 0) {
        R.summary->iterations = it;
        R.summary->epochs = epochs;
        R.summary->examined = examined;
        R.summary->pushes = pushes;
        R.summary->pulls = pulls;
        R.summary->init_ns = (int64_t)t_init;
    }
}

// Bit v of word v/32: vertex v has in-edges.
__global__ void k_ss_nzin(int64_t n, const int64_t *csc_off, uint32_t *bits) {
    const int64_t nwords = (n + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < nwords; wd += stride) {
        uint32_t word = 0;
        const int64_t v0 = wd * 32, v1 = min(n, v0 + 32);
        for (int64_t v = v0; v < v1; ++v)
            if (csc_off[v + 1] > csc_off[v]) word |= 1u << (v - v0);
        bits[wd] = word;
    }
}

// Flag (bit 0) when any weight is negative or not a number.
__global__ void k_ss_check_weights(int64_t m, const float *w, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int b = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) b |= !(w[e] >= 0.f);
    if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}

}  // namespace gp

// ------------------------------------------------------------------ driver

using namespace gp;

struct gp_sssp_work {
    bool ready = false;
    unsigned long long *key = nullptr;
    uint32_t *act[3] = {nullptr, nullptr, nullptr};
    uint32_t *pend = nullptr, *members = nullptr, *unset = nullptr, *nzin = nullptr;
    int32_t *hq = nullptr;
    SsCtr *ctr = nullptr;
    SsIterStat *stats = nullptr;
    SsSummary *summary = nullptr;
    GridSync *sync = nullptr;
    int8_t *dirs = nullptr;
    float *dist_dev = nullptr;
    int32_t *pred_dev = nullptr;
    void *host = nullptr;  // pinned: summary, iteration stats, barrier word
    int grid = 0;
    int weights_ok = -1;  // -1 unknown, 0 negative or NaN weight, 1 checked
    cudaEvent_t done_ev = nullptr;  // end of the last asynchronous search
    bool pending = false;           // its barrier status not yet checked
    Arena mem;
};

namespace gp {

// host mirror: summary, per-iteration statistics, barrier status
constexpr size_t SS_HOST_BYTES = sizeof(SsSummary) + GP_SSSP_MAX_ITERS * sizeof(SsIterStat) + sizeof(GridSync);

void release_sssp_work(gp_graph *g, cudaStream_t s) {
    if (!g->sssp) return;
    if (g->sssp->done_ev) {
        cudaEventSynchronize(g->sssp->done_ev);
        cudaEventDestroy(g->sssp->done_ev);
    }
    pinned_free(g->sssp->host, SS_HOST_BYTES);
    g->sssp->mem.release(s);
    delete g->sssp;
    g->sssp = nullptr;
}

}  // namespace gp

static int ensure_sssp_work(gp_graph *g, cudaStream_t s) {
    if (!g->sssp) g->sssp = new gp_sssp_work();
    gp_sssp_work &w = *g->sssp;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    GP_TRY(w.mem.alloc(w.key, n, s));
    for (int i = 0; i < 3; ++i) GP_TRY(w.mem.alloc(w.act[i], words, s));
    GP_TRY(w.mem.alloc(w.pend, words, s));
    GP_TRY(w.mem.alloc(w.members, words, s));
    GP_TRY(w.mem.alloc(w.unset, words, s));
    GP_TRY(w.mem.alloc(w.nzin, words, s));
    GP_TRY(w.mem.alloc(w.hq, (size_t)std::max<int64_t>(g->push_bins.nchunks, 1), s));
    GP_TRY(w.mem.alloc(w.ctr, 3, s));
    GP_TRY(w.mem.alloc(w.stats, GP_SSSP_MAX_ITERS, s));
    GP_TRY(w.mem.alloc(w.summary, 1, s));
    GP_TRY(w.mem.alloc(w.sync, 1, s));
    GP_TRY(w.mem.alloc(w.dirs, GP_SSSP_MAX_ITERS, s));
    if (g->n > 0) {
        k_ss_nzin<<<(int)std::min<size_t>((words + 255) / 256, 4096), 256, 0, s>>>(g->n, g->csc_off, w.nzin);
        GP_CUDA(cudaGetLastError());
    }
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp_persistent, SS_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "SSSP kernel does not fit on an SM");
    w.grid = per_sm * g->num_sms;
    GP_TRY(pinned_alloc(&w.host, SS_HOST_BYTES));
    GP_CUDA(cudaEventCreateWithFlags(&w.done_ev, cudaEventDisableTiming));
    w.ready = true;
    return GP_OK;
}

static int sssp_check_weights(gp_graph *g, cudaStream_t s) {
    gp_sssp_work &w = *g->sssp;
    if (w.weights_ok >= 0) return w.weights_ok ? GP_OK : set_error(GP_ERR_INVALID, "gp_sssp: negative or NaN edge weight");
    if (!g->csr_w || g->m == 0) {
        w.weights_ok = 1;
        return GP_OK;
    }
    Arena tmp;
    int *bad = nullptr;
    GP_TRY(tmp.alloc(bad, 1, s));
    int hb = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    const int blocks = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)g->num_sms * 8);
    if (e == cudaSuccess) {
        k_ss_check_weights<<<blocks, 256, 0, s>>>(g->m, g->csr_w, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    tmp.release(s);
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_sssp: %s", cudaGetErrorString(e));
    w.weights_ok = hb ? 0 : 1;
    return hb ? set_error(GP_ERR_INVALID, "gp_sssp: negative or NaN edge weight") : GP_OK;
}

extern "C" int gp_sssp(const gp_graph *gc, int32_t src, float delta, int mode, const int8_t *dirs, int ndirs,
                       float *dist_out, int32_t *pred_out, gp_sssp_stats *stats, void *stream) {
    clear_error();
    if (!gc) return set_error(GP_ERR_INVALID, "gp_sssp: graph is NULL");
    gp_graph *g = const_cast<gp_graph *>(gc);
    cudaStream_t s = (cudaStream_t)stream;
    if (src < 0 || (int64_t)src >= g->n) return set_error(GP_ERR_INVALID, "gp_sssp: source %d outside [0, %lld)", src, (long long)g->n);
    if (!(delta > 0.f) || !std::isfinite(delta)) return set_error(GP_ERR_INVALID, "gp_sssp: delta %g is not a positive number", (double)delta);
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "gp_sssp: bad mode %d", mode);
    if (dirs && ndirs < 1) return set_error(GP_ERR_INVALID, "gp_sssp: dirs given with ndirs < 1");
    for (int i = 0; dirs && i < ndirs; ++i)
        if (dirs[i] != GP_PUSH && dirs[i] != GP_PULL) return set_error(GP_ERR_INVALID, "gp_sssp: dirs[%d] = %d", i, dirs[i]);
    if (!dist_out) return set_error(GP_ERR_INVALID, "gp_sssp: dist_out is NULL");
    if (g->csr_w && !g->csc_w) return set_error(GP_ERR_INVALID, "gp_sssp: weighted graph without in-edge weights");
    GP_TRY(ensure_sssp_work(g, s));
    gp_sssp_work &w = *g->sssp;
    GP_TRY(sssp_check_weights(g, s));
    char *h = (char *)w.host;
    SsSummary *hs = (SsSummary *)h;
    SsIterStat *hl = (SsIterStat *)(h + sizeof(SsSummary));
    GridSync *hsync = (GridSync *)(h + sizeof(SsSummary) + GP_SSSP_MAX_ITERS * sizeof(SsIterStat));
    if (w.pending) {  // the barrier status of the previous, asynchronous search
        GP_CUDA(cudaEventSynchronize(w.done_ev));
        w.pending = false;
        const int err = hsync->err;
        hsync->err = 0;
        if (err == 2) return set_error(GP_ERR_INVALID, "gp_sssp: iteration limit reached in the previous asynchronous search");
        if (err) return set_error(GP_ERR_TIMEOUT, "gp_sssp: a grid barrier wait ran out in the previous asynchronous search");
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    const int64_t n = g->n;
    float *dist = dist_out;
    int32_t *pred = pred_out;
    const bool dist_dev = is_device_ptr(dist_out), pred_dev = !pred_out || is_device_ptr(pred_out);
    if (!dist_dev) {
        if (!w.dist_dev) GP_TRY(w.mem.alloc(w.dist_dev, (size_t)n, s));
        dist = w.dist_dev;
    }
    if (!pred_dev) {
        if (!w.pred_dev) GP_TRY(w.mem.alloc(w.pred_dev, (size_t)n, s));
        pred = w.pred_dev;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    SsRun R;
    memset(&R, 0, sizeof(R));
    R.n = n;
    R.m = g->m;
    R.csr_off = g->csr_off;
    R.csc_off = g->csc_off;
    R.csr_idx = g->csr_idx;
    R.csc_idx = g->csc_idx;
    R.csr_w = g->csr_w;
    R.csc_w = g->csc_w;
    R.push_rank = g->push_bins.rank;
    R.push_cstart = g->push_bins.cstart;
    R.push_chunks = g->push_bins.chunks;
    R.pull_rank = g->pull_bins.rank;
    R.pull_chunks = g->pull_bins.chunks;
    R.pull_nchunks = g->pull_bins.nchunks;
    R.key = w.key;
    for (int i = 0; i < 3; ++i) R.act[i] = w.act[i];
    R.pend = w.pend;
    R.members = w.members;
    R.unset = w.unset;
    R.nzin = w.nzin;
    R.hq = w.hq;
    R.ctr = w.ctr;
    R.delta = delta;
    R.alpha = g->opt.sssp_alpha;
    R.mode = mode;
    R.src = src;
    // each epoch needs at most n + 1 iterations and there are at most n epochs:
    // the guard only catches a defect, it is never reached on valid input
    R.max_iters = n < (int64_t)1 << 30 ? (n + 2) * (n + 2) : ((int64_t)1 << 62);
    R.dist_out = dist;
    R.pred_out = pred;
    R.stats = w.stats;
    R.summary = w.summary;
    R.sync = w.sync;
    if (dirs) {
        const int nd = std::min(ndirs, GP_SSSP_MAX_ITERS);
        GP_CUDA(cudaMemcpyAsync(w.dirs, dirs, nd, cudaMemcpyHostToDevice, s));
        R.dirs = w.dirs;
        R.ndirs = nd;
    }
    GP_CUDA(cudaMemsetAsync(w.sync, 0, sizeof(GridSync), s));
    GP_CUDA(cudaMemsetAsync(w.summary, 0, sizeof(SsSummary), s));
    {
        ProfScope ps("sssp_persistent", s);
        void *args[] = {&R};
        GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_sssp_persistent, dim3((unsigned)w.grid), dim3(SS_THREADS),
                                            args, 0, s));
    }
    if (!dist_dev) GP_CUDA(cudaMemcpyAsync(dist_out, dist, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (!pred_dev) GP_CUDA(cudaMemcpyAsync(pred_out, pred, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hsync, w.sync, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    if (!stats && dist_dev && pred_dev) {
        // nothing for the host to read: return without waiting; the barrier
        // status is checked by the next search on this graph
        GP_CUDA(cudaEventRecord(w.done_ev, s));
        w.pending = true;
        return GP_OK;
    }
    if (stats) {
        GP_CUDA(cudaMemcpyAsync(hs, w.summary, sizeof(SsSummary), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaMemcpyAsync(hl, w.stats, GP_SSSP_MAX_ITERS * sizeof(SsIterStat), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaEventRecord(ev1, s));
    }
    GP_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->iterations = (int32_t)hs->iterations;
        stats->epochs = (int32_t)hs->epochs;
        stats->reached = hs->reached;
        stats->edges_examined = hs->examined;
        stats->pushes = (int32_t)hs->pushes;
        stats->pulls = (int32_t)hs->pulls;
        stats->ms = ms;
        stats->init_ns = (int32_t)std::min<int64_t>(hs->init_ns, INT32_MAX);
        const int L = (int)std::min<int64_t>(hs->iterations, GP_SSSP_MAX_ITERS);
        for (int i = 0; i < L; ++i) {
            stats->direction[i] = (int8_t)hl[i].direction;
            stats->bucket[i] = hl[i].bucket;
            stats->active[i] = hl[i].active;
            stats->examined[i] = hl[i].examined;
            stats->iter_ns[i] = hl[i].ns;
        }
    }
    if (hsync->err == 2) return set_error(GP_ERR_INVALID, "gp_sssp: iteration limit reached");
    if (hsync->err) return set_error(GP_ERR_TIMEOUT, "gp_sssp: a grid barrier wait ran out");
    return GP_OK;
}
