// bc.cu -- betweenness centrality by Brandes' scheme with push- and
// pull-based steps (the paper's Section 3 BC listing), a batch of sources per
// persistent cooperative launch.
//
// Forward phase of a source s: a level-synchronous BFS that counts shortest
// paths, sigma(w) = sum of sigma(u) over the in-neighbours u one level closer.
//   push: every vertex u of the frontier Q_l walks its out-edges; an unvisited
//         w is claimed by a CAS on its level, and every w at level l+1 gets
//         sigma(u) added with an FP64 atomic;
//   pull: every unvisited vertex sums sigma(u) over its in-edges from Q_l (no
//         early exit: each predecessor counts), written by its own lane; hub
//         in-lists are split into warp chunks whose sums are added atomically.
// Backward phase, from the deepest level up.  With
//   S(u) = sum over successors w (one level further) of c(w),
//   c(w) = (1 + delta(w)) / sigma(w),
// the dependency is delta(u) = sigma(u) S(u) and c(u) = 1/sigma(u) + S(u): one
// division per vertex and one addition per shortest-path DAG edge.  Step l
// finishes the vertices of Q_l (bc += sigma S) and passes their coefficients to
// Q_{l-1}:
//   push: each w of Q_l adds c(w) to S(u) of its in-neighbours u in Q_{l-1}
//         (FP64 atomics), in the same pass that finishes w;
//   pull: Q_l is finished (c stored) first; after a grid barrier each u of
//         Q_{l-1} sums c(w) over its out-neighbours in Q_l.
// Direction per step: pull when the push side's edges times alpha exceed the
// pull side's, or a caller-given sequence.
//
// Level sets are bitmaps in a ring of four (level x in slot x mod 4): a
// forward step sets the bits of the vertices it claims, a compaction pass then
// appends them to the visit order `order` (so Q_l is a contiguous range) and
// counts their degrees; the backward phase rebuilds Q_{l-2}'s bitmap from the
// order one step ahead and clears the slot of Q_{l+1}.  Three tiers by the
// degree of the list a step walks, so that no warp gets far more edges than
// another: light lists (<= BC_LIGHT) are summed one lane per vertex (pull) or
// walked 32 vertices per warp as one merged edge stream (push, four 32-edge
// windows in flight); medium lists (<= BC_HUB) by groups of BC_G lanes, or a
// warp each when a level has few of them, from per-level lists the compaction
// writes; hub lists are cut into chunks that every step scans, taking those
// whose vertex is in the step's set.  Per-step counters are deltas in a ring of
// three records (the next one zeroed a step ahead); every block keeps the
// cumulative values.  Per vertex: level (int32), sigma, S and c (FP64), bc
// (FP64); all reset for the visited vertices after each source.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "gp_internal.cuh"

namespace gp {

constexpr int BC_THREADS = 512;
constexpr int64_t BC_BATCH = 4096;  // sources per launch
constexpr int BC_W = 4;             // 32-edge windows of a merged stream in flight per lane
constexpr int BC_WL = 8;            // list entries in flight per lane (chunks, medium and light lists)
constexpr int32_t BC_LIGHT = 32;    // lists up to this: merged warp streams
constexpr int32_t BC_HUB = 1024;    // lists above this: chunks; between: a warp each
constexpr int32_t BC_CHUNK = 256;   // edges per hub chunk
constexpr int BC_G = 8;               // lanes per medium list (32 / BC_G lists per warp at once)
constexpr int BC_HOT = 256;           // backward push: targets summed in shared memory per block

struct BcCtr {  // what one step added
    unsigned long long tail;     // vertices appended to the visit order
    unsigned long long med_out;  // ... of them with a medium out-list
    unsigned long long med_in;   // ... of them with a medium in-list
    unsigned long long in;       // in-degree sum of the appended vertices
    unsigned long long out;      // out-degree sum of the appended vertices
    unsigned long long examined;
    unsigned long long pad[2];
};

struct BcCum {  // cumulative counters of a source: the state at a level's start
    long long start, med_out, med_in, in, out;
};

struct BcStepStat {
    int32_t direction;
    int32_t phase;
    int32_t level;
    int32_t ns;
    int64_t frontier;
    int64_t examined;
};

struct BcSummary {
    int64_t levels, reached, examined, pushes, pulls, steps;
};

struct BcRun {
    int64_t n, m;
    const int64_t *csr_off, *csc_off;
    const int32_t *csr_idx, *csc_idx;
    const Chunk *hub_out, *hub_in;  // chunks of the lists above BC_HUB
    int64_t n_hub_out, n_hub_in;
    const int32_t *csc_enc;         // CSC indices, the BC_HOT largest out-degrees as HOT_BIT | slot
    const int32_t *hot_id;          // [nhot] vertex of each slot
    int32_t nhot;
    const int32_t *med_in_all;      // every vertex with a medium in-list
    int64_t n_med_in_all;
    int32_t *dist;
    double *sigma, *S, *coef, *bc;
    int32_t *order;             // visit order, level by level
    int32_t *med_out, *med_in;  // the visited vertices with medium lists, level by level
    uint32_t *unvis;
    const uint32_t *nzin;
    uint32_t *lbits[4];  // level bitmaps, level x in lbits[x & 3]
    BcCum *lev;          // [n + 2]
    BcCtr *ctr;          // [3]
    const int32_t *sources;
    int64_t nsrc;
    int32_t mode, ndirs;
    const int8_t *dirs;
    float alpha;
    int32_t record;  // record the first source's steps
    BcStepStat *stats;
    BcSummary *summary;
    GridSync *sync;
};

struct BcLocal {  // per-thread contributions of a step
    unsigned long long in = 0, out = 0, examined = 0;
};

__device__ __forceinline__ unsigned long long bc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool bit_of(const uint32_t *bits, int32_t v) { return (bits[v >> 5] >> (v & 31)) & 1u; }

__device__ __forceinline__ int64_t warp_id_global() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warps_total() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

__device__ void bc_flush(BcCtr *nx, const BcLocal &c) {
    __shared__ unsigned long long sm[32];
    const unsigned long long a = block_sum(c.in, sm), b = block_sum(c.out, sm), e = block_sum(c.examined, sm);
    if (threadIdx.x == 0) {
        if (a) atomicAdd(&nx->in, a);
        if (b) atomicAdd(&nx->out, b);
        if (e) atomicAdd(&nx->examined, e);
    }
}

// Lane index o of the 32 whose exclusive prefix `excl` is the largest not above
// id (lanes of degree 0 share their successor's prefix, so o has edges).
__device__ __forceinline__ int warp_owner(int excl, int id) {
    int o = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
        const int ek = __shfl_sync(FULL, excl, o + st);
        if (ek <= id) o += st;
    }
    return o;
}

// A warp's merged edge stream: lane k holds a vertex whose list is
// idx[eb_k, eb_k + deg_k) (deg 0: none).  Visits the combined lists BC_W
// windows of 32 edges at a time: f(base, u, own, excl, incl) gets each lane's
// neighbours u[q] (-1 past the end) of windows base + 32 q with their owner
// lanes, all loads issued.  Returns the number of edges (warp-uniform).
template <class F>
__device__ __forceinline__ int warp_stream(const int32_t *__restrict__ idx, int64_t eb, int deg, F f) {
    const int lane = lane_id();
    const int incl = warp_incl_scan(deg);
    const int excl = incl - deg;
    const int E = __shfl_sync(FULL, incl, 31);
    for (int base = 0; base < E; base += 32 * BC_W) {
        int32_t u[BC_W];
        int own[BC_W];
#pragma unroll
        for (int q = 0; q < BC_W; ++q) {
            const int eid = base + 32 * q + lane;
            const int o = warp_owner(excl, eid);
            const int64_t ob = __shfl_sync(FULL, eb, o);
            const int oex = __shfl_sync(FULL, excl, o);
            own[q] = o;
            u[q] = eid < E ? __ldcs(idx + ob + (eid - oex)) : -1;
        }
        f(base, u, own, excl, incl);
    }
    return E;
}

// Sum of val[u] over the entries u of idx[b, e) set in `bits`, one lane over
// its own list with BC_W loads in flight.
__device__ __forceinline__ double lane_gather(const int32_t *__restrict__ idx, int64_t b, int64_t e,
                                              const uint32_t *bits, const double *val) {
    double s = 0.0;
    for (int64_t p = b; p < e; p += BC_WL) {
        int32_t u[BC_WL];
        uint32_t wd[BC_WL];
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) u[q] = p + q < e ? __ldcs(idx + p + q) : -1;
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) wd[q] = u[q] >= 0 ? bits[u[q] >> 5] : 0u;
#pragma unroll
        for (int q = 0; q < BC_WL; ++q)
            if ((wd[q] >> (u[q] & 31)) & 1u) s += val[u[q]];
    }
    return s;
}

// Sum of val[u] over the entries u of idx[b, e) set in `bits`, the warp's
// lanes striding the list (every lane gets the sum).
__device__ __forceinline__ double list_gather(const int32_t *__restrict__ idx, int64_t b, int64_t e,
                                              const uint32_t *bits, const double *val) {
    double s = 0.0;
    for (int64_t i0 = b + lane_id(); i0 < e; i0 += 32 * BC_WL) {
        int32_t u[BC_WL];
        uint32_t wd[BC_WL];
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) u[q] = i0 + 32 * q < e ? __ldcs(idx + i0 + 32 * q) : -1;
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) wd[q] = u[q] >= 0 ? bits[u[q] >> 5] : 0u;
#pragma unroll
        for (int q = 0; q < BC_WL; ++q)
            if ((wd[q] >> (u[q] & 31)) & 1u) s += val[u[q]];
    }
    return warp_sum(s);
}

// Apply f(u) to the entries of idx[b, e), the warp's lanes striding the list:
// f gets BC_W entries at a time (-1 past the end), all loads issued.
template <class F>
__device__ __forceinline__ void list_each(const int32_t *__restrict__ idx, int64_t b, int64_t e, F f) {
    for (int64_t i0 = b + lane_id(); i0 < e; i0 += 32 * BC_WL) {
        int32_t u[BC_WL];
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) u[q] = i0 + 32 * q < e ? __ldcs(idx + i0 + 32 * q) : -1;
        f(u);
    }
}

// The lanes of a group of G (aligned) stride one list idx[b, e) each: f gets
// BC_WL entries at a time (-1 past the end), all loads issued.  Groups finish
// at different times; f must not use warp-wide operations.
template <int G, class F>
__device__ __forceinline__ void group_list_each(const int32_t *__restrict__ idx, int64_t b, int64_t e, F f) {
    for (int64_t i0 = b + (lane_id() & (G - 1)); i0 < e; i0 += G * BC_WL) {
        int32_t u[BC_WL];
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) u[q] = i0 + G * q < e ? __ldcs(idx + i0 + G * q) : -1;
        f(u);
    }
}

// Sum of val[u] over the entries u of idx[b, e) set in `bits`, per group of G
// lanes (every lane of the group gets its list's sum).
template <int G>
__device__ __forceinline__ double group_gather(const int32_t *__restrict__ idx, int64_t b, int64_t e,
                                               const uint32_t *bits, const double *val) {
    double s = 0.0;
    group_list_each<G>(idx, b, e, [&](const int32_t *u) {
        uint32_t wd[BC_WL];
#pragma unroll
        for (int q = 0; q < BC_WL; ++q) wd[q] = u[q] >= 0 ? bits[u[q] >> 5] : 0u;
#pragma unroll
        for (int q = 0; q < BC_WL; ++q)
            if ((wd[q] >> (u[q] & 31)) & 1u) s += val[u[q]];
    });
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o, G);
    return s;
}

// The items [b, e) of a list, 32/G per warp at once: group g of the warp gets
// item it or -1 (all lanes call work together).
template <int G, class F>
__device__ __forceinline__ void warp_groups_each(long long b, long long e, F work) {
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    constexpr int NG = 32 / G;
    const int g = lane_id() / G;
    for (long long i0 = b + warp * NG; i0 < e; i0 += nwarps * NG) {
        const long long it = i0 + g;
        work(it < e ? it : -1);
    }
}

// As warp_select_each, the selected items taken 32/G at a time, one per group
// of G lanes (-1 for a group without one; all lanes call work together).
template <int G, class P, class F>
__device__ __forceinline__ void warp_select_groups(int64_t count, P pred, F work) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    constexpr int NG = 32 / G;
    const int g = lane / G;
    for (int64_t k0 = 0; warp + nwarps * k0 < count; k0 += 32) {
        const int64_t i = warp + nwarps * (k0 + lane);
        const bool sel = i < count && pred(i);
        unsigned bsel = __ballot_sync(FULL, sel);
        while (bsel) {
            // the group's pick: the g-th set bit of bsel (none past the count)
            unsigned x = bsel;
            for (int r = 0; r < g && x; ++r) x &= x - 1;
            const int64_t it = x ? warp + nwarps * (k0 + (__ffs(x) - 1)) : -1;
            work(it);
            for (int r = 0; r < NG && bsel; ++r) bsel &= bsel - 1;
        }
    }
}

// Warp-strided selection: lane i of warp w tests item w + nwarps (k + i) with
// pred (32 tests per load round, consecutive items on different warps); the
// selected items are then taken one by one by the whole warp.
template <class P, class F>
__device__ __forceinline__ void warp_select_each(int64_t count, P pred, F work) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    for (int64_t k0 = 0; warp + nwarps * k0 < count; k0 += 32) {
        const int64_t i = warp + nwarps * (k0 + lane);
        const bool sel = i < count && pred(i);
        for (unsigned bsel = __ballot_sync(FULL, sel); bsel; bsel &= bsel - 1)
            work(warp + nwarps * (k0 + (__ffs(bsel) - 1)));
    }
}

// Forward, push: edges u->w[q], q < N, from the frontier (level l, path counts
// su[q]; w[q] = -1: none).  An unvisited w is claimed by a CAS on its level (all of
// them issued before any result is used); the winner marks it in the next
// level's bitmap; every w at level l+1 gets su added.
template <int N>
__device__ __forceinline__ void bc_visit(const BcRun &R, const int32_t *w, const double *su, int32_t l1,
                                         uint32_t *next_bits) {
    int32_t d[N], old[N];
#pragma unroll
    for (int q = 0; q < N; ++q) d[q] = w[q] >= 0 ? R.dist[w[q]] : -2;
#pragma unroll
    for (int q = 0; q < N; ++q) old[q] = d[q] == -1 ? atomicCAS(R.dist + w[q], -1, l1) : d[q];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const bool won = d[q] == -1 && old[q] == -1;
        if (won) atomicOr(next_bits + (w[q] >> 5), 1u << (w[q] & 31));
        if (won || old[q] == l1) atomicAdd(R.sigma + w[q], su[q]);
    }
}

__device__ void bc_fwd_push(const BcRun &R, int32_t l, const BcCum &a, const BcCum &b, BcLocal &c) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    const int32_t l1 = l + 1;
    const uint32_t *fb = R.lbits[l & 3];
    uint32_t *nb = R.lbits[l1 & 3];
    // hubs of the frontier: every hub chunk whose vertex is in Q_l
    warp_select_each(R.n_hub_out, [&](int64_t j) { return bit_of(fb, R.hub_out[j].v); }, [&](int64_t j) {
        const Chunk ch = R.hub_out[j];
        double su[BC_WL];
        su[0] = R.sigma[ch.v];
#pragma unroll
        for (int q = 1; q < BC_WL; ++q) su[q] = su[0];
        list_each(R.csr_idx, ch.beg, ch.beg + ch.len, [&](const int32_t *w) { bc_visit<BC_WL>(R, w, su, l1, nb); });
        if (lane == 0) c.examined += (unsigned long long)ch.len;
    });
    // medium lists: BC_G lanes per vertex when there are enough of them, else a warp each
    auto med_push = [&](auto gsz) {
        constexpr int G = decltype(gsz)::value;
        warp_groups_each<G>(a.med_out, b.med_out, [&](long long i) {
            if (i < 0) return;
            const int32_t u = R.med_out[i];
            double su[BC_WL];
            su[0] = R.sigma[u];
#pragma unroll
            for (int q = 1; q < BC_WL; ++q) su[q] = su[0];
            const int64_t eb = R.csr_off[u], ee = R.csr_off[u + 1];
            group_list_each<G>(R.csr_idx, eb, ee, [&](const int32_t *w) { bc_visit<BC_WL>(R, w, su, l1, nb); });
            if ((lane & (G - 1)) == 0) c.examined += (unsigned long long)(ee - eb);
        });
    };
    if (b.med_out - a.med_out >= (32 / BC_G) * nwarps)
        med_push(std::integral_constant<int, BC_G>());
    else
        med_push(std::integral_constant<int, 32>());
    // light lists: 32 queue entries per warp, their out-edges as one stream
    for (long long base = a.start + warp * 32; base < b.start; base += nwarps * 32) {
        const long long qi = base + lane;
        int deg = 0;
        int64_t eb = 0;
        double su = 0.0;
        if (qi < b.start) {
            const int32_t u = R.order[qi];
            eb = R.csr_off[u];
            const int64_t d = R.csr_off[u + 1] - eb;
            if (d <= BC_LIGHT) {
                deg = (int)d;
                su = R.sigma[u];
            }
        }
        const int E = warp_stream(R.csr_idx, eb, deg, [&](int, const int32_t *w, const int *own, int, int) {
            double s[BC_W];
#pragma unroll
            for (int q = 0; q < BC_W; ++q) s[q] = __shfl_sync(FULL, su, own[q]);
            bc_visit<BC_W>(R, w, s, l1, nb);
        });
        if (lane == 0) c.examined += (unsigned long long)E;
    }
}

__device__ void bc_fwd_pull(const BcRun &R, int32_t l, BcLocal &c) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    const int32_t l1 = l + 1;
    const uint32_t *fb = R.lbits[l & 3];
    uint32_t *nb = R.lbits[l1 & 3];
    // the candidate set (unvis) does not change during the step
    // hub in-lists by chunks, sums added atomically, claimed by CAS
    warp_select_each(R.n_hub_in, [&](int64_t j) { return bit_of(R.unvis, R.hub_in[j].v); }, [&](int64_t j) {
        const Chunk ch = R.hub_in[j];
        const double s = list_gather(R.csc_idx, ch.beg, ch.beg + ch.len, fb, R.sigma);
        if (lane == 0) {
            c.examined += (unsigned long long)ch.len;
            if (s > 0.0) {
                atomicAdd(R.sigma + ch.v, s);
                if (atomicCAS(R.dist + ch.v, -1, l1) == -1) atomicOr(nb + (ch.v >> 5), 1u << (ch.v & 31));
            }
        }
    });
    // medium in-lists: BC_G lanes per vertex
    warp_select_groups<BC_G>(R.n_med_in_all, [&](int64_t i) { return bit_of(R.unvis, R.med_in_all[i]); }, [&](int64_t i) {
        const int32_t v = i >= 0 ? R.med_in_all[i] : 0;
        const int64_t eb = i >= 0 ? R.csc_off[v] : 0, ee = i >= 0 ? R.csc_off[v + 1] : 0;
        const double s = group_gather<BC_G>(R.csc_idx, eb, ee, fb, R.sigma);
        if (i >= 0 && (lane & (BC_G - 1)) == 0) {
            c.examined += (unsigned long long)(ee - eb);
            if (s > 0.0) {
                R.sigma[v] = s;  // its own group: the only writer
                R.dist[v] = l1;
                atomicOr(nb + (v >> 5), 1u << (v & 31));
            }
        }
    });
    // light in-lists: one candidate word (32 vertices) at a time per warp, as one stream
    const int64_t nwords = (R.n + 31) >> 5;
    warp_select_each(nwords, [&](int64_t wd) { return R.unvis[wd] != 0u; }, [&](int64_t wd) {
        const uint32_t word = R.unvis[wd];
        const int32_t v = (int32_t)(wd * 32 + lane);
        int deg = 0;
        int64_t eb = 0;
        if ((word >> lane) & 1u) {
            eb = R.csc_off[v];
            const int64_t d = R.csc_off[v + 1] - eb;
            deg = d <= BC_LIGHT ? (int)d : 0;
        }
        const double s = lane_gather(R.csc_idx, eb, eb + deg, fb, R.sigma);
        c.examined += (unsigned long long)deg;
        const bool take = deg > 0 && s > 0.0;
        if (take) {
            R.sigma[v] = s;  // its own lane: the only writer
            R.dist[v] = l1;
        }
        const unsigned got = __ballot_sync(FULL, take);
        if (lane == 0 && got) atomicOr(nb + wd, got);
    });
}

// After a forward step: append the vertices of the new level's bitmap to the
// visit order and the medium ones to their level lists (one atomic per list,
// warp and 32 words), take them out of the pull candidates and count degrees.
__device__ void bc_compact(const BcRun &R, const uint32_t *bits, BcCtr *nx, const BcCum &cur, BcLocal &c) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    const int64_t nwords = (R.n + 31) >> 5;
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t word = wd < nwords ? bits[wd] : 0u;
        if (!__any_sync(FULL, word != 0u)) continue;  // uniform
        uint32_t mo = 0, mi = 0;  // vertices of the word with medium out- / in-lists
        for (uint32_t x = word; x; x &= x - 1) {
            const int b = __ffs(x) - 1;
            const int64_t v = wd * 32 + b;
            const int64_t dout = R.csr_off[v + 1] - R.csr_off[v], din = R.csc_off[v + 1] - R.csc_off[v];
            c.out += (unsigned long long)dout;
            c.in += (unsigned long long)din;
            if (dout > BC_LIGHT && dout <= BC_HUB) mo |= 1u << b;
            if (din > BC_LIGHT && din <= BC_HUB) mi |= 1u << b;
        }
        const int n0 = __popc(word), n1 = __popc(mo), n2 = __popc(mi);
        const int i0 = warp_incl_scan(n0), i1 = warp_incl_scan(n1), i2 = warp_incl_scan(n2);
        unsigned long long p0 = 0, p1 = 0, p2 = 0;
        if (lane == 31) {
            p0 = atomicAdd(&nx->tail, (unsigned long long)i0);
            if (i1) p1 = atomicAdd(&nx->med_out, (unsigned long long)i1);
            if (i2) p2 = atomicAdd(&nx->med_in, (unsigned long long)i2);
        }
        long long q0 = cur.start + (long long)(__shfl_sync(FULL, p0, 31) + (unsigned long long)(i0 - n0));
        long long q1 = cur.med_out + (long long)(__shfl_sync(FULL, p1, 31) + (unsigned long long)(i1 - n1));
        long long q2 = cur.med_in + (long long)(__shfl_sync(FULL, p2, 31) + (unsigned long long)(i2 - n2));
        if (!word) continue;
        R.unvis[wd] &= ~word;  // the word's only writer
        for (uint32_t x = word; x; x &= x - 1) {
            const int b = __ffs(x) - 1;
            const int32_t v = (int32_t)(wd * 32 + b);
            R.order[q0++] = v;
            if ((mo >> b) & 1u) R.med_out[q1++] = v;
            if ((mi >> b) & 1u) R.med_in[q2++] = v;
        }
    }
}

// Backward step l: finish the vertices of Q_l (bc += sigma S; c = 1/sigma + S,
// stored when `store_coef`) and, when `scatter`, add c to S of their
// in-neighbours in Q_{l-1}.  The scatter walks the hot-encoded CSC: the targets
// of largest out-degree (most updated) are summed in the block's shared memory
// `acc` and added to S once per block at the end, the others with FP64 RED.
__device__ void bc_bwd_push(const BcRun &R, int32_t l, const BcCum &a, const BcCum &b, bool scatter, bool store_coef,
                            double *acc, BcLocal &c) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    const uint32_t *qb = R.lbits[l & 3];        // Q_l
    const uint32_t *pb = R.lbits[(l - 1) & 3];  // Q_{l-1}
    // N entries u[q] of the encoded CSC (-1: none) receive cw[q] when in Q_{l-1}
    auto scatter_n = [&](auto nn, const int32_t *u, const double *cw) {
        constexpr int N = decltype(nn)::value;
        int32_t v[N];
        uint32_t wd[N];
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] = u[q] < -1 ? R.hot_id[u[q] & 0x7fffffff] : u[q];
#pragma unroll
        for (int q = 0; q < N; ++q) wd[q] = v[q] >= 0 ? pb[v[q] >> 5] : 0u;
#pragma unroll
        for (int q = 0; q < N; ++q)
            if ((wd[q] >> (v[q] & 31)) & 1u) {
                if (u[q] < -1)
                    atomicAdd(acc + (u[q] & 0x7fffffff), cw[q]);
                else
                    atomicAdd(R.S + v[q], cw[q]);
            }
    };
    if (scatter) {
        for (int i = threadIdx.x; i < R.nhot; i += blockDim.x) acc[i] = 0.0;
        __syncthreads();
        warp_select_each(R.n_hub_in, [&](int64_t j) { return bit_of(qb, R.hub_in[j].v); }, [&](int64_t j) {
            const Chunk ch = R.hub_in[j];
            double cw[BC_WL];
            cw[0] = 1.0 / R.sigma[ch.v] + R.S[ch.v];
#pragma unroll
            for (int q = 1; q < BC_WL; ++q) cw[q] = cw[0];
            list_each(R.csc_enc, ch.beg, ch.beg + ch.len,
                      [&](const int32_t *u) { scatter_n(std::integral_constant<int, BC_WL>(), u, cw); });
            if (lane == 0) c.examined += (unsigned long long)ch.len;
        });
        auto med_scatter = [&](auto gsz) {
            constexpr int G = decltype(gsz)::value;
            warp_groups_each<G>(a.med_in, b.med_in, [&](long long i) {
                if (i < 0) return;
                const int32_t w = R.med_in[i];
                double cw[BC_WL];
                cw[0] = 1.0 / R.sigma[w] + R.S[w];
#pragma unroll
                for (int q = 1; q < BC_WL; ++q) cw[q] = cw[0];
                const int64_t eb = R.csc_off[w], ee = R.csc_off[w + 1];
                group_list_each<G>(R.csc_enc, eb, ee,
                                   [&](const int32_t *u) { scatter_n(std::integral_constant<int, BC_WL>(), u, cw); });
                if ((lane & (G - 1)) == 0) c.examined += (unsigned long long)(ee - eb);
            });
        };
        if (b.med_in - a.med_in >= (32 / BC_G) * nwarps)
            med_scatter(std::integral_constant<int, BC_G>());
        else
            med_scatter(std::integral_constant<int, 32>());
    }
    for (long long base = a.start + warp * 32; base < b.start; base += nwarps * 32) {
        const long long qi = base + lane;
        int deg = 0;
        int64_t eb = 0;
        double cw = 0.0;
        if (qi < b.start) {
            const int32_t w = R.order[qi];
            const double sg = R.sigma[w], sw = R.S[w];
            cw = 1.0 / sg + sw;
            R.bc[w] += sg * sw;
            if (store_coef) R.coef[w] = cw;
            eb = R.csc_off[w];
            const int64_t d = R.csc_off[w + 1] - eb;
            deg = scatter && d <= BC_LIGHT ? (int)d : 0;
        }
        if (!scatter) continue;  // uniform
        const int E = warp_stream(R.csc_enc, eb, deg, [&](int, const int32_t *u, const int *own, int, int) {
            double cv[BC_W];
#pragma unroll
            for (int q = 0; q < BC_W; ++q) cv[q] = __shfl_sync(FULL, cw, own[q]);
            scatter_n(std::integral_constant<int, BC_W>(), u, cv);
        });
        if (lane == 0) c.examined += (unsigned long long)E;
    }
    if (scatter) {  // the block's sums of the hot targets, once per block
        __syncthreads();
        for (int i = threadIdx.x; i < R.nhot; i += blockDim.x)
            if (acc[i] != 0.0) atomicAdd(R.S + R.hot_id[i], acc[i]);
    }
}

// Backward pull for step l: each u of Q_{l-1} (levels p..a) sums c(w) over its
// out-neighbours in Q_l.
__device__ void bc_bwd_pull(const BcRun &R, int32_t l, const BcCum &p, const BcCum &a, BcLocal &c) {
    const int lane = lane_id();
    const int64_t warp = warp_id_global(), nwarps = warps_total();
    const uint32_t *qb = R.lbits[l & 3];        // Q_l
    const uint32_t *pb = R.lbits[(l - 1) & 3];  // Q_{l-1}
    warp_select_each(R.n_hub_out, [&](int64_t j) { return bit_of(pb, R.hub_out[j].v); }, [&](int64_t j) {
        const Chunk ch = R.hub_out[j];
        const double s = list_gather(R.csr_idx, ch.beg, ch.beg + ch.len, qb, R.coef);
        if (lane == 0) {
            c.examined += (unsigned long long)ch.len;
            if (s != 0.0) atomicAdd(R.S + ch.v, s);
        }
    });
    auto med_gather = [&](auto gsz) {
        constexpr int G = decltype(gsz)::value;
        warp_groups_each<G>(p.med_out, a.med_out, [&](long long i) {
            const int32_t u = i >= 0 ? R.med_out[i] : 0;
            const int64_t eb = i >= 0 ? R.csr_off[u] : 0, ee = i >= 0 ? R.csr_off[u + 1] : 0;
            const double s = group_gather<G>(R.csr_idx, eb, ee, qb, R.coef);
            if (i >= 0 && (lane & (G - 1)) == 0) {
                c.examined += (unsigned long long)(ee - eb);
                R.S[u] = s;  // its own group: the only writer
            }
        });
    };
    if (a.med_out - p.med_out >= (32 / BC_G) * nwarps)
        med_gather(std::integral_constant<int, BC_G>());
    else
        med_gather(std::integral_constant<int, 32>());
    for (long long base = p.start + warp * 32; base < a.start; base += nwarps * 32) {
        const long long qi = base + lane;
        int32_t u = -1;
        int deg = 0;
        int64_t eb = 0;
        if (qi < a.start) {
            u = R.order[qi];
            eb = R.csr_off[u];
            const int64_t d = R.csr_off[u + 1] - eb;
            if (d <= BC_LIGHT) deg = (int)d;
            else u = -1;  // medium or hub: done above
        }
        const double s = lane_gather(R.csr_idx, eb, eb + deg, qb, R.coef);
        c.examined += (unsigned long long)deg;
        if (u >= 0) R.S[u] = s;  // its own lane: the only writer
    }
}

// Set the bits of order[b, e) in `bits` (one level's bitmap, from its vertex range).
__device__ __forceinline__ void bc_mark(const BcRun &R, long long b, long long e, uint32_t *bits) {
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (long long i = b + gthread; i < e; i += nthreads) {
        const int32_t v = R.order[i];
        atomicOr(bits + (v >> 5), 1u << (v & 31));
    }
}

__device__ __forceinline__ void bc_clear(uint32_t *bits, int64_t nwords) {
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gthread; i < nwords; i += nthreads) bits[i] = 0u;
}

__device__ __forceinline__ BcCum bc_load_lev(const BcCum *p) {
    BcCum a;
    a.start = __ldcg(&p->start);
    a.med_out = __ldcg(&p->med_out);
    a.med_in = __ldcg(&p->med_in);
    a.in = __ldcg(&p->in);
    a.out = __ldcg(&p->out);
    return a;
}

__global__ void __launch_bounds__(BC_THREADS, 2) k_bc_persistent(BcRun R) {
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t nwords = (R.n + 31) >> 5;
    constexpr int CW = (int)(sizeof(BcCtr) / sizeof(unsigned long long));
    __shared__ unsigned long long s_c[CW];
    __shared__ double s_acc[BC_HOT];  // backward push: the block's sums of the hot targets
    auto read_ctr = [&](int slot) {  // one thread per block reads, the block shares
        if (threadIdx.x < CW) s_c[threadIdx.x] = ((volatile unsigned long long *)(R.ctr + slot))[threadIdx.x];
        __syncthreads();
    };
    for (int64_t i = gthread; i < nwords; i += nthreads) {
        R.unvis[i] = R.nzin[i];
        for (int q = 0; q < 4; ++q) R.lbits[q][i] = 0u;
    }
    if (!grid_sync(R.sync, gridDim.x)) return;
    int64_t levels = 0, reached = 0, examined = 0, pushes = 0, pulls = 0;
    for (int64_t k = 0; k < R.nsrc; ++k) {
        const int32_t src = R.sources[k];
        if (src < 0 || (int64_t)src >= R.n) {  // every block reads the same source: all return here
            if (gthread == 0) atomicExch(&R.sync->err, 3);
            return;
        }
        const bool rec = R.record && k == 0;
        // the source: level 0, one path; its record goes to ctr[0], the others start at zero
        if (blockIdx.x == 0) {
            const int64_t dout = R.csr_off[src + 1] - R.csr_off[src], din = R.csc_off[src + 1] - R.csc_off[src];
            const bool mo = dout > BC_LIGHT && dout <= BC_HUB, mi = din > BC_LIGHT && din <= BC_HUB;
            if (threadIdx.x < 3 * CW) {
                unsigned long long v = 0;
                if (threadIdx.x == 0) v = 1;
                if (threadIdx.x == 1) v = mo;
                if (threadIdx.x == 2) v = mi;
                if (threadIdx.x == 3) v = (unsigned long long)din;
                if (threadIdx.x == 4) v = (unsigned long long)dout;
                ((unsigned long long *)R.ctr)[threadIdx.x] = v;
            }
            if (threadIdx.x == 0) {
                R.dist[src] = 0;
                R.sigma[src] = 1.0;
                R.order[0] = src;
                if (mo) R.med_out[0] = src;
                if (mi) R.med_in[0] = src;
                R.unvis[src >> 5] &= ~(1u << (src & 31));
                R.lbits[0][src >> 5] |= 1u << (src & 31);
            }
        }
        if (!grid_sync(R.sync, gridDim.x)) return;
        read_ctr(0);
        BcCum prev = {0, 0, 0, 0, 0};
        BcCum cur = {(long long)s_c[0], (long long)s_c[1], (long long)s_c[2], (long long)s_c[3], (long long)s_c[4]};
        if (gthread == 0) {
            R.lev[0] = prev;
            R.lev[1] = cur;
        }
        int64_t t = 0;  // steps of this source: the counter ring's position
        unsigned long long t_step = bc_now();
        auto decide = [&](bool pull_rule) -> int {
            if (R.dirs) return R.dirs[t < R.ndirs ? t : R.ndirs - 1];
            if (R.mode == GP_PUSH || R.mode == GP_PULL) return R.mode;
            return pull_rule ? GP_PULL : GP_PUSH;
        };
        auto end_step = [&](int dir, int phase, int32_t level, long long frontier, unsigned long long ex) {
            if (rec && gthread == 0 && t < GP_BC_MAX_STEPS) {
                const unsigned long long now = bc_now();
                BcStepStat &st = R.stats[t];
                st.direction = dir;
                st.phase = phase;
                st.level = level;
                st.ns = (int32_t)min(now - t_step, 0x7fffffffull);
                st.frontier = frontier;
                st.examined = (int64_t)ex;
                t_step = now;
            }
            examined += (int64_t)ex;
            if (dir == GP_PUSH)
                ++pushes;
            else
                ++pulls;
            ++t;
        };
        // forward: Q_l = order[prev.start, cur.start)
        int32_t l = 0;
        while (cur.start > prev.start) {
            const long long mf = cur.out - prev.out, mu = (long long)R.m - cur.in;
            const int dir = decide((double)mf * R.alpha > (double)(mu > 0 ? mu : 0));
            BcCtr *nx = R.ctr + (t + 1) % 3;
            if (gthread < CW) ((unsigned long long *)(R.ctr + (t + 2) % 3))[gthread] = 0;
            bc_clear(R.lbits[(l + 2) & 3], nwords);  // Q_{l-2}: no longer read
            BcLocal c;
            if (dir == GP_PUSH)
                bc_fwd_push(R, l, prev, cur, c);
            else
                bc_fwd_pull(R, l, c);
            if (!grid_sync(R.sync, gridDim.x)) return;
            bc_compact(R, R.lbits[(l + 1) & 3], nx, cur, c);
            bc_flush(nx, c);
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr((int)((t + 1) % 3));
            const BcCum nxt = {cur.start + (long long)s_c[0], cur.med_out + (long long)s_c[1],
                               cur.med_in + (long long)s_c[2], cur.in + (long long)s_c[3], cur.out + (long long)s_c[4]};
            end_step(dir, 0, l, cur.start - prev.start, s_c[5]);
            ++l;
            prev = cur;
            cur = nxt;
            if (gthread == 0) R.lev[l + 1] = cur;
        }
        const int32_t L = l - 1;  // deepest non-empty level
        levels += L + 1;
        reached += cur.start;
        // backward: step lb finishes Q_lb and passes its coefficients to Q_{lb-1}
        for (int32_t lb = L; lb >= 1; --lb) {
            const BcCum p = bc_load_lev(R.lev + lb - 1), a = bc_load_lev(R.lev + lb), b = bc_load_lev(R.lev + lb + 1);
            const long long push_cost = b.in - a.in, pull_cost = a.out - p.out;
            const int dir = decide((double)push_cost * R.alpha > (double)pull_cost);
            BcCtr *nx = R.ctr + (t + 1) % 3;
            if (gthread < CW) ((unsigned long long *)(R.ctr + (t + 2) % 3))[gthread] = 0;
            // one step ahead: Q_{lb-2}'s bitmap into the slot cleared last step; Q_{lb+1}'s cleared
            bc_clear(R.lbits[(lb + 1) & 3], nwords);
            if (lb >= 2) bc_mark(R, bc_load_lev(R.lev + lb - 2).start, p.start, R.lbits[(lb - 2) & 3]);
            BcLocal c;
            if (dir == GP_PUSH) {
                bc_bwd_push(R, lb, a, b, true, false, s_acc, c);
            } else {
                bc_bwd_push(R, lb, a, b, false, true, s_acc, c);
                if (!grid_sync(R.sync, gridDim.x)) return;
                bc_bwd_pull(R, lb, p, a, c);
            }
            bc_flush(nx, c);
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr((int)((t + 1) % 3));
            end_step(dir, 1, lb, b.start - a.start, s_c[5]);
        }
        if (rec && gthread == 0) R.summary->steps = t;
        // reset the visited vertices, the pull candidates and the level bitmaps
        for (long long i = gthread; i < cur.start; i += nthreads) {
            const int32_t v = R.order[i];
            R.dist[v] = -1;
            R.sigma[v] = 0.0;
            R.S[v] = 0.0;
        }
        for (int64_t i = gthread; i < nwords; i += nthreads) {
            R.unvis[i] = R.nzin[i];
            for (int q = 0; q < 4; ++q) R.lbits[q][i] = 0u;
        }
        if (!grid_sync(R.sync, gridDim.x)) return;
    }
    if (gthread == 0) {
        R.summary->levels = levels;
        R.summary->reached = reached;
        R.summary->examined = examined;
        R.summary->pushes = pushes;
        R.summary->pulls = pulls;
    }
}

// Bit v of word v/32: vertex v has in-edges.
__global__ void k_bc_nzin(int64_t n, const int64_t *csc_off, uint32_t *bits) {
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

}  // namespace gp

// ------------------------------------------------------------------ driver

using namespace gp;

struct gp_bc_work {
    bool ready = false;
    int32_t *dist = nullptr, *order = nullptr, *med_out = nullptr, *med_in = nullptr;
    int32_t *med_in_all = nullptr;  // every vertex with a medium in-list
    int64_t n_med_in_all = 0;
    BigBins hub_out, hub_in;  // lists above BC_HUB cut into BC_CHUNK-edge chunks
    HotSet hot;               // the BC_HOT largest out-degrees, CSC encoded
    double *sigma = nullptr, *S = nullptr, *coef = nullptr, *bc = nullptr;
    uint32_t *unvis = nullptr, *nzin = nullptr;
    uint32_t *lbits[4] = {nullptr, nullptr, nullptr, nullptr};
    BcCum *lev = nullptr;
    BcCtr *ctr = nullptr;
    BcStepStat *stats = nullptr;
    BcSummary *summary = nullptr;  // [one per launch of a call, up to BC_MAX_LAUNCH_SUMMARIES]
    GridSync *sync = nullptr;
    int8_t *dirs = nullptr;
    int32_t *src_dev = nullptr;
    int64_t src_cap = 0;
    void *host = nullptr;  // pinned: summary, step stats, barrier word
    int grid = 0;
    cudaEvent_t done_ev = nullptr;
    bool pending = false;
    Arena mem, src_mem;
};

namespace gp {

// host mirror: summary, per-step statistics, barrier status
constexpr size_t BC_HOST_BYTES = sizeof(BcSummary) + GP_BC_MAX_STEPS * sizeof(BcStepStat) + sizeof(GridSync);

void release_bc_work(gp_graph *g, cudaStream_t s) {
    if (!g->bc) return;
    if (g->bc->done_ev) {
        cudaEventSynchronize(g->bc->done_ev);
        cudaEventDestroy(g->bc->done_ev);
    }
    pinned_free(g->bc->host, BC_HOST_BYTES);
    g->bc->mem.release(s);
    g->bc->src_mem.release(s);
    g->bc->hub_out.mem.release(s);
    g->bc->hub_in.mem.release(s);
    g->bc->hot.mem.release(s);
    delete g->bc;
    g->bc = nullptr;
}

}  // namespace gp

static int ensure_bc_work(gp_graph *g, cudaStream_t s) {
    if (!g->bc) g->bc = new gp_bc_work();
    gp_bc_work &w = *g->bc;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    GP_TRY(w.mem.alloc(w.dist, n, s));
    GP_TRY(w.mem.alloc(w.order, n, s));
    GP_TRY(w.mem.alloc(w.med_out, n, s));
    GP_TRY(w.mem.alloc(w.med_in, n, s));
    GP_TRY(build_bins(g, w.hub_out, g->csr_off, BC_HUB, BC_CHUNK, s));
    GP_TRY(build_bins(g, w.hub_in, g->csc_off, BC_HUB, BC_CHUNK, s));
    GP_TRY(build_hot(g, w.hot, BC_HOT, g->csr_off, g->csc_idx, s));
    GP_TRY(select_by_degree(g->csc_off, g->n, BC_LIGHT + 1, BC_HUB, w.mem, w.med_in_all, w.n_med_in_all, INT64_MAX,
                            nullptr, s));
    GP_TRY(w.mem.alloc(w.sigma, n, s));
    GP_TRY(w.mem.alloc(w.S, n, s));
    GP_TRY(w.mem.alloc(w.coef, n, s));
    GP_TRY(w.mem.alloc(w.unvis, words, s));
    GP_TRY(w.mem.alloc(w.nzin, words, s));
    for (int q = 0; q < 4; ++q) GP_TRY(w.mem.alloc(w.lbits[q], words, s));
    GP_TRY(w.mem.alloc(w.lev, n + 2, s));
    GP_TRY(w.mem.alloc(w.ctr, 3, s));
    GP_TRY(w.mem.alloc(w.stats, GP_BC_MAX_STEPS, s));
    GP_TRY(w.mem.alloc(w.summary, 1, s));
    GP_TRY(w.mem.alloc(w.sync, 1, s));
    GP_TRY(w.mem.alloc(w.dirs, GP_BC_MAX_STEPS, s));
    if (g->n > 0) {
        k_bc_nzin<<<(int)std::min<size_t>((words + 255) / 256, 4096), 256, 0, s>>>(g->n, g->csc_off, w.nzin);
        GP_CUDA(cudaGetLastError());
    }
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bc_persistent, BC_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "BC kernel does not fit on an SM");
    w.grid = per_sm * g->num_sms;
    GP_TRY(pinned_alloc(&w.host, BC_HOST_BYTES));
    GP_CUDA(cudaEventCreateWithFlags(&w.done_ev, cudaEventDisableTiming));
    w.ready = true;
    return GP_OK;
}

static int bc_barrier_status(int err, const char *when) {
    if (err == 3) return set_error(GP_ERR_INVALID, "gp_bc: a source outside [0, n)%s", when);
    if (err) return set_error(GP_ERR_TIMEOUT, "gp_bc: a grid barrier wait ran out%s", when);
    return GP_OK;
}

extern "C" int gp_bc(const gp_graph *gc, const int32_t *sources, int64_t nsources, int mode, const int8_t *dirs,
                     int ndirs, double *bc_out, gp_bc_stats *stats, void *stream) {
    clear_error();
    if (!gc) return set_error(GP_ERR_INVALID, "gp_bc: graph is NULL");
    gp_graph *g = const_cast<gp_graph *>(gc);
    cudaStream_t s = (cudaStream_t)stream;
    if (nsources < 0) return set_error(GP_ERR_INVALID, "gp_bc: nsources %lld < 0", (long long)nsources);
    if (nsources > 0 && !sources) return set_error(GP_ERR_INVALID, "gp_bc: sources is NULL");
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "gp_bc: bad mode %d", mode);
    if (dirs && ndirs < 1) return set_error(GP_ERR_INVALID, "gp_bc: dirs given with ndirs < 1");
    for (int i = 0; dirs && i < ndirs; ++i)
        if (dirs[i] != GP_PUSH && dirs[i] != GP_PULL) return set_error(GP_ERR_INVALID, "gp_bc: dirs[%d] = %d", i, dirs[i]);
    if (!bc_out) return set_error(GP_ERR_INVALID, "gp_bc: bc_out is NULL");
    const bool src_dev = nsources > 0 && is_device_ptr(sources);
    if (!src_dev)
        for (int64_t i = 0; i < nsources; ++i)
            if (sources[i] < 0 || (int64_t)sources[i] >= g->n)
                return set_error(GP_ERR_INVALID, "gp_bc: sources[%lld] = %d outside [0, %lld)", (long long)i, sources[i],
                                 (long long)g->n);
    GP_TRY(ensure_bc_work(g, s));
    gp_bc_work &w = *g->bc;
    char *h = (char *)w.host;
    BcSummary *hs = (BcSummary *)h;
    BcStepStat *hl = (BcStepStat *)(h + sizeof(BcSummary));
    GridSync *hsync = (GridSync *)(h + sizeof(BcSummary) + GP_BC_MAX_STEPS * sizeof(BcStepStat));
    if (w.pending) {  // the barrier status of the previous, asynchronous call
        GP_CUDA(cudaEventSynchronize(w.done_ev));
        w.pending = false;
        const int err = hsync->err;
        hsync->err = 0;
        GP_TRY(bc_barrier_status(err, " in the previous asynchronous call"));
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    const int64_t n = g->n;
    const bool out_dev = is_device_ptr(bc_out);
    if (!out_dev && !w.bc) GP_TRY(w.mem.alloc(w.bc, (size_t)std::max<int64_t>(n, 1), s));
    double *bc = out_dev ? bc_out : w.bc;
    const int32_t *src = sources;
    if (nsources > 0 && !src_dev) {
        if (w.src_cap < nsources) {
            GP_CUDA(cudaStreamSynchronize(s));  // an earlier call may still read the old copy
            w.src_mem.release(s);
            w.src_cap = 0;
            GP_TRY(w.src_mem.alloc(w.src_dev, (size_t)nsources, s));
            w.src_cap = nsources;
        }
        GP_CUDA(cudaMemcpyAsync(w.src_dev, sources, (size_t)nsources * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        src = w.src_dev;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    if (n > 0) {
        GP_CUDA(cudaMemsetAsync(bc, 0, (size_t)n * sizeof(double), s));
        // clean per-vertex state: every launch leaves it so, this covers an aborted one
        GP_CUDA(cudaMemsetAsync(w.dist, 0xff, (size_t)n * sizeof(int32_t), s));
        GP_CUDA(cudaMemsetAsync(w.sigma, 0, (size_t)n * sizeof(double), s));
        GP_CUDA(cudaMemsetAsync(w.S, 0, (size_t)n * sizeof(double), s));
    }
    BcRun R;
    memset(&R, 0, sizeof(R));
    R.n = n;
    R.m = g->m;
    R.csr_off = g->csr_off;
    R.csc_off = g->csc_off;
    R.csr_idx = g->csr_idx;
    R.csc_idx = g->csc_idx;
    R.csc_enc = w.hot.nhot > 0 ? w.hot.enc_idx : g->csc_idx;
    R.hot_id = w.hot.hot_id;
    R.nhot = (int32_t)w.hot.nhot;
    R.med_in_all = w.med_in_all;
    R.n_med_in_all = w.n_med_in_all;
    R.med_out = w.med_out;
    R.med_in = w.med_in;
    R.hub_out = w.hub_out.chunks;
    R.hub_in = w.hub_in.chunks;
    R.n_hub_out = w.hub_out.nchunks;
    R.n_hub_in = w.hub_in.nchunks;
    R.dist = w.dist;
    R.sigma = w.sigma;
    R.S = w.S;
    R.coef = w.coef;
    R.bc = bc;
    R.order = w.order;
    R.unvis = w.unvis;
    R.nzin = w.nzin;
    for (int q = 0; q < 4; ++q) R.lbits[q] = w.lbits[q];
    R.lev = w.lev;
    R.ctr = w.ctr;
    R.mode = mode;
    R.alpha = g->opt.bc_alpha;
    R.stats = w.stats;
    R.summary = w.summary;
    R.sync = w.sync;
    if (dirs) {
        const int nd = std::min(ndirs, GP_BC_MAX_STEPS);
        GP_CUDA(cudaMemcpyAsync(w.dirs, dirs, nd, cudaMemcpyHostToDevice, s));
        R.dirs = w.dirs;
        R.ndirs = nd;
    }
    GP_CUDA(cudaMemsetAsync(w.sync, 0, sizeof(GridSync), s));
    BcSummary total;
    memset(&total, 0, sizeof(total));
    const bool wait = stats || !out_dev || (nsources > 0 && !src_dev);
    for (int64_t k0 = 0; k0 < nsources && n > 0; k0 += BC_BATCH) {
        R.sources = src + k0;
        R.nsrc = std::min<int64_t>(BC_BATCH, nsources - k0);
        R.record = stats && k0 == 0;
        GP_CUDA(cudaMemsetAsync(w.summary, 0, sizeof(BcSummary), s));
        {
            ProfScope ps("bc_persistent", s);
            void *args[] = {&R};
            GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_bc_persistent, dim3((unsigned)w.grid),
                                                dim3(BC_THREADS), args, 0, s));
        }
        if (stats) {  // per-launch summaries are summed on the host
            GP_CUDA(cudaMemcpyAsync(hs, w.summary, sizeof(BcSummary), cudaMemcpyDeviceToHost, s));
            if (k0 == 0) GP_CUDA(cudaMemcpyAsync(hl, w.stats, GP_BC_MAX_STEPS * sizeof(BcStepStat), cudaMemcpyDeviceToHost, s));
            GP_CUDA(cudaMemcpyAsync(hsync, w.sync, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
            GP_CUDA(cudaStreamSynchronize(s));
            if (hsync->err) break;
            if (k0 == 0) total.steps = hs->steps;
            total.levels += hs->levels;
            total.reached += hs->reached;
            total.examined += hs->examined;
            total.pushes += hs->pushes;
            total.pulls += hs->pulls;
        }
    }
    if (!out_dev && n > 0) GP_CUDA(cudaMemcpyAsync(bc_out, bc, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hsync, w.sync, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    if (!wait) {
        // nothing for the host to read: return without waiting; the barrier
        // status is checked by the next call on this graph
        GP_CUDA(cudaEventRecord(w.done_ev, s));
        w.pending = true;
        return GP_OK;
    }
    if (stats) GP_CUDA(cudaEventRecord(ev1, s));
    GP_CUDA(cudaStreamSynchronize(s));
    const int err = hsync->err;
    hsync->err = 0;
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->sources = nsources;
        stats->levels = total.levels;
        stats->reached = total.reached;
        stats->edges_examined = total.examined;
        stats->pushes = total.pushes;
        stats->pulls = total.pulls;
        stats->ms = ms;
        const int L = (int)std::min<int64_t>(total.steps, GP_BC_MAX_STEPS);
        stats->steps = L;
        for (int i = 0; i < L; ++i) {
            stats->direction[i] = (int8_t)hl[i].direction;
            stats->phase[i] = (int8_t)hl[i].phase;
            stats->level[i] = hl[i].level;
            stats->frontier[i] = hl[i].frontier;
            stats->examined[i] = hl[i].examined;
            stats->step_ns[i] = hl[i].ns;
        }
    }
    return bc_barrier_status(err, "");
}
