// tc.cu -- per-vertex triangle counts by the push- and pull-based
// NodeIterator of the paper's Section 3 listing.
//
// For every vertex v, every neighbour w1 and every neighbour w2 of v with w1
// adjacent to w2, pull adds one to tc[v] (only v's owner writes it) and push
// adds one to tc[w1] (fetch-and-add: the listing's FAA atomics); both halve at
// the end.  The inner loop over w2 is counted at once as |N(v) n N(w1)| minus v
// and w1 themselves: the number of w2 it accepts.  One warp handles one edge
// (v, w1) at a time: its lanes take the elements of the shorter of the two
// sorted lists in turn and binary-search the longer one.  Work units: each
// light vertex (degree <= push_light_max) is one unit, each chunk of a heavy
// vertex's list is one; pull adds a heavy vertex's chunk sums in a second
// kernel, so every count still has a single writer.
#include <algorithm>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {

struct TcArgs {
    int64_t n;
    const int64_t *off;
    const int32_t *idx;
    const int32_t *rank;    // [n] rank among heavy vertices, -1 light
    const int64_t *cstart;  // heavy vertex r's chunks: [cstart[r], cstart[r+1])
    const Chunk *chunks;
    const int32_t *big;     // heavy vertex of rank r
    int64_t nchunks, nbig;
    int push;
    unsigned long long *tc;       // [n] counts (push: atomics; pull: owner writes)
    unsigned long long *chunk_part;  // pull: [nchunks] sums of heavy vertices' chunks
    unsigned long long *probes;   // elements searched (statistic)
};

// |a n b| \ {x0, x1} for sorted a[0..na), b[0..nb); every lane gets the count.
__device__ __forceinline__ unsigned long long warp_intersect(const int32_t *__restrict__ a, int na,
                                                             const int32_t *__restrict__ b, int nb, int32_t x0,
                                                             int32_t x1) {
    unsigned long long cnt = 0;
    for (int i = lane_id(); i < na; i += 32) {
        const int32_t x = __ldg(a + i);
        if (x == x0 || x == x1) continue;
        int lo = 0, hi = nb;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(b + mid) < x)
                lo = mid + 1;
            else
                hi = mid;
        }
        cnt += lo < nb && __ldg(b + lo) == x;
    }
    return warp_sum(cnt);
}

// Triangle-closing count of the edge slots [e0, e1) of v, summed; push also
// credits each w1 with its own count.
__device__ unsigned long long tc_edges(const TcArgs &a, int32_t v, int64_t e0, int64_t e1, unsigned long long &probes) {
    const int64_t bv = a.off[v];
    const int dv = (int)(a.off[v + 1] - bv);
    unsigned long long sum = 0;
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t w1 = __ldg(a.idx + e);
        if (w1 == v) continue;  // self-loop
        const int64_t bw = a.off[w1];
        const int dw = (int)(a.off[w1 + 1] - bw);
        const bool vshort = dv <= dw;
        const unsigned long long k = vshort ? warp_intersect(a.idx + bv, dv, a.idx + bw, dw, v, w1)
                                            : warp_intersect(a.idx + bw, dw, a.idx + bv, dv, v, w1);
        if (lane_id() == 0) probes += (unsigned long long)(vshort ? dv : dw);
        if (a.push) {
            if (k && lane_id() == 0) atomicAdd(a.tc + w1, k);
        } else {
            sum += k;
        }
    }
    return sum;
}

__global__ void __launch_bounds__(256) k_tc(TcArgs a) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long probes = 0;
    // heavy vertices: one chunk of the list per unit
    for (int64_t j = warp; j < a.nchunks; j += nwarps) {
        const Chunk ch = a.chunks[j];
        const unsigned long long s = tc_edges(a, ch.v, ch.beg, ch.beg + ch.len, probes);
        if (!a.push && lane == 0) a.chunk_part[j] = s;
    }
    // light vertices: the whole list per unit
    for (int64_t v = warp; v < a.n; v += nwarps) {
        if (a.rank[v] >= 0) continue;
        const int64_t b = a.off[v], e = a.off[v + 1];
        if (b == e) {
            if (!a.push && lane == 0) a.tc[v] = 0;
            continue;
        }
        const unsigned long long s = tc_edges(a, (int32_t)v, b, e, probes);
        if (!a.push && lane == 0) a.tc[v] = s / 2;
    }
    probes = warp_sum(probes);
    if (lane == 0 && probes) atomicAdd(a.probes, probes);
}

// pull: heavy vertices add their chunk sums (one writer per count).
__global__ void k_tc_combine(TcArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.nbig; r += stride) {
        unsigned long long s = 0;
        for (int64_t j = a.cstart[r]; j < a.cstart[r + 1]; ++j) s += a.chunk_part[j];
        a.tc[a.big[r]] = s / 2;
    }
}

// push: every count was met twice; halve, and sum for the total.
__global__ void k_tc_finish(int64_t n, int push, unsigned long long *tc, unsigned long long *total) {
    __shared__ unsigned long long sm[32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long s = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        unsigned long long c = tc[v];
        if (push) {
            c /= 2;
            tc[v] = c;
        }
        s += c;
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0 && s) atomicAdd(total, s);
}

}  // namespace gp

using namespace gp;

extern "C" int gp_triangles(const gp_graph *gc, int mode, int64_t *tc_out, int64_t *total_out, gp_tc_stats *stats,
                            void *stream) {
    clear_error();
    if (!gc) return set_error(GP_ERR_INVALID, "gp_triangles: graph is NULL");
    gp_graph *g = const_cast<gp_graph *>(gc);
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "gp_triangles: bad mode %d", mode);
    if (!g->symmetric) return set_error(GP_ERR_INVALID, "gp_triangles: the graph must be undirected (uploaded as symmetric)");
    if (!tc_out && !total_out) return set_error(GP_ERR_INVALID, "gp_triangles: no output");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    if (stats) memset(stats, 0, sizeof(*stats));
    const bool push = mode == GP_PUSH;
    Arena tmp;
    unsigned long long *tc = nullptr, *cp = nullptr, *scal = nullptr;
    const bool dev_out = tc_out && is_device_ptr(tc_out);
    if (dev_out) {
        tc = (unsigned long long *)tc_out;
    } else {
        GP_TRY(tmp.alloc(tc, (size_t)std::max<int64_t>(n, 1), s));
    }
    int st = tmp.alloc(scal, 2, s);  // [0] total, [1] probes
    if (st == GP_OK && !push) st = tmp.alloc(cp, (size_t)std::max<int64_t>(g->push_bins.nchunks, 1), s);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (st == GP_OK && stats) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, s);
    }
    unsigned long long host[2] = {0, 0};
    cudaError_t e = cudaSuccess;
    if (st == GP_OK) {
        e = cudaMemsetAsync(scal, 0, 2 * sizeof(unsigned long long), s);
        if (e == cudaSuccess && push && n > 0) e = cudaMemsetAsync(tc, 0, (size_t)n * sizeof(unsigned long long), s);
    }
    if (st == GP_OK && e == cudaSuccess && n > 0) {
        TcArgs a;
        memset(&a, 0, sizeof(a));
        a.n = n;
        a.off = g->csr_off;
        a.idx = g->csr_idx;
        a.rank = g->push_bins.rank;
        a.cstart = g->push_bins.cstart;
        a.chunks = g->push_bins.chunks;
        a.big = g->push_bins.big;
        a.nchunks = g->push_bins.nchunks;
        a.nbig = g->push_bins.nbig;
        a.push = push;
        a.tc = tc;
        a.chunk_part = cp;
        a.probes = scal + 1;
        const int grid = grid_blocks(g, 256);
        GP_LAUNCH("tc", s, (k_tc<<<grid, 256, 0, s>>>(a)));
        e = cudaGetLastError();
        if (e == cudaSuccess && !push && a.nbig > 0) {
            const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((a.nbig + 255) / 256, grid));
            GP_LAUNCH("tc_combine", s, (k_tc_combine<<<gb, 256, 0, s>>>(a)));
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            const int gf = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, grid));
            GP_LAUNCH("tc_finish", s, (k_tc_finish<<<gf, 256, 0, s>>>(n, push, tc, scal)));
            e = cudaGetLastError();
        }
    }
    if (st == GP_OK && e == cudaSuccess && tc_out && !dev_out && n > 0)
        e = cudaMemcpyAsync(tc_out, tc, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (st == GP_OK && e == cudaSuccess) e = cudaMemcpyAsync(host, scal, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (st == GP_OK && e == cudaSuccess && stats) e = cudaEventRecord(ev1, s);
    if (st == GP_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (stats && ev0) {
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->ms = ms;
        stats->probes = (int64_t)host[1];
        stats->triangles = (int64_t)(host[0] / 3);
        stats->mode_used = push ? GP_PUSH : GP_PULL;
    }
    tmp.release(s);
    if (st != GP_OK) return st;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_triangles: %s", cudaGetErrorString(e));
    if (total_out) *total_out = (int64_t)(host[0] / 3);
    return GP_OK;
}
