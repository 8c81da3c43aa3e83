// pr_fe.cu -- Frontier-Exploit PageRank (Section 5's Frontier-Exploit strategy
// applied to the PageRank of Section 3.1) with a push/pull switch per
// iteration (Generic-Switch), the whole run in one persistent cooperative
// launch.
//
// Residual form: ranks x start at s (1/n uniform), residuals r at (1-d) s +
// d P x - x, the change one PageRank sweep would make.  Iteration k's
// frontier is F = {u : |r_u| > eps}; each u in F moves its residual into x_u
// and sends d * P_vu * r_u to its out-neighbours, all from the residuals at the
// iteration's start:  r'_v = [v not in F] r_v + d * sum_{u in F, u->v} P_vu r_u.
// x + (I - dP)^-1 r stays the fixed point, so when F is empty (every
// |r_u| <= eps) ||x - x*||_1 <= ||r||_1 / (1 - d) for column-substochastic P.
//   push: F's vertices scatter c_u = d r_u / S_u (times w_uv) over their
//         out-edges with FP64 atomics into L2 (a hub's thousands of updates
//         stay exact to FP32 rounding), rounded once to FP32 in the epilogue
//         (light sources as one merged edge stream per warp, heavy ones as
//         queued chunk ids);
//   pull: every vertex gathers c over its in-edges (c_u = 0 outside F): light
//         vertices by their own lane, heavy ones by chunk sums combined by the
//         owner in the epilogue -- no atomics.
// Both end in one epilogue over all vertices: x, r, the next frontier (bitmap
// ring of three, owner-written words), its c and counters.  Direction: pull
// when the frontier's out-edges times fe_alpha exceed m, else push, or a
// caller-given sequence.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {

constexpr int FE_WARPS = 32;
constexpr int FE_THREADS = FE_WARPS * 32;

struct FeCtr {
    unsigned long long nf;     // frontier vertices
    unsigned long long mf;     // their out-degree sum
    unsigned long long h_len;  // push: heavy chunk ids queued
    unsigned long long examined;
    double res;                // L1 norm of the residuals after the iteration
    unsigned long long pad[3];
};

struct FeIterStat {
    int32_t direction;
    int32_t ns;
    int64_t frontier;
    int64_t examined;
};

struct FeSummary {
    int64_t iterations, pushes, pulls;
    double residual;
    int64_t init_ns;
    int64_t left;  // frontier size when the run stopped (0: converged)
};

struct FeRun {
    int64_t n, m;
    const int64_t *csr_off, *csc_off;
    const int32_t *csr_idx, *csc_idx;
    const float *csr_w, *csc_w;
    const float *inv_deg;
    const int32_t *push_rank;
    const int64_t *push_cstart;
    const Chunk *push_chunks;
    const int32_t *pull_rank;
    const int64_t *pull_cstart;
    const Chunk *pull_chunks;
    int64_t pull_nchunks;
    float d, eps, alpha;
    const float *s;  // personalization or nullptr (uniform)
    int32_t mode;
    const int8_t *dirs;
    int32_t ndirs, iters;
    float *x, *r;
    double *acc;  // incoming sums (push: FP64 atomics; pull: the owner's sum)
    float *c[2];
    float *part;  // pull: chunk sums of heavy vertices
    uint32_t *act[3];
    int32_t *hq;
    FeCtr *ctr;  // [3]
    FeIterStat *stats;
    FeSummary *summary;
    GridSync *sync;
};

__device__ __forceinline__ unsigned long long fe_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Push, phase A: a warp ranks the frontier vertices of 32 bitmap words; light
// ones scatter over their out-edges as one merged edge stream, heavy ones
// queue their chunk ids for phase B.
__device__ void fe_push_a(const FeRun &R, const uint32_t *act, const float *c, FeCtr *cur, unsigned long long &ex) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwords = (R.n + 31) >> 5;
    for (int64_t base = warp * 32; base < nwords; base += nwarps * 32) {
        const int64_t wd = base + lane;
        const uint32_t word = wd < nwords ? act[wd] : 0u;
        const int cnt = __popc(word);
        const int incl = warp_incl_scan(cnt);
        const int excl = incl - cnt;
        const int total = __shfl_sync(FULL, incl, 31);
        for (int rr = 0; rr < total; rr += 32) {
            const int id = rr + lane;
            int k = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ek = __shfl_sync(FULL, excl, k + st);
                if (ek <= id) k += st;
            }
            const uint32_t kw = __shfl_sync(FULL, word, k);
            const int kex = __shfl_sync(FULL, excl, k);
            int deg = 0;
            int64_t eb = 0;
            float cu = 0.f;
            if (id < total) {
                const int32_t u = (int32_t)((base + k) * 32 + nth_set_bit(kw, id - kex));
                const int32_t rk = R.push_rank[u];
                if (rk >= 0) {
                    const int64_t c0 = R.push_cstart[rk], c1 = R.push_cstart[rk + 1];
                    const unsigned long long pos = atomicAdd(&cur->h_len, (unsigned long long)(c1 - c0));
                    for (int64_t j = c0; j < c1; ++j) R.hq[pos + (j - c0)] = (int32_t)j;
                } else {
                    eb = R.csr_off[u];
                    deg = (int)(R.csr_off[u + 1] - eb);
                    cu = c[u];
                }
            }
            const int dincl = warp_incl_scan(deg);
            const int dexcl = dincl - deg;
            const int E = __shfl_sync(FULL, dincl, 31);
            for (int e0 = 0; e0 < E; e0 += 32) {
                const int eid = e0 + lane;
                int o = 0;
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int ek = __shfl_sync(FULL, dexcl, o + st);
                    if (ek <= eid) o += st;
                }
                const int64_t ob = __shfl_sync(FULL, eb, o);
                const int oex = __shfl_sync(FULL, dexcl, o);
                const float oc = __shfl_sync(FULL, cu, o);
                if (eid < E) {
                    const int64_t pos = ob + (eid - oex);
                    const int32_t v = __ldcs(R.csr_idx + pos);
                    atomicAdd(R.acc + v, (double)(R.csr_w ? oc * __ldcs(R.csr_w + pos) : oc));
                    ++ex;
                }
            }
        }
    }
}

// Push, phase B: heavy frontier vertices' chunks, one warp each.
__device__ void fe_push_b(const FeRun &R, const float *c, int64_t h_len, unsigned long long &ex) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < h_len; j += nwarps) {
        const Chunk ch = R.push_chunks[R.hq[j]];
        const float cu = c[ch.v];
        for (int i = lane; i < ch.len; i += 32) {
            const int32_t v = __ldcs(R.csr_idx + ch.beg + i);
            atomicAdd(R.acc + v, (double)(R.csr_w ? cu * __ldcs(R.csr_w + ch.beg + i) : cu));
            ++ex;
        }
    }
}

// Pull: heavy vertices' in-lists by chunks (a warp sum per chunk), light
// vertices by their own lane over their in-edges; c is zero outside F.
__device__ void fe_pull(const FeRun &R, const float *c, unsigned long long &ex) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < R.pull_nchunks; j += nwarps) {
        const Chunk ch = R.pull_chunks[j];
        float a = 0.f;
        for (int i = lane; i < ch.len; i += 32) {
            const int32_t u = __ldcs(R.csc_idx + ch.beg + i);
            const float cu = c[u];
            a += R.csc_w ? cu * __ldcs(R.csc_w + ch.beg + i) : cu;
        }
        a = warp_sum(a);
        if (lane == 0) {
            R.part[j] = a;
            ex += (unsigned long long)ch.len;
        }
    }
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < R.n; v += nth) {
        if (R.pull_rank[v] >= 0) continue;
        const int64_t b = R.csc_off[v], e = R.csc_off[v + 1];
        float a = 0.f;
        for (int64_t p = b; p < e; ++p) {
            const float cu = c[__ldcs(R.csc_idx + p)];
            a += R.csc_w ? cu * __ldcs(R.csc_w + p) : cu;
        }
        R.acc[v] = (double)a;
        ex += (unsigned long long)(e - b);
    }
}

__global__ void __launch_bounds__(FE_THREADS) k_pr_fe(FeRun R) {
    const unsigned long long t_start = fe_now();
    const int64_t n = R.n;
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t nwords = (n + 31) >> 5;
    const int lane = lane_id();
    constexpr int CW = (int)(sizeof(FeCtr) / sizeof(unsigned long long));
    __shared__ unsigned long long s_c[CW];
    __shared__ unsigned long long sm[32];
    __shared__ double smd[32];
    volatile FeCtr *vc = (volatile FeCtr *)R.ctr;
    auto read_ctr = [&](int slot) {
        if (threadIdx.x < CW) s_c[threadIdx.x] = ((volatile unsigned long long *)(vc + slot))[threadIdx.x];
        __syncthreads();
    };
    // Epilogue over every vertex (the same for both directions): x += r on the
    // frontier, r' = [v not in F] r + incoming, the next frontier (bitmap word
    // written by the lane-0 owner of the warp's 32 vertices), c for it, counters.
    auto epilogue = [&](const uint32_t *act, uint32_t *act_next, float *c_next, FeCtr *nx, bool pull) {
        unsigned long long nf = 0, mf = 0;
        double res = 0.0;
        for (int64_t base = (gthread >> 5) * 32; base < n; base += (nthreads >> 5) * 32) {
            const int64_t v = base + lane;
            bool inf = false;
            if (v < n) {
                float a = f64_to_f32_rn(R.acc[v]);
                R.acc[v] = 0.0;
                if (pull) {
                    const int32_t rk = R.pull_rank[v];
                    if (rk >= 0)
                        for (int64_t j = R.pull_cstart[rk]; j < R.pull_cstart[rk + 1]; ++j) a += R.part[j];
                }
                const bool in_f = (act[v >> 5] >> (v & 31)) & 1u;
                const float ro = R.r[v];
                if (in_f) R.x[v] += ro;
                const float rn = (in_f ? 0.f : ro) + a;
                R.r[v] = rn;
                inf = R.eps < 0.f ? true : fabsf(rn) > R.eps;
                c_next[v] = inf ? R.d * rn * R.inv_deg[v] : 0.f;
                res += fabs((double)rn);
                if (inf) {
                    nf += 1;
                    mf += (unsigned long long)(R.csr_off[v + 1] - R.csr_off[v]);
                }
            }
            const unsigned word = __ballot_sync(FULL, inf);
            if (lane == 0) act_next[base >> 5] = word;
        }
        nf = block_sum(nf, sm);
        mf = block_sum(mf, sm);
        res = block_sum(res, smd);
        if (threadIdx.x == 0) {
            if (nf) atomicAdd(&nx->nf, nf);
            if (mf) atomicAdd(&nx->mf, mf);
            atomicAdd(&nx->res, res);
        }
    };
    // initial state: x = s (1/n when uniform), r = (1-d) s + d P x - x (the
    // change one PageRank sweep would make), frontier {|r| > eps}
    for (int64_t i = gthread; i < 3 * CW; i += nthreads) ((unsigned long long *)R.ctr)[i] = 0;
    for (int64_t i = gthread; i < nwords; i += nthreads) {
        R.act[1][i] = 0u;
        R.act[2][i] = 0u;
    }
    for (int64_t v = gthread; v < n; v += nthreads) {
        const float xv = R.s ? R.s[v] : 1.f / (float)n;
        R.x[v] = xv;
        R.acc[v] = 0.0;
        R.c[1][v] = xv * R.inv_deg[v];
    }
    if (!grid_sync(R.sync, gridDim.x)) return;
    {
        unsigned long long ex0 = 0;
        fe_pull(R, R.c[1], ex0);  // (P x)_v into acc (light) and the chunk sums (heavy)
    }
    if (!grid_sync(R.sync, gridDim.x)) return;
    {
        unsigned long long nf = 0, mf = 0;
        for (int64_t base = (gthread >> 5) * 32; base < n; base += (nthreads >> 5) * 32) {
            const int64_t v = base + lane;
            bool inf = false;
            if (v < n) {
                float a = f64_to_f32_rn(R.acc[v]);
                R.acc[v] = 0.0;
                const int32_t rk = R.pull_rank[v];
                if (rk >= 0)
                    for (int64_t j = R.pull_cstart[rk]; j < R.pull_cstart[rk + 1]; ++j) a += R.part[j];
                const float sv = R.s ? R.s[v] : 1.f / (float)n;
                const float r0 = (1.f - R.d) * sv + R.d * a - R.x[v];
                R.r[v] = r0;
                inf = R.eps < 0.f ? true : fabsf(r0) > R.eps;
                R.c[0][v] = inf ? R.d * r0 * R.inv_deg[v] : 0.f;
                if (inf) {
                    nf += 1;
                    mf += (unsigned long long)(R.csr_off[v + 1] - R.csr_off[v]);
                }
            }
            const unsigned word = __ballot_sync(FULL, inf);
            if (lane == 0) R.act[0][base >> 5] = word;
        }
        nf = block_sum(nf, sm);
        mf = block_sum(mf, sm);
        if (threadIdx.x == 0) {
            if (nf) atomicAdd(&R.ctr[0].nf, nf);
            if (mf) atomicAdd(&R.ctr[0].mf, mf);
        }
    }
    if (!grid_sync(R.sync, gridDim.x)) return;
    unsigned long long t_iter = fe_now();
    const unsigned long long t_init = t_iter - t_start;
    read_ctr(0);
    unsigned long long nf = s_c[0], mf = s_c[1];
    double res = 0.0;
    int it = 0, pushes = 0, pulls = 0;
    while (nf > 0 && it < R.iters) {
        int dir;
        if (R.dirs) {
            dir = R.dirs[it < R.ndirs ? it : R.ndirs - 1];
        } else if (R.mode == GP_PUSH || R.mode == GP_PULL) {
            dir = R.mode;
        } else {
            dir = ((float)mf * R.alpha > (float)R.m) ? GP_PULL : GP_PUSH;
        }
        const int cur = it % 3, nxt = (it + 1) % 3, spare = (it + 2) % 3;
        const float *c = R.c[it & 1];
        float *c_next = R.c[(it + 1) & 1];
        if (gthread < CW) ((unsigned long long *)(R.ctr + spare))[gthread] = 0;
        for (int64_t i = gthread; i < nwords; i += nthreads) R.act[spare][i] = 0u;
        unsigned long long ex = 0;
        if (dir == GP_PUSH) {
            fe_push_a(R, R.act[cur], c, R.ctr + cur, ex);
            if (!grid_sync(R.sync, gridDim.x)) return;
            read_ctr(cur);
            if (s_c[2] > 0) {
                fe_push_b(R, c, (int64_t)s_c[2], ex);
            }
            ++pushes;
        } else {
            fe_pull(R, c, ex);
            ++pulls;
        }
        ex = block_sum(ex, sm);
        if (threadIdx.x == 0 && ex) atomicAdd(&R.ctr[nxt].examined, ex);
        if (!grid_sync(R.sync, gridDim.x)) return;
        epilogue(R.act[cur], R.act[nxt], c_next, R.ctr + nxt, dir == GP_PULL);
        if (!grid_sync(R.sync, gridDim.x)) return;
        read_ctr(nxt);
        nf = s_c[0];
        mf = s_c[1];
        res = __longlong_as_double((long long)s_c[4]);
        if (gthread == 0 && it < GP_FE_MAX_ITERS) {
            const unsigned long long t = fe_now();
            R.stats[it].direction = dir;
            R.stats[it].ns = (int32_t)min(t - t_iter, 0x7fffffffull);
            R.stats[it].frontier = (int64_t)(vc[cur].nf);
            R.stats[it].examined = (int64_t)s_c[3];
            t_iter = t;
        }
        ++it;
    }
    if (gthread == 0) {
        // with no iteration run the residual is the initial one
        if (it == 0) {
            double r0 = 0.0;
            for (int64_t v = 0; v < n; ++v) r0 += fabs((double)R.r[v]);
            res = r0;
        }
        R.summary->iterations = it;
        R.summary->pushes = pushes;
        R.summary->pulls = pulls;
        R.summary->residual = res;
        R.summary->init_ns = (int64_t)t_init;
        R.summary->left = (int64_t)nf;
    }
}

}  // namespace gp

// ------------------------------------------------------------------ driver

using namespace gp;

struct gp_fe_work {
    bool ready = false;
    float *r = nullptr, *c[2] = {nullptr, nullptr}, *part = nullptr, *x_dev = nullptr;
    double *acc = nullptr;
    uint32_t *act[3] = {nullptr, nullptr, nullptr};
    int32_t *hq = nullptr;
    FeCtr *ctr = nullptr;
    FeIterStat *stats = nullptr;
    FeSummary *summary = nullptr;
    GridSync *sync = nullptr;
    int8_t *dirs = nullptr;
    void *host = nullptr;
    int grid = 0;
    Arena mem;
};

namespace gp {

// host mirror: summary, per-iteration statistics, barrier status
constexpr size_t FE_HOST_BYTES = sizeof(FeSummary) + GP_FE_MAX_ITERS * sizeof(FeIterStat) + sizeof(GridSync);

void release_fe_work(gp_graph *g, cudaStream_t s) {
    if (!g->fe) return;
    pinned_free(g->fe->host, FE_HOST_BYTES);
    g->fe->mem.release(s);
    delete g->fe;
    g->fe = nullptr;
}

}  // namespace gp

static int ensure_fe_work(gp_graph *g, cudaStream_t s) {
    if (!g->fe) g->fe = new gp_fe_work();
    gp_fe_work &w = *g->fe;
    if (w.ready) return GP_OK;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    const size_t words = (n + 31) / 32;
    GP_TRY(w.mem.alloc(w.r, n, s));
    GP_TRY(w.mem.alloc(w.acc, n, s));
    GP_TRY(w.mem.alloc(w.c[0], n, s));
    GP_TRY(w.mem.alloc(w.c[1], n, s));
    GP_TRY(w.mem.alloc(w.part, (size_t)std::max<int64_t>(g->pull_bins.nchunks, 1), s));
    for (int i = 0; i < 3; ++i) GP_TRY(w.mem.alloc(w.act[i], words, s));
    GP_TRY(w.mem.alloc(w.hq, (size_t)std::max<int64_t>(g->push_bins.nchunks, 1), s));
    GP_TRY(w.mem.alloc(w.ctr, 3, s));
    GP_TRY(w.mem.alloc(w.stats, GP_FE_MAX_ITERS, s));
    GP_TRY(w.mem.alloc(w.summary, 1, s));
    GP_TRY(w.mem.alloc(w.sync, 1, s));
    GP_TRY(w.mem.alloc(w.dirs, GP_FE_MAX_ITERS, s));
    int per_sm = 0;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pr_fe, FE_THREADS, 0));
    if (per_sm < 1) return set_error(GP_ERR_UNSUPPORTED, "Frontier-Exploit PageRank kernel does not fit on an SM");
    w.grid = per_sm * g->num_sms;
    GP_TRY(pinned_alloc(&w.host, FE_HOST_BYTES));
    w.ready = true;
    return GP_OK;
}

extern "C" int gp_pagerank_fe(const gp_graph *gc, int mode, float damping, double eps, int iters, const int8_t *dirs,
                              int ndirs, const float *personalization, float *ranks_out, gp_fe_stats *stats,
                              void *stream) {
    clear_error();
    if (!gc) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: graph is NULL");
    gp_graph *g = const_cast<gp_graph *>(gc);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode != GP_PUSH && mode != GP_PULL && mode != GP_AUTO) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: bad mode %d", mode);
    if (!(damping > 0.f && damping < 1.f)) return set_error(GP_ERR_INVALID, "damping %g outside (0, 1)", (double)damping);
    if (!(eps == eps) || iters < 0) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: bad eps or iteration cap");
    if (dirs && ndirs < 1) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: dirs given with ndirs < 1");
    for (int i = 0; dirs && i < ndirs; ++i)
        if (dirs[i] != GP_PUSH && dirs[i] != GP_PULL) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: dirs[%d] = %d", i, dirs[i]);
    if (!ranks_out) return set_error(GP_ERR_INVALID, "gp_pagerank_fe: ranks_out is NULL");
    if (g->n == 0) return GP_OK;
    GP_TRY(ensure_fe_work(g, s));
    gp_fe_work &w = *g->fe;
    const int64_t n = g->n;
    float *x = ranks_out;
    const bool x_dev = is_device_ptr(ranks_out);
    if (!x_dev) {
        if (!w.x_dev) GP_TRY(w.mem.alloc(w.x_dev, (size_t)n, s));
        x = w.x_dev;
    }
    const float *sp = personalization;
    DevBuf sbuf;
    if (sp && !is_device_ptr(sp)) {
        GP_TRY(dev_alloc(sbuf, (size_t)n * sizeof(float), s));
        GP_CUDA(cudaMemcpyAsync(sbuf.ptr, sp, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
        sp = (const float *)sbuf.ptr;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        GP_CUDA(cudaEventCreate(&ev0));
        GP_CUDA(cudaEventCreate(&ev1));
        GP_CUDA(cudaEventRecord(ev0, s));
    }
    FeRun R;
    memset(&R, 0, sizeof(R));
    R.n = n;
    R.m = g->m;
    R.csr_off = g->csr_off;
    R.csc_off = g->csc_off;
    R.csr_idx = g->csr_idx;
    R.csc_idx = g->csc_idx;
    R.csr_w = g->csr_w;
    R.csc_w = g->csc_w;
    R.inv_deg = g->inv_deg;
    R.push_rank = g->push_bins.rank;
    R.push_cstart = g->push_bins.cstart;
    R.push_chunks = g->push_bins.chunks;
    R.pull_rank = g->pull_bins.rank;
    R.pull_cstart = g->pull_bins.cstart;
    R.pull_chunks = g->pull_bins.chunks;
    R.pull_nchunks = g->pull_bins.nchunks;
    R.d = damping;
    R.eps = (float)eps;
    R.alpha = g->opt.fe_alpha;
    R.s = sp;
    R.mode = mode;
    R.iters = iters;
    R.x = x;
    R.r = w.r;
    R.acc = w.acc;
    R.c[0] = w.c[0];
    R.c[1] = w.c[1];
    R.part = w.part;
    for (int i = 0; i < 3; ++i) R.act[i] = w.act[i];
    R.hq = w.hq;
    R.ctr = w.ctr;
    R.stats = w.stats;
    R.summary = w.summary;
    R.sync = w.sync;
    if (dirs) {
        const int nd = std::min(ndirs, GP_FE_MAX_ITERS);
        GP_CUDA(cudaMemcpyAsync(w.dirs, dirs, nd, cudaMemcpyHostToDevice, s));
        R.dirs = w.dirs;
        R.ndirs = nd;
    }
    GP_CUDA(cudaMemsetAsync(w.sync, 0, sizeof(GridSync), s));
    {
        ProfScope ps("pr_fe_persistent", s);
        void *args[] = {&R};
        GP_CUDA(cudaLaunchCooperativeKernel((const void *)k_pr_fe, dim3((unsigned)w.grid), dim3(FE_THREADS), args, 0, s));
    }
    if (!x_dev) GP_CUDA(cudaMemcpyAsync(ranks_out, x, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    char *h = (char *)w.host;
    FeSummary *hs = (FeSummary *)h;
    FeIterStat *hl = (FeIterStat *)(h + sizeof(FeSummary));
    GridSync *hsync = (GridSync *)(h + sizeof(FeSummary) + GP_FE_MAX_ITERS * sizeof(FeIterStat));
    GP_CUDA(cudaMemcpyAsync(hsync, w.sync, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(hs, w.summary, sizeof(FeSummary), cudaMemcpyDeviceToHost, s));
    if (stats) {
        GP_CUDA(cudaMemcpyAsync(hl, w.stats, GP_FE_MAX_ITERS * sizeof(FeIterStat), cudaMemcpyDeviceToHost, s));
        GP_CUDA(cudaEventRecord(ev1, s));
    }
    GP_CUDA(cudaStreamSynchronize(s));
    dev_free(sbuf, s);
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats->iterations = (int32_t)hs->iterations;
        stats->pushes = (int32_t)hs->pushes;
        stats->pulls = (int32_t)hs->pulls;
        stats->residual_l1 = hs->residual;
        stats->error_bound = hs->residual / (1.0 - (double)damping);
        stats->ms = ms;
        stats->init_ns = (int32_t)std::min<int64_t>(hs->init_ns, INT32_MAX);
        stats->frontier_left = hs->left;
        const int L = (int)std::min<int64_t>(hs->iterations, GP_FE_MAX_ITERS);
        for (int i = 0; i < L; ++i) {
            stats->direction[i] = (int8_t)hl[i].direction;
            stats->frontier[i] = hl[i].frontier;
            stats->examined[i] = hl[i].examined;
            stats->iter_ns[i] = hl[i].ns;
        }
    }
    if (hsync->err) return set_error(GP_ERR_TIMEOUT, "gp_pagerank_fe: a grid barrier wait ran out");
    if (hs->left > 0 && eps >= 0.0)  // the cap was reached first: the ranks are the last iterate
        return set_error(GP_ERR_NOT_CONVERGED, "gp_pagerank_fe: %lld vertices still in the frontier after %d iterations",
                         (long long)hs->left, iters);
    return GP_OK;
}
