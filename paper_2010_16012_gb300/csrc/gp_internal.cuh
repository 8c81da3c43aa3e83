// gp_internal.cuh -- shared internals of libgp: the graph handle, error and
// allocation plumbing, launch/profiling helpers and warp/block primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gp.h"

namespace gp {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP = 32;

// ------------------------------------------------------------------ errors

int set_error(int status, const char *fmt, ...);  // records the message, returns status
void clear_error();

#define GP_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return ::gp::set_error(GP_ERR_CUDA, "%s failed: %s (%s:%d)", #call,              \
                                   cudaGetErrorString(_e), __FILE__, __LINE__);                \
    } while (0)

#define GP_TRY(expr)              \
    do {                          \
        int _s = (expr);          \
        if (_s != GP_OK) return _s; \
    } while (0)

// ------------------------------------------------------------------ memory

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    gp_free_fn free_fn = nullptr;  // nullptr = cudaFreeAsync
    void *ctx = nullptr;
};

// Allocate `bytes` of device memory through the registered allocator.
int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s);
void dev_free(DevBuf &b, cudaStream_t s);
// Page-locked host blocks (status mirrors), reused across graphs.
int pinned_alloc(void **p, size_t bytes);
void pinned_free(void *p, size_t bytes);
// The address under which kernels on the current device write a pinned block.
int pinned_device_ptr(void *host, void **dev);
// Device-to-host read of a result the host waits for (sizes, counts, flags):
// a kernel on `s` writes it into a mapped page-locked block, then `s` is
// synchronised.  No copy-engine transfer is involved, so the read never waits
// behind large copies the caller has in flight on other streams.
cudaError_t read_mapped(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Owned allocations of a handle (freed together).
struct Arena {
    std::vector<DevBuf> bufs;
    size_t total = 0;
    template <class T>
    int alloc(T *&out, size_t count, cudaStream_t s) {
        DevBuf b;
        int st = dev_alloc(b, (count ? count : 1) * sizeof(T), s);
        if (st != GP_OK) return st;
        bufs.push_back(b);
        total += b.bytes;
        out = static_cast<T *>(b.ptr);
        return GP_OK;
    }
    void release(cudaStream_t s) {
        for (auto &b : bufs) dev_free(b, s);
        bufs.clear();
        total = 0;
    }
};

// Memory kind of a user pointer: true if the device can dereference it as device memory.
bool is_device_ptr(const void *p);

// ------------------------------------------------------------------ profiling

// Launch bookkeeping: with profiling on, brackets a launch with CUDA events.
struct ProfScope {
    int slot = -1;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
};

#define GP_LAUNCH(name, stream, ...)                      \
    do {                                                  \
        ::gp::ProfScope _ps(name, stream);                \
        __VA_ARGS__;                                      \
    } while (0)

int check_launch(const char *what);  // cudaGetLastError -> status

// ------------------------------------------------------------------ graph handle

// A contiguous piece of one vertex's adjacency list processed by one warp.
struct __align__(16) Chunk {
    int64_t beg;  // first edge slot
    int32_t len;  // edges in the piece (<= chunk_edges)
    int32_t v;    // vertex whose list it is
};

// Vertices whose degree exceeds the light limit, split into warp-sized chunks.
struct BigBins {
    int64_t nbig = 0;
    int64_t nchunks = 0;
    int32_t *big = nullptr;     // [nbig] ascending vertex ids
    int64_t *cstart = nullptr;  // [nbig + 1] first chunk of each big vertex
    Chunk *chunks = nullptr;    // [nchunks]
    int32_t *rank = nullptr;    // [n] position of v in `big`, -1 for light vertices
    int32_t light_max = 0;
    int32_t chunk_edges = 0;
    Arena mem;
};

// Contributions of the H most gathered vertices (largest out-degree), kept in
// shared memory by the pull kernels: enc_idx is the CSC index array with each
// such vertex u replaced by HOT_BIT | slot(u); c_hot[slot] mirrors c[u].
constexpr uint32_t HOT_BIT = 0x80000000u;
struct HotSet {
    int32_t slots = 0;  // requested H (0 = off)
    int64_t nhot = 0;
    int32_t *hot_id = nullptr;   // [nhot] vertex of each slot
    float *c_hot = nullptr;      // [nhot]
    int32_t *enc_idx = nullptr;  // [m]
    Arena mem;
};

// Cached PageRank workspace (sized for the graph; reused across calls).
struct PrWork {
    bool ready = false;
    float *r1 = nullptr;           // second rank buffer
    float *c0 = nullptr, *c1 = nullptr;  // contribution buffers x*P-scale
    float *s_dev = nullptr;        // personalization copy (host input)
    float *x0_dev = nullptr;       // start vector copy (host input)
    float *out_dev = nullptr;      // output buffer when ranks_out is host memory
    double *partials = nullptr;    // per-block residual partials
    float *chunk_part = nullptr;   // per-chunk partial sums (pull, big vertices)
    double *acc64 = nullptr;       // FP64 accumulator of the push scatter
    float *lam = nullptr;          // adjoint solution
    float *gw_dev = nullptr;       // weight gradient when the output is host memory
    void *status = nullptr;        // device PrStatus
    void *status_host = nullptr;   // pinned mirror (written by the kernels)
    void *status_mirror = nullptr; // its device-side address
    int max_blocks = 0;
    Arena mem;
};

// Cached BFS workspace.
struct BfsWork {
    bool ready = false;
    int32_t *queue[2] = {nullptr, nullptr};  // light frontier vertices
    int32_t *hchunk[2] = {nullptr, nullptr}; // heavy frontier: indices into the push chunk table
    uint32_t *bits[3] = {nullptr, nullptr, nullptr};  // frontier bitmaps, a ring: level k in bits[k % 3]
    uint32_t *unvis = nullptr;               // vertices possibly unvisited with in-edges (bottom-up candidates)
    uint32_t *nzin = nullptr;                // vertices with in-edges (the initial candidates)
    int32_t *level_dev = nullptr, *parent_dev = nullptr;  // when outputs are host memory
    void *ctr = nullptr;                     // device counters
    void *ctr_host = nullptr;                // pinned mirror of the summary, level stats and barrier word
    void *stats = nullptr;                   // per-level statistics (device)
    void *summary = nullptr;                 // search summary (device)
    void *sync = nullptr;                    // grid barrier word
    int8_t *dirs = nullptr;                  // forced directions (device copy)
    int dirs_cap = 0;                        // entries `dirs` holds
    int grid = 0;                            // blocks of the cooperative launch
    cudaEvent_t done_ev = nullptr;           // end of the last asynchronous search
    bool pending = false;                    // its barrier status not yet checked
    Arena mem;
    // gp_bfs_multi: one frontier workspace per group of blocks, and the tables
    // of one call (group runs, sources, output pointers) staged through pinned memory
    struct Group {
        int32_t *queue[2], *hchunk[2];
        uint32_t *bits[3], *unvis;
        void *ctr;
    };
    std::vector<Group> mgrp;
    int msrc_cap = 0;                        // searches the tables hold
    void *mtab = nullptr;                    // device copy of the staged tables
    void *msummary = nullptr;                // per-search summaries (device)
    void *msync = nullptr;                   // a barrier word per group (device)
    int32_t *mdraw = nullptr;                // the next search to hand out, then two slots per group (device)
    void *mhost = nullptr;                   // pinned: staged tables, then summaries and barrier words
    size_t mhost_bytes = 0;
    cudaEvent_t mdone_ev = nullptr;          // end of the last asynchronous gp_bfs_multi
    bool mpending = false;                   // its barrier status not yet checked
    Arena mmem;
};

}  // namespace gp

struct gp_sssp_work;  // shortest-path workspace (sssp.cu)
struct gp_fe_work;    // Frontier-Exploit PageRank workspace (pr_fe.cu)
struct gp_bc_work;    // betweenness-centrality workspace (bc.cu)

struct gp_graph {
    int device = 0;
    int num_sms = 0;
    int64_t l2_bytes = 0;  // the device's L2 cache size
    int64_t n = 0, m = 0;
    bool symmetric = false, weighted = false, normalized = false;
    const int64_t *csr_off = nullptr, *csc_off = nullptr;
    const int32_t *csr_idx = nullptr, *csc_idx = nullptr;
    const float *csr_w = nullptr, *csc_w = nullptr;
    float *inv_deg = nullptr;  // [n]: 1/deg_out, 1/sum(w) (NORMALIZE) or 1 (weighted as given); 0 if dangling
    int64_t max_out = 0, max_in = 0, isolated = 0;
    gp_options opt;
    gp::BigBins pull_bins;  // by in-degree (CSC)
    gp::BigBins push_bins;  // by out-degree (CSR)
    gp::BigBins bfs_bins;   // by out-degree at bfs_light_max (BFS top-down), when it differs from push_light_max
    gp::HotSet pull_hot;    // shared-memory contribution cache of the pull sweep
    gp::HotSet push_hot;    // shared-memory accumulators of the push scatter
    gp::PrWork pr;
    gp::BfsWork bfs;
    gp_sssp_work *sssp = nullptr;
    gp_fe_work *fe = nullptr;
    gp_bc_work *bc = nullptr;
    gp::Arena mem;          // copies of the arrays and degree data
    cudaStream_t home = nullptr;
};

namespace gp {

int build_bins(gp_graph *g, BigBins &b, const int64_t *off, int32_t light_max, int32_t chunk_edges,
               cudaStream_t s);
// The `slots` vertices of largest degree by sel_off, and enc_src (an index array
// of m entries) with each of them replaced by HOT_BIT | slot.
int build_hot(gp_graph *g, HotSet &h, int32_t slots, const int64_t *sel_off, const int32_t *enc_src,
              cudaStream_t s);
int build_pull_hot(gp_graph *g, int32_t slots, cudaStream_t s);
int build_push_hot(gp_graph *g, int32_t slots, cudaStream_t s);
int select_by_degree(const int64_t *off, int64_t n, int64_t lo, int64_t hi, Arena &mem, int32_t *&list,
                     int64_t &count, int64_t cap, int32_t *rank, cudaStream_t s);
int grid_blocks(const gp_graph *g, int threads_per_block);

// ------------------------------------------------------------------ device primitives

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T t = __shfl_xor_sync(FULL, v, o);
        v = t > v ? t : v;
    }
    return v;
}

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
template <class T>
__device__ __forceinline__ T block_sum(T v, T *smem /* >= 32 entries */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane_id() == 0) smem[w] = v;
    __syncthreads();
    T r = T(0);
    if (w == 0) {
        r = lane_id() < nw ? smem[lane_id()] : T(0);
        r = warp_sum(r);
    }
    return r;
}

// Per-thread part of the L1 residual sum |y - x|: compensated (Kahan) FP32
// summation, whose error does not grow with the number of terms, converted to
// FP64 for the cross-thread reduction (warp, block, grid partials are FP64).
// FP64 arithmetic per vertex would run on this GPU's narrow FP64 pipe.
struct ResSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void push(float v) {
        v -= c;
        const float t = s + v;
        c = (t - s) - v;
        s = t;
    }
    __device__ __forceinline__ void add(float y, float x) { push(fabsf(y - x)); }
    __device__ __forceinline__ float getf() const { return s - c; }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
    // Warp total (valid in every lane): compensated pairwise sums in FP32, one
    // conversion to FP64 at the end.
    __device__ __forceinline__ double warp_total() const {
        float hi = s, lo = -c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ohi = __shfl_xor_sync(0xffffffffu, hi, o), olo = __shfl_xor_sync(0xffffffffu, lo, o);
            const float t = hi + ohi;  // error-free: t + e == hi + ohi (Knuth's two-sum)
            const float bp = t - hi;
            const float e = (hi - (t - bp)) + (ohi - bp);
            hi = t;
            lo = lo + olo + e;
        }
        return (double)hi + (double)lo;
    }
};

// Block total of per-thread residual sums (valid in thread 0): warp totals
// from warp_total, then an FP64 sum over the block's warps in warp order.
__device__ __forceinline__ double block_residual(const ResSum &r, double *smem /* >= 32 entries */) {
    const double wt = r.warp_total();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) smem[w] = wt;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t += smem[i];
    return t;
}

// binary64 -> binary32, round to nearest (ties to even), by integer operations
// on the IEEE 754 encodings (1 sign, 11/8 exponent bits with bias 1023/127,
// 52/23 fraction bits).  Results below the binary32 normal range (|v| < 2^-126)
// become signed zero; results above it become infinity; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e11 = (int)((b >> 52) & 0x7ff);
    const unsigned long long frac = b & 0xfffffffffffffull;
    if (e11 == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u));
    const int e8 = e11 - 1023 + 127;
    if (e8 <= 0) return __uint_as_float(sign);
    if (e8 >= 0xff) return __uint_as_float(sign | 0x7f800000u);
    const unsigned keep = (unsigned)(frac >> 29);                // top 23 fraction bits
    const unsigned rest = (unsigned)(frac & 0x1fffffffull);       // 29 dropped bits
    unsigned r = ((unsigned)e8 << 23) | keep;
    if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) ++r;  // a carry into the exponent is exact
    return __uint_as_float(sign | r);  // a carry out of e8 = 254 gives 0x7f800000: infinity
}

// Position of the j-th (0-based) set bit of x (j < popc(x)).
__device__ __forceinline__ int nth_set_bit(uint32_t x, int j) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(x & ((1u << s) - 1u));
        if (j >= c) {
            j -= c;
            x >>= s;
            pos += s;
        }
    }
    return pos;
}

// ------------------------------------------------------------------ grid barrier

// Grid-wide barrier for cooperative launches (all blocks co-resident).  The
// spin-wait has an iteration limit: a block that gives up sets `err`, every
// other waiting block sees it and gives up too, and all of them return false so
// the kernel can return; the host then reports GP_ERR_TIMEOUT.
struct GridSync {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

constexpr unsigned long long GRID_SPIN_LIMIT = 1ull << 24;  // ~2 s of 128 ns sleeps

// Returns false (and sets gs->err for every block) when a wait runs past
// `limit` sleeps or another block has already given up.
__device__ __forceinline__ bool grid_sync(GridSync *gs, unsigned nblocks, unsigned long long limit = GRID_SPIN_LIMIT) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gs->gen;
        volatile int *verr = &gs->err;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gs->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == g0) {
                if (*verr || ++spins > limit) {
                    atomicExch(&gs->err, 1);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = *verr == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace gp
