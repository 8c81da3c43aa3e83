// runtime.cu -- libgp runtime: status/error text, allocator hook, kernel timing,
// options, and gp_graph_upload (validation, degree preparation, degree bins).
//
// Graph layout: Section 2.2 of the paper (contiguous neighbour arrays plus
// per-vertex offsets); CSR = out-edges (push), CSC = in-edges (pull), as the
// paper's Section 4.8 ("Directed Graphs") distinguishes them.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "gp_internal.cuh"

namespace gp {

// ------------------------------------------------------------------ errors

static thread_local std::string t_last_error;

int set_error(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return status;
}

void clear_error() { t_last_error.clear(); }

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return GP_OK;
}

// ------------------------------------------------------------------ allocator

static std::mutex g_alloc_mu;
static gp_alloc_fn g_alloc = nullptr;
static gp_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

// Without a registered allocator, workspace comes from a memory pool of the
// library's own per device, which keeps freed memory for reuse (release
// threshold: no limit) instead of returning it to the driver at every stream
// synchronisation: a graph uploaded again (same sizes) then costs no new
// mappings.  Process-local; nullptr where the device has no pool support.
constexpr int GP_MAX_DEVICES = 64;
static cudaMemPool_t g_pool[GP_MAX_DEVICES];
static bool g_pool_tried[GP_MAX_DEVICES];

static cudaMemPool_t lib_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= GP_MAX_DEVICES) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (!g_pool_tried[dev]) {
        g_pool_tried[dev] = true;
        int ok = 0;
        cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev);
        cudaMemPool_t pool = nullptr;
        if (ok) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
                unsigned long long keep = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            } else {
                pool = nullptr;
            }
        }
        cudaGetLastError();
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

// Page-locked host blocks.  Every graph takes a few small ones (the host
// mirrors of the kernels' status words); page-locking is a driver call that
// pins pages and now and then takes milliseconds, so a freed block is kept and
// handed out again for the same size (gp_pool_trim releases the kept ones).
// Portable: one block may serve graphs on any device.  Mapped: kernels may
// write a block directly (pinned_device_ptr), so a status the host polls
// needs no copy, which would queue behind any large transfer the caller has
// in flight on the copy engines.
static std::mutex g_pin_mu;
static std::vector<std::pair<size_t, void *>> g_pin_free;
constexpr size_t PIN_KEEP_MAX = 256;

int pinned_alloc(void **p, size_t bytes) {
    *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_pin_free.size(); ++i) {
            if (g_pin_free[i].first == bytes) {
                *p = g_pin_free[i].second;
                g_pin_free[i] = g_pin_free.back();
                g_pin_free.pop_back();
                return GP_OK;
            }
        }
    }
    GP_CUDA(cudaHostAlloc(p, bytes, cudaHostAllocPortable | cudaHostAllocMapped));
    return GP_OK;
}

int pinned_device_ptr(void *host, void **dev) {
    GP_CUDA(cudaHostGetDevicePointer(dev, host, 0));
    return GP_OK;
}

void pinned_free(void *p, size_t bytes) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (g_pin_free.size() < PIN_KEEP_MAX) {
            g_pin_free.emplace_back(bytes, p);
            return;
        }
    }
    cudaFreeHost(p);
}

static __global__ void k_copy_bytes(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst,
                                    size_t bytes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < bytes; i += stride) dst[i] = src[i];
    __threadfence_system();
}

cudaError_t read_mapped(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaStreamSynchronize(s);
    const size_t cap = (bytes + 4095) & ~size_t(4095);  // pooled by size: a few distinct sizes
    void *h = nullptr, *d = nullptr;
    if (pinned_alloc(&h, cap) != GP_OK) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)std::min<size_t>((bytes + 4095) / 4096, 64);
        k_copy_bytes<<<blocks, 256, 0, s>>>((const unsigned char *)src, (unsigned char *)d, bytes);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) memcpy(dst, h, bytes);
    pinned_free(h, cap);
    return e;
}

static void pinned_release_all() {
    std::vector<std::pair<size_t, void *>> blocks;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        blocks.swap(g_pin_free);
    }
    for (auto &b : blocks) cudaFreeHost(b.second);
}

int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s) {
    gp_alloc_fn fn;
    gp_free_fn ffn;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fn = g_alloc;
        ffn = g_free;
        ctx = g_alloc_ctx;
    }
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (fn) {
        p = fn(bytes, (void *)s, ctx);
        if (!p) return set_error(GP_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
    } else {
        cudaMemPool_t pool = lib_pool();
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(GP_ERR_OOM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    b.ptr = p;
    b.bytes = bytes;
    b.free_fn = fn ? ffn : nullptr;
    b.ctx = ctx;
    return GP_OK;
}

void dev_free(DevBuf &b, cudaStream_t s) {
    if (!b.ptr) return;
    if (b.free_fn)
        b.free_fn(b.ptr, b.bytes, (void *)s, b.ctx);
    else
        cudaFreeAsync(b.ptr, s);
    b.ptr = nullptr;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ kernel timing

struct ProfEntry {
    std::string name;
    int64_t launches = 0;
    double total_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfEntry> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t get_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

ProfScope::ProfScope(const char *name, cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    for (size_t i = 0; i < g_prof.size(); ++i)
        if (g_prof[i].name == name) slot = (int)i;
    if (slot < 0) {
        g_prof.push_back(ProfEntry());
        g_prof.back().name = name;
        slot = (int)g_prof.size() - 1;
    }
    a = get_event();
    b = get_event();
    if (!a || !b) {
        slot = -1;
        return;
    }
    cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
    if (slot < 0) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof[slot].pending.emplace_back(a, b);
    g_prof[slot].launches++;
}

// ------------------------------------------------------------------ scans (upload only)

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ int64_t block_excl_scan_i64(int64_t v, int64_t *smem, int64_t &total) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < nw ? smem[lane] : 0;
        int64_t si = warp_incl_scan(s);
        if (lane < nw) smem[lane] = si - s;
        if (lane == nw - 1) smem[32] = si;
    }
    __syncthreads();
    int64_t r = smem[w] + inc - v;
    total = smem[32];
    __syncthreads();
    return r;
}

__global__ void k_tile_sums(const int64_t *in, int64_t N, int64_t *sums) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t j = base + i;
        if (j < N) acc += in[j];
    }
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Exclusive scan of one tile per block; adds offs[blockIdx] (if given); the
// block holding the last element also writes the grand total to out[N].
__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t N, const int64_t *offs) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t vals[SCAN_ITEMS];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i;
        vals[i] = j < N ? in[j] : 0;
        local += vals[i];
    }
    int64_t total;
    int64_t pre = block_excl_scan_i64(local, sm, total);
    if (offs) pre += offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i;
        if (j < N) out[j] = pre;
        pre += vals[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[N] = (offs ? offs[blockIdx.x] : 0) + total;
}

// out[0..N] = exclusive prefix sums of in[0..N) and the total at out[N].  out may alias in.
static int exclusive_scan(const int64_t *in, int64_t *out, int64_t N, Arena &tmp, cudaStream_t s) {
    if (N <= 0) {
        GP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return GP_OK;
    }
    int64_t nb = (N + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        GP_LAUNCH("scan_tiles", s, (k_scan_tiles<<<1, SCAN_THREADS, 0, s>>>(in, out, N, nullptr)));
        return check_launch("scan");
    }
    int64_t *sums;
    GP_TRY(tmp.alloc(sums, nb + 1, s));
    GP_LAUNCH("tile_sums", s, (k_tile_sums<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, N, sums)));
    GP_TRY(check_launch("scan sums"));
    GP_TRY(exclusive_scan(sums, sums, nb, tmp, s));
    GP_LAUNCH("scan_tiles", s, (k_scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, N, sums)));
    return check_launch("scan tiles");
}

// ------------------------------------------------------------------ validation kernels

enum : unsigned {
    BAD_OFF_FIRST = 1u,
    BAD_OFF_LAST = 2u,
    BAD_OFF_ORDER = 4u,
    BAD_INDEX = 8u,
};

__global__ void k_check_offsets(const int64_t *off, int64_t n, int64_t m, unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (off[i + 1] < off[i]) atomicOr(err, BAD_OFF_ORDER);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (off[0] != 0) atomicOr(err, BAD_OFF_FIRST);
        if (off[n] != m) atomicOr(err, BAD_OFF_LAST);
    }
}

__global__ void k_check_indices(const int32_t *idx, int64_t m, int64_t n, unsigned *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        int32_t v = idx[i];
        bad |= (v < 0) | ((int64_t)v >= n);
    }
    if (__any_sync(FULL, bad) && lane_id() == 0) atomicOr(err, BAD_INDEX);
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Order-independent fingerprint of an edge multiset: sum over edges of
// mix64(key(u, v, weight bits)), warp per vertex.  by_column: the list of
// vertex x holds tails (edges idx -> x) instead of heads (x -> idx); swap:
// fingerprint the reversed edges (symmetry check).
__global__ void k_edge_fingerprint(const int64_t *off, const int32_t *idx, const float *w, int64_t n,
                                   int by_column, int swap, unsigned long long *out) {
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t x = warp; x < n; x += nwarps) {
        for (int64_t j = off[x] + lane; j < off[x + 1]; j += 32) {
            unsigned long long u = by_column ? (unsigned)idx[j] : (unsigned long long)x;
            unsigned long long v = by_column ? (unsigned long long)x : (unsigned)idx[j];
            if (swap) {
                unsigned long long t = u;
                u = v;
                v = t;
            }
            unsigned long long key = (u << 32) | v;
            unsigned long long h = mix64(key * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull);
            if (w) h += mix64((unsigned long long)__float_as_uint(w[j]) + key * 0x94D049BB133111EBull);
            acc += h;
        }
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc) atomicAdd(out, acc);
}

// ------------------------------------------------------------------ degree preparation

struct DegStats {
    unsigned long long max_out, max_in, isolated;
};

// inv_deg[u] = 1/deg_out(u) (unweighted), 1/sum_v w_uv (NORMALIZE) or 1 (weights as given); 0 if dangling.
__global__ void k_degree_prep(const int64_t *csr_off, const int64_t *csc_off, const float *csr_w, int64_t n,
                              int weighted, int normalize, float *inv_deg, DegStats *st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long mo = 0, mi = 0, iso = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t b = csr_off[u], e = csr_off[u + 1];
        const int64_t dout = e - b, din = csc_off[u + 1] - csc_off[u];
        float inv = 0.f;
        if (dout > 0) {
            if (!weighted) {
                inv = 1.0f / (float)dout;
            } else if (normalize) {
                double sw = 0.0;
                for (int64_t j = b; j < e; ++j) sw += (double)csr_w[j];
                inv = sw > 0.0 ? (float)(1.0 / sw) : 0.f;
            } else {
                inv = 1.f;
            }
        }
        inv_deg[u] = inv;
        mo = max(mo, (unsigned long long)dout);
        mi = max(mi, (unsigned long long)din);
        iso += (dout == 0 && din == 0);
    }
    mo = warp_max(mo);
    mi = warp_max(mi);
    iso = warp_sum(iso);
    if (lane_id() == 0) {
        atomicMax(&st->max_out, mo);
        atomicMax(&st->max_in, mi);
        if (iso) atomicAdd(&st->isolated, iso);
    }
}

// ------------------------------------------------------------------ degree bins

constexpr int BIN_SEG = 2048;  // vertices per block segment in the selection kernels

// Vertices v with lo <= off[v+1] - off[v] <= hi, per block segment: count, then
// write them in ascending order (and rank[v], -1 for the others, if given).
__global__ void k_count_deg(const int64_t *off, int64_t n, int64_t lo, int64_t hi, int64_t *counts) {
    __shared__ int64_t sm[33];
    const int64_t base = (int64_t)blockIdx.x * BIN_SEG;
    int64_t c = 0;
    for (int i = threadIdx.x; i < BIN_SEG; i += blockDim.x) {
        int64_t v = base + i;
        if (v < n) {
            const int64_t d = off[v + 1] - off[v];
            c += (d >= lo && d <= hi);
        }
    }
    c = block_sum(c, sm);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void k_write_deg(const int64_t *off, int64_t n, int64_t lo, int64_t hi, const int64_t *seg_off, int64_t cap,
                            int32_t *list, int32_t *rank) {
    __shared__ int32_t warp_cnt[32];
    __shared__ int64_t running;
    const int64_t base = (int64_t)blockIdx.x * BIN_SEG;
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) running = seg_off[blockIdx.x];
    __syncthreads();
    for (int i0 = 0; i0 < BIN_SEG; i0 += blockDim.x) {
        int64_t v = base + i0 + threadIdx.x;
        bool sel = false;
        if (v < n) {
            const int64_t d = off[v + 1] - off[v];
            sel = d >= lo && d <= hi;
        }
        unsigned bal = __ballot_sync(FULL, sel);
        if (lane == 0) warp_cnt[w] = __popc(bal);
        __syncthreads();
        int64_t pos = running;
        for (int k = 0; k < w; ++k) pos += warp_cnt[k];
        pos += __popc(bal & ((1u << lane) - 1u));
        if (rank && v < n) rank[v] = sel ? (int32_t)pos : -1;
        if (sel && pos < cap) list[pos] = (int32_t)v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t t = 0;
            for (int k = 0; k < nw; ++k) t += warp_cnt[k];
            running += t;
        }
        __syncthreads();
    }
}

int select_by_degree(const int64_t *off, int64_t n, int64_t lo, int64_t hi, Arena &mem, int32_t *&list,
                     int64_t &count, int64_t cap, int32_t *rank, cudaStream_t s) {
    count = 0;
    list = nullptr;
    if (n == 0) return GP_OK;
    const int64_t nseg = (n + BIN_SEG - 1) / BIN_SEG;
    Arena tmp;
    int64_t *segc;
    int st = tmp.alloc(segc, nseg + 1, s);
    if (st == GP_OK) {
        GP_LAUNCH("count_deg", s, (k_count_deg<<<(unsigned)nseg, 256, 0, s>>>(off, n, lo, hi, segc)));
        st = check_launch("count_deg");
    }
    if (st == GP_OK) st = exclusive_scan(segc, segc, nseg, tmp, s);
    int64_t total = 0;
    if (st == GP_OK) {
        cudaError_t e = read_mapped(&total, segc + nseg, sizeof(int64_t), s);
        if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "selection count read-back: %s", cudaGetErrorString(e));
    }
    const int64_t keep = std::min(total, cap);
    if (st == GP_OK) st = mem.alloc(list, (size_t)std::max<int64_t>(keep, 1), s);
    if (st == GP_OK) {
        GP_LAUNCH("write_deg", s, (k_write_deg<<<(unsigned)nseg, 256, 0, s>>>(off, n, lo, hi, segc, keep, list, rank)));
        st = check_launch("write_deg");
    }
    tmp.release(s);
    count = keep;
    return st;
}

__global__ void k_chunk_counts(const int32_t *big, int64_t nbig, const int64_t *off, int32_t C, int64_t *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nbig; r += stride) {
        const int32_t v = big[r];
        const int64_t d = off[v + 1] - off[v];
        cnt[r] = (d + C - 1) / C;
    }
}

__global__ void k_fill_chunks(const int32_t *big, int64_t nbig, const int64_t *off, const int64_t *cstart,
                              int32_t C, Chunk *chunks) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nbig; r += stride) {
        const int32_t v = big[r];
        const int64_t b = off[v], e = off[v + 1];
        int64_t j = cstart[r];
        for (int64_t p = b; p < e; p += C, ++j) {
            Chunk ch;
            ch.beg = p;
            ch.len = (int32_t)((e - p) < (int64_t)C ? (e - p) : (int64_t)C);
            ch.v = v;
            chunks[j] = ch;
        }
    }
}

constexpr int HOT_HIST = 65536;  // out-degree histogram buckets (the last one collects all larger degrees)

constexpr int HOT_HIST_SMEM = 8192;  // low buckets counted per block in shared memory

// Degree histogram; the low buckets, which almost every vertex falls into, are
// counted in shared memory first so the global atomics are one per bucket and block.
__global__ void k_deg_hist(const int64_t *off, int64_t n, unsigned long long *hist) {
    __shared__ unsigned sh[HOT_HIST_SMEM];
    for (int i = threadIdx.x; i < HOT_HIST_SMEM; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = off[v + 1] - off[v];
        if (d <= 0) continue;
        if (d < HOT_HIST_SMEM)
            atomicAdd(sh + d, 1u);
        else
            atomicAdd(hist + (d < HOT_HIST - 1 ? d : HOT_HIST - 1), 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HOT_HIST_SMEM; i += blockDim.x)
        if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
}

__global__ void k_fill_slots(const int32_t *hot_id, int64_t nhot, int32_t *slot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nhot; i += stride) slot[hot_id[i]] = (int32_t)i;
}

__global__ void k_encode_hot(const int32_t *idx, int64_t m, const int32_t *slot, int32_t *enc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t u = idx[e];
        const int32_t sl = slot[u];
        enc[e] = sl >= 0 ? (int32_t)(HOT_BIT | (uint32_t)sl) : u;
    }
}

// Picks the `slots` vertices with the largest degree by `sel_off` (ties: lowest
// ids), builds the copy of `enc_src` (an index array of the graph) with those
// vertices encoded as HOT_BIT | slot, and the slot -> vertex table.
int build_hot(gp_graph *g, HotSet &h, int32_t slots, const int64_t *sel_off, const int32_t *enc_src,
              cudaStream_t s) {
    h.mem.release(s);
    h = HotSet();
    h.slots = slots;
    const int64_t n = g->n, m = g->m;
    if (slots <= 0 || n == 0 || m == 0) return GP_OK;
    Arena tmp;
    unsigned long long *hist = nullptr;
    int st = tmp.alloc(hist, HOT_HIST, s);
    std::vector<unsigned long long> hh(HOT_HIST);
    if (st == GP_OK) {
        cudaError_t e = cudaMemsetAsync(hist, 0, HOT_HIST * sizeof(unsigned long long), s);
        int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->num_sms * 8));
        if (e == cudaSuccess) {
            GP_LAUNCH("deg_hist", s, (k_deg_hist<<<blocks, 256, 0, s>>>(sel_off, n, hist)));
            e = read_mapped(hh.data(), hist, HOT_HIST * sizeof(unsigned long long), s);
        }
        if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "hot-set histogram: %s", cudaGetErrorString(e));
    }
    // bucket B: every vertex above B is taken, then the lowest ids of bucket B until `slots`
    int64_t above = 0;
    int B = 0;
    if (st == GP_OK) {
        for (int b = HOT_HIST - 1; b >= 1; --b) {
            if (above + (int64_t)hh[b] > slots) {
                B = b;
                break;
            }
            above += (int64_t)hh[b];
        }
    }
    int32_t *list1 = nullptr, *list2 = nullptr;
    int64_t c1 = 0, c2 = 0;
    const int64_t top_lo = B > 0 ? (int64_t)B + 1 : 1;
    if (st == GP_OK && top_lo <= HOT_HIST - 1)
        st = select_by_degree(sel_off, n, top_lo, INT64_MAX, tmp, list1, c1, slots, nullptr, s);
    if (st == GP_OK && B > 0) {
        const int64_t hi = B == HOT_HIST - 1 ? INT64_MAX : (int64_t)B;
        st = select_by_degree(sel_off, n, B, hi, tmp, list2, c2, slots - c1, nullptr, s);
    }
    const int64_t nhot = c1 + c2;
    int32_t *slot = nullptr;
    if (st == GP_OK) st = h.mem.alloc(h.hot_id, (size_t)std::max<int64_t>(nhot, 1), s);
    if (st == GP_OK) st = h.mem.alloc(h.c_hot, (size_t)std::max<int64_t>(nhot, 4), s);
    if (st == GP_OK) st = h.mem.alloc(h.enc_idx, (size_t)m, s);
    if (st == GP_OK) st = tmp.alloc(slot, (size_t)n, s);
    if (st == GP_OK) {
        cudaError_t e = cudaSuccess;
        if (c1) e = cudaMemcpyAsync(h.hot_id, list1, c1 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && c2)
            e = cudaMemcpyAsync(h.hot_id + c1, list2, c2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(slot, 0xff, (size_t)n * sizeof(int32_t), s);
        if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "hot-set copy: %s", cudaGetErrorString(e));
    }
    if (st == GP_OK && nhot > 0) {
        int b1 = (int)std::max<int64_t>(1, std::min<int64_t>((nhot + 255) / 256, 65535));
        GP_LAUNCH("fill_slots", s, (k_fill_slots<<<b1, 256, 0, s>>>(h.hot_id, nhot, slot)));
        int b2 = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 8));
        GP_LAUNCH("encode_hot", s, (k_encode_hot<<<b2, 256, 0, s>>>(enc_src, m, slot, h.enc_idx)));
        st = check_launch("encode_hot");
    }
    if (st == GP_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "hot-set build: %s", cudaGetErrorString(e));
    }
    tmp.release(s);
    if (st != GP_OK) {
        h.mem.release(s);
        h = HotSet();
        return st;
    }
    h.nhot = nhot;
    return GP_OK;
}

// Pull: the most gathered contributions are those of the largest out-degrees;
// the gathered index array is CSC.
int build_pull_hot(gp_graph *g, int32_t slots, cudaStream_t s) {
    return build_hot(g, g->pull_hot, slots, g->csr_off, g->csc_idx, s);
}

// Push: the most updated vertices are those of the largest in-degrees; the
// scattered index array is CSR.
int build_push_hot(gp_graph *g, int32_t slots, cudaStream_t s) {
    return build_hot(g, g->push_hot, slots, g->csc_off, g->csr_idx, s);
}

int grid_blocks(const gp_graph *g, int threads_per_block) {
    int per_sm = std::max(1, g->opt.blocks_per_sm * 256 / std::max(32, threads_per_block));
    return std::max(1, g->num_sms * per_sm);
}

int build_bins(gp_graph *g, BigBins &b, const int64_t *off, int32_t light_max, int32_t chunk_edges,
               cudaStream_t s) {
    b.mem.release(s);
    b.nbig = b.nchunks = 0;
    b.big = nullptr;
    b.cstart = nullptr;
    b.chunks = nullptr;
    b.rank = nullptr;
    b.light_max = light_max;
    b.chunk_edges = chunk_edges;
    const int64_t n = g->n;
    int32_t *rank = nullptr;
    GP_TRY(b.mem.alloc(rank, (size_t)std::max<int64_t>(n, 1), s));
    b.rank = rank;
    if (n == 0) return GP_OK;
    int64_t nbig = 0;
    GP_TRY(select_by_degree(off, n, (int64_t)light_max + 1, INT64_MAX, b.mem, b.big, nbig, INT64_MAX, rank, s));
    Arena tmp;
    int st = b.mem.alloc(b.cstart, (size_t)nbig + 1, s);
    int64_t nchunks = 0;
    if (st == GP_OK && nbig > 0) {
        int blocks = (int)std::min<int64_t>((nbig + 255) / 256, 65535);
        GP_LAUNCH("chunk_counts", s, (k_chunk_counts<<<blocks, 256, 0, s>>>(b.big, nbig, off, chunk_edges, b.cstart)));
        st = check_launch("chunk_counts");
        if (st == GP_OK) st = exclusive_scan(b.cstart, b.cstart, nbig, tmp, s);
        if (st == GP_OK) {
            cudaError_t e = read_mapped(&nchunks, b.cstart + nbig, sizeof(int64_t), s);
            if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "chunk count read-back: %s", cudaGetErrorString(e));
        }
        if (st == GP_OK) st = b.mem.alloc(b.chunks, (size_t)std::max<int64_t>(nchunks, 1), s);
        if (st == GP_OK) {
            GP_LAUNCH("fill_chunks", s, (k_fill_chunks<<<blocks, 256, 0, s>>>(b.big, nbig, off, b.cstart, chunk_edges, b.chunks)));
            st = check_launch("fill_chunks");
        }
    } else if (st == GP_OK) {
        cudaError_t e = cudaMemsetAsync(b.cstart, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) st = set_error(GP_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    }
    tmp.release(s);
    if (st != GP_OK) return st;
    b.nbig = nbig;
    b.nchunks = nchunks;
    return GP_OK;
}

}  // namespace gp

namespace gp {
void release_pr_work(gp_graph *g, cudaStream_t s);
void release_bfs_work(gp_graph *g, cudaStream_t s);
void release_bfs_multi(gp_graph *g, cudaStream_t s);
void release_sssp_work(gp_graph *g, cudaStream_t s);
void release_fe_work(gp_graph *g, cudaStream_t s);
void release_bc_work(gp_graph *g, cudaStream_t s);
}  // namespace gp

using namespace gp;

template <class T>
static int copy_in(gp_graph *g, const T *src, size_t count, const T *&dst, cudaStream_t s) {
    T *p = nullptr;
    GP_TRY(g->mem.alloc(p, count, s));
    if (count) GP_CUDA(cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyDefault, s));
    dst = p;
    return GP_OK;
}


// ================================================================== C ABI

extern "C" {

const char *gp_status_string(int status) {
    switch (status) {
        case GP_OK: return "GP_OK";
        case GP_ERR_INVALID: return "GP_ERR_INVALID: invalid argument or malformed graph";
        case GP_ERR_OOM: return "GP_ERR_OOM: device allocation failed";
        case GP_ERR_CUDA: return "GP_ERR_CUDA: CUDA runtime error";
        case GP_ERR_NOT_CONVERGED: return "GP_ERR_NOT_CONVERGED: sweep cap reached before tol";
        case GP_ERR_TIMEOUT: return "GP_ERR_TIMEOUT: bounded device wait ran out";
        case GP_ERR_UNSUPPORTED: return "GP_ERR_UNSUPPORTED: not supported for this input";
        default: return "unknown gp status";
    }
}

const char *gp_last_error(void) { return t_last_error.c_str(); }

int gp_version(void) { return GP_VERSION; }

int gp_set_allocator(gp_alloc_fn alloc, gp_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return set_error(GP_ERR_INVALID, "gp_set_allocator: give both callbacks or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return GP_OK;
}

int gp_pool_usage(int64_t *reserved_bytes, int64_t *used_bytes) {
    clear_error();
    if (!reserved_bytes || !used_bytes) return set_error(GP_ERR_INVALID, "gp_pool_usage: NULL output");
    *reserved_bytes = 0;
    *used_bytes = 0;
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        if (dev >= 0 && dev < GP_MAX_DEVICES && g_pool_tried[dev]) pool = g_pool[dev];
    }
    if (!pool) return GP_OK;  // never used on this device (or no pool support)
    unsigned long long r = 0, u = 0;
    GP_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    GP_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    *reserved_bytes = (int64_t)r;
    *used_bytes = (int64_t)u;
    return GP_OK;
}

int gp_pool_trim(int64_t keep_bytes) {
    clear_error();
    if (keep_bytes < 0) return set_error(GP_ERR_INVALID, "gp_pool_trim: keep_bytes %lld < 0", (long long)keep_bytes);
    pinned_release_all();
    int dev = 0;
    GP_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        if (dev >= 0 && dev < GP_MAX_DEVICES && g_pool_tried[dev]) pool = g_pool[dev];
    }
    if (!pool) return GP_OK;
    // frees enqueued on streams complete before the trim sees them
    GP_CUDA(cudaDeviceSynchronize());
    GP_CUDA(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
    return GP_OK;
}

int gp_options_default(gp_options *opt) {
    if (!opt) return set_error(GP_ERR_INVALID, "gp_options_default: NULL");
    memset(opt, 0, sizeof(*opt));
    opt->pull_light_max = 16;
    opt->push_light_max = 32;
    opt->chunk_edges = 256;
    opt->blocks_per_sm = 4;
    opt->poll_interval = 8;
    opt->pr_auto_mode = -1;
    opt->bfs_alpha = 14.0f;
    opt->bfs_beta = 24.0f;
    opt->push_fp64_accum = -1;
    opt->pull_hot_slots = 20480;
    opt->push_hot_slots = 32768;
    opt->sssp_alpha = 1.0f;
    opt->fe_alpha = 8.0f;
    opt->bc_alpha = 1.0f;
    opt->bfs_light_max = 32;
    return GP_OK;
}

static __global__ void k_selftest_narrow(int64_t n, const double *in, float *ours, float *hw) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        ours[i] = f64_to_f32_rn(in[i]);
        hw[i] = __double2float_rn(in[i]);
    }
}

int gp_selftest_narrow(int64_t n, const double *in, float *ours, float *hw, void *stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!in || !ours || !hw))) return set_error(GP_ERR_INVALID, "gp_selftest_narrow: bad arguments");
    if (n == 0) return GP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_selftest_narrow<<<blocks, 256, 0, s>>>(n, in, ours, hw);
    GP_CUDA(cudaGetLastError());
    return GP_OK;
}

// Every block but `absent` enters one grid barrier whose waits give up after
// `spins` sleeps.
static __global__ void k_selftest_barrier(GridSync *gs, int absent, unsigned long long spins) {
    if ((int)blockIdx.x == absent) return;
    grid_sync(gs, gridDim.x, spins);
}

int gp_selftest_barrier(int absent, void *stream) {
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, coop = 0;
    GP_CUDA(cudaGetDevice(&dev));
    GP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return set_error(GP_ERR_UNSUPPORTED, "gp_selftest_barrier: no cooperative launch on this device");
    if (absent >= sms) return set_error(GP_ERR_INVALID, "gp_selftest_barrier: block %d outside the grid of %d", absent, sms);
    GridSync *gs = nullptr;
    GP_CUDA(cudaMalloc(&gs, sizeof(GridSync)));
    GridSync host = {};
    cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GridSync), s);
    unsigned long long spins = 1ull << 16;  // a few tens of milliseconds
    void *args[] = {&gs, &absent, &spins};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)k_selftest_barrier, dim3((unsigned)sms), dim3(128), args, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(gs);
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_selftest_barrier: %s", cudaGetErrorString(e));
    if (host.err) return set_error(GP_ERR_TIMEOUT, "gp_selftest_barrier: a grid barrier wait ran out");
    return GP_OK;
}

int gp_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return GP_OK;
}

int gp_profile_read(gp_kernel_time *out, int cap, int *count, int reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_prof) {
        for (auto &ev : p.pending) {
            cudaError_t e = cudaEventSynchronize(ev.second);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_error(GP_ERR_CUDA, "gp_profile_read: %s", cudaGetErrorString(e));
            }
            p.total_ms += ms;
            g_event_pool.push_back(ev.first);
            g_event_pool.push_back(ev.second);
        }
        p.pending.clear();
    }
    std::vector<int> order(g_prof.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [](int a, int b) { return g_prof[a].total_ms > g_prof[b].total_ms; });
    int k = 0;
    for (int i : order) {
        if (k >= cap || !out) break;
        memset(&out[k], 0, sizeof(gp_kernel_time));
        strncpy(out[k].name, g_prof[i].name.c_str(), sizeof(out[k].name) - 1);
        out[k].launches = g_prof[i].launches;
        out[k].total_ms = g_prof[i].total_ms;
        ++k;
    }
    if (count) *count = k;
    if (reset) g_prof.clear();
    return GP_OK;
}

static int upload_fail(gp_graph *g, cudaStream_t s, int st) {
    g->pull_bins.mem.release(s);
    g->push_bins.mem.release(s);
    g->bfs_bins.mem.release(s);
    g->pull_hot.mem.release(s);
    g->push_hot.mem.release(s);
    g->mem.release(s);
    delete g;
    return st;
}

int gp_graph_upload(gp_graph **out, int64_t n, int64_t m, const int64_t *csr_off, const int32_t *csr_idx,
                    const float *csr_w, const int64_t *csc_off, const int32_t *csc_idx, const float *csc_w,
                    unsigned flags, void *stream) {
    clear_error();
    if (!out) return set_error(GP_ERR_INVALID, "gp_graph_upload: out is NULL");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const bool sym = flags & GP_UPLOAD_SYMMETRIC;
    if (n < 0 || n >= (int64_t(1) << 31)) return set_error(GP_ERR_INVALID, "n = %lld outside [0, 2^31)", (long long)n);
    if (m < 0) return set_error(GP_ERR_INVALID, "m = %lld < 0", (long long)m);
    if (!csr_off || (m > 0 && !csr_idx)) return set_error(GP_ERR_INVALID, "CSR arrays missing");
    if (!sym && (!csc_off || (m > 0 && !csc_idx))) return set_error(GP_ERR_INVALID, "CSC arrays missing (no GP_UPLOAD_SYMMETRIC)");
    if (!sym && ((csr_w == nullptr) != (csc_w == nullptr)))
        return set_error(GP_ERR_INVALID, "give weights for both CSR and CSC or for neither");
    if (sym && csc_off) {
        if ((csr_w == nullptr) != (csc_w == nullptr))
            return set_error(GP_ERR_INVALID, "give weights for both CSR and CSC or for neither");
    }
    const bool copy = flags & GP_UPLOAD_COPY;
    if (!copy) {
        if (!is_device_ptr(csr_off) || (m > 0 && !is_device_ptr(csr_idx)) || (csr_w && !is_device_ptr(csr_w)))
            return set_error(GP_ERR_INVALID, "CSR arrays must be device memory without GP_UPLOAD_COPY");
        if (csc_off && (!is_device_ptr(csc_off) || (m > 0 && !is_device_ptr(csc_idx)) || (csc_w && !is_device_ptr(csc_w))))
            return set_error(GP_ERR_INVALID, "CSC arrays must be device memory without GP_UPLOAD_COPY");
    }
    gp_graph *g = new gp_graph();
    GP_CUDA(cudaGetDevice(&g->device));
    GP_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    {
        int l2 = 0;
        GP_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device));
        g->l2_bytes = l2;
    }
    gp_options_default(&g->opt);
    g->n = n;
    g->m = m;
    g->symmetric = sym;
    g->weighted = csr_w != nullptr;
    g->normalized = g->weighted && (flags & GP_UPLOAD_NORMALIZE);
    g->home = s;
    int st = GP_OK;
    if (copy) {
        st = copy_in(g, csr_off, (size_t)n + 1, g->csr_off, s);
        if (st == GP_OK) st = copy_in(g, csr_idx, (size_t)m, g->csr_idx, s);
        if (st == GP_OK && csr_w) st = copy_in(g, csr_w, (size_t)m, g->csr_w, s);
        if (st == GP_OK && csc_off) {
            st = copy_in(g, csc_off, (size_t)n + 1, g->csc_off, s);
            if (st == GP_OK) st = copy_in(g, csc_idx, (size_t)m, g->csc_idx, s);
            if (st == GP_OK && csc_w) st = copy_in(g, csc_w, (size_t)m, g->csc_w, s);
        }
        if (st != GP_OK) return upload_fail(g, s, st);
    } else {
        g->csr_off = csr_off;
        g->csr_idx = csr_idx;
        g->csr_w = csr_w;
        g->csc_off = csc_off;
        g->csc_idx = csc_idx;
        g->csc_w = csc_w;
    }
    if (!g->csc_off) {
        g->csc_off = g->csr_off;
        g->csc_idx = g->csr_idx;
        g->csc_w = g->csr_w;
    }
    // Offsets and index ranges are always checked: later kernels index with them.
    unsigned *err = nullptr;
    DegStats *dst = nullptr;
    st = g->mem.alloc(err, 4, s);
    if (st == GP_OK) st = g->mem.alloc(dst, 1, s);
    if (st != GP_OK) return upload_fail(g, s, st);
    unsigned herr[4] = {0, 0, 0, 0};
    {
        cudaError_t e = cudaMemsetAsync(err, 0, 4 * sizeof(unsigned), s);
        int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->num_sms * 8));
        if (e == cudaSuccess) {
            GP_LAUNCH("check_offsets", s, (k_check_offsets<<<blocks, 256, 0, s>>>(g->csr_off, n, m, err)));
            if (g->csc_off != g->csr_off)
                GP_LAUNCH("check_offsets", s, (k_check_offsets<<<blocks, 256, 0, s>>>(g->csc_off, n, m, err + 1)));
            e = read_mapped(herr, err, 4 * sizeof(unsigned), s);
        }
        if (e != cudaSuccess) return upload_fail(g, s, set_error(GP_ERR_CUDA, "offset check: %s", cudaGetErrorString(e)));
        if (herr[0] | herr[1])
            return upload_fail(g, s, set_error(GP_ERR_INVALID, "malformed %s offsets (code %u): need off[0]=0, off[n]=m, non-decreasing",
                                               herr[0] ? "CSR" : "CSC", herr[0] ? herr[0] : herr[1]));
        int eb = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 8));
        if (m > 0) {
            GP_LAUNCH("check_indices", s, (k_check_indices<<<eb, 256, 0, s>>>(g->csr_idx, m, n, err + 2)));
            if (g->csc_idx != g->csr_idx)
                GP_LAUNCH("check_indices", s, (k_check_indices<<<eb, 256, 0, s>>>(g->csc_idx, m, n, err + 3)));
        }
        e = read_mapped(herr, err, 4 * sizeof(unsigned), s);
        if (e != cudaSuccess) return upload_fail(g, s, set_error(GP_ERR_CUDA, "index check: %s", cudaGetErrorString(e)));
        if (herr[2] | herr[3])
            return upload_fail(g, s, set_error(GP_ERR_INVALID, "%s index outside [0, n)", herr[2] ? "CSR" : "CSC"));
    }
    if ((flags & GP_UPLOAD_VALIDATE) && m > 0) {
        unsigned long long *fp = nullptr;
        st = g->mem.alloc(fp, 2, s);
        if (st != GP_OK) return upload_fail(g, s, st);
        unsigned long long hfp[2] = {0, 0};
        cudaError_t e = cudaMemsetAsync(fp, 0, 2 * sizeof(unsigned long long), s);
        int blocks = grid_blocks(g, 256);
        if (e == cudaSuccess) {
            GP_LAUNCH("edge_fingerprint", s, (k_edge_fingerprint<<<blocks, 256, 0, s>>>(g->csr_off, g->csr_idx, g->csr_w, n, 0, 0, fp)));
            if (g->csc_off != g->csr_off)
                GP_LAUNCH("edge_fingerprint", s, (k_edge_fingerprint<<<blocks, 256, 0, s>>>(g->csc_off, g->csc_idx, g->csc_w, n, 1, 0, fp + 1)));
            else  // symmetric: the reversed edge multiset must equal the edge multiset
                GP_LAUNCH("edge_fingerprint", s, (k_edge_fingerprint<<<blocks, 256, 0, s>>>(g->csr_off, g->csr_idx, g->csr_w, n, 0, 1, fp + 1)));
            e = read_mapped(hfp, fp, sizeof(hfp), s);
        }
        if (e != cudaSuccess) return upload_fail(g, s, set_error(GP_ERR_CUDA, "fingerprint: %s", cudaGetErrorString(e)));
        if (hfp[0] != hfp[1])
            return upload_fail(g, s, set_error(GP_ERR_INVALID, g->csc_off != g->csr_off
                                                                   ? "CSR and CSC do not hold the same edges"
                                                                   : "graph flagged symmetric is not symmetric"));
    }
    st = g->mem.alloc(g->inv_deg, (size_t)std::max<int64_t>(n, 1), s);
    if (st != GP_OK) return upload_fail(g, s, st);
    if (n > 0) {
        DegStats hs = {0, 0, 0};
        cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(DegStats), s);
        int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)g->num_sms * 8));
        if (e == cudaSuccess) {
            GP_LAUNCH("degree_prep", s, (k_degree_prep<<<blocks, 256, 0, s>>>(g->csr_off, g->csc_off, g->csr_w, n,
                                                                             g->weighted, g->normalized, g->inv_deg, dst)));
            e = read_mapped(&hs, dst, sizeof(hs), s);
        }
        if (e != cudaSuccess) return upload_fail(g, s, set_error(GP_ERR_CUDA, "degree prep: %s", cudaGetErrorString(e)));
        g->max_out = (int64_t)hs.max_out;
        g->max_in = (int64_t)hs.max_in;
        g->isolated = (int64_t)hs.isolated;
    }
    st = build_bins(g, g->pull_bins, g->csc_off, g->opt.pull_light_max, g->opt.chunk_edges, s);
    if (st == GP_OK) st = build_bins(g, g->push_bins, g->csr_off, g->opt.push_light_max, g->opt.chunk_edges, s);
    if (st != GP_OK) return upload_fail(g, s, st);
    *out = g;
    return GP_OK;
}

int gp_graph_free(gp_graph *g) {
    clear_error();
    if (!g) return GP_OK;
    cudaStream_t s = g->home;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != g->device) cudaSetDevice(g->device);
    // work queued on other streams must finish before the memory goes back
    cudaDeviceSynchronize();
    release_pr_work(g, s);
    release_bfs_work(g, s);
    release_sssp_work(g, s);
    release_fe_work(g, s);
    release_bc_work(g, s);
    g->pull_bins.mem.release(s);
    g->push_bins.mem.release(s);
    g->bfs_bins.mem.release(s);
    g->pull_hot.mem.release(s);
    g->push_hot.mem.release(s);
    g->mem.release(s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (dev != g->device && dev >= 0) cudaSetDevice(dev);
    delete g;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_graph_free: %s", cudaGetErrorString(e));
    return GP_OK;
}

int gp_graph_info_get(const gp_graph *g, gp_graph_info *info) {
    clear_error();
    if (!g || !info) return set_error(GP_ERR_INVALID, "gp_graph_info_get: NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->m = g->m;
    info->max_out_degree = g->max_out;
    info->max_in_degree = g->max_in;
    info->pull_big_vertices = g->pull_bins.nbig;
    info->pull_big_chunks = g->pull_bins.nchunks;
    info->push_big_vertices = g->push_bins.nbig;
    info->push_big_chunks = g->push_bins.nchunks;
    info->isolated = g->isolated;
    info->symmetric = g->symmetric;
    info->weighted = g->weighted;
    info->device_bytes = (int64_t)(g->mem.total + g->pull_bins.mem.total + g->push_bins.mem.total +
                                   g->bfs_bins.mem.total + g->pr.mem.total + g->bfs.mem.total + g->bfs.mmem.total);
    return GP_OK;
}

int gp_graph_get_options(const gp_graph *g, gp_options *opt) {
    clear_error();
    if (!g || !opt) return set_error(GP_ERR_INVALID, "gp_graph_get_options: NULL argument");
    *opt = g->opt;
    return GP_OK;
}

int gp_graph_set_options(gp_graph *g, const gp_options *opt, void *stream) {
    clear_error();
    if (!g || !opt) return set_error(GP_ERR_INVALID, "gp_graph_set_options: NULL argument");
    if (opt->pull_light_max < 0 || opt->push_light_max < 0 || opt->pull_light_max > (1 << 20) ||
        opt->push_light_max > (1 << 20) || opt->chunk_edges < 32 || opt->chunk_edges > (1 << 24) ||
        opt->blocks_per_sm < 1 || opt->blocks_per_sm > 32 || opt->poll_interval < 1 ||
        !(opt->bfs_alpha > 0.f) || !(opt->bfs_beta > 0.f) || !(opt->sssp_alpha > 0.f) || !(opt->fe_alpha > 0.f) || !(opt->bc_alpha > 0.f) || opt->pr_auto_mode < -1 || opt->pr_auto_mode > 1 ||
        opt->push_fp64_accum < -1 || opt->push_fp64_accum > 1 || opt->pull_hot_slots < 0 ||
        opt->pull_hot_slots > 49152 || opt->push_hot_slots < 0 || opt->push_hot_slots > 49152 ||
        opt->bfs_light_max < 0 || opt->bfs_light_max > (1 << 20) || opt->bfs_groups < 0 || opt->bfs_groups > 32)
        return set_error(GP_ERR_INVALID, "gp_graph_set_options: option out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const gp_options old = g->opt;
    g->opt = *opt;
    int st = GP_OK;
    if (old.pull_light_max != opt->pull_light_max || old.chunk_edges != opt->chunk_edges)
        st = build_bins(g, g->pull_bins, g->csc_off, opt->pull_light_max, opt->chunk_edges, s);
    if (st == GP_OK && (old.push_light_max != opt->push_light_max || old.chunk_edges != opt->chunk_edges))
        st = build_bins(g, g->push_bins, g->csr_off, opt->push_light_max, opt->chunk_edges, s);
    if (st == GP_OK && (old.blocks_per_sm != opt->blocks_per_sm || old.chunk_edges != opt->chunk_edges ||
                        old.pull_light_max != opt->pull_light_max || old.bfs_light_max != opt->bfs_light_max ||
                        old.push_light_max != opt->push_light_max)) {
        // workspace sizes depend on the grid and the chunk count: rebuild lazily
        release_pr_work(g, s);
        release_bfs_work(g, s);
        release_sssp_work(g, s);
        release_fe_work(g, s);
        release_bc_work(g, s);
    } else if (st == GP_OK && old.bfs_groups != opt->bfs_groups) {
        release_bfs_multi(g, s);  // sized for the old group count
    }
    if (st != GP_OK) {
        g->opt = old;
        return st;
    }
    return GP_OK;
}

}  // extern "C"
