// noalloc.cu -- one pull PageRank sweep that allocates no device memory.
//
// Who needs this: callers that must not allocate device memory while they run
// the sweep -- for example code executing inside a framework hook that may
// only use buffers the framework hands it, real-time pipelines that reserve
// all memory at start-up and forbid allocation afterwards, or processes whose
// device memory is already fully claimed by another allocator, so that a
// cudaMalloc would fail or stall.  They pass inputs and outputs; the
// intermediate data lives in a fixed-size array compiled into this library.
//
// The sweep is the light-tile pull kernel of pagerank.cu run over every vertex
// (no degree bins, since those are built by gp_graph_upload, which allocates):
// 32 consecutive vertices per warp, their in-edges walked as one stream,
// segmented warp sums, owner-only writes.  Its scratch -- the contribution
// vector c[u] = x[u] * inv_deg[u] and the per-block residual partials -- sits
// in g_noalloc_scratch below, so the graph may have at most
// GP_NOALLOC_MAX_VERTICES vertices.
//
// Every call reuses the same array, and it keeps the previous call's contents.
// Nothing in it needs to start at zero: each call writes every entry it reads
// (the error flag is cleared by the call's first kernel).  Two calls whose
// kernels overlap on the GPU -- on different streams, or from different host
// threads -- race on the array and corrupt each other's results; serialise them.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int64_t NA_MAX_N = GP_NOALLOC_MAX_VERTICES;
constexpr int NA_MAX_BLOCKS = 1024;

struct NoallocScratch {
    float c[NA_MAX_N];               // contributions x[u] * inv_deg[u]
    double partials[NA_MAX_BLOCKS];  // residual per block of the sweep
    unsigned bad;                    // malformed-input flag of the current call
};

// The static scratch: 4 MiB + 8 KiB, resident on every device that loads the library.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device ordinal (host code may not use
// the symbol itself as a device pointer: it names a host-side shadow).
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
NoallocScratch *g_na_ptr[NA_MAX_DEVICES] = {};

int scratch_on_current_device(NoallocScratch **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(GP_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, NA_MAX_DEVICES);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(GP_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) on device %d: %s", dev,
                             cudaGetErrorString(e));
        g_na_ptr[dev] = (NoallocScratch *)p;
    }
    *out = g_na_ptr[dev];
    return GP_OK;
}

__global__ void k_na_contrib(int64_t n, const float *x, const float *inv_deg, NoallocScratch *sc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->bad = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) sc->c[u] = x[u] * inv_deg[u];
}

// y[v] = base(v) + d * sum_{u in in(v)} c[u] (* w), residual partial |y - x|.
// Offsets and indices are range-checked: an out-of-range value is skipped and
// flagged instead of being dereferenced.
__global__ void __launch_bounds__(256) k_na_sweep(int64_t n, int64_t m, const int64_t *off, const int32_t *idx,
                                                   const float *w, const float *x, const float *s, float base_uniform,
                                                   float one_minus_d, float d, float *y, NoallocScratch *sc) {
    __shared__ double red[32];
    const int lane = lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = (n + 31) >> 5;
    ResSum res;
    bool bad = false;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int64_t v = t * 32 + lane;
        int64_t b = 0, e = 0;
        if (v < n) {
            b = off[v];
            e = off[v + 1];
            if (b < 0 || e < b || e > m) {
                bad = true;
                b = e = 0;
            }
        }
        // The 32-bit scan below is exact while the tile's degrees sum to at most
        // m (< 2^31), which monotone offsets guarantee.  Offsets that rise and
        // fall pass the per-vertex check yet can sum past 2^31, so the tile's
        // total is formed in 64 bits first and a tile above m is skipped.
        int64_t tile_sum = e - b;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) tile_sum += __shfl_xor_sync(FULL, tile_sum, st);
        if (tile_sum > m) {
            bad = true;
            b = e = 0;
        }
        const int deg = (int)(e - b);
        const int incl = warp_incl_scan(deg);
        const int excl = incl - deg;
        const int E = __shfl_sync(FULL, incl, 31);
        float acc = 0.f;
        for (int base = 0; base < E; base += 32) {
            const int eid = base + lane;
            int k = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ex = __shfl_sync(FULL, excl, k + st);
                if (ex <= eid) k += st;
            }
            const int64_t kb = __shfl_sync(FULL, b, k);
            const int kex = __shfl_sync(FULL, excl, k);
            float val = 0.f;
            if (eid < E) {
                const int64_t pos = kb + (eid - kex);
                const int32_t u = __ldg(idx + pos);
                if (u >= 0 && (int64_t)u < n) {
                    val = sc->c[u];
                    if (w) val *= __ldg(w + pos);
                } else {
                    bad = true;
                }
            }
            const int head = max(kex, base) - base;
#pragma unroll
            for (int st = 1; st < 32; st <<= 1) {
                const float tv = __shfl_up_sync(FULL, val, st);
                if (lane - st >= head) val += tv;
            }
            const bool has = deg > 0 && excl < base + 32 && incl > base;
            const int tail = has ? min(incl, base + 32) - base - 1 : 0;
            const float segsum = __shfl_sync(FULL, val, tail);
            if (has) acc += segsum;
        }
        if (v < n) {
            const float yv = (s ? one_minus_d * s[v] : base_uniform) + d * acc;
            res.add(yv, x[v]);
            y[v] = yv;
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(&sc->bad, 1u);
    const double r = block_residual(res, red);
    if (threadIdx.x == 0) sc->partials[blockIdx.x] = r;
}

// Sums the block partials in block order; NaN signals malformed input.
__global__ void k_na_reduce(int nblocks, NoallocScratch *sc, double *residual_out) {
    __shared__ double red[32];
    double r = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) r += sc->partials[i];
    r = block_sum(r, red);
    if (threadIdx.x == 0) *residual_out = sc->bad ? __longlong_as_double(0x7FF8000000000000LL) : r;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" int gp_pull_sweep_noalloc(int64_t n, int64_t m, const int64_t *csc_off, const int32_t *csc_idx,
                                     const float *csc_w, const float *inv_deg, const float *x, float damping,
                                     const float *personalization, float *y, double *residual_out, void *stream) {
    clear_error();
    if (n < 1 || n > NA_MAX_N)
        return set_error(GP_ERR_INVALID, "gp_pull_sweep_noalloc: n = %lld outside [1, %lld] (the static scratch holds "
                                         "GP_NOALLOC_MAX_VERTICES contributions)", (long long)n, (long long)NA_MAX_N);
    if (m < 0 || m >= (int64_t(1) << 31))
        return set_error(GP_ERR_INVALID, "gp_pull_sweep_noalloc: m = %lld outside [0, 2^31)", (long long)m);
    if (!csc_off || (m > 0 && !csc_idx) || !inv_deg || !x || !y || !residual_out)
        return set_error(GP_ERR_INVALID, "gp_pull_sweep_noalloc: NULL array");
    if (!(damping > 0.f && damping < 1.f))
        return set_error(GP_ERR_INVALID, "gp_pull_sweep_noalloc: damping %g outside (0, 1)", (double)damping);
    NoallocScratch *sc = nullptr;
    GP_TRY(scratch_on_current_device(&sc));
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    GP_CUDA(cudaGetDevice(&dev));
    GP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = (n + 31) / 32;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)NA_MAX_BLOCKS, (int64_t)sms * 4,
                                                                     (ntiles + 7) / 8}));
    const int cb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4);
    const float one_minus_d = 1.0f - damping;
    const float base_uniform = (float)((1.0 - (double)damping) / (double)n);
    // plain launches: no profiling events are created on this path
    k_na_contrib<<<cb, 256, 0, s>>>(n, x, inv_deg, sc);
    GP_TRY(check_launch("noalloc_contrib"));
    k_na_sweep<<<blocks, 256, 0, s>>>(n, m, csc_off, csc_idx, csc_w, x, personalization, base_uniform, one_minus_d,
                                      damping, y, sc);
    GP_TRY(check_launch("noalloc_sweep"));
    k_na_reduce<<<1, 256, 0, s>>>(blocks, sc, residual_out);
    return check_launch("noalloc_reduce");
}
