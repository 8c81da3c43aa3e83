// probe.cu -- rates of the memory operations the sweeps are built from
// (random gathers from L2, shared memory and a cluster's distributed shared
// memory; random FP64/FP32 atomic adds into L2 and into shared memory), for
// the roofline bounds of the gather-, scatter- and atomic-bound kernels.
#include <cstring>

#include "gp_internal.cuh"

namespace gp {

constexpr int PR_THREADS = 1024;
constexpr uint32_t PR_GLOBAL_N = 1u << 22;  // 16 MB of floats, 32 MB of doubles: L2-resident
constexpr uint32_t PR_SLICE = 16384;        // floats per block (64 KB)
constexpr uint32_t PR_TABLE = 8192;         // shared-memory atomic table entries

// Integer hash (multiply-xorshift) giving each step of each thread an address.
__device__ __forceinline__ uint32_t pr_mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(PR_THREADS, 2) k_probe_gather_global(const float *a, int iters, float *out) {
    float s = 0.f;
    uint32_t h = blockIdx.x * PR_THREADS + threadIdx.x;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        h = pr_mix(h + i);
        s += __ldg(a + (h & (PR_GLOBAL_N - 1)));
    }
    out[blockIdx.x * PR_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PR_THREADS, 2) k_probe_gather_shared(const float *a, int iters, float *out) {
    extern __shared__ float sh[];
    for (uint32_t i = threadIdx.x; i < PR_SLICE; i += PR_THREADS) sh[i] = a[i];
    __syncthreads();
    float s = 0.f;
    uint32_t h = blockIdx.x * PR_THREADS + threadIdx.x;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        h = pr_mix(h + i);
        s += sh[h & (PR_SLICE - 1)];
    }
    out[blockIdx.x * PR_THREADS + threadIdx.x] = s;
}

// Cluster of 8 blocks: each step reads a random entry of a random block's slice.
__global__ void __launch_bounds__(PR_THREADS, 2) k_probe_gather_cluster(const float *a, int iters, float *out) {
    extern __shared__ float sh[];
    for (uint32_t i = threadIdx.x; i < PR_SLICE; i += PR_THREADS) sh[i] = a[i];
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(sh);
    float s = 0.f;
    uint32_t h = blockIdx.x * PR_THREADS + threadIdx.x;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        h = pr_mix(h + i);
        const uint32_t rank = (h >> 14) & 7u;
        const uint32_t laddr = base + 4u * (h & (PR_SLICE - 1));
        uint32_t raddr;
        float v;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
        asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(raddr) : "memory");
        s += v;
    }
    // no block leaves while another may still read its shared memory
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    out[blockIdx.x * PR_THREADS + threadIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(PR_THREADS, 2) k_probe_red(T *a, int iters) {
    uint32_t h = blockIdx.x * PR_THREADS + threadIdx.x;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        h = pr_mix(h + i);
        atomicAdd(a + (h & (PR_GLOBAL_N - 1)), (T)1);
    }
}

template <class T>
__global__ void __launch_bounds__(PR_THREADS, 2) k_probe_atom_shared(T *out, int iters) {
    __shared__ T acc[PR_TABLE];
    for (uint32_t i = threadIdx.x; i < PR_TABLE; i += PR_THREADS) acc[i] = (T)0;
    __syncthreads();
    uint32_t h = blockIdx.x * PR_THREADS + threadIdx.x;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
        h = pr_mix(h + i);
        atomicAdd(acc + (h & (PR_TABLE - 1)), (T)1);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < PR_TABLE; i += PR_THREADS) out[blockIdx.x * PR_TABLE + i] = acc[i];
}

template <class T>
__global__ void k_probe_sum(const T *a, int64_t n, double *out) {
    __shared__ double sm[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

}  // namespace gp

using namespace gp;

extern "C" int gp_probe_rates(int kind, int iters, double *rate_out, double *check_out, void *stream) {
    clear_error();
    if (kind < 0 || kind >= GP_PROBE_KINDS) return set_error(GP_ERR_INVALID, "gp_probe_rates: bad kind %d", kind);
    if (iters < 1 || iters > 65536) return set_error(GP_ERR_INVALID, "gp_probe_rates: iters %d outside [1, 65536]", iters);
    if (!rate_out) return set_error(GP_ERR_INVALID, "gp_probe_rates: rate_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    GP_CUDA(cudaGetDevice(&dev));
    GP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = 2 * sms - (2 * sms) % 8;  // a whole number of 8-block clusters
    Arena tmp;
    float *fa = nullptr, *fout = nullptr;
    double *da = nullptr, *dsum = nullptr;
    const size_t nout = (size_t)grid * std::max<uint32_t>(PR_THREADS, PR_TABLE);
    int st = tmp.alloc(fa, PR_GLOBAL_N, s);
    if (st == GP_OK) st = tmp.alloc(da, PR_GLOBAL_N, s);
    if (st == GP_OK) st = tmp.alloc(fout, nout * 2, s);  // room for FP64 tables too
    if (st == GP_OK) st = tmp.alloc(dsum, 1, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    float ms = 0.f;
    if (st == GP_OK) {
        e = cudaMemsetAsync(fa, 0, PR_GLOBAL_N * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(da, 0, PR_GLOBAL_N * sizeof(double), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(double), s);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_probe_gather_shared, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)(PR_SLICE * sizeof(float)));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_probe_gather_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)(PR_SLICE * sizeof(float)));
        if (e == cudaSuccess && kind == GP_PROBE_GATHER_CLUSTER) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3(PR_THREADS);
            cfg.dynamicSmemBytes = PR_SLICE * sizeof(float);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 8;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            e = cudaOccupancyMaxActiveClusters(&nclusters, (const void *)k_probe_gather_cluster, &cfg);
            if (e == cudaSuccess && nclusters < 1) st = set_error(GP_ERR_UNSUPPORTED, "gp_probe_rates: no 8-block cluster fits");
        }
    }
    if (st == GP_OK && e == cudaSuccess) {
        e = cudaEventRecord(e0, s);
        switch (kind) {
            case GP_PROBE_GATHER_GLOBAL:
                k_probe_gather_global<<<grid, PR_THREADS, 0, s>>>(fa, iters, fout);
                break;
            case GP_PROBE_GATHER_SHARED:
                k_probe_gather_shared<<<grid, PR_THREADS, PR_SLICE * sizeof(float), s>>>(fa, iters, fout);
                break;
            case GP_PROBE_GATHER_CLUSTER: {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)grid);
                cfg.blockDim = dim3(PR_THREADS);
                cfg.dynamicSmemBytes = PR_SLICE * sizeof(float);
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 8;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, k_probe_gather_cluster, (const float *)fa, iters, fout);
                break;
            }
            case GP_PROBE_RED_F64:
                k_probe_red<double><<<grid, PR_THREADS, 0, s>>>(da, iters);
                break;
            case GP_PROBE_RED_F32:
                k_probe_red<float><<<grid, PR_THREADS, 0, s>>>(fa, iters);
                break;
            case GP_PROBE_ATOM_SHARED_F64:
                k_probe_atom_shared<double><<<grid, PR_THREADS, 0, s>>>((double *)fout, iters);
                break;
            default:
                k_probe_atom_shared<float><<<grid, PR_THREADS, 0, s>>>(fout, iters);
                break;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess && check_out) {
            switch (kind) {
                case GP_PROBE_RED_F64:
                    k_probe_sum<double><<<256, 256, 0, s>>>(da, PR_GLOBAL_N, dsum);
                    break;
                case GP_PROBE_RED_F32:
                    k_probe_sum<float><<<256, 256, 0, s>>>(fa, PR_GLOBAL_N, dsum);
                    break;
                case GP_PROBE_ATOM_SHARED_F64:
                    k_probe_sum<double><<<256, 256, 0, s>>>((const double *)fout, (int64_t)grid * PR_TABLE, dsum);
                    break;
                case GP_PROBE_ATOM_SHARED_F32:
                    k_probe_sum<float><<<256, 256, 0, s>>>(fout, (int64_t)grid * PR_TABLE, dsum);
                    break;
                default:
                    k_probe_sum<float><<<256, 256, 0, s>>>(fout, (int64_t)grid * PR_THREADS, dsum);
                    break;
            }
            e = cudaGetLastError();
        }
        double h = 0.0;
        if (e == cudaSuccess && check_out) e = cudaMemcpyAsync(&h, dsum, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) {
            *rate_out = (double)grid * PR_THREADS * iters / (ms * 1e-3);
            if (check_out) *check_out = h;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    tmp.release(s);
    if (st != GP_OK) return st;
    if (e != cudaSuccess) return set_error(GP_ERR_CUDA, "gp_probe_rates: %s", cudaGetErrorString(e));
    return GP_OK;
}
