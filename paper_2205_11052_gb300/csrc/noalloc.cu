// pic_field_energy_noalloc: the FP64 field-energy / total-charge reduction
// with no device allocation anywhere on its path.
//
// Who needs it: a caller that must not allocate device memory at run time,
// for example a host application that gives this code a fixed memory budget
// it manages itself, or a time-critical loop in which a cudaMalloc (which
// may synchronise the device, and may fail once memory is fragmented) is not
// allowed.  Such a caller cannot size and bind a workspace arena, so the
// reduction's scratch space lives in this file instead: a statically sized
// __device__ array that every GPU loading the library holds until exit.
//
// Scratch: one FP64 partial (4 values) per block, each block reducing a
// fixed span of kSpan nodes, at most kMaxBlocks blocks, so inputs of up to
// kMaxBlocks * kSpan nodes are accepted (PIC_NOALLOC_MAX_NODES in pic.h).
// Every partial the second kernel reads is written by the first kernel of
// the same call, so nothing has to be cleared between calls; the array keeps
// the last call's partials.  All calls share that one array: calls whose
// kernels overlap on the GPU (for instance on two streams without ordering)
// race on it and must be serialised by the caller.
#include <stdio.h>

#include "pic_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kSpan = 16384;                       // nodes per block
constexpr int kMaxBlocks = 8192;                   // partial slots in the scratch
static_assert((long long)kSpan * kMaxBlocks == PIC_NOALLOC_MAX_NODES, "size contract");

// 8192 blocks x 4 doubles = 256 KiB per device
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 4];

__global__ void __launch_bounds__(kThreads) k_energy_partials(const float *__restrict__ rho,
                                                              const float4 *__restrict__ E4,
                                                              long long n, double *part) {
    const long long g0 = (long long)blockIdx.x * kSpan;
    const long long g1 = g0 + kSpan < n ? g0 + kSpan : n;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long g = g0 + threadIdx.x; g < g1; g += kThreads) {
        const float4 e = E4[g];
        const double ex = e.x, ey = e.y, ez = e.z;
        s[0] += ex * ex;
        s[1] += ey * ey;
        s[2] += ez * ez;
        s[3] += (double)rho[g];
    }
    __shared__ double red[4][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        double t = s[q];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[threadIdx.x][w];
        part[4 * blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_energy_combine(const double *__restrict__ part,
                                                             int nblocks, double dV,
                                                             double *out) {
    __shared__ double red[4][kThreads];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < 4; ++q) s[q] += part[4 * b + q];
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = dV * red[threadIdx.x][0];
}

int noalloc_fail(int code, const char *msg, cudaError_t e = cudaSuccess) {
    return pic::record_error(code, "pic_field_energy_noalloc: %s%s%s", msg,
                             e != cudaSuccess ? ": " : "",
                             e != cudaSuccess ? cudaGetErrorString(e) : "");
}

// Device address of the scratch array on the current device.  It is looked
// up on every call (cudaGetSymbolAddress allocates nothing), so a context
// that was reset or replaced since an earlier call is never handed a stale
// address; the first lookup on a device also loads this library's device
// code there.
int scratch_for_current_device(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) return noalloc_fail(PIC_ERR_CUDA, "cudaGetSymbolAddress failed", e);
    *out = static_cast<double *>(p);
    return PIC_OK;
}

}  // namespace

extern "C" int pic_field_energy_noalloc(const float *rho, const float *E, int64_t n_nodes,
                                        double cell_volume, double *out, void *stream) {
    if (!rho || !E || !out) return noalloc_fail(PIC_ERR_ARG, "null pointer");
    if (n_nodes < 1) return noalloc_fail(PIC_ERR_ARG, "n_nodes must be >= 1");
    if (n_nodes > PIC_NOALLOC_MAX_NODES)
        return noalloc_fail(PIC_ERR_CAPACITY,
                            "n_nodes above PIC_NOALLOC_MAX_NODES (134,217,728 = 512^3)");
    if (!(cell_volume > 0.0)) return noalloc_fail(PIC_ERR_ARG, "cell_volume must be > 0");
    if ((uintptr_t)E % 16) return noalloc_fail(PIC_ERR_ARG, "E must be 16-byte aligned");
    double *scratch = nullptr;
    int r = scratch_for_current_device(&scratch);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblocks = (int)((n_nodes + kSpan - 1) / kSpan);
    k_energy_partials<<<nblocks, kThreads, 0, st>>>(rho, reinterpret_cast<const float4 *>(E),
                                                    (long long)n_nodes, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "partials launch failed", e);
    k_energy_combine<<<1, kThreads, 0, st>>>(scratch, nblocks, cell_volume, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "combine launch failed", e);
    return PIC_OK;
}
