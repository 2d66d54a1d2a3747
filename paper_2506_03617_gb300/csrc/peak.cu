// Arithmetic ceilings of the device, measured: the FP32 and FP64 fused
// multiply-add throughput.  The roofline of the sweep kernels whose vectors stay
// on chip (2D grids up to ~1100^2 held in shared memory and L2) is the FMA pipe,
// and the complex128 path is bound by the FP64 pipe, so both are timed here
// with CUDA events the same way the kernels themselves are (no clock or power
// setting is touched).  No counterpart in the paper.
#include <algorithm>

#include "mxp_internal.h"

namespace mxp {

// Each thread runs kChains independent FMA chains for `iters` rounds; every
// chain's value depends on the previous one, so nothing can be folded away, and
// the final sum is stored only under a condition the host makes impossible.
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T seed, T mult, int iters, T never, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], mult, seed);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == never) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t time_fma(int blocks, int iters, double *flops_per_s)
{
    T *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, (size_t)blocks * 256 * sizeof(T));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    // mult slightly below 1 keeps every chain finite; `never` is negative while
    // all chains stay positive
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        count_launch();
        k_fma_chain<T><<<blocks, 256>>>((T)1.0, (T)0.999999, iters, (T)-1.0, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);     // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    const double fmas = (double)blocks * 256 * iters * kUnroll * kChains;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace mxp

extern "C" mxp_status mxp_measure_fma_peak(int device, double *fp32_flops, double *fp64_flops)
{
    if (!fp32_flops || !fp64_flops) {
        mxp::note_error("NULL argument");
        return MXP_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        mxp::note_error("no such CUDA device");
        return MXP_EINVAL;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    const int blocks = mxp::sm_count() * 8;     // eight 256-thread blocks per SM
    cudaError_t e = mxp::time_fma<float>(blocks, 4096, fp32_flops);
    if (e == cudaSuccess) e = mxp::time_fma<double>(blocks, 256, fp64_flops);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        mxp::note_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MXP_ENOMEM : MXP_ECUDA;
    }
    return MXP_OK;
}
