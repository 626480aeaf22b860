// Measured roof of the kernels that the FP64 pipe bounds: the device's fused multiply-add rate in
// FP64 and FP32.  Each thread runs eight independent FMA chains (enough to cover the pipe's
// latency), the grid fills every SM several times over, and the kernel is timed with CUDA events
// on the caller's stream.  The paper has no counterpart: it is the measurement the FP64 PCG's
// ALU roofline is stated against.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/vofp.h"

namespace {

constexpr int kChains = 8;
// the sink is written only by a branch the inputs never take; it must still be a valid address,
// so it is one static element per precision (no allocation)
__device__ double g_sink64[1];
__device__ float g_sink32[1];
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(T* __restrict__ sink, T m, T a, int iters) {
    T v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) v[i] = fma(v[i], m, a);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += v[i];
    // the store is never taken for the multipliers the host passes (|m| < 1 keeps s finite), but
    // the compiler cannot know that, so every chain is computed
    if (s == (T)-1.2345e30) sink[0] = s;
}

template <typename T>
cudaError_t time_fma(cudaStream_t st, int blocks, int iters, T* sink, double* tflops) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_fma_chains<T><<<blocks, kPeakThreads, 0, st>>>(sink, (T)0.999999, (T)1e-7, iters);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, ms);   // launch 0 is the warm-up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) {
        const double fmas = (double)blocks * kPeakThreads * kChains * (double)iters;
        *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    }
    return e;
}

}  // namespace

extern "C" vofp_status vofp_measure_fma_peaks(vofp_stream stream, double* fp64_tflops, double* fp32_tflops) {
    if (!fp64_tflops || !fp32_tflops) return VOFP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return VOFP_ERR_CUDA;
    double* s64 = nullptr;
    float* s32 = nullptr;
    if (cudaGetSymbolAddress((void**)&s64, g_sink64) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&s32, g_sink32) != cudaSuccess)
        return VOFP_ERR_CUDA;
    const int blocks = sms * 8;
    // about 10 ms per launch at each precision's rate on a 152-SM part
    if (time_fma<double>(st, blocks, 1536, s64, fp64_tflops) != cudaSuccess) return VOFP_ERR_CUDA;
    if (time_fma<float>(st, blocks, 65536, s32, fp32_tflops) != cudaSuccess) return VOFP_ERR_CUDA;
    return VOFP_OK;
}
