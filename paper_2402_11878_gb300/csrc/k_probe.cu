// Arithmetic-throughput probe: the measured FMA rate of this GPU in FP64
// and FP32, the denominator of the "alu" roofline of the FP64 pass kernels.
//
// Every thread runs kChains independent fused multiply-add chains
// a <- a * x + y for `iters` steps (x just below 1, so the chains converge
// to y / (1 - x) and never overflow); the grid fills every SM with enough
// warps to hide the FMA latency.  The result of each thread is stored, so
// no chain can be removed by the compiler.  Time is taken with CUDA events
// on the caller's stream after one untimed launch; nothing about the GPU's
// clocks or power settings is changed.
#include "vqe_probe.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T x, T y, int iters, T *out) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], x, y);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[size_t(blockIdx.x) * kThreads + threadIdx.x] = s;
}

template <typename T>
vqe_status run_probe(int blocks, int iters, cudaStream_t s, double *tflops) {
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * size_t(blocks) * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return VQE_ERR_OOM;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    vqe_status st = VQE_OK;
    float ms = 0.f;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        st = VQE_ERR_CUDA;
    } else {
        const T x = T(0.999999), y = T(1e-6);
        k_fma_chains<T><<<blocks, kThreads, 0, s>>>(x, y, iters, out);   // warm-up
        cudaEventRecord(a, s);
        k_fma_chains<T><<<blocks, kThreads, 0, s>>>(x, y, iters, out);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess ||
            ms <= 0.f)
            st = VQE_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) st = VQE_ERR_CUDA;
    if (st == VQE_OK) {
        const double flops = 2.0 * kChains * double(iters) * double(blocks) * kThreads;
        *tflops = flops / (double(ms) * 1e-3) / 1e12;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    return st;
}

}  // namespace

extern "C" vqe_status vqe_measure_fma_peak(int fp64, void *cuda_stream, double *tflops) {
    if (!tflops || (fp64 != 0 && fp64 != 1)) return VQE_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return VQE_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // 8 blocks of 256 threads per SM (64 warps); FP64 runs fewer steps since
    // its rate is a small fraction of FP32's
    const int blocks = sms * 8;
    return fp64 ? run_probe<double>(blocks, 1 << 14, s, tflops)
                : run_probe<float>(blocks, 1 << 18, s, tflops);
}
