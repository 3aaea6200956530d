// Throughput of this GPU's FP32 and FP64 fused multiply-add pipes, measured by the library's own kernel. The
// per-voxel local Newton solve is the step of the method that does the most arithmetic per byte; its pipe
// utilisation is reported against these measured rates rather than against nominal figures.
#include <cuda_runtime.h>

#include "../../include/evp.h"

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread (covers the FMA latency)
constexpr int kThreadsFma = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreadsFma) k_fma_chain(int iters, T m, T b, T *__restrict__ sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1) sink[0] = s;   // never true for the inputs used; keeps every chain live
}

}  // namespace

extern "C" int evp_fma_throughput(int precision, int iters, void *sink_dev, double *tflops, void *cuda_stream) {
    if (!sink_dev || !tflops || iters < 1 || precision < EVP_FP64 || precision > EVP_MIXED_FAST) return EVP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EVP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return EVP_ERR_CUDA;
    const int blocks = nsm * kBlocksPerSm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return EVP_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EVP_ERR_CUDA;
    }
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        if (precision == EVP_FP64)
            k_fma_chain<double><<<blocks, kThreadsFma, 0, s>>>(iters, 0.9999999, 1e-9, (double *)sink_dev);
        else
            k_fma_chain<float><<<blocks, kThreadsFma, 0, s>>>(iters, 0.9999999f, 1e-9f, (float *)sink_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return EVP_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)iters * kThreadsFma * (double)blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return EVP_OK;
}
