// Measured FMA throughput of the GPU for the roofline denominators: FP32 and
// FP64 fused multiply-adds in independent chains on every SM, timed with
// CUDA events on the caller's stream.  Changes no device setting.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/mrcm.h"

namespace {

constexpr int PK_CHAINS = 8;      // independent FMA chains per thread
constexpr int PK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(T* out, int iters, T m, T a) {
    T v[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) v[c] = T(1) + T(1e-3) * (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = v[c] * m + a;   // one FMA
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += v[c];
    if (s == T(12345)) out[blockIdx.x] = s;   // keeps the chains live; never true
}

template <typename T>
int measure(int blocks, int iters, cudaStream_t st, double* tflops) {
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return MRCM_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ms;
    k_fma_peak<T><<<blocks, PK_THREADS, 0, st>>>(out, iters / 8, T(0.999999), T(1e-7));   // warm-up
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        k_fma_peak<T><<<blocks, PK_THREADS, 0, st>>>(out, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms.push_back(t);
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return MRCM_ERR_CUDA;
    std::sort(ms.begin(), ms.end());
    const double flops = 2.0 * (double)blocks * PK_THREADS * PK_CHAINS * (double)iters;
    *tflops = flops / (ms[1] * 1e-3) / 1e12;
    return MRCM_OK;
}

}  // namespace

extern "C" int mrcm_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* cuda_stream) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MRCM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = MRCM_OK;
    // eight 256-thread blocks per SM: enough warps to cover the FMA latency on every sub-partition
    if (fp32_tflops && (rc = measure<float>(8 * sms, 1 << 16, st, fp32_tflops))) return rc;
    if (fp64_tflops && (rc = measure<double>(8 * sms, 1 << 12, st, fp64_tflops))) return rc;
    return MRCM_OK;
}
