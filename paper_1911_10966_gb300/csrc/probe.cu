// Measurement helpers: FMA-throughput probes (the ALU roofline denominators) and CUDA-event timing
// of the residual kernels inside a context.
#include <cuda_runtime.h>

#include <vector>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace {

// Eight independent FMA chains per thread; the result is stored only if it is a NaN so that the
// compiler keeps the work and the store almost never happens.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe(T* out, int iters, T seed) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + (T)(threadIdx.x * 8 + i) * (T)1e-7;
    const T b = (T)0.999999, c = (T)1e-9;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s != s) out[blockIdx.x] = s;
}

}  // namespace

cudaError_t probe_fma(int kind, double* flops_per_s, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256;
    const int iters = kind == 0 ? 2048 : 65536;
    void* buf = nullptr;
    e = cudaMalloc(&buf, blocks * sizeof(double));
    if (e != cudaSuccess) return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(t0, s);
        if (kind == 0) fma_probe<double><<<blocks, threads, 0, s>>>((double*)buf, iters, 1.0);
        else fma_probe<float><<<blocks, threads, 0, s>>>((float*)buf, iters, 1.0f);
        cudaEventRecord(t1, s);
        e = cudaEventSynchronize(t1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(buf);
    *flops_per_s = (double)blocks * threads * iters * 8 * 2 / (best * 1e-3);
    return e;
}

}  // namespace esdc
