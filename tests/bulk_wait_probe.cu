// Test-only probe of the bulk-copy helpers the float32 element kernel uses (csrc/bulk_copy.cuh):
// one CTA copies n floats from global memory to shared memory by one bulk copy completed on an
// mbarrier, waits with the bounded wait, and writes the shared copy back out.  With extra > 0 the
// barrier also expects `extra` bytes that no copy delivers, so its phase never completes and the
// bounded wait must give up: the probe then records status bit 1 and leaves dst untouched.  Built
// and run by tests/test_gpu_bulk_wait.py; not part of the library.
#include <cuda_runtime.h>

#include "../paper_1911_10966_gb300/csrc/bulk_copy.cuh"

namespace {

__global__ void bulk_probe(const float* __restrict__ src, float* __restrict__ dst, int n, unsigned extra,
                           int* __restrict__ status) {
    extern __shared__ float4 sm4[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int failed;
    float* sm = reinterpret_cast<float*>(sm4);
    if (threadIdx.x == 0) {
        esdc::mbar_init(&bar, 1);
        failed = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        esdc::mbar_expect_tx(&bar, (unsigned)n * 4u + extra);
        esdc::bulk_g2s(sm, src, (unsigned)n * 4u, &bar);
    }
    if (!esdc::mbar_wait_bounded(&bar, 0)) failed = 1;
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, esdc::kStatusBulkWait);
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = sm[i];
}

}  // namespace

// n: a multiple of 4 floats, at most 8192; src and dst 16-byte aligned device pointers.  Returns the
// CUDA error code of the launch and the synchronisation.
extern "C" int probe_bulk_copy(const float* src, float* dst, int n, unsigned extra, int* status) {
    if (n <= 0 || n % 4 != 0 || n > 8192) return (int)cudaErrorInvalidValue;
    bulk_probe<<<1, 128, (size_t)n * sizeof(float)>>>(src, dst, n, extra, status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return (int)e;
}
