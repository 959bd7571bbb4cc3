// Float64 <-> float32 state kernels of the mixed-precision form.
//   shadow:  dq = float(q - q_ref) with q_ref = (rho0, 0, 0, 0, E0): the float32 perturbation state
//            the float32 residual reads (float64 subtraction before rounding).
//   final:   q += sum_j c_j k_j accumulated in float64 (the Runge-Kutta solution update), then the
//            new shadow of q is written.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "fpconv.cuh"
#include "kernels.h"

namespace esdc {
namespace {

// Variable index (0..4) of entry i of a [K][5][N3] array: (i / N3) mod 5 by invariant division.
__device__ __forceinline__ int var_of(int64_t i, DivU64 div_n3, DivU64 div_5) {
    const unsigned long long row = div_n3((unsigned long long)i);
    return (int)(row - 5ull * div_5(row));
}

__global__ void __launch_bounds__(256) shadow_kernel(const double* __restrict__ q, float* __restrict__ dq,
                                                     int64_t n_nodes, DivU64 div_n3, DivU64 div_5, double rho0,
                                                     double E0) {
    const int64_t n = n_nodes * 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int v = var_of(i, div_n3, div_5);
        double x = q[i];
        if (v == 0) x -= rho0;
        else if (v == 4) x -= E0;
        dq[i] = d2f_int(x);
    }
}

__global__ void __launch_bounds__(256) final_kernel(double* __restrict__ q, float* __restrict__ dq_new,
                                                    const Combine64F cb, int64_t n_nodes, DivU64 div_n3,
                                                    DivU64 div_5, double rho0, double E0) {
    const int64_t n = n_nodes * 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        // all stage loads issued together (fixed trip count, predicated), summed in stage order
        float kv[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) kv[j] = j < cb.nk ? __ldg(cb.k[j] + i) : 0.0f;
        const double q0 = q[i];
        double inc = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (j < cb.nk) inc = fma(cb.coef[j], f2d_int(kv[j]), inc);
        const double qn = q0 + inc;
        q[i] = qn;
        const int v = var_of(i, div_n3, div_5);
        double x = qn;
        if (v == 0) x -= rho0;
        else if (v == 4) x -= E0;
        dq_new[i] = d2f_int(x);
    }
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_shadow(const esdc_ctx* c, const double* q, float* dq, cudaStream_t s) {
    const double E0 = c->phys.R / (c->phys.gamma - 1.0);
    shadow_kernel<<<grid_for(c->n_nodes * 5), 256, 0, s>>>(q, dq, c->n_nodes, DivU64::make(c->N3), DivU64::make(5),
                                                           1.0, E0);
    return cudaGetLastError();
}

cudaError_t launch_final_f32(const esdc_ctx* c, double* q, float* dq_new, const Combine64F& cb, cudaStream_t s) {
    const double E0 = c->phys.R / (c->phys.gamma - 1.0);
    final_kernel<<<grid_for(c->n_nodes * 5), 256, 0, s>>>(q, dq_new, cb, c->n_nodes, DivU64::make(c->N3),
                                                          DivU64::make(5), 1.0, E0);
    return cudaGetLastError();
}

}  // namespace esdc
