// Float64 <-> float32 state kernels of the mixed-precision form.
//   shadow:  dq = float(q - q_ref) with q_ref = (rho0, 0, 0, 0, E0): the float32 perturbation state
//            the float32 residual reads (float64 subtraction before rounding).
//   final:   q += sum_j c_j k_j accumulated in float64 (the Runge-Kutta solution update), then the
//            new shadow of q is written.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace {

__global__ void __launch_bounds__(256) shadow_kernel(const double* __restrict__ q, float* __restrict__ dq,
                                                     int64_t n_nodes, int N3, double rho0, double E0) {
    const int64_t n = n_nodes * 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int v = (int)((i / N3) % 5);
        const double off = v == 0 ? rho0 : (v == 4 ? E0 : 0.0);
        dq[i] = (float)(q[i] - off);
    }
}

__global__ void __launch_bounds__(256) final_kernel(double* __restrict__ q, float* __restrict__ dq_new,
                                                    const Combine64F cb, int64_t n_nodes, int N3, double rho0,
                                                    double E0) {
    const int64_t n = n_nodes * 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double inc = 0.0;
        for (int j = 0; j < cb.nk; ++j) inc += cb.coef[j] * (double)cb.k[j][i];
        const double qn = q[i] + inc;
        q[i] = qn;
        const int v = (int)((i / N3) % 5);
        const double off = v == 0 ? rho0 : (v == 4 ? E0 : 0.0);
        dq_new[i] = (float)(qn - off);
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
    shadow_kernel<<<grid_for(c->n_nodes * 5), 256, 0, s>>>(q, dq, c->n_nodes, c->N3, 1.0, E0);
    return cudaGetLastError();
}

cudaError_t launch_final_f32(const esdc_ctx* c, double* q, float* dq_new, const Combine64F& cb, cudaStream_t s) {
    const double E0 = c->phys.R / (c->phys.gamma - 1.0);
    final_kernel<<<grid_for(c->n_nodes * 5), 256, 0, s>>>(q, dq_new, cb, c->n_nodes, c->N3, 1.0, E0);
    return cudaGetLastError();
}

}  // namespace esdc
