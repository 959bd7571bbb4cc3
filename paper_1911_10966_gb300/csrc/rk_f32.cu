// Float64 <-> float32 state kernels of the mixed-precision form, and its float32 stage states.
//   stage:   y = base + sum_j c_j k_j in float32 (the input of a stage's residual).
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

// q - q_ref for variable v of the layout (rho0 for the density, E0 for the energy)
__device__ __forceinline__ double less_ref(double x, int v, double rho0, double E0) {
    if (v == 0) return x - rho0;
    if (v == 4) return x - E0;
    return x;
}

// Four consecutive entries per thread and iteration (two 16-byte state loads, one 16-byte shadow
// store); the remaining n mod 4 entries are done by one thread.  Several independent entries per
// thread keep the float64 pipe busy despite its latency.
__global__ void __launch_bounds__(256) shadow_kernel(const double* __restrict__ q, float* __restrict__ dq,
                                                     int64_t n_nodes, DivU64 div_n3, DivU64 div_5, double rho0,
                                                     double E0) {
    const int64_t n = n_nodes * 5, n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        const int64_t i = 4 * t;
        const double2 x0 = reinterpret_cast<const double2*>(q)[2 * t], x1 = reinterpret_cast<const double2*>(q)[2 * t + 1];
        const double x[4] = {x0.x, x0.y, x1.x, x1.y};
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) r[e] = d2f_int(less_ref(x[e], var_of(i + e, div_n3, div_5), rho0, E0));
        reinterpret_cast<float4*>(dq)[t] = make_float4(r[0], r[1], r[2], r[3]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = 4 * n4; i < n; ++i) dq[i] = d2f_int(less_ref(q[i], var_of(i, div_n3, div_5), rho0, E0));
}

// The update of NK stage terms, four consecutive entries per thread and iteration; all loads of an
// iteration are issued together and each entry's terms are summed in stage order in float64.
template <int NK>
__device__ __forceinline__ double stage_sum(const Combine64F& cb, const float* kv) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < NK; ++j) acc = fma(cb.coef[j], f2d_int(kv[j]), acc);
    return acc;
}

template <int NK>
__global__ void __launch_bounds__(256) final_kernel(double* __restrict__ q, float* __restrict__ dq_new,
                                                    const Combine64F cb, int64_t n_nodes, DivU64 div_n3,
                                                    DivU64 div_5, double rho0, double E0) {
    const int64_t n = n_nodes * 5, n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        const int64_t i = 4 * t;
        float4 k4[NK];
#pragma unroll
        for (int j = 0; j < NK; ++j) k4[j] = __ldg(reinterpret_cast<const float4*>(cb.k[j]) + t);
        const double2 q0 = reinterpret_cast<const double2*>(q)[2 * t], q1 = reinterpret_cast<const double2*>(q)[2 * t + 1];
        float kx[NK], ky[NK], kz[NK], kw[NK];
#pragma unroll
        for (int j = 0; j < NK; ++j) {
            kx[j] = k4[j].x;
            ky[j] = k4[j].y;
            kz[j] = k4[j].z;
            kw[j] = k4[j].w;
        }
        const double qn[4] = {q0.x + stage_sum<NK>(cb, kx), q0.y + stage_sum<NK>(cb, ky), q1.x + stage_sum<NK>(cb, kz),
                              q1.y + stage_sum<NK>(cb, kw)};
        reinterpret_cast<double2*>(q)[2 * t] = make_double2(qn[0], qn[1]);
        reinterpret_cast<double2*>(q)[2 * t + 1] = make_double2(qn[2], qn[3]);
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) r[e] = d2f_int(less_ref(qn[e], var_of(i + e, div_n3, div_5), rho0, E0));
        reinterpret_cast<float4*>(dq_new)[t] = make_float4(r[0], r[1], r[2], r[3]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = 4 * n4; i < n; ++i) {
            float kv[NK];
#pragma unroll
            for (int j = 0; j < NK; ++j) kv[j] = cb.k[j][i];
            const double qi = q[i] + stage_sum<NK>(cb, kv);
            q[i] = qi;
            dq_new[i] = d2f_int(less_ref(qi, var_of(i, div_n3, div_5), rho0, E0));
        }
}

// y = base + sum_j c_j k_j: a float32 stage state of the mixed-precision step, the terms added in
// stage order with float32 fused multiply-adds; four entries per thread and iteration (16-byte
// accesses; workspace buffers), all loads of an iteration issued together.
template <int NK>
__global__ void __launch_bounds__(256) stage_kernel(float* __restrict__ y, const StageF in, int64_t n) {
    const int64_t n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        float4 kv[NK];
#pragma unroll
        for (int j = 0; j < NK; ++j) kv[j] = __ldg(reinterpret_cast<const float4*>(in.k[j]) + t);
        float4 a = __ldg(reinterpret_cast<const float4*>(in.base) + t);
#pragma unroll
        for (int j = 0; j < NK; ++j) {
            a.x = fmaf(in.c[j], kv[j].x, a.x);
            a.y = fmaf(in.c[j], kv[j].y, a.y);
            a.z = fmaf(in.c[j], kv[j].z, a.z);
            a.w = fmaf(in.c[j], kv[j].w, a.w);
        }
        reinterpret_cast<float4*>(y)[t] = a;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = 4 * n4; i < n; ++i) {
            float a = in.base[i];
#pragma unroll
            for (int j = 0; j < NK; ++j) a = fmaf(in.c[j], in.k[j][i], a);
            y[i] = a;
        }
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > grid_cap()) b = grid_cap();
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_shadow(const esdc_ctx* c, const double* q, float* dq, cudaStream_t s) {
    const double E0 = c->phys.R / (c->phys.gamma - 1.0);
    shadow_kernel<<<grid_for(c->n_nodes * 5 / 4), 256, 0, s>>>(q, dq, c->n_nodes, DivU64::make(c->N3),
                                                               DivU64::make(5), 1.0, E0);
    return cudaGetLastError();
}

cudaError_t launch_stage_f32(const esdc_ctx* c, const StageF& in, float* y, cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    const unsigned g = grid_for(n / 4);
    switch (in.nk) {
        case 1: stage_kernel<1><<<g, 256, 0, s>>>(y, in, n); break;
        case 2: stage_kernel<2><<<g, 256, 0, s>>>(y, in, n); break;
        case 3: stage_kernel<3><<<g, 256, 0, s>>>(y, in, n); break;
        case 4: stage_kernel<4><<<g, 256, 0, s>>>(y, in, n); break;
        case 5: stage_kernel<5><<<g, 256, 0, s>>>(y, in, n); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_final_f32(const esdc_ctx* c, double* q, float* dq_new, const Combine64F& cb, cudaStream_t s) {
    const double E0 = c->phys.R / (c->phys.gamma - 1.0);
    const unsigned g = grid_for(c->n_nodes * 5 / 4);
    const DivU64 d3 = DivU64::make(c->N3), d5 = DivU64::make(5);
    switch (cb.nk) {
        case 1: final_kernel<1><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        case 2: final_kernel<2><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        case 3: final_kernel<3><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        case 4: final_kernel<4><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        case 5: final_kernel<5><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        case 6: final_kernel<6><<<g, 256, 0, s>>>(q, dq_new, cb, c->n_nodes, d3, d5, 1.0, E0); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace esdc
