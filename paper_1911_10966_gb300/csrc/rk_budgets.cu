// Runge-Kutta stage combination (HBM-bound axpy), deterministic float64 budget reductions and the
// CFL reduction.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace {

constexpr int kRedThreads = 256;

// out[i] = q0[i] + sum_j coef_j k_j[i]; two doubles per thread per iteration (16-byte accesses)
__global__ void __launch_bounds__(256) combine_kernel(double* __restrict__ out, const double* __restrict__ q0,
                                                      const Combine cb, int64_t n) {
    const int64_t n2 = n / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        double2 acc = reinterpret_cast<const double2*>(q0)[i];
        for (int j = 0; j < cb.nk; ++j) {
            const double2 kv = reinterpret_cast<const double2*>(cb.k[j])[i];
            acc.x += cb.coef[j] * kv.x;
            acc.y += cb.coef[j] * kv.y;
        }
        reinterpret_cast<double2*>(out)[i] = acc;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        double acc = q0[n - 1];
        for (int j = 0; j < cb.nk; ++j) acc += cb.coef[j] * cb.k[j][n - 1];
        out[n - 1] = acc;
    }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    // fixed-order tree over the block (deterministic)
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Per block: sums of P J S, P J KE, P J w.dq, P J dKE.dq and the count of non-physical nodes.
template <typename TD>
__global__ void __launch_bounds__(kRedThreads) budgets_kernel(const double* __restrict__ q, const TD* __restrict__ dq,
                                                               const double* __restrict__ geom, int64_t K, int N,
                                                               const Ops ops, const Phys ph, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    const int N3 = N * N * N;
    const int64_t n = K * N3;
    double aS = 0.0, aK = 0.0, aW = 0.0, aE = 0.0, bad = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const int64_t e = g / N3;
        const int node = (int)(g - e * N3);
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / (N * N);
        const double PJ = ops.w[i1] * ops.w[i2] * ops.w[i3] * geom[e * 10 * N3 + node];
        double qv[5];
        for (int v = 0; v < 5; ++v) qv[v] = q[(e * 5 + v) * N3 + node];
        const double rho = qv[0];
        const double ri = 1.0 / rho;
        const double u0 = qv[1] * ri, u1 = qv[2] * ri, u2 = qv[3] * ri;
        const double usq = u0 * u0 + u1 * u1 + u2 * u2;
        const double p = (ph.gamma - 1.0) * (qv[4] - 0.5 * rho * usq);
        const bool ok = rho > 0.0 && p > 0.0 && isfinite(qv[0] + qv[1] + qv[2] + qv[3] + qv[4]);
        if (!ok) {
            bad += 1.0;
            continue;
        }
        const double s = log(p) - ph.gamma * log(rho);
        aS += PJ * (-rho * s * ph.inv_gm1);
        aK += PJ * 0.5 * rho * usq;
        if (dq) {
            double d[5];
            for (int v = 0; v < 5; ++v) d[v] = (double)dq[(e * 5 + v) * N3 + node];
            const double rp = rho / p;
            const double w1 = (ph.gamma - s) * ph.inv_gm1 - 0.5 * rp * usq;
            aW += PJ * (w1 * d[0] + rp * (u0 * d[1] + u1 * d[2] + u2 * d[3]) - rp * d[4]);
            aE += PJ * (-0.5 * usq * d[0] + u0 * d[1] + u1 * d[2] + u2 * d[3]);
            if (!isfinite(d[0] + d[1] + d[2] + d[3] + d[4])) bad += 1.0;
        }
    }
    const double r0 = block_sum(aS, sh), r1 = block_sum(aK, sh), r2 = block_sum(aW, sh), r3 = block_sum(aE, sh),
                 r4 = block_sum(bad, sh);
    if (threadIdx.x == 0) {
        double* o = part + blockIdx.x * 5;
        o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3; o[4] = r4;
    }
}

// Sum nparts rows of width `width` in a fixed order (one block).
__global__ void __launch_bounds__(kRedThreads) finish_sum(const double* __restrict__ part, int nparts, int width,
                                                          double* __restrict__ out) {
    __shared__ double sh[kRedThreads];
    for (int c = 0; c < width; ++c) {
        double a = 0.0;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += part[i * width + c];
        const double r = block_sum(a, sh);
        if (threadIdx.x == 0) out[c] = r;
    }
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = fmax(sh[t], sh[t + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Per block: max(|u| + c), max(-rho) and the non-physical count (as a max of a 0/1 flag sum).
__global__ void __launch_bounds__(kRedThreads) cfl_kernel(const double* __restrict__ q, int64_t n_nodes, int N3,
                                                           const Phys ph, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double smax = 0.0, nrmin = -1e300, bad = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_nodes; g += stride) {
        const int64_t e = g / N3;
        const int node = (int)(g - e * N3);
        double qv[5];
        for (int v = 0; v < 5; ++v) qv[v] = q[(e * 5 + v) * N3 + node];
        const double rho = qv[0];
        const double u0 = qv[1] / rho, u1 = qv[2] / rho, u2 = qv[3] / rho;
        const double usq = u0 * u0 + u1 * u1 + u2 * u2;
        const double p = (ph.gamma - 1.0) * (qv[4] - 0.5 * rho * usq);
        if (!(rho > 0.0 && p > 0.0 && isfinite(usq + p))) {
            bad = 1.0;
            continue;
        }
        smax = fmax(smax, sqrt(usq) + sqrt(ph.gamma * p / rho));
        nrmin = fmax(nrmin, -rho);
    }
    const double r0 = block_max(smax, sh), r1 = block_max(nrmin, sh), r2 = block_max(bad, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = r0;
        part[blockIdx.x * 3 + 1] = r1;
        part[blockIdx.x * 3 + 2] = r2;
    }
}

__global__ void __launch_bounds__(kRedThreads) finish_max(const double* __restrict__ part, int nparts, int width,
                                                          double* __restrict__ out) {
    __shared__ double sh[kRedThreads];
    for (int c = 0; c < width; ++c) {
        double a = -1e300;
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) a = fmax(a, part[i * width + c]);
        const double r = block_max(a, sh);
        if (threadIdx.x == 0) out[c] = r;
    }
}

__global__ void __launch_bounds__(256) scale_kernel(double* __restrict__ out, const double* __restrict__ x, double a,
                                                    int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = a * x[i];
}

// d/dq of sum P J rho|u|^2/2: P J (-|u|^2/2, u, 0)
__global__ void __launch_bounds__(256) ke_grad_kernel(const double* __restrict__ q, const double* __restrict__ geom,
                                                      int64_t K, int N, const Ops ops, double* __restrict__ g) {
    const int N3 = N * N * N;
    const int64_t n = K * N3;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t e = i / N3;
        const int node = (int)(i - e * N3);
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / (N * N);
        const double PJ = ops.w[i1] * ops.w[i2] * ops.w[i3] * geom[e * 10 * N3 + node];
        const double* qe = q + e * 5 * N3 + node;
        const double ri = 1.0 / qe[0];
        const double u0 = qe[N3] * ri, u1 = qe[2 * N3] * ri, u2 = qe[3 * N3] * ri;
        double* ge = g + e * 5 * N3 + node;
        ge[0] = -0.5 * PJ * (u0 * u0 + u1 * u1 + u2 * u2);
        ge[N3] = PJ * u0;
        ge[2 * N3] = PJ * u1;
        ge[3 * N3] = PJ * u2;
        ge[4 * N3] = 0.0;
    }
}

}  // namespace

cudaError_t launch_scale(double* out, const double* x, double a, int64_t n, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    scale_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, x, a, n);
    return cudaGetLastError();
}

cudaError_t launch_ke_gradient(const esdc_ctx* c, const double* q, double* grad, cudaStream_t s) {
    int64_t blocks = (c->n_nodes + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    ke_grad_kernel<<<(unsigned)blocks, 256, 0, s>>>(q, c->d_geom, c->K, c->N, c->ops, grad);
    return cudaGetLastError();
}

cudaError_t launch_combine(double* out, const double* q0, const Combine& cb, int64_t n, cudaStream_t s) {
    int64_t blocks = (n / 2 + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, q0, cb, n);
    return cudaGetLastError();
}

cudaError_t launch_budgets(const esdc_ctx* c, const double* q, const void* dqdt, int dq_f32, cudaStream_t s) {
    if (dq_f32)
        budgets_kernel<float><<<c->red_blocks, kRedThreads, 0, s>>>(q, (const float*)dqdt, c->d_geom, c->K, c->N,
                                                                     c->ops, c->phys, c->d_red);
    else
        budgets_kernel<double><<<c->red_blocks, kRedThreads, 0, s>>>(q, (const double*)dqdt, c->d_geom, c->K, c->N,
                                                                      c->ops, c->phys, c->d_red);
    finish_sum<<<1, kRedThreads, 0, s>>>(c->d_red, c->red_blocks, 5, c->d_red_out);
    return cudaGetLastError();
}

cudaError_t launch_cfl(const esdc_ctx* c, const double* q, cudaStream_t s) {
    cfl_kernel<<<c->red_blocks, kRedThreads, 0, s>>>(q, c->n_nodes, c->N3, c->phys, c->d_red);
    finish_max<<<1, kRedThreads, 0, s>>>(c->d_red, c->red_blocks, 3, c->d_red_out);
    return cudaGetLastError();
}

}  // namespace esdc
