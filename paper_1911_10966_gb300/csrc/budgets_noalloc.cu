// esdc_budgets_noalloc: the float64 budget reduction for callers that must not allocate device
// memory.  Its scratch (per-block partial sums and the final sums) lives in a file-scope static
// device array, so the call itself performs no cudaMalloc/cudaFree and needs no context.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "esdc_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 16;                 // each block reduces 4096 consecutive nodes
constexpr int64_t kMaxRows = 65536;                 // partial rows the scratch holds
constexpr int64_t kMaxNodes = kMaxRows * kThreads * kNodesPerThread;   // 268,435,456 nodes
constexpr int kWidth = 5;                           // S, KE, w.dq, dKE.dq, non-physical count

// Scratch shared by every call on a device: kMaxRows rows of 5 partial sums (2.6 MB per device,
// resident until process exit; the final sums go to the caller's out array).  Every row a call
// reads was written earlier by the same call, so nothing needs clearing between calls.  Calls
// that overlap on the GPU race on it.
static __device__ __align__(256) double g_scratch[kMaxRows * kWidth];

struct W {
    double w[esdc::kMaxN];
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) partial_kernel(const double* __restrict__ q, const double* __restrict__ dq,
                                                           const double* __restrict__ J, int64_t n, int N,
                                                           double gamma, const W w, double* __restrict__ part) {
    __shared__ double sh[kThreads];
    const int N3 = N * N * N;
    const double inv_gm1 = 1.0 / (gamma - 1.0);
    double acc[kWidth] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t base = (int64_t)blockIdx.x * kThreads * kNodesPerThread;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const int64_t g = base + (int64_t)k * kThreads + threadIdx.x;
        if (g >= n) break;
        const int64_t e = g / N3;
        const int node = (int)(g - e * N3);
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / (N * N);
        const double PJ = w.w[i1] * w.w[i2] * w.w[i3] * J[g];
        double qv[5];
        for (int v = 0; v < 5; ++v) qv[v] = q[(e * 5 + v) * N3 + node];
        const double rho = qv[0];
        const double u0 = qv[1] / rho, u1 = qv[2] / rho, u2 = qv[3] / rho;
        const double usq = u0 * u0 + u1 * u1 + u2 * u2;
        const double p = (gamma - 1.0) * (qv[4] - 0.5 * rho * usq);
        if (!(rho > 0.0 && p > 0.0 && isfinite(qv[0] + qv[1] + qv[2] + qv[3] + qv[4]))) {
            acc[4] += 1.0;
            continue;
        }
        const double s = log(p) - gamma * log(rho);
        acc[0] += PJ * (-rho * s * inv_gm1);
        acc[1] += PJ * 0.5 * rho * usq;
        if (dq) {
            double d[5];
            for (int v = 0; v < 5; ++v) d[v] = dq[(e * 5 + v) * N3 + node];
            const double rp = rho / p;
            const double w1 = (gamma - s) * inv_gm1 - 0.5 * rp * usq;
            acc[2] += PJ * (w1 * d[0] + rp * (u0 * d[1] + u1 * d[2] + u2 * d[3]) - rp * d[4]);
            acc[3] += PJ * (-0.5 * usq * d[0] + u0 * d[1] + u1 * d[2] + u2 * d[3]);
            if (!isfinite(d[0] + d[1] + d[2] + d[3] + d[4])) acc[4] += 1.0;
        }
    }
    for (int c = 0; c < kWidth; ++c) {
        const double r = block_sum(acc[c], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kWidth + c] = r;
    }
}

// One block: sum the rows in a fixed order and write the five totals to out (caller memory).
__global__ void __launch_bounds__(kThreads) final_kernel(const double* __restrict__ part, int64_t rows,
                                                         double* __restrict__ out) {
    __shared__ double sh[kThreads];
    for (int c = 0; c < kWidth; ++c) {
        double a = 0.0;
        for (int64_t i = threadIdx.x; i < rows; i += kThreads) a += part[i * kWidth + c];
        const double r = block_sum(a, sh);
        if (threadIdx.x == 0) out[c] = r;
    }
}

// Device address of g_scratch per device (with that device current).  Outside stream capture the
// address is looked up again on every call, so a device reset (which reloads the module and moves
// the array) never leaves a stale pointer behind; during capture the last looked-up address is used.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {nullptr};

int scratch_for_current_device(bool refresh, double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        esdc::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return ESDC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        esdc::set_last_error("device index beyond the supported range");
        return ESDC_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (refresh || !g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            esdc::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return ESDC_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return ESDC_OK;
}

}  // namespace

extern "C" int esdc_budgets_noalloc(int N, int64_t K, double gamma, const double* w_host, const double* q_dev,
                                    const double* dqdt_dev, const double* J_dev, double* out_dev, void* stream) {
    if (N < 2 || N > esdc::kMaxN || K < 1 || !(gamma > 1.0) || !w_host || !q_dev || !J_dev || !out_dev) {
        esdc::set_last_error("esdc_budgets_noalloc: need 2 <= N <= 8, K >= 1, gamma > 1 and non-null w, q, J, out");
        return ESDC_ERR_ARG;
    }
    const int64_t n = K * (int64_t)N * N * N;
    if (n > kMaxNodes) {
        esdc::set_last_error("esdc_budgets_noalloc: " + std::to_string((long long)n) +
                             " nodes exceed the static scratch limit of " + std::to_string((long long)kMaxNodes) +
                             " nodes");
        return ESDC_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) {
        esdc::set_last_error(std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
        return ESDC_ERR_CUDA;
    }
    double* scratch = nullptr;
    int st = scratch_for_current_device(cs == cudaStreamCaptureStatusNone, &scratch);
    if (st) return st;
    W w{};
    for (int i = 0; i < N; ++i) w.w[i] = w_host[i];
    const int64_t rows = (n + (int64_t)kThreads * kNodesPerThread - 1) / ((int64_t)kThreads * kNodesPerThread);
    partial_kernel<<<(unsigned)rows, kThreads, 0, s>>>(q_dev, dqdt_dev, J_dev, n, N, gamma, w, scratch);
    final_kernel<<<1, kThreads, 0, s>>>(scratch, rows, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        esdc::set_last_error(std::string("esdc_budgets_noalloc launch: ") + cudaGetErrorString(e));
        return ESDC_ERR_CUDA;
    }
    return ESDC_OK;
}

