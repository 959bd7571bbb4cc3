// Initial states of the workloads evaluated on the device at the element node coordinates: the
// Taylor-Green vortex (Sec. 5.2), the isentropic vortex (Sec. 5.1.1, eq. iv_sol, about an arbitrary
// axis with a uniform drift) and a uniform state, in the library's nondimensionalisation
// (rho_inf = T_inf = 1, R = 1/(gamma Ma^2)).
#include <cmath>

#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

__global__ void __launch_bounds__(256) init_kernel(int ic, const InitParams prm, const double* __restrict__ xyz,
                                                   double* __restrict__ q, int64_t K, int N3, double gamma, double Ma,
                                                   double R) {
    const int64_t n = K * N3;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const int64_t el = g / N3;
        const int node = (int)(g - el * N3);
        const double* x = xyz + el * 3 * N3 + node;
        const double x1 = x[0], x2 = x[N3], x3 = x[2 * N3];
        double rho, u[3], p;
        if (ic == ESDC_IC_TGV) {
            rho = 1.0 + gamma * Ma * Ma / 16.0 * (cos(2.0 * x1) + cos(2.0 * x2)) * (cos(2.0 * x3) + 2.0);
            u[0] = sin(x1) * cos(x2) * cos(x3);
            u[1] = -cos(x1) * sin(x2) * cos(x3);
            u[2] = 0.0;
            p = rho * R;                                     // T = 1
        } else if (ic == ESDC_IC_VORTEX) {
            const double* a = prm.v + 4;                     // unit axis
            const double d[3] = {x1 - prm.v[1], x2 - prm.v[2], x3 - prm.v[3]};
            const double along = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
            const double r[3] = {d[0] - along * a[0], d[1] - along * a[1], d[2] - along * a[2]};
            const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            const double beta = prm.v[0];
            const double T = 1.0 - (gamma - 1.0) * Ma * Ma * beta * beta / (8.0 * kPi * kPi) * exp(1.0 - r2);
            rho = pow(T, 1.0 / (gamma - 1.0));
            const double amp = beta / (2.0 * kPi) * exp(0.5 * (1.0 - r2));      // u_t / r
            u[0] = prm.v[7] + amp * (a[1] * r[2] - a[2] * r[1]);
            u[1] = prm.v[8] + amp * (a[2] * r[0] - a[0] * r[2]);
            u[2] = prm.v[9] + amp * (a[0] * r[1] - a[1] * r[0]);
            p = rho * R * T;
        } else {
            rho = prm.v[0];
            u[0] = prm.v[1];
            u[1] = prm.v[2];
            u[2] = prm.v[3];
            p = prm.v[4];
        }
        double* qe = q + el * 5 * N3 + node;
        qe[0] = rho;
        qe[N3] = rho * u[0];
        qe[2 * N3] = rho * u[1];
        qe[3 * N3] = rho * u[2];
        qe[4 * N3] = p / (gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
}

}  // namespace

cudaError_t launch_init_state(const esdc_ctx* c, int ic, const InitParams& prm, double* q, cudaStream_t s) {
    int64_t blocks = (c->n_nodes + 255) / 256;
    if (blocks > grid_cap()) blocks = grid_cap();
    if (blocks < 1) blocks = 1;
    init_kernel<<<(unsigned)blocks, 256, 0, s>>>(ic, prm, c->d_xyz, q, c->K, c->N3, c->phys.gamma, c->setup.Ma,
                                                 c->phys.R);
    return cudaGetLastError();
}

}  // namespace esdc
