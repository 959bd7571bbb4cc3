// Runge-Kutta stage combination (HBM-bound axpy), deterministic float64 budget reductions and the
// CFL reduction.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace {

constexpr int kRedThreads = 256;

// out[i] = q0[i] + sum_j coef_j k_j[i]; with V2 two doubles per thread per iteration (16-byte accesses,
// every pointer 16-byte aligned), else one.  NK, the number of terms, is a template parameter so that
// the stage pointers stay in parameter space, all loads of an iteration are issued together and no
// float64 work is spent on absent terms; terms are summed in stage order.
template <int NK, bool V2>
__global__ void __launch_bounds__(256) combine_kernel(double* __restrict__ out, const double* __restrict__ q0,
                                                      const Combine cb, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (V2) {
        const int64_t n2 = n / 2;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
            double2 kv[NK];
#pragma unroll
            for (int j = 0; j < NK; ++j) kv[j] = reinterpret_cast<const double2*>(cb.k[j])[i];
            double2 acc = reinterpret_cast<const double2*>(q0)[i];
#pragma unroll
            for (int j = 0; j < NK; ++j) {
                acc.x = fma(cb.coef[j], kv[j].x, acc.x);
                acc.y = fma(cb.coef[j], kv[j].y, acc.y);
            }
            reinterpret_cast<double2*>(out)[i] = acc;
        }
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            double acc = q0[n - 1];
#pragma unroll
            for (int j = 0; j < NK; ++j) acc = fma(cb.coef[j], cb.k[j][n - 1], acc);
            out[n - 1] = acc;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            double kv[NK];
#pragma unroll
            for (int j = 0; j < NK; ++j) kv[j] = cb.k[j][i];
            double acc = q0[i];
#pragma unroll
            for (int j = 0; j < NK; ++j) acc = fma(cb.coef[j], kv[j], acc);
            out[i] = acc;
        }
    }
}

// out[i] = sum_j c_j x_j[i] over NT terms, terms in j order (the first one a product, the rest fused
// multiply-adds); with V2 two doubles per thread and iteration (every pointer 16-byte aligned), else
// one.  Each thread reads all its terms before writing, so out may alias an input.
template <int NT, bool V2>
__global__ void __launch_bounds__(256) lincomb_kernel(double* __restrict__ out, const LinComb lc, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (V2) {
        const int64_t n2 = n / 2;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
            double2 xv[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) xv[j] = reinterpret_cast<const double2*>(lc.x[j])[i];
            double2 acc = make_double2(lc.c[0] * xv[0].x, lc.c[0] * xv[0].y);
#pragma unroll
            for (int j = 1; j < NT; ++j) {
                acc.x = fma(lc.c[j], xv[j].x, acc.x);
                acc.y = fma(lc.c[j], xv[j].y, acc.y);
            }
            reinterpret_cast<double2*>(out)[i] = acc;
        }
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            double acc = lc.c[0] * lc.x[0][n - 1];
#pragma unroll
            for (int j = 1; j < NT; ++j) acc = fma(lc.c[j], lc.x[j][n - 1], acc);
            out[n - 1] = acc;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            double xv[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) xv[j] = lc.x[j][i];
            double acc = lc.c[0] * xv[0];
#pragma unroll
            for (int j = 1; j < NT; ++j) acc = fma(lc.c[j], xv[j], acc);
            out[i] = acc;
        }
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

__device__ __forceinline__ double rcp_nr(double x) {
    // hardware reciprocal estimate refined by two Newton steps y <- y + y (1 - x y)
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}

// ln x for a positive finite double by table reduction (Tang's method, ACM TOMS 15, 1989): with
// x = m 2^e, m in [1, 2), and k the top 7 bits of m's fraction, r = m T_k - 1 (one FMA, |r| <= 2^-8
// since m lies within 1/256 of c_k), and
//   ln x = e ln 2 - ln T_k + ln(1 + r),  ln(1 + r) = r - r^2/2 + r^3/3 - ... + r^7/7,
// the first omitted term r^8/8 being below 2^-67.  The error is about one unit in the last place of
// the larger of e ln 2 and ln c_k; near x = 1 from below the two nearly cancel, so the error there is
// absolute (~1e-16), which is what the entropy sums need.  tab: shared-memory copy of the table
// (T_k, head, tail of -ln T_k).
__device__ __forceinline__ double ln_pos(double x, const double* __restrict__ tab, double ln2_hi, double ln2_lo) {
    long long b = __double_as_longlong(x);
    int e = 0;
    if (b < 0x0010000000000000LL) {            // subnormal: scale by 2^54 first
        x *= 18014398509481984.0;
        b = __double_as_longlong(x);
        e = -54;
    }
    e += (int)(b >> 52) - 1023;
    const int k = (int)((b >> 45) & (kLnTab - 1));
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);   // [1, 2)
    const double r = fma(m, tab[3 * k], -1.0);
    double c = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    c = fma(r, c, 1.0 / 5.0);
    c = fma(r, c, -1.0 / 4.0);
    c = fma(r, c, 1.0 / 3.0);
    c = fma(r, c, -1.0 / 2.0);
    const double p = fma(r * r, c, r);
    const double ed = (double)e;
    return fma(ed, ln2_hi, tab[3 * k + 1]) + (fma(ed, ln2_lo, tab[3 * k + 2]) + p);
}

struct Ln2 {
    double hi, lo;
};

// true when x is neither infinite nor NaN (exponent field not all ones), tested on the integer pipe
__device__ __forceinline__ bool finite_bits(double x) { return (__double2hiint(x) & 0x7FF00000) != 0x7FF00000; }

// Per block: sums of P J S, P J KE, P J w.dq, P J dKE.dq and the count of non-physical nodes.
template <typename TD>
__global__ void __launch_bounds__(kRedThreads) budgets_kernel(const double* __restrict__ q, const TD* __restrict__ dq,
                                                              const double* __restrict__ geom, int64_t K, int N,
                                                              DivU64 div_n3, const Ops ops, const Phys ph, Ln2 ln2,
                                                              const double* __restrict__ lntab, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    __shared__ double sw[kMaxN * kMaxN * kMaxN];     // tensor-product LGL weights w_i1 w_i2 w_i3
    __shared__ double stab[3 * kLnTab];
    const int N3 = N * N * N;
    const bool table = N3 <= kMaxN * kMaxN * kMaxN;   // p = 15: weights formed per node below
    if (table)
        for (int node = threadIdx.x; node < N3; node += blockDim.x)
            sw[node] = ops.w[node % N] * ops.w[(node / N) % N] * ops.w[node / (N * N)];
    for (int i = threadIdx.x; i < 3 * kLnTab; i += blockDim.x) stab[i] = lntab[i];
    __syncthreads();
    const int64_t n = K * N3;
    double aS = 0.0, aK = 0.0, aW = 0.0, aE = 0.0, bad = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const int64_t e = (int64_t)div_n3((unsigned long long)g);
        const int node = (int)(g - e * N3);
        const double wn = table ? sw[node] : ops.w[node % N] * ops.w[(node / N) % N] * ops.w[node / (N * N)];
        const double PJ = wn * geom[e * 10 * N3 + node];
        double qv[5];
        for (int v = 0; v < 5; ++v) qv[v] = q[(e * 5 + v) * N3 + node];
        const double rho = qv[0];
        const bool pos = rho > 0.0 && finite_bits(qv[0]) && finite_bits(qv[1]) && finite_bits(qv[2]) &&
                         finite_bits(qv[3]) && finite_bits(qv[4]);
        const double ri = rcp_nr(pos ? rho : 1.0);
        const double u0 = qv[1] * ri, u1 = qv[2] * ri, u2 = qv[3] * ri;
        const double usq = u0 * u0 + u1 * u1 + u2 * u2;
        const double p = (ph.gamma - 1.0) * (qv[4] - 0.5 * rho * usq);
        if (!(pos && p > 0.0)) {
            bad += 1.0;
            continue;
        }
        const double s = ln_pos(p, stab, ln2.hi, ln2.lo) - ph.gamma * ln_pos(rho, stab, ln2.hi, ln2.lo);
        aS += PJ * (-rho * s * ph.inv_gm1);
        aK += PJ * 0.5 * rho * usq;
        if (dq) {
            double d[5];
            bool fin = true;
            for (int v = 0; v < 5; ++v) {
                d[v] = (double)dq[(e * 5 + v) * N3 + node];
                fin = fin && finite_bits(d[v]);
            }
            const double rp = rho * rcp_nr(p);
            const double w1 = (ph.gamma - s) * ph.inv_gm1 - 0.5 * rp * usq;
            aW += PJ * (w1 * d[0] + rp * (u0 * d[1] + u1 * d[2] + u2 * d[3]) - rp * d[4]);
            aE += PJ * (-0.5 * usq * d[0] + u0 * d[1] + u1 * d[2] + u2 * d[3]);
            if (!fin) bad += 1.0;
        }
    }
    const double r0 = block_sum(aS, sh), r1 = block_sum(aK, sh), r2 = block_sum(aW, sh), r3 = block_sum(aE, sh),
                 r4 = block_sum(bad, sh);
    if (threadIdx.x == 0) {
        double* o = part + blockIdx.x * 5;
        o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3; o[4] = r4;
    }
}

// Embedded error estimate of one Dormand-Prince 5(4) step (Dormand & Prince 1980): per element
// e = sum_j d_j k_j (d_j = dt (b_j - bhat_j), NT nonzero terms), sc = atol + rtol max(|q0|, |q1|),
// and the block sums of (e/sc)^2 (the weighted RMS norm of Hairer, Norsett & Wanner, eq. II.4.11,
// before the mean and square root).
template <int NT, typename LC>
__global__ void __launch_bounds__(kRedThreads) dp54_err_kernel(const double* __restrict__ q0,
                                                               const double* __restrict__ q1, const LC lc,
                                                               double rtol, double atol, int64_t n,
                                                               double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double kv[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) kv[j] = (double)lc.x[j][i];
        const double a = q0[i], b = q1[i];
        double e = lc.c[0] * kv[0];
#pragma unroll
        for (int j = 1; j < NT; ++j) e = fma(lc.c[j], kv[j], e);
        const double sc = fma(rtol, fmax(fabs(a), fabs(b)), atol);
        const double r = e * rcp_nr(sc);
        acc = fma(r, r, acc);
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Sum nparts rows of width `width` in a fixed order (one block): warp w sums columns w, w + 8, ...;
// each lane adds rows lane, lane + 32, ... in order, then a fixed butterfly combines the lanes.
__global__ void __launch_bounds__(kRedThreads) finish_sum(const double* __restrict__ part, int nparts, int width,
                                                          double* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < width; c += kRedThreads / 32) {
        double a = 0.0;
        for (int i = lane; i < nparts; i += 32) a += part[i * width + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[c] = a;
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
    if (blocks > grid_cap()) blocks = grid_cap();
    if (blocks < 1) blocks = 1;
    scale_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, x, a, n);
    return cudaGetLastError();
}

cudaError_t launch_ke_gradient(const esdc_ctx* c, const double* q, double* grad, cudaStream_t s) {
    int64_t blocks = (c->n_nodes + 255) / 256;
    if (blocks > grid_cap()) blocks = grid_cap();
    if (blocks < 1) blocks = 1;
    ke_grad_kernel<<<(unsigned)blocks, 256, 0, s>>>(q, c->d_geom, c->K, c->N, c->ops, grad);
    return cudaGetLastError();
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int NK>
void combine_any(unsigned g, bool v2, double* out, const double* q0, const Combine& cb, int64_t n, cudaStream_t s) {
    if (v2)
        combine_kernel<NK, true><<<g, 256, 0, s>>>(out, q0, cb, n);
    else
        combine_kernel<NK, false><<<g, 256, 0, s>>>(out, q0, cb, n);
}

// Stage states inside caller arrays (checkpoints, stored stages) start at multiples of the state
// size, only 8-byte aligned when K N^3 is odd: such calls take the one-double-per-thread kernels.
cudaError_t launch_combine(double* out, const double* q0, const Combine& cb, int64_t n, cudaStream_t s) {
    bool v2 = aligned16(out) && aligned16(q0);
    for (int j = 0; j < cb.nk && j < 6; ++j) v2 = v2 && aligned16(cb.k[j]);
    int64_t blocks = ((v2 ? n / 2 : n) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > grid_cap()) blocks = grid_cap();
    const unsigned g = (unsigned)blocks;
    switch (cb.nk) {
        case 1: combine_any<1>(g, v2, out, q0, cb, n, s); break;
        case 2: combine_any<2>(g, v2, out, q0, cb, n, s); break;
        case 3: combine_any<3>(g, v2, out, q0, cb, n, s); break;
        case 4: combine_any<4>(g, v2, out, q0, cb, n, s); break;
        case 5: combine_any<5>(g, v2, out, q0, cb, n, s); break;
        case 6: combine_any<6>(g, v2, out, q0, cb, n, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

void fill_ln_table(double* tab) {
    for (int k = 0; k < kLnTab; ++k) {
        const double c = 1.0 + (k + 0.5) / kLnTab;
        const double T = 1.0 / c;
        const long double L = -std::log((long double)T);
        const double hi = (double)L;
        tab[3 * k] = T;
        tab[3 * k + 1] = hi;
        tab[3 * k + 2] = (double)(L - (long double)hi);
    }
}

Ln2 ln2_split() {
    // ln 2 as a head with the low 20 bits of its significand cleared and the tail ln 2 - head
    const double l = std::log(2.0);
    unsigned long long bits;
    std::memcpy(&bits, &l, sizeof bits);
    bits &= ~0xFFFFFull;
    double hi;
    std::memcpy(&hi, &bits, sizeof hi);
    return Ln2{hi, (double)(std::log(2.0L) - (long double)hi)};
}

template <int NT>
void lincomb_any(unsigned g, bool v2, double* out, const LinComb& lc, int64_t n, cudaStream_t s) {
    if (v2)
        lincomb_kernel<NT, true><<<g, 256, 0, s>>>(out, lc, n);
    else
        lincomb_kernel<NT, false><<<g, 256, 0, s>>>(out, lc, n);
}

cudaError_t launch_lincomb(double* out, const LinComb& lc, int64_t n, cudaStream_t s) {
    bool v2 = aligned16(out);
    for (int j = 0; j < lc.n && j < 7; ++j) v2 = v2 && aligned16(lc.x[j]);
    int64_t blocks = ((v2 ? n / 2 : n) + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > grid_cap()) blocks = grid_cap();
    const unsigned g = (unsigned)blocks;
    switch (lc.n) {
        case 1: lincomb_any<1>(g, v2, out, lc, n, s); break;
        case 2: lincomb_any<2>(g, v2, out, lc, n, s); break;
        case 3: lincomb_any<3>(g, v2, out, lc, n, s); break;
        case 4: lincomb_any<4>(g, v2, out, lc, n, s); break;
        case 5: lincomb_any<5>(g, v2, out, lc, n, s); break;
        case 6: lincomb_any<6>(g, v2, out, lc, n, s); break;
        case 7: lincomb_any<7>(g, v2, out, lc, n, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename LC>
cudaError_t dp54_error_any(const esdc_ctx* c, const double* q0, const double* q1, const LC& lc, double rtol,
                           double atol, cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    switch (lc.n) {
        case 5: dp54_err_kernel<5, LC><<<c->red_blocks, kRedThreads, 0, s>>>(q0, q1, lc, rtol, atol, n, c->d_red); break;
        case 6: dp54_err_kernel<6, LC><<<c->red_blocks, kRedThreads, 0, s>>>(q0, q1, lc, rtol, atol, n, c->d_red); break;
        case 7: dp54_err_kernel<7, LC><<<c->red_blocks, kRedThreads, 0, s>>>(q0, q1, lc, rtol, atol, n, c->d_red); break;
        default: return cudaErrorInvalidValue;
    }
    finish_sum<<<1, kRedThreads, 0, s>>>(c->d_red, c->red_blocks, 1, c->d_red_out);
    return cudaGetLastError();
}

cudaError_t launch_dp54_error(const esdc_ctx* c, const double* q0, const double* q1, const LinComb& lc, double rtol,
                              double atol, cudaStream_t s) {
    return dp54_error_any(c, q0, q1, lc, rtol, atol, s);
}

cudaError_t launch_dp54_error_f32(const esdc_ctx* c, const double* q0, const double* q1, const LinCombF& lc,
                                  double rtol, double atol, cudaStream_t s) {
    return dp54_error_any(c, q0, q1, lc, rtol, atol, s);
}

cudaError_t launch_budgets(const esdc_ctx* c, const double* q, const void* dqdt, int dq_f32, double* out,
                           cudaStream_t s) {
    static const Ln2 ln2 = ln2_split();
    const DivU64 dn3 = DivU64::make((unsigned long long)c->N3);
    if (dq_f32)
        budgets_kernel<float><<<c->red_blocks, kRedThreads, 0, s>>>(q, (const float*)dqdt, c->d_geom, c->K, c->N, dn3,
                                                                     c->ops, c->phys, ln2, c->d_lntab, c->d_red);
    else
        budgets_kernel<double><<<c->red_blocks, kRedThreads, 0, s>>>(q, (const double*)dqdt, c->d_geom, c->K, c->N,
                                                                      dn3, c->ops, c->phys, ln2, c->d_lntab, c->d_red);
    finish_sum<<<1, kRedThreads, 0, s>>>(c->d_red, c->red_blocks, 5, out ? out : c->d_red_out);
    return cudaGetLastError();
}

cudaError_t launch_cfl(const esdc_ctx* c, const double* q, cudaStream_t s) {
    cfl_kernel<<<c->red_blocks, kRedThreads, 0, s>>>(q, c->n_nodes, c->N3, c->phys, c->d_red);
    finish_max<<<1, kRedThreads, 0, s>>>(c->d_red, c->red_blocks, 3, c->d_red_out);
    return cudaGetLastError();
}

}  // namespace esdc
