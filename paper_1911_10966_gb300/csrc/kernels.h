// Kernel launchers (one per translation unit) used by the C ABI layer.
#pragma once

#include <cuda_runtime.h>

#include "esdc_internal.h"

namespace esdc {

// Quotient by a run-time invariant divisor d >= 2 as the high 64 bits of x * M with M = ceil(2^64 / d)
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994).  Writing
// M d = 2^64 + delta, 0 <= delta < d, the product over 2^64 is x/d + x delta / (d 2^64), which keeps
// the floor of x/d for every x < 2^64 / d.
struct DivU64 {
    unsigned long long m;
    static DivU64 make(unsigned long long d) { return DivU64{~0ull / d + 1ull}; }
    __device__ __forceinline__ unsigned long long operator()(unsigned long long x) const { return __umul64hi(x, m); }
};

cudaError_t prepare_rhs_f64(const esdc_ctx* c);
// ev: NULL, or four events recorded around the element kernel and the face kernel
cudaError_t launch_rhs_f64(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev);
// the p = 15 float64 residual (N = kLargeN), called by the two above
cudaError_t prepare_rhs_large(const esdc_ctx* c);
cudaError_t launch_rhs_large(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev);

// out = q0 + sum_j coef[j] * k[j]   (n doubles; k pointers may alias nothing but each other)
struct Combine {
    const double* k[6];
    double coef[6];
    int nk;
};
cudaError_t launch_combine(double* out, const double* q0, const Combine& cb, int64_t n, cudaStream_t s);

// out = sum_j c[j] * x[j] (n doubles, up to 7 terms, summed in j order; out may alias an x[j])
struct LinComb {
    const double* x[7];
    double c[7];
    int n;
};
cudaError_t launch_lincomb(double* out, const LinComb& lc, int64_t n, cudaStream_t s);
// sum over all elements of ((sum_j c_j x_j) / (atol + rtol max(|q0|, |q1|)))^2 into c->d_red_out[0]
// (5 to 7 terms)
cudaError_t launch_dp54_error(const esdc_ctx* c, const double* q0, const double* q1, const LinComb& lc, double rtol,
                              double atol, cudaStream_t s);
// the same with float32 stage derivatives (the float32-mixed form)
struct LinCombF {
    const float* x[7];
    double c[7];
    int n;
};
cudaError_t launch_dp54_error_f32(const esdc_ctx* c, const double* q0, const double* q1, const LinCombF& lc,
                                  double rtol, double atol, cudaStream_t s);

// Reductions: budgets (4 sums + non-physical count) and CFL inputs (max |u|+c, min rho).
// Table of the budgets' logarithm: entry k (0 <= k < kLnTab) holds T_k = 1/c_k rounded to double,
// c_k = 1 + (k + 1/2)/kLnTab, and -ln T_k as a head and a tail double (host, long double).
constexpr int kLnTab = 128;
void fill_ln_table(double* tab);
// out: 5 doubles of device memory (NULL: the context's d_red_out)
cudaError_t launch_budgets(const esdc_ctx* c, const double* q, const void* dqdt, int dq_f32, double* out,
                           cudaStream_t s);
cudaError_t launch_cfl(const esdc_ctx* c, const double* q, cudaStream_t s);

cudaError_t probe_fma(int kind, double* flops_per_s, cudaStream_t s);

// initial states at the node coordinates (ESDC_IC_*); v as documented for esdc_init_state, the
// vortex axis normalised
struct InitParams {
    double v[10];
};
cudaError_t launch_init_state(const esdc_ctx* c, int ic, const InitParams& prm, double* q, cudaStream_t s);

// adjoint (float64)
size_t adjoint_mu_blocks(const esdc_ctx* c);
cudaError_t prepare_adjoint(const esdc_ctx* c);
// grad = (dR/dq)^T lam; if mu_acc != NULL, *mu_acc += lam . dR/dmu (device scalar)
cudaError_t launch_rhs_vjp(const esdc_ctx* c, const double* q, const double* lam, double* grad, double* mu_acc,
                           cudaStream_t s);
cudaError_t launch_scale(double* out, const double* x, double a, int64_t n, cudaStream_t s);
cudaError_t launch_ke_gradient(const esdc_ctx* c, const double* q, double* grad, cudaStream_t s);

// mixed-precision form
struct StageF {             // a stage state base + sum_j c_j k_j (float32 perturbation state); the
                            // residual kernels take nk = 0, launch_stage_f32 forms the others
    const float* base;
    const float* k[6];
    float c[6];
    int nk;
};
cudaError_t prepare_rhs_f32(const esdc_ctx* c);
cudaError_t launch_rhs_f32(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev);
// the ES-C float32 residual with packed (f32x2) pair evaluation (rhs_f32_pairs.cu; built for N = 4,
// 6, 8, taken for N = 4, 8), called by the two above where supported
bool pairs_f32_supported(const esdc_ctx* c);
cudaError_t prepare_rhs_f32_pairs(const esdc_ctx* c);
cudaError_t launch_rhs_f32_pairs(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev);
struct Combine64F {         // float64 accumulation of float32 stage derivatives
    const float* k[6];
    double coef[6];
    int nk;
};
cudaError_t launch_shadow(const esdc_ctx* c, const double* q, float* dq, cudaStream_t s);
// y = in.base + sum_j in.c[j] in.k[j] (float32, 1 <= in.nk <= 5; y, base, k 16-byte aligned)
cudaError_t launch_stage_f32(const esdc_ctx* c, const StageF& in, float* y, cudaStream_t s);
cudaError_t launch_final_f32(const esdc_ctx* c, double* q, float* dq_new, const Combine64F& cb, cudaStream_t s);

}  // namespace esdc
