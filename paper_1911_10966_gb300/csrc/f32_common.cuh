// Device helpers shared by the float32 residual kernels of the mixed-precision form (rhs_f32.cu and
// rhs_f32_pairs.cu): the reference state, per-node primitives of the perturbation state, the split
// Chandrashekar two-point flux and the on-load formation of Runge-Kutta stage states.
#pragma once

#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"

namespace esdc {
namespace f32 {

// Per-node primitives in the form the pair loop consumes: half the density perturbation and half the
// velocity (so that averages are single additions), the velocity itself, and the perturbation of
// beta = rho/(2p) relative to beta0, dbn = beta/beta0 - 1 (so that the reference values are 1).
struct PrimF {
    float hdr, hu0, hu1, hu2, dbn, u0, u1, u2;
    float hdp, eh;   // SF-KG: half the pressure perturbation, (RT - RT0)/(2(gamma-1)) + |u|^2/4
};

struct Ref {
    float rho0, p0, RT0, H0, gm1, gamma;
    float hrho0;     // rho0 / 2
    float two_RT0;   // 2 RT0
    float c5;        // RT0 / (gamma - 1)
    float inv_rho0;
    float two_beta0; // rho0 / p0
    double rho0d, E0d;   // the reference density and energy in float64 (exterior states)
    float e0;            // RT0 / (gamma - 1)
    float inv_2gm1;      // 1 / (2 (gamma - 1))
};

// approximate reciprocal and square root (about 1 ulp): the float32 residual's rounding is
// dominated by the flux differencing, not by these
__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fsqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// primitives from the float32 perturbation state; with p = p0 + dp,
// beta/beta0 - 1 = (drho p0 - rho0 dp) / (rho0 p)
__device__ __forceinline__ void to_prim_f(const float dq[5], const Ref& r, PrimF& s) {
    const float rho = r.rho0 + dq[0];
    const float ri = frcp(rho);
    s.u0 = dq[1] * ri;
    s.u1 = dq[2] * ri;
    s.u2 = dq[3] * ri;
    const float usq = s.u0 * s.u0 + s.u1 * s.u1 + s.u2 * s.u2;
    const float dp = r.gm1 * (dq[4] - 0.5f * rho * usq);
    s.dbn = (dq[0] * r.p0 - r.rho0 * dp) * frcp(r.p0 + dp) * r.inv_rho0;
    s.hdp = 0.5f * dp;
    s.eh = (r.rho0 * dp - r.p0 * dq[0]) * ri * r.inv_rho0 * r.inv_2gm1 + 0.25f * usq;   // RT - RT0 = (rho0 dp - p0 drho)/(rho rho0)
    s.hdr = 0.5f * dq[0];
    s.hu0 = 0.5f * s.u0;
    s.hu1 = 0.5f * s.u1;
    s.hu2 = 0.5f * s.u2;
}

// 2 beta of a node (the entropy variables are 2 beta u and -2 beta) and RT = 1/(2 beta)
__device__ __forceinline__ float two_beta(const PrimF& s, const Ref& r) { return r.two_beta0 * (1.0f + s.dbn); }
__device__ __forceinline__ float node_RT(float dbn, const Ref& r) { return r.RT0 * frcp(1.0f + dbn); }

// perturbation part of the two-point flux (df[0..4]) and ubar.n (the linear reference part).  a
// supplies u (the full velocity), b half of it, both the halved density perturbation and dbn.
//   density: rho_bar = rho0 + dbar with dbar the mean perturbation, f = (drho_a - drho_b)/(rho_a + rho_b),
//     drho_ln = dbar + rho_bar (G(f^2) - 1), G = 1 - u/3 - 4u^2/45 - 44u^3/945 for f^2 < 1e-2
//   beta (in units of beta0): 1/(2 beta_ln) - RT0 = RT0 dIn, dIn = (2 (F - 1) - dbs)/(2 + dbs) with
//     dbs = dbn_a + dbn_b and F = 1 + u/3 + u^2/5 + u^3/7 in u = ((dbn_a - dbn_b)/(2 + dbs))^2
//   p_t - p0 = rho_bar/(2 beta_bar) - p0 = 2 RT0 (dbar - rho0 dbs / 2) / (2 + dbs)
//   df5 = RT0/(gamma-1) ubar.n (rho0 dIn + drho_ln (1 + dIn)) + f1 (u_a.u_b)/2 + (p_t - p0) ubar.n
__device__ __forceinline__ void ec_flux_pert(const PrimF& a, const PrimF& b, float n0, float n1, float n2,
                                             const Ref& r, float df[5], float& un) {
    const float dbar = a.hdr + b.hdr;
    const float rb = r.rho0 + dbar;
    const float f = (a.hdr - b.hdr) * frcp(rb);
    const float uu = f * f;
    float drl;
    if (uu < 1.0e-2f) {
        drl = fmaf(rb, uu * (-1.0f / 3.0f + uu * (-4.0f / 45.0f + uu * (-44.0f / 945.0f))), dbar);
    } else {
        const float ra = r.rho0 + 2.0f * a.hdr, rbb = r.rho0 + 2.0f * b.hdr;
        drl = (ra - rbb) * frcp(logf(ra * frcp(rbb))) - r.rho0;
    }
    const float dbs = a.dbn + b.dbn;
    const float rsb = frcp(2.0f + dbs);
    const float db = a.dbn - b.dbn;
    const float fb = db * rsb;
    const float ub = fb * fb;
    float dIn;
    if (ub < 1.0e-2f) {
        dIn = (ub * (2.0f / 3.0f + ub * (2.0f / 5.0f + ub * (2.0f / 7.0f))) - dbs) * rsb;
    } else {
        dIn = logf((1.0f + a.dbn) * frcp(1.0f + b.dbn)) * frcp(db) - 1.0f;
    }
    const float dpt = (r.two_RT0 * rsb) * fmaf(-r.hrho0, dbs, dbar);
    const float ub0 = a.hu0 + b.hu0, ub1 = a.hu1 + b.hu1, ub2 = a.hu2 + b.hu2;
    un = ub0 * n0 + ub1 * n1 + ub2 * n2;
    const float rr = r.rho0 + drl;
    const float f1 = rr * un;
    df[0] = drl * un;
    df[1] = f1 * ub0 + dpt * n0;
    df[2] = f1 * ub1 + dpt * n1;
    df[3] = f1 * ub2 + dpt * n2;
    const float hab = a.u0 * b.hu0 + a.u1 * b.hu1 + a.u2 * b.hu2;
    df[4] = fmaf(r.c5 * un, fmaf(dIn, rr, drl), fmaf(f1, hab, dpt * un));
}

template <int N>
__device__ __forceinline__ int line_base_f(int l, int t1, int t2) {
    return l == 0 ? (t1 * N + t2 * N * N) : (l == 1 ? (t1 + t2 * N * N) : (t1 + t2 * N));
}

template <int N>
__device__ __forceinline__ int dir_stride_f(int l) {
    return l == 0 ? 1 : (l == 1 ? N : N * N);
}



// The reference constants of the split flux for a float32-mixed context.
inline Ref make_ref(const esdc_ctx* c) {
    const PhysF& ph = c->physf;
    Ref ref;
    ref.rho0 = ph.rho0;
    ref.p0 = ph.p0;
    ref.RT0 = ph.p0 / ph.rho0;
    ref.H0 = ph.gamma * ph.p0 / (ph.gamma - 1.0f);
    ref.gm1 = ph.gamma - 1.0f;
    ref.gamma = ph.gamma;
    ref.hrho0 = 0.5f * ph.rho0;
    ref.two_RT0 = 2.0f * ref.RT0;
    ref.c5 = ref.RT0 * ph.inv_gm1;
    ref.inv_rho0 = 1.0f / ph.rho0;
    ref.two_beta0 = ph.rho0 / ph.p0;
    ref.rho0d = 1.0;                                      // the float64 reference of the shadow state
    ref.E0d = c->phys.R / (c->phys.gamma - 1.0);
    ref.e0 = ref.RT0 * ph.inv_gm1;
    ref.inv_2gm1 = 0.5f * ph.inv_gm1;
    return ref;
}

}  // namespace f32
}  // namespace esdc
