// Float64 device functions shared by the residual kernels (rhs_f64.cu for p <= 7, rhs_large_f64.cu
// for p = 15): primitive variables, reciprocals, the Chandrashekar, Kennedy-Gruber and Euler fluxes
// contracted with a direction (Sec. 4), the face jump/average quantities and the matrix dissipation,
// and the line indexing of an element's tensor-product nodes.
#pragma once

#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "rcp_f64.cuh"

namespace esdc {
namespace {

// Per-node primitives in the form the pair loop consumes: half density and half velocity (so that
// averages are single additions), beta = rho/(2p) and a quarter of |u|^2.
struct Prim {
    double hr, hu0, hu1, hu2, beta, qq;
};


// Primitives of a conserved state, plus RT = p/rho and the sound speed c = sqrt(gamma p/rho).
__device__ __forceinline__ void to_prim(const double* q, const Phys& ph, Prim& s, double& RT, double& c) {
    const double ri = rcp_newton2(q[0]);
    const double u0 = q[1] * ri, u1 = q[2] * ri, u2 = q[3] * ri;
    const double usq = u0 * u0 + u1 * u1 + u2 * u2;
    const double p = (ph.gamma - 1.0) * (q[4] - 0.5 * q[0] * usq);
    s.hr = 0.5 * q[0];
    s.hu0 = 0.5 * u0;
    s.hu1 = 0.5 * u1;
    s.hu2 = 0.5 * u2;
    s.beta = s.hr * rcp_newton2(p);
    s.qq = 0.25 * usq;
    RT = p * ri;
    c = sqrt(ph.gamma * RT);
}

// u = ((a-b)/(a+b))^2 < 1e-4, tested on the high word (integer pipe): the threshold moves by less
// than 1e-6 relative, and both branches are accurate to float64 round-off around it.
__device__ __forceinline__ bool small_jump(double u) { return __double2hiint(u) < 0x3F1A36E2; }

// Chandrashekar two-point flux contracted with a direction vector n (Sec. 4):
// f1 = rho_ln ubar.n, f_m = f1 ubar + p_t n, f5 = f1 (1/(2(g-1) beta_ln) - avg|u|^2/2) + ubar.f_m,
// p_t = avg(rho)/(2 avg(beta)).  Log means by the artanh series in u = f^2, f = (a-b)/(a+b)
// (Ismail-Roe style): L = (a+b)/2 G(u), G = 1 - u/3 - 4u^2/45 - 44u^3/945, and
// 1/L = 2/(a+b) (1 + u/3 + u^2/5 + u^3/7) for u < 1e-4 (truncation below 1e-17), else the
// logarithmic form.  The flux is linear in n: the volume loop passes n_i + n_j (twice the averaged
// metric) and takes S, half of the pair coefficient 2S, instead.
__device__ __forceinline__ void ec_flux(const Prim& a, const Prim& b, double n0, double n1, double n2,
                                        const Phys& ph, double f[5]) {
    // density log mean from half densities: L = (hr_a + hr_b) G(u)
    const double sh = a.hr + b.hr;
    const double fr = (a.hr - b.hr) * rcp_newton1(sh);
    const double ur = fr * fr;
    double rho_ln;
    if (small_jump(ur)) rho_ln = sh * fma(ur, fma(ur, fma(ur, -44.0 / 945.0, -4.0 / 45.0), -1.0 / 3.0), 1.0);
    else rho_ln = 2.0 * (a.hr - b.hr) / log(a.hr / b.hr);
    // 1/beta_ln and p_t share 1/(beta_a + beta_b)
    const double rsb = rcp_newton2(a.beta + b.beta);
    const double fb = (a.beta - b.beta) * rsb;
    const double ub = fb * fb;
    double ibeta_ln;
    if (small_jump(ub)) ibeta_ln = rsb * fma(ub, fma(ub, fma(ub, 2.0 / 7.0, 2.0 / 5.0), 2.0 / 3.0), 2.0);
    else ibeta_ln = log(a.beta / b.beta) / (a.beta - b.beta);
    const double ub0 = a.hu0 + b.hu0, ub1 = a.hu1 + b.hu1, ub2 = a.hu2 + b.hu2;
    const double un = fma(ub2, n2, fma(ub1, n1, ub0 * n0));
    const double pt = sh * rsb;
    const double f1 = rho_ln * un;
    f[0] = f1;
    f[1] = fma(f1, ub0, pt * n0);
    f[2] = fma(f1, ub1, pt * n1);
    f[3] = fma(f1, ub2, pt * n2);
    const double c5 = fma(0.5 * ph.inv_gm1, ibeta_ln, -(a.qq + b.qq));
    f[4] = fma(ub2, f[3], fma(ub1, f[2], fma(ub0, f[1], f1 * c5)));
}

template <int N>
__device__ __forceinline__ int line_base(int l, int t1, int t2) {
    return l == 0 ? (t1 * N + t2 * N * N) : (l == 1 ? (t1 + t2 * N * N) : (t1 + t2 * N));
}

template <int N>
__device__ __forceinline__ int dir_stride(int l) {
    return l == 0 ? 1 : (l == 1 ? N : N * N);
}

__device__ __forceinline__ void load_prim(const double* sP, int N3, int idx, Prim& s) {
    s.hr = sP[idx];
    s.hu0 = sP[N3 + idx];
    s.hu1 = sP[2 * N3 + idx];
    s.hu2 = sP[3 * N3 + idx];
    s.beta = sP[4 * N3 + idx];
    s.qq = sP[5 * N3 + idx];
}

// Face quantities shared by the matrix dissipation and the interior penalty: the jump of the entropy
// variables w = ((gamma - s)/(gamma - 1) - beta |u|^2, 2 beta u, -2 beta) across the face (its
// logarithms taken as log(p_a/p_b) and log(rho_a/rho_b)), and dq/dw times that jump at the averaged
// state (rho_ln, ubar, p = rho_bar/(2 beta_bar)), from which a, H and rho E follow.
struct FaceAvg {
    double rho, u0, u1, u2, p, c2, H, E, ujw;
};

__device__ __forceinline__ void face_jump_avg(const Prim& a, double RTa, const Prim& b, double RTb, const Phys& ph,
                                              double jw[5], double r[5], FaceAvg& st) {
    const double ra = 2.0 * a.hr, rb = 2.0 * b.hr;
    const double pa = ra * RTa, pb = rb * RTb;
    const double ds = log(pa / pb) - ph.gamma * log(ra / rb);
    jw[0] = -ds * ph.inv_gm1 - 4.0 * (a.beta * a.qq - b.beta * b.qq);
    jw[1] = 4.0 * (a.beta * a.hu0 - b.beta * b.hu0);
    jw[2] = 4.0 * (a.beta * a.hu1 - b.beta * b.hu1);
    jw[3] = 4.0 * (a.beta * a.hu2 - b.beta * b.hu2);
    jw[4] = -2.0 * (a.beta - b.beta);
    const double sh = a.hr + b.hr;
    const double fr = (a.hr - b.hr) * rcp_newton1(sh);
    const double ur = fr * fr;
    if (small_jump(ur)) st.rho = sh * fma(ur, fma(ur, fma(ur, -44.0 / 945.0, -4.0 / 45.0), -1.0 / 3.0), 1.0);
    else st.rho = 2.0 * (a.hr - b.hr) / log(a.hr / b.hr);
    st.p = sh * rcp_newton2(a.beta + b.beta);
    st.u0 = a.hu0 + b.hu0;
    st.u1 = a.hu1 + b.hu1;
    st.u2 = a.hu2 + b.hu2;
    const double usq = st.u0 * st.u0 + st.u1 * st.u1 + st.u2 * st.u2;
    st.c2 = ph.gamma * st.p / st.rho;
    st.H = fma(st.c2, ph.inv_gm1, 0.5 * usq);
    st.E = fma(st.p, ph.inv_gm1, 0.5 * st.rho * usq);
    // dq/dw jw
    const double m0 = st.rho * st.u0, m1 = st.rho * st.u1, m2 = st.rho * st.u2;
    st.ujw = st.u0 * jw[1] + st.u1 * jw[2] + st.u2 * jw[3];
    const double t = jw[0] + st.ujw + st.H * jw[4];
    r[0] = st.rho * jw[0] + m0 * jw[1] + m1 * jw[2] + m2 * jw[3] + st.E * jw[4];
    r[1] = fma(m0, t, st.p * jw[1]);
    r[2] = fma(m1, t, st.p * jw[2]);
    r[3] = fma(m2, t, st.p * jw[3]);
    r[4] = st.E * jw[0] + st.rho * st.H * st.ujw + (st.rho * st.H * st.H - st.c2 * st.p * ph.inv_gm1) * jw[4];
}

// Roe-type entropy-stable interface dissipation D (w_a - w_b) (the matrix alternative to local
// Lax-Friedrichs).  D = R |Lambda| R^T in the direction n at the averaged state, with R the
// eigenvectors of the flux Jacobian scaled so that R R^T = dq/dw.  The three eigenvalues u.n share an
// eigenspace, so D = |u.n| dq/dw + s (|u.n - a|n|| - |u.n|) r1 r1^T + s (|u.n + a|n|| - |u.n|) r5 r5^T,
// r1,5 = (1, u -+ a nhat, H -+ a u.nhat), s = rho/(2 gamma).  r = dq/dw jw from face_jump_avg.
__device__ __forceinline__ void matrix_dissipation(const FaceAvg& st, const double jw[5], const double r[5],
                                                   double n0, double n1, double n2, const Phys& ph, double dm[5]) {
    const double c = sqrt(st.c2);
    const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const double inn = 1.0 / nn;
    const double un = st.u0 * n0 + st.u1 * n1 + st.u2 * n2;
    const double unh = un * inn;
    const double l2 = fabs(un), l1 = fabs(un - c * nn), l5 = fabs(un + c * nn);
    const double cn0 = c * n0 * inn, cn1 = c * n1 * inn, cn2 = c * n2 * inn;
    const double njw = cn0 * jw[1] + cn1 * jw[2] + cn2 * jw[3];
    const double c1 = jw[0] + st.ujw - njw + (st.H - c * unh) * jw[4];
    const double c5 = jw[0] + st.ujw + njw + (st.H + c * unh) * jw[4];
    const double sc = st.rho / (2.0 * ph.gamma);
    const double k1 = sc * (l1 - l2) * c1, k5 = sc * (l5 - l2) * c5;
    dm[0] = l2 * r[0] + k1 + k5;
    dm[1] = l2 * r[1] + k1 * (st.u0 - cn0) + k5 * (st.u0 + cn0);
    dm[2] = l2 * r[2] + k1 * (st.u1 - cn1) + k5 * (st.u1 + cn1);
    dm[3] = l2 * r[3] + k1 * (st.u2 - cn2) + k5 * (st.u2 + cn2);
    dm[4] = l2 * r[4] + k1 * (st.H - c * unh) + k5 * (st.H + c * unh);
}

// Volume-flux variants of the kernel (the paper's comparison, Sec. 4): the entropy-stable
// Chandrashekar flux (ES-C), the Kennedy-Gruber split form (SF-KG) and standard collocation (DC).
enum : int { kFluxESC = 0, kFluxKG = 1, kFluxDC = 2 };

// Kennedy-Gruber two-point flux contracted with n: f1 = rho_bar ubar.n, f_m = f1 ubar_m + p_bar n_m,
// f5 = f1 e_bar + p_bar ubar.n with arithmetic means of rho, u, p = rho RT and the specific total
// energy e = RT/(gamma-1) + |u|^2/2 (halved primitives: rho_bar = hr_a + hr_b, ubar = hu_a + hu_b).
__device__ __forceinline__ void kg_flux(const Prim& a, const Prim& b, double RTa, double RTb, double n0, double n1,
                                        double n2, const Phys& ph, double f[5]) {
    const double rb = a.hr + b.hr;
    const double ub0 = a.hu0 + b.hu0, ub1 = a.hu1 + b.hu1, ub2 = a.hu2 + b.hu2;
    const double pb = fma(a.hr, RTa, b.hr * RTb);
    const double eb = fma(0.5 * ph.inv_gm1, RTa + RTb, a.qq + b.qq);
    const double un = fma(ub2, n2, fma(ub1, n1, ub0 * n0));
    const double f1 = rb * un;
    f[0] = f1;
    f[1] = fma(f1, ub0, pb * n0);
    f[2] = fma(f1, ub1, pb * n1);
    f[3] = fma(f1, ub2, pb * n2);
    f[4] = fma(f1, eb, pb * un);
}

// Euler flux of one state contracted with n, from the halved primitives and RT = p/rho:
// f1 = rho u.n, f_m = f1 u_m + p n_m, f5 = f1 H with H = gamma/(gamma-1) RT + |u|^2/2.
__device__ __forceinline__ void euler_flux_prim(const Prim& s, double RT, double n0, double n1, double n2,
                                                const Phys& ph, double f[5]) {
    const double rho = 2.0 * s.hr;
    const double u0 = 2.0 * s.hu0, u1 = 2.0 * s.hu1, u2 = 2.0 * s.hu2;
    const double p = rho * RT;
    const double un = fma(u2, n2, fma(u1, n1, u0 * n0));
    const double f1 = rho * un;
    f[0] = f1;
    f[1] = fma(f1, u0, p * n0);
    f[2] = fma(f1, u1, p * n1);
    f[3] = fma(f1, u2, p * n2);
    f[4] = f1 * fma(ph.gamma * ph.inv_gm1, RT, 2.0 * s.qq);
}

}  // namespace
}  // namespace esdc
