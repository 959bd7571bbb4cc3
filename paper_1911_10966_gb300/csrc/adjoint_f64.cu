// Vector-Jacobian product of the float64 residual: grad = (dR/dq)^T lambda and
// grad_mu = lambda . dR/dmu, for R = dq/dt of rhs_f64.cu (same discretization, same readings).
//
// The forward residual is a sum of terms, each local to one element except the face couplings:
//   volume   r_i -= 2 S_ij f(q_i,q_j)/w_i, r_j += 2 S_ij f(q_i,q_j)/w_j     (pairs on xi_l lines)
//   inviscid r_o += (-E f(q_o,q_n) - lam/2 (q_o - q_n))/w_end               (face nodes)
//   viscous  r += sum_l D_l Ft_l + (E/2)(Ft_l,nbr - Ft_l,own)/w_end, Ft built from theta_a =
//            D_a w + (E/2)(w_nbr - w_own)/w_end
//   dq/dt = r / J.
// With lt = lambda / J the transposes are: pair cotangent mu = 2 S_ij (lt_j/w_j - lt_i/w_i) pulled
// back through the two-point flux to both nodes; the interface cotangent lt_o/w_end pulled back to
// the own node and (through the face buffer gbuf) to the neighbour; the viscous chain reversed
// node by node with the transposed derivative D_l^T along lines, the lifted-gradient cotangent on
// faces written to tbuf for the neighbour.  Kernel adj_main does everything inside an element,
// kernel adj_face adds what the neighbours wrote for this element's face nodes.
// On a bounded box a boundary face (neighbour -1) takes the exterior state q_ext, which does not
// depend on q, as its neighbour: the interface cotangent stays with the own node, the lift keeps its
// own part, and the viscous interface term, zero on such faces, has no transpose.
// Non-smooth points follow the convention of reverse-mode differentiation: d|x| = sign(x) with
// sign(0) = 0, and max(a, b) splits its cotangent in half at a tie.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"
#include "rcp_f64.cuh"

namespace esdc {
namespace {

constexpr int kAdjRed = 256;

// Float64 reciprocal square root by Newton-Raphson on g(y) = 1/y^2 - x from the hardware
// approximation (about 23 bits): each step y <- y (3/2 - x y^2/2) doubles the number of correct bits.
__device__ __forceinline__ double rsqrt_newton2(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}

template <int N>
struct CfgA {
    static constexpr int N2 = N * N, N3 = N * N * N;
    // (two elements per CTA at N = 5, one CTA of 250 threads per SM, made the VJP 8.5% slower on
    // 16^3 elements and 17% faster on 8^3: fewer warps per SM against fuller ones and fewer waves)
    static constexpr int EPB = N3 >= 96 ? 1 : (N3 >= 48 ? 2 : (N3 >= 24 ? 4 : 16));
    static constexpr int THREADS = EPB * N3;
    // shared doubles per element: prim/w and the pair form 14 | lt 5 | geometry 10 | prim-bar 6 | q-bar 5
    // | theta-bar 12
    // (also the own side's interface cotangents, 30 N2, which exceed 12 N3 only at N = 2)
    // | neighbour face w 24 N2
    static constexpr int TSZ = 12 * N3 > 30 * N2 ? 12 * N3 : 30 * N2;
    static constexpr int SM = 40 * N3 + TSZ + 24 * N2;
    // resident CTAs the register allocation is sized for (3 at N = 4, 5 measured faster than 2)
    static constexpr int MINB = (N == 4 || N == 5) ? 3 : 1;
};

struct Prim {
    double rho, u0, u1, u2, beta, usq;
};
struct PBar {   // cotangents of (rho, u0, u1, u2, beta, usq)
    double rho, u0, u1, u2, beta, usq;
};

__device__ __forceinline__ void to_prim(const double* q, const Phys& ph, Prim& s) {
    const double ri = rcp_newton2(q[0]);
    s.rho = q[0];
    s.u0 = q[1] * ri;
    s.u1 = q[2] * ri;
    s.u2 = q[3] * ri;
    s.usq = s.u0 * s.u0 + s.u1 * s.u1 + s.u2 * s.u2;
    const double p = (ph.gamma - 1.0) * (q[4] - 0.5 * q[0] * s.usq);
    s.beta = 0.5 * q[0] * rcp_newton2(p);
}

// pull a primitive cotangent back to the conserved variables at state s
__device__ __forceinline__ void pbar_to_q(const Prim& s, const PBar& b, const Phys& ph, double qb[5]) {
    const double gm1 = ph.gamma - 1.0;
    const double ut0 = b.u0 + 2.0 * s.u0 * b.usq, ut1 = b.u1 + 2.0 * s.u1 * b.usq, ut2 = b.u2 + 2.0 * s.u2 * b.usq;
    const double ri = rcp_newton2(s.rho);
    // beta = rho/(2p): d beta = beta/rho d rho - beta/p d p, and beta/p = 2 beta^2/rho
    const double pb = -b.beta * 2.0 * s.beta * s.beta * ri;
    qb[0] = b.rho + b.beta * s.beta * ri + pb * gm1 * 0.5 * s.usq - (ut0 * s.u0 + ut1 * s.u1 + ut2 * s.u2) * ri;
    qb[1] = ut0 * ri - pb * gm1 * s.u0;
    qb[2] = ut1 * ri - pb * gm1 * s.u1;
    qb[3] = ut2 * ri - pb * gm1 * s.u2;
    qb[4] = pb * gm1;
}

// Logarithmic mean, its partial derivatives and its reciprocal, given rs = 1/(a+b).  Series branch
// (u = ((a-b)/(a+b))^2 < 1e-4): with F(u) = artanh(f)/f = 1 + u/3 + u^2/5 + u^3/7 + u^4/9 and
// G = 1/F = 1 - u/3 - 4u^2/45 - 44u^3/945, L = (a+b) G/2, 1/L = 2 F/(a+b) and
// dL/da = G/2 - 2 f b F'(u) G^2/(a+b), dL/db = G/2 + 2 f a F'(u) G^2/(a+b); otherwise L = (a-b)/l,
// l = log(a/b), dL/da = (1 - L/a)/l, dL/db = (L/b - 1)/l.
__device__ __forceinline__ void ln_mean_d(double a, double b, double rs, double& L, double& La, double& Lb,
                                          double& IL) {
    const double d = a - b, s = a + b;
    const double f = d * rs;
    const double u = f * f;
    if (u < 1.0e-4) {
        const double G = fma(u, fma(u, fma(u, -44.0 / 945.0, -4.0 / 45.0), -1.0 / 3.0), 1.0);
        const double Fp = fma(u, fma(u, fma(u, 4.0 / 9.0, 3.0 / 7.0), 2.0 / 5.0), 1.0 / 3.0);
        const double F = fma(u, fma(u, fma(u, fma(u, 1.0 / 9.0, 1.0 / 7.0), 1.0 / 5.0), 1.0 / 3.0), 1.0);
        L = 0.5 * s * G;
        const double t = 2.0 * f * Fp * G * G * rs;
        La = fma(-t, b, 0.5 * G);
        Lb = fma(t, a, 0.5 * G);
        IL = 2.0 * F * rs;
    } else {
        const double l = log(a / b);
        L = d / l;
        La = (1.0 - L / a) / l;
        Lb = (L / b - 1.0) / l;
        IL = l / d;
    }
}

// Pair form of a node's primitives for the ES-C reverse: half velocities and a quarter of |u|^2, so
// that the averages of the two-point flux are single additions.
struct PrimH {
    double rho, h0, h1, h2, beta, qsq;
};
// Cotangent accumulators of the ES-C reverse in pair form: rho and beta as in PBar, u twice the
// velocity cotangent, c the sum of the cotangents of c5 (the |u|^2 cotangent is -c/4); raw_to_pbar
// converts.
struct PRaw {
    double rho, u0, u1, u2, beta, c;
};

__device__ __forceinline__ void raw_to_pbar(const PRaw& r, PBar& b) {
    b.rho += r.rho;
    b.u0 += 0.5 * r.u0;
    b.u1 += 0.5 * r.u1;
    b.u2 += 0.5 * r.u2;
    b.beta += r.beta;
    b.usq += -0.25 * r.c;
}

// Reverse of the contracted Chandrashekar flux f(a, b; n) for the cotangent mu[5]: adds the pair-form
// cotangents of both states to ab, bb.  Two reciprocals, 1/(rho_a + rho_b) (one Newton step: it only
// forms f = (a - b)/(a + b)) and 1/(beta_a + beta_b), which serves p_t and the reciprocal of the beta
// log mean.  Logarithmic means (series branch, u = f^2 < 1e-4, F(u) = artanh(f)/f = 1 + u/3 + u^2/5 +
// u^3/7 + u^4/9, G = 1/F = 1 - u/3 - 4u^2/45 - 44u^3/945):
//   rho:  L = (a + b) G/2,  dL/da = G/2 - f F'(u) G^2 (1 - f),  dL/db = G/2 + f F'(u) G^2 (1 + f);
//   beta: only 1/L enters the flux, IL = 2 F/(a + b), dIL/da = 2 (2 f F'(u) (1 - f) - F)/(a + b)^2,
//         dIL/db = -2 (2 f F'(u) (1 + f) + F)/(a + b)^2;
// otherwise, with l = log(a/b): L = (a - b)/l, dL/da = (1 - L/a)/l, dL/db = (L/b - 1)/l, and
// IL = l/(a - b), dIL/da = (1/a - IL)/(a - b), dIL/db = (IL - 1/b)/(a - b).
__device__ __forceinline__ void ec_pair_vjp(const PrimH& a, const PrimH& b, double n0, double n1, double n2,
                                            const double mu[5], const Phys& ph, PRaw& ab, PRaw& bb) {
    const double sr = a.rho + b.rho, sb = a.beta + b.beta;
    const double rsb = rcp_newton2(sb);
    // rho log mean and its partial derivatives
    double Lr, Lra, Lrb;
    {
        const double d = a.rho - b.rho;
        const double f = d * rcp_newton1(sr);
        const double u = f * f;
        if (u < 1.0e-4) {
            const double hG = fma(u, fma(u, fma(u, -22.0 / 945.0, -2.0 / 45.0), -1.0 / 6.0), 0.5);          // G/2
            const double Fp4 = fma(u, fma(u, fma(u, 16.0 / 9.0, 12.0 / 7.0), 8.0 / 5.0), 4.0 / 3.0);     // 4 F'
            const double W = f * Fp4 * (hG * hG);                                                          // f F' G^2
            const double Y = W * f;
            Lr = sr * hG;
            Lra = hG - W + Y;
            Lrb = hG + W + Y;
        } else {
            const double ra = rcp_newton2(a.rho), rb = rcp_newton2(b.rho);
            const double rl = rcp_newton2(log(a.rho * rb));
            Lr = d * rl;
            Lra = fma(-Lr, ra, 1.0) * rl;
            Lrb = fma(Lr, rb, -1.0) * rl;
        }
    }
    // reciprocal of the beta log mean and its partial derivatives: dIL/da = sc Ab, dIL/db = sc Bb
    double IB, sc, Ab, Bb;
    {
        const double d = a.beta - b.beta;
        const double f = d * rsb;
        const double u = f * f;
        if (u < 1.0e-4) {
            const double F = fma(u, fma(u, fma(u, fma(u, 1.0 / 9.0, 1.0 / 7.0), 1.0 / 5.0), 1.0 / 3.0), 1.0);
            const double Fp2 = fma(u, fma(u, fma(u, 8.0 / 9.0, 6.0 / 7.0), 4.0 / 5.0), 2.0 / 3.0);      // 2 F'
            const double w = f * Fp2;
            const double X = w * f;
            IB = 2.0 * F * rsb;
            sc = 2.0 * rsb * rsb;
            Ab = w - X - F;
            Bb = -(w + X + F);
        } else {
            const double ra = rcp_newton2(a.beta), rb = rcp_newton2(b.beta);
            sc = rcp_newton2(d);
            IB = log(a.beta * rb) * sc;
            Ab = ra - IB;
            Bb = IB - rb;
        }
    }
    const double hig = 0.5 * ph.inv_gm1;
    const double ub0 = a.h0 + b.h0, ub1 = a.h1 + b.h1, ub2 = a.h2 + b.h2;
    const double un = ub0 * n0 + ub1 * n1 + ub2 * n2;
    const double pt = 0.5 * sr * rsb;
    const double f1 = Lr * un;
    const double c5 = fma(hig, IB, -(a.qsq + b.qsq));
    // reverse
    const double fmb0 = fma(mu[4], ub0, mu[1]), fmb1 = fma(mu[4], ub1, mu[2]), fmb2 = fma(mu[4], ub2, mu[3]);
    const double f1b = mu[0] + mu[4] * c5 + fmb0 * ub0 + fmb1 * ub1 + fmb2 * ub2;
    const double c5b = mu[4] * f1;
    const double ptb = fmb0 * n0 + fmb1 * n1 + fmb2 * n2;
    const double unb = f1b * Lr;
    const double Lrb_ = f1b * un;
    // pt = (rho_a + rho_b)/(2 (beta_a + beta_b)): d pt/d rho = 1/(2 sb), d pt/d beta = -pt/sb
    const double ptr = ptb * rsb;
    const double hp = 0.5 * ptr;
    const double bp = -pt * ptr;
    const double S = c5b * hig * sc;
    ab.rho += fma(Lrb_, Lra, hp);
    bb.rho += fma(Lrb_, Lrb, hp);
    ab.beta += fma(S, Ab, bp);
    bb.beta += fma(S, Bb, bp);
    ab.c += c5b;
    bb.c += c5b;
    // ubar cotangent mu_5 f_m + fmb f1 + unb n with f_m = f1 ubar + p_t n:
    // f1 (mu_5 ubar + fmb) + (mu_5 p_t + unb) n
    const double An = fma(mu[4], pt, unb);
    const double ubb0 = fma(f1, fma(mu[4], ub0, fmb0), An * n0);
    const double ubb1 = fma(f1, fma(mu[4], ub1, fmb1), An * n1);
    const double ubb2 = fma(f1, fma(mu[4], ub2, fmb2), An * n2);
    ab.u0 += ubb0;
    ab.u1 += ubb1;
    ab.u2 += ubb2;
    bb.u0 += ubb0;
    bb.u1 += ubb1;
    bb.u2 += ubb2;
}

__device__ __forceinline__ PrimH to_pair_form(const Prim& s) {
    return PrimH{s.rho, 0.5 * s.u0, 0.5 * s.u1, 0.5 * s.u2, s.beta, 0.25 * s.usq};
}

// The same reverse for full-form states and cotangents (the interface terms).
__device__ __forceinline__ void ec_flux_vjp(const Prim& a, const Prim& b, double n0, double n1, double n2,
                                            const double mu[5], const Phys& ph, PBar& ab, PBar& bb) {
    PRaw ra{0, 0, 0, 0, 0, 0}, rb{0, 0, 0, 0, 0, 0};
    ec_pair_vjp(to_pair_form(a), to_pair_form(b), n0, n1, n2, mu, ph, ra, rb);
    raw_to_pbar(ra, ab);
    raw_to_pbar(rb, bb);
}

// Reverse of the contracted Kennedy-Gruber flux (the SF-KG variant): with arithmetic means
// rho_bar, u_bar, p_bar = (p_a + p_b)/2 (p = rho RT, RT = 1/(2 beta)) and e_bar = (RT_a + RT_b)/
// (2 (gamma-1)) + (|u_a|^2 + |u_b|^2)/4, f1 = rho_bar u_bar.n, f_m = f1 u_bar_m + p_bar n_m,
// f5 = f1 e_bar + p_bar u_bar.n.  Adds the primitive cotangents of both states to ab, bb.
__device__ __forceinline__ void kg_flux_vjp(const Prim& a, const Prim& b, double n0, double n1, double n2,
                                            const double mu[5], const Phys& ph, PBar& ab, PBar& bb) {
    const double RTa = 0.5 * rcp_newton2(a.beta), RTb = 0.5 * rcp_newton2(b.beta);
    const double rb = 0.5 * (a.rho + b.rho);
    const double ub0 = 0.5 * (a.u0 + b.u0), ub1 = 0.5 * (a.u1 + b.u1), ub2 = 0.5 * (a.u2 + b.u2);
    const double pb = 0.5 * (a.rho * RTa + b.rho * RTb);
    const double eb = 0.5 * ph.inv_gm1 * (RTa + RTb) + 0.25 * (a.usq + b.usq);
    const double un = ub0 * n0 + ub1 * n1 + ub2 * n2;
    const double f1 = rb * un;
    // reverse
    const double f1b = mu[0] + mu[1] * ub0 + mu[2] * ub1 + mu[3] * ub2 + mu[4] * eb;
    const double pbb = mu[1] * n0 + mu[2] * n1 + mu[3] * n2 + mu[4] * un;
    const double ebb = mu[4] * f1;
    const double unb = mu[4] * pb + f1b * rb;
    const double rbb = f1b * un;
    const double ubb0 = mu[1] * f1 + unb * n0, ubb1 = mu[2] * f1 + unb * n1, ubb2 = mu[3] * f1 + unb * n2;
    const double RTab = 0.5 * pbb * a.rho + 0.5 * ph.inv_gm1 * ebb;
    const double RTbb = 0.5 * pbb * b.rho + 0.5 * ph.inv_gm1 * ebb;
    ab.rho += 0.5 * rbb + 0.5 * pbb * RTa;
    bb.rho += 0.5 * rbb + 0.5 * pbb * RTb;
    ab.u0 += 0.5 * ubb0;
    ab.u1 += 0.5 * ubb1;
    ab.u2 += 0.5 * ubb2;
    bb.u0 += 0.5 * ubb0;
    bb.u1 += 0.5 * ubb1;
    bb.u2 += 0.5 * ubb2;
    ab.usq += 0.25 * ebb;
    bb.usq += 0.25 * ebb;
    ab.beta += RTab * (-2.0 * RTa * RTa);      // dRT/dbeta = -1/(2 beta^2) = -2 RT^2
    bb.beta += RTbb * (-2.0 * RTb * RTb);
}

// Reverse of the Euler flux of one state contracted with n (the DC variant differentiates nodal
// fluxes): f1 = rho u.n, f_m = rho u_m u.n + p n_m, f5 = rho u.n H, with p = rho RT, RT = 1/(2 beta)
// and H = gamma/(gamma-1) RT + |u|^2/2.  Adds the primitive cotangents of the state to sb.
__device__ __forceinline__ void euler_flux_vjp(const Prim& s, double n0, double n1, double n2, const double mu[5],
                                               const Phys& ph, PBar& sb) {
    const double RT = 0.5 * rcp_newton2(s.beta);
    const double un = s.u0 * n0 + s.u1 * n1 + s.u2 * n2;
    const double H = ph.gamma * ph.inv_gm1 * RT + 0.5 * s.usq;
    const double A = s.rho * un;                                   // mass flux
    const double Ab = mu[0] + mu[1] * s.u0 + mu[2] * s.u1 + mu[3] * s.u2 + mu[4] * H;
    const double pb = mu[1] * n0 + mu[2] * n1 + mu[3] * n2;
    const double Hb = mu[4] * A;
    const double unb = Ab * s.rho;
    const double RTb = Hb * ph.gamma * ph.inv_gm1 + pb * s.rho;
    sb.rho += Ab * un + pb * RT;
    sb.u0 += mu[1] * A + unb * n0;
    sb.u1 += mu[2] * A + unb * n1;
    sb.u2 += mu[3] * A + unb * n2;
    sb.usq += 0.5 * Hb;
    sb.beta += RTb * (-2.0 * RT * RT);         // dRT/dbeta = -2 RT^2
}

// volume-flux variants of the adjoint kernel (the values of ESDC_FLUX_ESC, _KG and _DC)
enum : int { kAdjESC = 0, kAdjKG = 1, kAdjDC = 2 };

template <int VF>
__device__ __forceinline__ void flux_vjp(const Prim& a, const Prim& b, double n0, double n1, double n2,
                                         const double mu[5], const Phys& ph, PBar& ab, PBar& bb) {
    if constexpr (VF == kAdjKG) {
        kg_flux_vjp(a, b, n0, n1, n2, mu, ph, ab, bb);
    } else if constexpr (VF == kAdjDC) {
        // central interface flux (f(a) + f(b))/2
        double h[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) h[v] = 0.5 * mu[v];
        euler_flux_vjp(a, n0, n1, n2, h, ph, ab);
        euler_flux_vjp(b, n0, n1, n2, h, ph, bb);
    } else {
        ec_flux_vjp(a, b, n0, n1, n2, mu, ph, ab, bb);
    }
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
    s.rho = sP[idx];
    s.u0 = sP[N3 + idx];
    s.u1 = sP[2 * N3 + idx];
    s.u2 = sP[3 * N3 + idx];
    s.beta = sP[4 * N3 + idx];
    s.usq = sP[5 * N3 + idx];
}

// the pair form (half velocities, |u|^2/4) kept at rows 10..13 of the primitive array
__device__ __forceinline__ PrimH load_pair_form(const double* sP, int N3, int idx) {
    return PrimH{sP[idx], sP[10 * N3 + idx], sP[11 * N3 + idx], sP[12 * N3 + idx], sP[4 * N3 + idx],
                 sP[13 * N3 + idx]};
}

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// Reverse of the interface terms built on the face-averaged state: the matrix dissipation
// (1/2) D (w_own - w_nbr) (D = R |Lambda| R^T in the direction n, split into |u.n| dq/dw and the two
// acoustic rank-one parts) and the interior penalty cip dq/dw (w_own - w_nbr).  The forward quantities
// are recomputed: the entropy-variable jump jw (with s = log p - gamma log rho), the averaged state
// (rho_ln, ubar, p = avg(rho)/(2 avg(beta)), c^2 = gamma p/rho_ln, H, rho E) and r = dq/dw jw.  dmb
// is the cotangent of the sum of the two terms; the primitive cotangents of both states are added
// to ab, bb.  Returns dmb . (interior-penalty term), the term's share of lambda . R (linear in mu).
// Kept out of line: only contexts with these options call it.
__device__ __noinline__ double face_avg_vjp(const Prim& a, const Prim& b, double n0, double n1, double n2,
                                            const Phys& ph, bool matrix, double cip, const double dmb[5], PBar& ab,
                                            PBar& bb) {
    const double g = ph.gamma, igm1 = ph.inv_gm1;
    const double ua[3] = {a.u0, a.u1, a.u2}, uv[3] = {b.u0, b.u1, b.u2};
    const double nv[3] = {n0, n1, n2};
    // ---- forward
    const double ds = log((a.rho / a.beta) / (b.rho / b.beta)) - g * log(a.rho / b.rho);
    double jw[5];
    jw[0] = -ds * igm1 - (a.beta * a.usq - b.beta * b.usq);
    for (int k = 0; k < 3; ++k) jw[1 + k] = 2.0 * (a.beta * ua[k] - b.beta * uv[k]);
    jw[4] = -2.0 * (a.beta - b.beta);
    double L, La, Lb;
    double IL;
    ln_mean_d(a.rho, b.rho, 1.0 / (a.rho + b.rho), L, La, Lb, IL);
    const double sb = a.beta + b.beta;
    const double p = 0.5 * (a.rho + b.rho) / sb;
    double u[3], m[3];
    for (int k = 0; k < 3; ++k) u[k] = 0.5 * (ua[k] + uv[k]);
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double c2 = g * p / L;
    const double H = c2 * igm1 + 0.5 * usq;
    const double E = p * igm1 + 0.5 * L * usq;
    for (int k = 0; k < 3; ++k) m[k] = L * u[k];
    const double ujw = u[0] * jw[1] + u[1] * jw[2] + u[2] * jw[3];
    const double t = jw[0] + ujw + H * jw[4];
    double r[5];
    r[0] = L * jw[0] + m[0] * jw[1] + m[1] * jw[2] + m[2] * jw[3] + E * jw[4];
    for (int k = 0; k < 3; ++k) r[1 + k] = m[k] * t + p * jw[1 + k];
    r[4] = E * jw[0] + L * H * ujw + (L * H * H - c2 * p * igm1) * jw[4];
    // ---- reverse
    double rb[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, jb[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, ubar[3] = {0.0, 0.0, 0.0};
    double Lbar = 0.0, Hb = 0.0, c2b = 0.0, pb = 0.0, ujwb = 0.0;
    double ip_dot = 0.0;
    if (cip != 0.0) {
        for (int v = 0; v < 5; ++v) {
            rb[v] += cip * dmb[v];
            ip_dot += dmb[v] * cip * r[v];
        }
    }
    if (matrix) {
        double D[5];
        for (int v = 0; v < 5; ++v) D[v] = 0.5 * dmb[v];
        const double c = sqrt(c2);
        const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        const double inn = 1.0 / nn;
        const double un = u[0] * n0 + u[1] * n1 + u[2] * n2;
        const double unh = un * inn;
        const double e1 = un - c * nn, e5 = un + c * nn;
        const double l2 = fabs(un), l1 = fabs(e1), l5 = fabs(e5);
        double cn[3];
        for (int k = 0; k < 3; ++k) cn[k] = c * nv[k] * inn;
        const double njw = cn[0] * jw[1] + cn[1] * jw[2] + cn[2] * jw[3];
        const double cu = c * unh;
        const double c1 = jw[0] + ujw - njw + (H - cu) * jw[4];
        const double c5 = jw[0] + ujw + njw + (H + cu) * jw[4];
        const double sc = L / (2.0 * g);
        const double k1 = sc * (l1 - l2) * c1, k5 = sc * (l5 - l2) * c5;
        // dm = l2 r + k1 (1, u - cn, H - cu) + k5 (1, u + cn, H + cu)
        double l2b = 0.0;
        for (int v = 0; v < 5; ++v) {
            l2b += D[v] * r[v];
            rb[v] += l2 * D[v];
        }
        double k1b = D[0] + D[4] * (H - cu), k5b = D[0] + D[4] * (H + cu);
        double cnb[3];
        for (int k = 0; k < 3; ++k) {
            k1b += D[1 + k] * (u[k] - cn[k]);
            k5b += D[1 + k] * (u[k] + cn[k]);
            ubar[k] += (k1 + k5) * D[1 + k];
            cnb[k] = (k5 - k1) * D[1 + k];
        }
        Hb += (k1 + k5) * D[4];
        double cub = (k5 - k1) * D[4];
        const double scb = k1b * (l1 - l2) * c1 + k5b * (l5 - l2) * c5;
        const double l1b = k1b * sc * c1, l5b = k5b * sc * c5;
        l2b -= k1b * sc * c1 + k5b * sc * c5;
        const double c1b = k1b * sc * (l1 - l2), c5b = k5b * sc * (l5 - l2);
        jb[0] += c1b + c5b;
        ujwb += c1b + c5b;
        const double njwb = c5b - c1b;
        Hb += (c1b + c5b) * jw[4];
        cub += (c5b - c1b) * jw[4];
        jb[4] += c1b * (H - cu) + c5b * (H + cu);
        for (int k = 0; k < 3; ++k) {
            cnb[k] += njwb * jw[1 + k];
            jb[1 + k] += njwb * cn[k];
        }
        Lbar += scb / (2.0 * g);
        double cb = cub * unh;
        for (int k = 0; k < 3; ++k) cb += cnb[k] * nv[k] * inn;
        const double unb = l2b * sgn(un) + l1b * sgn(e1) + l5b * sgn(e5) + cub * c * inn;
        cb += (l5b * sgn(e5) - l1b * sgn(e1)) * nn;
        for (int k = 0; k < 3; ++k) ubar[k] += unb * nv[k];
        c2b += cb / (2.0 * c);
    }
    // r = dq/dw jw at the averaged state
    const double Eb = rb[4] * jw[0] + rb[0] * jw[4];
    jb[0] += rb[4] * E + rb[0] * L;
    Lbar += rb[4] * (H * ujw + H * H * jw[4]) + rb[0] * jw[0];
    Hb += rb[4] * (L * ujw + 2.0 * L * H * jw[4]);
    ujwb += rb[4] * L * H;
    c2b -= rb[4] * p * jw[4] * igm1;
    pb -= rb[4] * c2 * jw[4] * igm1;
    jb[4] += rb[4] * (L * H * H - c2 * p * igm1) + rb[0] * E;
    double tb = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double mb = rb[1 + k] * t + rb[0] * jw[1 + k];
        tb += rb[1 + k] * m[k];
        pb += rb[1 + k] * jw[1 + k];
        jb[1 + k] += rb[1 + k] * p + rb[0] * m[k];
        Lbar += mb * u[k];
        ubar[k] += mb * L;
    }
    jb[0] += tb;
    ujwb += tb;
    Hb += tb * jw[4];
    jb[4] += tb * H;
    for (int k = 0; k < 3; ++k) {
        ubar[k] += ujwb * jw[1 + k];
        jb[1 + k] += ujwb * u[k];
    }
    pb += Eb * igm1;
    Lbar += 0.5 * Eb * usq;
    double usqb = 0.5 * Eb * L;
    c2b += Hb * igm1;
    usqb += 0.5 * Hb;
    pb += c2b * g / L;
    Lbar -= c2b * c2 / L;
    for (int k = 0; k < 3; ++k) ubar[k] += 2.0 * usqb * u[k];
    // back to the two states
    ab.u0 += 0.5 * ubar[0];
    ab.u1 += 0.5 * ubar[1];
    ab.u2 += 0.5 * ubar[2];
    bb.u0 += 0.5 * ubar[0];
    bb.u1 += 0.5 * ubar[1];
    bb.u2 += 0.5 * ubar[2];
    ab.rho += pb * 0.5 / sb + Lbar * La;
    bb.rho += pb * 0.5 / sb + Lbar * Lb;
    ab.beta -= pb * p / sb + 2.0 * jb[4];
    bb.beta += -pb * p / sb + 2.0 * jb[4];
    double aub[3] = {0.0, 0.0, 0.0}, bub[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        ab.beta += 2.0 * jb[1 + k] * ua[k];
        aub[k] = 2.0 * jb[1 + k] * a.beta;
        bb.beta -= 2.0 * jb[1 + k] * uv[k];
        bub[k] = -2.0 * jb[1 + k] * b.beta;
    }
    ab.u0 += aub[0];
    ab.u1 += aub[1];
    ab.u2 += aub[2];
    bb.u0 += bub[0];
    bb.u1 += bub[1];
    bb.u2 += bub[2];
    // jw0 = -ds/(gamma-1) - (beta_a |u_a|^2 - beta_b |u_b|^2), ds = (1-gamma) log(rho_a/rho_b) - log(beta_a/beta_b)
    const double dsb = -jb[0] * igm1;
    ab.beta -= jb[0] * a.usq;
    ab.usq -= jb[0] * a.beta;
    bb.beta += jb[0] * b.usq;
    bb.usq += jb[0] * b.beta;
    ab.rho += dsb * (1.0 - g) / a.rho;
    bb.rho -= dsb * (1.0 - g) / b.rho;
    ab.beta -= dsb / a.beta;
    bb.beta += dsb / b.beta;
    return ip_dot;
}

template <int N, int VF>
__global__ void __launch_bounds__(CfgA<N>::THREADS, CfgA<N>::MINB)
adj_main(const double* __restrict__ q, const double* __restrict__ lam, const double* __restrict__ geom,
         const int32_t* __restrict__ nbr, double* __restrict__ grad, double* __restrict__ gbuf,
         double* __restrict__ tbuf, double* __restrict__ mupart, int64_t K, const Ops ops, const Phys ph,
         const double* __restrict__ nsurf, const double* __restrict__ qext, const double* __restrict__ fnorm) {
    constexpr int N2 = CfgA<N>::N2, N3 = CfgA<N>::N3, EPB = CfgA<N>::EPB;
    extern __shared__ double smem[];
    __shared__ double red[CfgA<N>::THREADS];
    const int t = threadIdx.x;
    const int el_loc = t / N3;
    const int node = t - el_loc * N3;
    const int64_t el = (int64_t)blockIdx.x * EPB + el_loc;
    const bool active = el < K;
    double* sP = smem + (size_t)el_loc * CfgA<N>::SM;   // [14][N3] rho,u0,u1,u2,beta,usq,w2..w5,u/2,|u|^2/4
    double* sL = sP + 14 * N3;                          // [5][N3] lt = lambda / J
    double* sG = sL + 5 * N3;                           // [10][N3]
    double* sB = sG + 10 * N3;                          // [6][N3] primitive cotangents
    double* sQ = sB + 6 * N3;                           // [5][N3] direct conserved cotangents
    double* sT = sQ + 5 * N3;                           // [12][N3] theta-bar
    double* sWf = sT + CfgA<N>::TSZ;                    // [6][4][N2]
    const int64_t eoff = el * 5 * N3;
    double mu_acc = 0.0;

    if (active) {
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = q[eoff + v * N3 + node];
        Prim s;
        to_prim(qv, ph, s);
        sP[node] = s.rho;
        sP[N3 + node] = s.u0;
        sP[2 * N3 + node] = s.u1;
        sP[3 * N3 + node] = s.u2;
        sP[4 * N3 + node] = s.beta;
        sP[5 * N3 + node] = s.usq;
        sP[6 * N3 + node] = 2.0 * s.beta * s.u0;
        sP[7 * N3 + node] = 2.0 * s.beta * s.u1;
        sP[8 * N3 + node] = 2.0 * s.beta * s.u2;
        sP[9 * N3 + node] = -2.0 * s.beta;
        sP[10 * N3 + node] = 0.5 * s.u0;
        sP[11 * N3 + node] = 0.5 * s.u1;
        sP[12 * N3 + node] = 0.5 * s.u2;
        sP[13 * N3 + node] = 0.25 * s.usq;
#pragma unroll
        for (int c = 0; c < 10; ++c) sG[c * N3 + node] = geom[(el * 10 + c) * N3 + node];
        const double Jinv = rcp_newton2(sG[node]);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            sL[v * N3 + node] = lam[eoff + v * N3 + node] * Jinv;
            sQ[v * N3 + node] = 0.0;
        }
    }
    __syncthreads();

    // ---- volume term: the 3 N^2 lines of all directions at once, one per thread; direction l
    // assigns its primitive cotangents to its own array (sB for l = 0, the two halves of the
    // theta-bar buffer sT for l = 1, 2, which is free until the viscous part).  With several
    // elements per CTA their lines are numbered consecutively over the CTA's threads, so that the
    // lines fill whole warps (a warp instruction costs the float64 pipe its full time whatever its
    // active lanes).
    {
        for (int g = t; g < EPB * 3 * N2; g += CfgA<N>::THREADS) {
            const int eidx = g / (3 * N2);
            if ((int64_t)blockIdx.x * EPB + eidx >= K) continue;
            const int lt = g - eidx * (3 * N2);
            // the arrays of element eidx (the same layout as the thread's own element's above)
            double* const sP = smem + (size_t)eidx * CfgA<N>::SM;
            double* const sL = sP + 14 * N3;
            double* const sG = sL + 5 * N3;
            double* const sB = sG + 10 * N3;
            double* const sT = sB + 11 * N3;
            const int l = lt / N2, line = lt - l * N2;
            double* Bl = l == 0 ? sB : sT + (l - 1) * 6 * N3;
            const int base = line_base<N>(l, line % N, line / N);
            const int st = dir_stride<N>(l);
            const double* n0p = sG + (1 + 3 * l) * N3;
            const double* n1p = n0p + N3;
            const double* n2p = n1p + N3;
            // pair cotangent mu = S_ij (lt_j/w_j - lt_i/w_i) = SW_ij lt_j + SW_ji lt_i, half of the pair
            // term's 2 S_ij (...): the flux is linear in n, so it takes the sum of the two metrics
            if constexpr (VF == kAdjESC) {
                PRaw acc[N];
#pragma unroll
                for (int i = 0; i < N; ++i) acc[i] = PRaw{0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int i = 0; i < N - 1; ++i) {
                    const int ii = base + i * st;
                    const PrimH si = load_pair_form(sP, N3, ii);
                    const double a0 = n0p[ii], a1 = n1p[ii], a2 = n2p[ii];
                    double li[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) li[v] = sL[v * N3 + ii];
#pragma unroll
                    for (int j = i + 1; j < N; ++j) {
                        const int jj = base + j * st;
                        const PrimH sj = load_pair_form(sP, N3, jj);
                        double mu[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) mu[v] = fma(ops.SW[i][j], sL[v * N3 + jj], ops.SW[j][i] * li[v]);
                        ec_pair_vjp(si, sj, a0 + n0p[jj], a1 + n1p[jj], a2 + n2p[jj], mu, ph, acc[i], acc[j]);
                    }
                }
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int ii = base + i * st;
                    Bl[ii] = acc[i].rho;
                    Bl[N3 + ii] = 0.5 * acc[i].u0;
                    Bl[2 * N3 + ii] = 0.5 * acc[i].u1;
                    Bl[3 * N3 + ii] = 0.5 * acc[i].u2;
                    Bl[4 * N3 + ii] = acc[i].beta;
                    Bl[5 * N3 + ii] = -0.25 * acc[i].c;
                }
            } else {
                PBar acc[N];
#pragma unroll
                for (int i = 0; i < N; ++i) acc[i] = PBar{0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int i = 0; i < N - 1; ++i) {
                    const int ii = base + i * st;
                    Prim si;
                    load_prim(sP, N3, ii, si);
                    const double a0 = n0p[ii], a1 = n1p[ii], a2 = n2p[ii];
                    double li[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) li[v] = sL[v * N3 + ii];
#pragma unroll
                    for (int j = i + 1; j < N; ++j) {
                        const int jj = base + j * st;
                        Prim sj;
                        load_prim(sP, N3, jj, sj);
                        double mu[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) mu[v] = fma(ops.SW[i][j], sL[v * N3 + jj], ops.SW[j][i] * li[v]);
                        if constexpr (VF == kAdjDC) {
                            // the pair term is 2 S_ij times the central flux (F(q_i).Ja_l(i) + F(q_j).Ja_l(j))/2
                            // of the nodal contravariant fluxes (D applied to nodal fluxes)
                            euler_flux_vjp(si, a0, a1, a2, mu, ph, acc[i]);
                            euler_flux_vjp(sj, n0p[jj], n1p[jj], n2p[jj], mu, ph, acc[j]);
                        } else {
                            kg_flux_vjp(si, sj, a0 + n0p[jj], a1 + n1p[jj], a2 + n2p[jj], mu, ph, acc[i], acc[j]);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int ii = base + i * st;
                    Bl[ii] = acc[i].rho;
                    Bl[N3 + ii] = acc[i].u0;
                    Bl[2 * N3 + ii] = acc[i].u1;
                    Bl[3 * N3 + ii] = acc[i].u2;
                    Bl[4 * N3 + ii] = acc[i].beta;
                    Bl[5 * N3 + ii] = acc[i].usq;
                }
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int c = 0; c < 6; ++c) sB[c * N3 + node] += sT[c * N3 + node] + sT[(6 + c) * N3 + node];
    }
    __syncthreads();

    // ---- inviscid interface term, all six faces at once: the own side's conserved cotangents to a
    // face buffer (sT, free until the viscous part), gathered per node below; the neighbour's
    // cotangents to gbuf
    double* sFo = sT;                                   // [5][6 N2]
    const double igam = rcp_newton2(ph.gamma);
    if (active) {
#pragma unroll 1
        for (int fn = node; fn < 6 * N2; fn += N3) {
            const int l = fn / (2 * N2);
            const int rem = fn - l * 2 * N2;
            const int side = rem / N2, fi = rem - side * N2;
            const int st = dir_stride<N>(l);
            const int base = line_base<N>(l, fi % N, fi / N);
            const int own = base + (side ? (N - 1) * st : 0);
            const int nbn = base + (side ? 0 : (N - 1) * st);
            const int64_t nb = nbr[el * 6 + 2 * l + side];
            const bool bnd = nb < 0;        // bounded boxes only: the exterior state at the own nodes
            double qo[5], qn[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                qo[v] = q[eoff + v * N3 + own];
                qn[v] = bnd ? qext[eoff + v * N3 + own] : q[nb * 5 * N3 + v * N3 + nbn];
            }
            Prim so, sn;
            load_prim(sP, N3, own, so);
            to_prim(qn, ph, sn);
            double n0 = sG[(1 + 3 * l) * N3 + own], n1 = sG[(2 + 3 * l) * N3 + own], n2 = sG[(3 + 3 * l) * N3 + own];
            if (nsurf) {   // optimized metrics: the interface terms take the surface metrics
                const double* ns = nsurf + (el * 6 + 2 * l + side) * 3 * N2 + fi;
                n0 = ns[0];
                n1 = ns[N2];
                n2 = ns[2 * N2];
            }
            const double E = side ? 1.0 : -1.0;
            const double wi = ops.winv[side ? N - 1 : 0];
            double nu[5], muf[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                nu[v] = sL[v * N3 + own] * wi;
                muf[v] = -E * nu[v];
            }
            PBar bo{0, 0, 0, 0, 0, 0}, bn{0, 0, 0, 0, 0, 0};
            flux_vjp<VF>(so, sn, n0, n1, n2, muf, ph, bo, bn);
            double qbo[5] = {0, 0, 0, 0, 0}, qbn[5] = {0, 0, 0, 0, 0};
            if (ph.dissipation == 2 || ph.ip_coef > 0.0) {
                // matrix dissipation and interior penalty (out of line); their term enters as -dm wi
                double dmb[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) dmb[v] = -nu[v];
                double cip = 0.0;
                if (ph.ip_coef > 0.0) {
                    const double Jn = bnd ? sG[own] : geom[nb * 10 * N3 + nbn];
                    cip = ph.ip_coef * ph.mu * (n0 * n0 + n1 * n1 + n2 * n2) / (sG[own] + Jn);
                }
                mu_acc += face_avg_vjp(so, sn, n0, n1, n2, ph, ph.dissipation == 2, cip, dmb, bo, bn);
            }
            if (ph.dissipation == 1) {
                const double nn = fnorm[(el * 6 + 2 * l + side) * N2 + fi];     // |n_J|, as the forward
                const double uo = so.u0 * n0 + so.u1 * n1 + so.u2 * n2;
                const double un_ = sn.u0 * n0 + sn.u1 * n1 + sn.u2 * n2;
                // c = sqrt(gamma/(2 beta)) = (2 beta/gamma)^(-1/2), and dc/dbeta = -c/(2 beta) = -c^3/gamma
                const double co = rsqrt_newton2(2.0 * so.beta * igam), cn = rsqrt_newton2(2.0 * sn.beta * igam);
                const double lo = fabs(uo) + co * nn, ln = fabs(un_) + cn * nn;
                const double lam2 = 0.5 * fmax(lo, ln);
                double lb = 0.0;
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    qbo[v] -= lam2 * nu[v];
                    qbn[v] += lam2 * nu[v];
                    lb -= nu[v] * (qo[v] - qn[v]);
                }
                const double lob = lo > ln ? 0.5 * lb : (lo < ln ? 0.0 : 0.25 * lb);
                const double lnb = ln > lo ? 0.5 * lb : (ln < lo ? 0.0 : 0.25 * lb);
                const double so_ = sgn(uo) * lob, sn_ = sgn(un_) * lnb;
                bo.u0 += so_ * n0;
                bo.u1 += so_ * n1;
                bo.u2 += so_ * n2;
                bn.u0 += sn_ * n0;
                bn.u1 += sn_ * n1;
                bn.u2 += sn_ * n2;
                bo.beta -= lob * nn * (co * co * co * igam);
                bn.beta -= lnb * nn * (cn * cn * cn * igam);
            }
            double qb[5];
            pbar_to_q(so, bo, ph, qb);
#pragma unroll
            for (int v = 0; v < 5; ++v) sFo[v * 6 * N2 + fn] = qb[v] + qbo[v];
            pbar_to_q(sn, bn, ph, qb);
            double* gb = gbuf + ((el * 6 + 2 * l + side) * 5) * N2 + fi;
#pragma unroll
            for (int v = 0; v < 5; ++v) gb[v * N2] = qb[v] + qbn[v];
            double* wf = sWf + (2 * l + side) * 4 * N2 + fi;
            wf[0] = 2.0 * sn.beta * sn.u0;
            wf[N2] = 2.0 * sn.beta * sn.u1;
            wf[2 * N2] = 2.0 * sn.beta * sn.u2;
            wf[3 * N2] = -2.0 * sn.beta;
        }
    }
    __syncthreads();
    if (active) {
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
            if (ia == 0 || ia == N - 1) {
                const int fi = a == 0 ? (i2 + N * i3) : (a == 1 ? (i1 + N * i3) : (i1 + N * i2));
                const int fn = (2 * a + (ia == N - 1)) * N2 + fi;
#pragma unroll
                for (int v = 0; v < 5; ++v) sQ[v * N3 + node] += sFo[v * 6 * N2 + fn];
            }
        }
    }
    __syncthreads();

    // ---- viscous chain, reversed node by node
    if (ph.viscous) {
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
        double ub[3] = {0, 0, 0}, bb = 0.0;
        if (active) {
            // forward recompute: theta, g, du, FV
            const double wown[4] = {sP[6 * N3 + node], sP[7 * N3 + node], sP[8 * N3 + node], sP[9 * N3 + node]};
            double th[3][4];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
                const int st = dir_stride<N>(a);
                const int lb = node - ia * st;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
#pragma unroll
                    for (int j = 0; j < N; ++j) s += ops.D[ia][j] * sP[(6 + k) * N3 + lb + j * st];
                    th[a][k] = s;
                }
                if (ia == 0 || ia == N - 1) {
                    const int side = ia == N - 1;
                    const int fi = a == 0 ? (i2 + N * i3) : (a == 1 ? (i1 + N * i3) : (i1 + N * i2));
                    const double E = side ? 0.5 : -0.5;
                    const double* wf = sWf + (2 * a + side) * 4 * N2 + fi;
#pragma unroll
                    for (int k = 0; k < 4; ++k) th[a][k] += E * (wf[k * N2] - wown[k]) * ops.winv[ia];
                }
            }
            const double Jinv = rcp_newton2(sG[node]);
            double g[3][4];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    g[m][k] = Jinv * (sG[(1 + m) * N3 + node] * th[0][k] + sG[(4 + m) * N3 + node] * th[1][k] +
                                      sG[(7 + m) * N3 + node] * th[2][k]);
            const double beta = sP[4 * N3 + node];
            const double RT = 0.5 * rcp_newton2(beta);
            const double u[3] = {sP[N3 + node], sP[2 * N3 + node], sP[3 * N3 + node]};
            double du[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int m = 0; m < 3; ++m) du[k][m] = RT * (g[m][k] + u[k] * g[m][3]);
            const double div = du[0][0] + du[1][1] + du[2][2];
            const double hc = ph.kappa / ph.R * RT * RT;
            double FV[3][4];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    FV[m][i] = ph.mu * (du[i][m] + du[m][i] - (i == m ? (2.0 / 3.0) * div : 0.0));
                FV[m][3] = FV[m][0] * u[0] + FV[m][1] * u[1] + FV[m][2] * u[2] + hc * g[m][3];
            }
            // Phi_l = D_l^T lt (momentum, energy) plus the interface terms -(E/2)(lt_own + lt_nbr)/w_end
            double Phi[3][4];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                const int st = dir_stride<N>(l);
                const int lb = node - il * st;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
#pragma unroll
                    for (int i = 0; i < N; ++i) s += ops.D[i][il] * sL[(1 + k) * N3 + lb + i * st];
                    Phi[l][k] = s;
                }
                const int64_t nb = (il == 0 || il == N - 1) ? nbr[el * 6 + 2 * l + (il == N - 1)] : -1;
                if (nb >= 0) {     // interior face (a boundary face has no viscous interface term)
                    const int side = il == N - 1;
                    const int st2 = dir_stride<N>(l);
                    const int nbn = node + (side ? -(N - 1) * st2 : (N - 1) * st2);   // matching node in nb
                    const double Jn = rcp_newton2(geom[nb * 10 * N3 + nbn]);
                    const double E = side ? 0.5 : -0.5;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        Phi[l][k] -= E * ops.winv[il] * (sL[(1 + k) * N3 + node] + lam[(nb * 5 + 1 + k) * N3 + nbn] * Jn);
                }
            }
            double Psi[3][4];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    Psi[m][k] = sG[(1 + m) * N3 + node] * Phi[0][k] + sG[(4 + m) * N3 + node] * Phi[1][k] +
                                sG[(7 + m) * N3 + node] * Phi[2][k];
            // lambda . R_visc is linear in mu (kappa proportional to mu)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) mu_acc += Psi[m][k] * FV[m][k];
            // reverse FV -> tau, u, hc, g.  With Tb_mi = Psi_mi + Psi_m3 u_i, the cotangent of du is
            // mu (Tb + Tb^T) - (2/3) mu tr(Tb) I, symmetric; E = RT times it.  Since du = RT (g_mk +
            // u_k g_m3), E_km feeds g_mk directly, g_m3 through u_k, u_k through g_m3, and RT through
            // du_km / RT; with dRT/dbeta = -2 RT^2 that last part gives -2 sum du_km E_km.
            double Tb[3][3];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int i = 0; i < 3; ++i) Tb[m][i] = fma(Psi[m][3], u[i], Psi[m][i]);
#pragma unroll
            for (int i = 0; i < 3; ++i) ub[i] += Psi[0][3] * FV[0][i] + Psi[1][3] * FV[1][i] + Psi[2][3] * FV[2][i];
            const double hcb = Psi[0][3] * g[0][3] + Psi[1][3] * g[1][3] + Psi[2][3] * g[2][3];
            const double rm = RT * ph.mu;
            const double dtr = (-2.0 / 3.0) * (Tb[0][0] + Tb[1][1] + Tb[2][2]);
            double E[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                E[k][k] = rm * fma(2.0, Tb[k][k], dtr);
#pragma unroll
                for (int m = k + 1; m < 3; ++m) E[k][m] = E[m][k] = rm * (Tb[k][m] + Tb[m][k]);
            }
            double gb[3][4];
            double sdE = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
#pragma unroll
                for (int k = 0; k < 3; ++k) gb[m][k] = E[k][m];
                gb[m][3] = fma(Psi[m][3], hc, u[0] * E[0][m] + u[1] * E[1][m] + u[2] * E[2][m]);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ub[k] += g[0][3] * E[k][0] + g[1][3] * E[k][1] + g[2][3] * E[k][2];
#pragma unroll
                for (int m = 0; m < 3; ++m) sdE = fma(du[k][m], E[k][m], sdE);
            }
            // hc = kappa/R RT^2: its cotangent reaches beta as hcb (kappa/R) 2 RT (-2 RT^2)
            bb -= fma(4.0 * ph.kappa / ph.R * RT * RT * RT, hcb, 2.0 * sdE);
            // g = J^-1 sum_a Ja_am theta_a  ->  theta-bar
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    sT[(a * 4 + k) * N3 + node] =
                        Jinv * (sG[(1 + 3 * a) * N3 + node] * gb[0][k] + sG[(2 + 3 * a) * N3 + node] * gb[1][k] +
                                sG[(3 + 3 * a) * N3 + node] * gb[2][k]);
        }
        __syncthreads();
        if (active) {
            // w-bar: D_a^T theta-bar_a along lines and the own part of the lift; faces to tbuf
            double wb[4] = {0, 0, 0, 0};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
                const int st = dir_stride<N>(a);
                const int lb = node - ia * st;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
#pragma unroll
                    for (int i = 0; i < N; ++i) s += ops.D[i][ia] * sT[(a * 4 + k) * N3 + lb + i * st];
                    wb[k] += s;
                }
                if (ia == 0 || ia == N - 1) {
                    const int side = ia == N - 1;
                    const int fi = a == 0 ? (i2 + N * i3) : (a == 1 ? (i1 + N * i3) : (i1 + N * i2));
                    const double E = side ? 0.5 : -0.5;
                    double* tb = tbuf + ((el * 6 + 2 * a + side) * 4) * N2 + fi;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const double thb = sT[(a * 4 + k) * N3 + node];
                        wb[k] -= E * ops.winv[ia] * thb;
                        tb[k * N2] = thb;
                    }
                }
            }
            const double beta = sP[4 * N3 + node];
            const double u[3] = {sP[N3 + node], sP[2 * N3 + node], sP[3 * N3 + node]};
            // w = (2 beta u, -2 beta)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ub[k] += 2.0 * beta * wb[k];
                bb += 2.0 * u[k] * wb[k];
            }
            bb -= 2.0 * wb[3];
            sB[N3 + node] += ub[0];
            sB[2 * N3 + node] += ub[1];
            sB[3 * N3 + node] += ub[2];
            sB[4 * N3 + node] += bb;
        }
    }
    __syncthreads();
    if (active) {
        Prim s;
        load_prim(sP, N3, node, s);
        PBar b{sB[node], sB[N3 + node], sB[2 * N3 + node], sB[3 * N3 + node], sB[4 * N3 + node], sB[5 * N3 + node]};
        double qb[5];
        pbar_to_q(s, b, ph, qb);
#pragma unroll
        for (int v = 0; v < 5; ++v) grad[eoff + v * N3 + node] = qb[v] + sQ[v * N3 + node];
    }
    // deterministic block sum of the mu cotangent (lambda . R_visc)
    red[t] = mu_acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int i = 0; i < CfgA<N>::THREADS; ++i) s += red[i];
        mupart[blockIdx.x] = s;
    }
}

// Add the neighbours' contributions on this element's face nodes: the inviscid interface
// cotangent they computed for our state (gbuf) and the lift part of their gradient cotangent
// (tbuf), pulled back through w(q).  One thread per node: a node on up to three faces sums their
// contributions (the pull-back is linear, so once for the summed entropy-variable cotangent) and
// updates its gradient once, so no two threads touch the same entry.
template <int N>
__global__ void __launch_bounds__(CfgA<N>::THREADS)
adj_face(const double* __restrict__ q, const int32_t* __restrict__ nbr, const double* __restrict__ gbuf,
         const double* __restrict__ tbuf, double* __restrict__ grad, int64_t K, const Ops ops, const Phys ph) {
    constexpr int N2 = CfgA<N>::N2, N3 = CfgA<N>::N3;
    const int t = threadIdx.x;
    const int el_loc = t / N3;
    const int node = t - el_loc * N3;
    const int64_t el = (int64_t)blockIdx.x * CfgA<N>::EPB + el_loc;
    if (el >= K) return;
    const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
    double add[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, wb[4] = {0.0, 0.0, 0.0, 0.0};
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
        if (ia != 0 && ia != N - 1) continue;
        const int side = ia == N - 1;
        const int64_t nb = nbr[el * 6 + 2 * a + side];
        if (nb < 0) continue;               // a boundary face receives nothing
        any = true;
        const int fi = a == 0 ? (i2 + N * i3) : (a == 1 ? (i1 + N * i3) : (i1 + N * i2));
        const int nside = 1 - side;
        const double* gb = gbuf + ((nb * 6 + 2 * a + nside) * 5) * N2 + fi;
#pragma unroll
        for (int v = 0; v < 5; ++v) add[v] += gb[v * N2];
        if (ph.viscous) {
            const double* tb = tbuf + ((nb * 6 + 2 * a + nside) * 4) * N2 + fi;
            const double c = (nside ? 0.5 : -0.5) * ops.winv[nside ? N - 1 : 0];
#pragma unroll
            for (int k = 0; k < 4; ++k) wb[k] = fma(c, tb[k * N2], wb[k]);
        }
    }
    if (!any) return;
    if (ph.viscous) {
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = q[(el * 5 + v) * N3 + node];
        Prim s;
        to_prim(qv, ph, s);
        PBar b{0.0, 2.0 * s.beta * wb[0], 2.0 * s.beta * wb[1], 2.0 * s.beta * wb[2],
               2.0 * (s.u0 * wb[0] + s.u1 * wb[1] + s.u2 * wb[2]) - 2.0 * wb[3], 0.0};
        double qb[5];
        pbar_to_q(s, b, ph, qb);
#pragma unroll
        for (int v = 0; v < 5; ++v) add[v] += qb[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) grad[(el * 5 + v) * N3 + node] += add[v];
}

__global__ void __launch_bounds__(kAdjRed) finish_mu(const double* __restrict__ part, int64_t n, double scale,
                                                     double* __restrict__ acc) {
    __shared__ double sh[kAdjRed];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kAdjRed) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = kAdjRed / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) acc[0] += sh[0] * scale;
}

template <int N>
cudaError_t launch_adj_n(const esdc_ctx* c, const double* q, const double* lam, double* grad, double* mu_acc,
                         cudaStream_t s) {
    using C = CfgA<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(double);
    const unsigned grid = (unsigned)((c->K + C::EPB - 1) / C::EPB);
    if (c->setup.volume_flux == ESDC_FLUX_KG)
        adj_main<N, kAdjKG><<<grid, C::THREADS, smem, s>>>(q, lam, c->d_geom, c->d_nbr, grad, c->d_adj_g, c->d_adj_t,
                                                           c->d_adj_mu, c->K, c->ops, c->phys, c->d_nsurf, c->d_qext,
                                                           c->d_fnorm);
    else if (c->setup.volume_flux == ESDC_FLUX_DC)
        adj_main<N, kAdjDC><<<grid, C::THREADS, smem, s>>>(q, lam, c->d_geom, c->d_nbr, grad, c->d_adj_g, c->d_adj_t,
                                                           c->d_adj_mu, c->K, c->ops, c->phys, c->d_nsurf, c->d_qext,
                                                           c->d_fnorm);
    else
        adj_main<N, kAdjESC><<<grid, C::THREADS, smem, s>>>(q, lam, c->d_geom, c->d_nbr, grad, c->d_adj_g, c->d_adj_t,
                                                            c->d_adj_mu, c->K, c->ops, c->phys, c->d_nsurf, c->d_qext,
                                                           c->d_fnorm);
    adj_face<N><<<grid, C::THREADS, 0, s>>>(q, c->d_nbr, c->d_adj_g, c->d_adj_t, grad, c->K, c->ops, c->phys);
    if (mu_acc) {
        const double scale = c->phys.mu > 0.0 ? 1.0 / c->phys.mu : 0.0;
        finish_mu<<<1, kAdjRed, 0, s>>>(c->d_adj_mu, grid, scale, mu_acc);
    }
    return cudaGetLastError();
}

template <int N>
cudaError_t prepare_adj_n() {
    using C = CfgA<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(double);
    const cudaError_t e = cudaFuncSetAttribute(adj_main<N, kAdjESC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    const cudaError_t e2 = e != cudaSuccess ? e
                                            : cudaFuncSetAttribute(adj_main<N, kAdjKG>,
                                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                   (int)smem);
    return e2 != cudaSuccess ? e2
                             : cudaFuncSetAttribute(adj_main<N, kAdjDC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem);
}

}  // namespace

size_t adjoint_mu_blocks(const esdc_ctx* c) {
    int epb = 1;
    switch (c->N) {
        case 2: epb = CfgA<2>::EPB; break;
        case 3: epb = CfgA<3>::EPB; break;
        case 4: epb = CfgA<4>::EPB; break;
        case 5: epb = CfgA<5>::EPB; break;
        case 6: epb = CfgA<6>::EPB; break;
        case 7: epb = CfgA<7>::EPB; break;
        default: epb = CfgA<8>::EPB; break;
    }
    return (size_t)((c->K + epb - 1) / epb);
}

cudaError_t prepare_adjoint(const esdc_ctx* c) {
    switch (c->N) {
        case 2: return prepare_adj_n<2>();
        case 3: return prepare_adj_n<3>();
        case 4: return prepare_adj_n<4>();
        case 5: return prepare_adj_n<5>();
        case 6: return prepare_adj_n<6>();
        case 7: return prepare_adj_n<7>();
        case 8: return prepare_adj_n<8>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rhs_vjp(const esdc_ctx* c, const double* q, const double* lam, double* grad, double* mu_acc,
                           cudaStream_t s) {
    switch (c->N) {
        case 2: return launch_adj_n<2>(c, q, lam, grad, mu_acc, s);
        case 3: return launch_adj_n<3>(c, q, lam, grad, mu_acc, s);
        case 4: return launch_adj_n<4>(c, q, lam, grad, mu_acc, s);
        case 5: return launch_adj_n<5>(c, q, lam, grad, mu_acc, s);
        case 6: return launch_adj_n<6>(c, q, lam, grad, mu_acc, s);
        case 7: return launch_adj_n<7>(c, q, lam, grad, mu_acc, s);
        case 8: return launch_adj_n<8>(c, q, lam, grad, mu_acc, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace esdc
