// FP64 residual kernels: Chandrashekar flux differencing (eq. discEL), entropy-stable interface SAT,
// BR1 entropy-variable gradients, viscous fluxes and their divergence (eq. MacroForm, eq. NSL).
//
// Kernel rhs_main: one element per group of N^3 threads (EPB elements per CTA).  The element's
// state is loaded once, converted to primitive and entropy variables in shared memory, and then:
//   1. volume: for each direction l (sequentially) one thread per xi_l line evaluates the
//      N(N-1)/2 distinct node pairs of its line once each, using the skew part S of Q = S + E/2:
//      r_i -= 2 S_ij f_ij / w_i, r_j += 2 S_ij f_ij / w_j.  The E/2 boundary part of the volume
//      term, -E_ii f(q_i).n_J / w_i, cancels the own-flux part of the interface SAT and is dropped
//      on both sides.
//   2. interface: one thread per face node adds -(E_ii f_EC(own, nbr).n_J + lambda/2 (q_own - q_nbr))
//      / w_i and records the neighbour's entropy variables for the gradient lift.
//   3. viscous (mu > 0): one thread per node forms theta_a = D_a w + lift, the physical gradient,
//      tau and the heat flux, and the contravariant viscous flux Ftilde_l = sum_m Ja_lm F^V_m;
//      the normal component on each face is written to the trace buffer.
//   4. divergence sum_l D_l Ftilde_l; dq/dt = r / J is written.
// visc_sat_kernel (visc_sat.cuh) then adds the BR1 interface term (E_ii/2)(Ftilde_nbr - Ftilde_own)
// / (w_i J) on face nodes once every element's traces exist.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "kernels.h"
#include "visc_sat.cuh"
#include "flux_f64.cuh"

namespace esdc {
namespace {

template <int N>
struct Cfg {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int EPB = N3 >= 96 ? 1 : (N3 >= 48 ? 2 : (N3 >= 24 ? 4 : 16));
    static constexpr int THREADS = EPB * N3;
    // shared doubles per element: prim/w/Ftilde 12 x N3 | r 3 x 5 x N3 (one per line direction) |
    // geometry 10 x N3 | face w 24 x N2
    static constexpr int SM = 37 * N3 + 24 * N2;
    // resident CTAs per SM the register allocation is sized for (the float64 pipe needs few warps)
    static constexpr int MINB = N >= 7 ? 1 : (N == 6 ? 2 : (N >= 4 ? 3 : 4));
};

// XF: the kernel also handles the matrix dissipation, the interior penalty, boundary faces with an
// exterior state and a source term (compiled only into the instantiations of contexts that use
// them, so the default kernel carries none of it)
template <int N, int VF, bool XF>
__global__ void __launch_bounds__(Cfg<N>::THREADS, Cfg<N>::MINB)
rhs_main_f64(const double* __restrict__ q, double* __restrict__ dqdt, const double* __restrict__ geom,
             const int32_t* __restrict__ nbr, double* __restrict__ trace, int64_t K, const Ops ops,
             const Phys ph, const double* __restrict__ qext, const double* __restrict__ src,
             const double* __restrict__ nsurf, const double* __restrict__ fnorm) {
    constexpr int N2 = Cfg<N>::N2, N3 = Cfg<N>::N3, EPB = Cfg<N>::EPB;
    extern __shared__ double smem[];
    const int t = threadIdx.x;
    const int el_loc = t / N3;
    const int node = t - el_loc * N3;
    const int64_t el = (int64_t)blockIdx.x * EPB + el_loc;
    const bool active = el < K;
    double* sP = smem + (size_t)el_loc * Cfg<N>::SM;   // [12][N3]: rho/2,u/2 (3),beta,|u|^2/4,w2..w5,RT,c | Ftilde
    double* sR = sP + 12 * N3;                          // [3][5][N3] per-direction accumulators
    double* sG = sP + 27 * N3;                          // [10][N3]: J, Ja_lm
    double* sWf = sP + 37 * N3;                         // [6][4][N2]
    const int64_t eoff = el * 5 * N3;

    // ---- node-local precompute
    if (active) {
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = q[eoff + v * N3 + node];
        Prim s;
        double RT, cs;
        to_prim(qv, ph, s, RT, cs);
        sP[10 * N3 + node] = RT;
        sP[11 * N3 + node] = cs;
        sP[node] = s.hr;
        sP[N3 + node] = s.hu0;
        sP[2 * N3 + node] = s.hu1;
        sP[3 * N3 + node] = s.hu2;
        sP[4 * N3 + node] = s.beta;
        sP[5 * N3 + node] = s.qq;
        sP[6 * N3 + node] = 4.0 * s.beta * s.hu0;     // w2..w4 = 2 beta u
        sP[7 * N3 + node] = 4.0 * s.beta * s.hu1;
        sP[8 * N3 + node] = 4.0 * s.beta * s.hu2;
        sP[9 * N3 + node] = -2.0 * s.beta;
#pragma unroll
        for (int c = 0; c < 10; ++c) sG[c * N3 + node] = geom[(el * 10 + c) * N3 + node];
        if constexpr (VF == kFluxDC) {
            // nodal contravariant fluxes Ftilde_l = sum_m Ja_lm F_m(q), held in the direction-l
            // accumulator until the line through the node reads them
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                double f[5];
                euler_flux_prim(s, RT, sG[(1 + 3 * l) * N3 + node], sG[(2 + 3 * l) * N3 + node],
                                sG[(3 + 3 * l) * N3 + node], ph, f);
#pragma unroll
                for (int v = 0; v < 5; ++v) sR[(l * 5 + v) * N3 + node] = f[v];
            }
        }
    }
    __syncthreads();

    // ---- volume flux differencing: the 3 N^2 lines of all directions at once, one per thread, each
    // direction into its own accumulator (assigned, so no clearing is needed)
    if (active) {
        for (int lt = node; lt < 3 * N2; lt += N3) {
            const int l = lt / N2, line = lt - l * N2;
            const int base = line_base<N>(l, line % N, line / N);
            const int st = dir_stride<N>(l);
            const double* n0p = sG + (1 + 3 * l) * N3;
            const double* n1p = n0p + N3;
            const double* n2p = n1p + N3;
            double acc[N][5];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int v = 0; v < 5; ++v) acc[i][v] = 0.0;
            double* R = sR + l * 5 * N3;
            [[maybe_unused]] double Fl[N][5];
            if constexpr (VF == kFluxDC) {
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int v = 0; v < 5; ++v) Fl[i][v] = R[v * N3 + base + i * st];
            }
#pragma unroll
            for (int i = 0; i < N - 1; ++i) {
                const int ii = base + i * st;
                Prim si;
                if constexpr (VF != kFluxDC) load_prim(sP, N3, ii, si);
                const double a0 = n0p[ii], a1 = n1p[ii], a2 = n2p[ii];
#pragma unroll
                for (int j = i + 1; j < N; ++j) {
                    const int jj = base + j * st;
                    double f[5];
                    if constexpr (VF == kFluxESC) {
                        Prim sj;
                        load_prim(sP, N3, jj, sj);
                        ec_flux(si, sj, a0 + n0p[jj], a1 + n1p[jj], a2 + n2p[jj], ph, f);   // 2 x averaged metric
                    } else if constexpr (VF == kFluxKG) {
                        Prim sj;
                        load_prim(sP, N3, jj, sj);
                        kg_flux(si, sj, sP[10 * N3 + ii], sP[10 * N3 + jj], a0 + n0p[jj], a1 + n1p[jj], a2 + n2p[jj],
                                ph, f);
                    } else {
                        // twice the central flux of the nodal contravariant fluxes
#pragma unroll
                        for (int v = 0; v < 5; ++v) f[v] = Fl[i][v] + Fl[j][v];
                    }
                    const double c = ops.S[i][j];
#pragma unroll
                    for (int v = 0; v < 5; ++v) {
                        acc[i][v] = fma(-c, f[v], acc[i][v]);
                        acc[j][v] = fma(c, f[v], acc[j][v]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int ii = base + i * st;
#pragma unroll
                for (int v = 0; v < 5; ++v) R[v * N3 + ii] = acc[i][v] * ops.winv[i];
            }
        }
    }
    __syncthreads();

    // ---- inviscid interface SAT on all six faces at once (face nodes of direction l add into the
    // direction-l accumulator); neighbour entropy variables recorded for the gradient lift
    if (active) {
        for (int fn = node; fn < 6 * N2; fn += N3) {
            const int l = fn / (2 * N2);
            const int rem = fn - l * 2 * N2;
            const int side = rem / N2, fi = rem - side * N2;
            const int st = dir_stride<N>(l);
            const int base = line_base<N>(l, fi % N, fi / N);
            const int own = base + (side ? (N - 1) * st : 0);
            const int nbn = base + (side ? 0 : (N - 1) * st);
            const int64_t nb = nbr[el * 6 + 2 * l + side];
            double qo[5], qn[5];
            // a boundary face (neighbour -1, bounded boxes only) sees the exterior state at its own nodes
            bool bnd = false;
            if constexpr (XF) bnd = nb < 0;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                qo[v] = q[eoff + v * N3 + own];
                qn[v] = bnd ? qext[eoff + v * N3 + own] : q[nb * 5 * N3 + v * N3 + nbn];
            }
            Prim so, sn;
            double RTn, cn;
            load_prim(sP, N3, own, so);
            to_prim(qn, ph, sn, RTn, cn);
            double n0 = sG[(1 + 3 * l) * N3 + own], n1 = sG[(2 + 3 * l) * N3 + own], n2 = sG[(3 + 3 * l) * N3 + own];
            if constexpr (XF) {
                // optimized metrics: the interface terms take the analytic surface metrics (the own
                // flux, cancelled against the volume term's boundary part, keeps the volume metrics)
                if (nsurf) {
                    const double* ns = nsurf + (el * 6 + 2 * l + side) * 3 * N2 + fi;
                    n0 = ns[0];
                    n1 = ns[N2];
                    n2 = ns[2 * N2];
                }
            }
            double f[5];
            if constexpr (VF == kFluxESC) {
                ec_flux(so, sn, n0, n1, n2, ph, f);
            } else if constexpr (VF == kFluxKG) {
                kg_flux(so, sn, sP[10 * N3 + own], RTn, n0, n1, n2, ph, f);
            } else {
                double fo[5];
                euler_flux_prim(so, sP[10 * N3 + own], n0, n1, n2, ph, fo);
                euler_flux_prim(sn, RTn, n0, n1, n2, ph, f);
#pragma unroll
                for (int v = 0; v < 5; ++v) f[v] = 0.5 * (fo[v] + f[v]);
            }
            const double E = side ? 1.0 : -1.0;
            double lam = 0.0;
            double dm[5] = {0.0, 0.0, 0.0, 0.0, 0.0};      // 1/2 D (w_own - w_nbr) + interior penalty
            if constexpr (XF) {
                double jw[5], r[5];
                FaceAvg fa;
                face_jump_avg(so, sP[10 * N3 + own], sn, RTn, ph, jw, r, fa);
                if (ph.dissipation == 2) {
                    matrix_dissipation(fa, jw, r, n0, n1, n2, ph, dm);
#pragma unroll
                    for (int v = 0; v < 5; ++v) dm[v] *= 0.5;
                }
                if (ph.ip_coef > 0.0) {
                    // sigma mu |n_J| / h with h = (J_own + J_nbr)/|n_J|
                    const double nsq = n0 * n0 + n1 * n1 + n2 * n2;
                    const double Jn = bnd ? sG[own] : geom[nb * 10 * N3 + nbn];
                    const double cip = ph.ip_coef * ph.mu * nsq / (sG[own] + Jn);
#pragma unroll
                    for (int v = 0; v < 5; ++v) dm[v] = fma(cip, r[v], dm[v]);
                }
            }
            if (ph.dissipation == 1) {
                const double nn = fnorm[(el * 6 + 2 * l + side) * N2 + fi];     // |n_J|, from the setup
                const double lo = 2.0 * fabs(so.hu0 * n0 + so.hu1 * n1 + so.hu2 * n2) + sP[11 * N3 + own] * nn;
                const double ln = 2.0 * fabs(sn.hu0 * n0 + sn.hu1 * n1 + sn.hu2 * n2) + cn * nn;
                lam = 0.5 * fmax(lo, ln);
            }
            const double wi = ops.winv[side ? N - 1 : 0];
            double* R = sR + l * 5 * N3;
#pragma unroll
            for (int v = 0; v < 5; ++v) R[v * N3 + own] += (-E * f[v] - lam * (qo[v] - qn[v]) - dm[v]) * wi;
            double* wf = sWf + (2 * l + side) * 4 * N2 + fi;
            wf[0] = 4.0 * sn.beta * sn.hu0;
            wf[N2] = 4.0 * sn.beta * sn.hu1;
            wf[2 * N2] = 4.0 * sn.beta * sn.hu2;
            wf[3 * N2] = -2.0 * sn.beta;
        }
    }
    __syncthreads();
    // sum the three directions into the first accumulator
    if (active) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sR[v * N3 + node] += sR[(5 + v) * N3 + node] + sR[(10 + v) * N3 + node];
    }
    __syncthreads();

    const double Jinv = active ? 1.0 / sG[node] : 0.0;
    if (ph.viscous) {
        const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
        double Ft[3][4];
        if (active) {
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
            // physical gradient g[m][k] = J^-1 sum_a Ja_am theta_a[k]
            double g[3][4];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    g[m][k] = Jinv * (sG[(1 + m) * N3 + node] * th[0][k] + sG[(4 + m) * N3 + node] * th[1][k]
                                      + sG[(7 + m) * N3 + node] * th[2][k]);
            const double RT = sP[10 * N3 + node];
            const double u[3] = {2.0 * sP[N3 + node], 2.0 * sP[2 * N3 + node], 2.0 * sP[3 * N3 + node]};
            // du_k/dx_m = RT (g_m[k] + u_k g_m[3]); dT/dx_m = (RT)^2/R g_m[3]
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
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    Ft[l][k] = sG[(1 + 3 * l) * N3 + node] * FV[0][k] + sG[(2 + 3 * l) * N3 + node] * FV[1][k]
                             + sG[(3 + 3 * l) * N3 + node] * FV[2][k];
        }
        __syncthreads();   // every thread is done reading w / primitives
        if (active) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
#pragma unroll
                for (int k = 0; k < 4; ++k) sP[(l * 4 + k) * N3 + node] = Ft[l][k];
                const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                if (il == 0 || il == N - 1) {
                    const int side = il == N - 1;
                    const int fi = l == 0 ? (i2 + N * i3) : (l == 1 ? (i1 + N * i3) : (i1 + N * i2));
                    double* tr = trace + ((el * 6 + 2 * l + side) * 4) * N2 + fi;
#pragma unroll
                    for (int k = 0; k < 4; ++k) tr[k * N2] = Ft[l][k];
                }
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                const int st = dir_stride<N>(l);
                const int lb = node - il * st;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    double s = 0.0;
#pragma unroll
                    for (int j = 0; j < N; ++j) s += ops.D[il][j] * sP[(l * 4 + k) * N3 + lb + j * st];
                    sR[(1 + k) * N3 + node] += s;
                }
            }
        }
    }
    if (active) {
        if constexpr (XF) {
            if (src) {
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    dqdt[eoff + v * N3 + node] = fma(sR[v * N3 + node], Jinv, src[eoff + v * N3 + node]);
                return;
            }
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) dqdt[eoff + v * N3 + node] = sR[v * N3 + node] * Jinv;
    }
}

// ---- host-side launchers

template <int N, int VF, bool XF>
cudaError_t launch_rhs_n(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s,
                         cudaEvent_t* ev) {
    using C = Cfg<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(double);
    const unsigned grid = (unsigned)((c->K + C::EPB - 1) / C::EPB);
    if (ev) cudaEventRecord(ev[0], s);
    rhs_main_f64<N, VF, XF><<<grid, C::THREADS, smem, s>>>(q, dqdt, c->d_geom, c->d_nbr, (double*)c->d_trace, c->K,
                                                           c->ops, c->phys, c->d_qext, c->d_src, c->d_nsurf,
                                                           c->d_fnorm);
    if (ev) cudaEventRecord(ev[1], s);
    if (ev) cudaEventRecord(ev[2], s);
    if (c->phys.viscous) {
        const cudaError_t e = launch_visc_sat<double, N, true>(dqdt, c->d_jinv, c->d_nbr, (const double*)c->d_trace,
                                                               c->K, c->ops.winv[0], s);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

template <int N, bool XF>
cudaError_t prepare_xf(int vf) {
    using C = Cfg<N>;
    const int smem = (int)(C::EPB * C::SM * sizeof(double));
    constexpr cudaFuncAttribute kAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    switch (vf) {
        case kFluxESC: return cudaFuncSetAttribute(rhs_main_f64<N, kFluxESC, XF>, kAttr, smem);
        case kFluxKG: return cudaFuncSetAttribute(rhs_main_f64<N, kFluxKG, XF>, kAttr, smem);
        case kFluxDC: return cudaFuncSetAttribute(rhs_main_f64<N, kFluxDC, XF>, kAttr, smem);
        default: return cudaErrorInvalidValue;
    }
}

bool extra_face_terms(const esdc_ctx* c) {
    return c->phys.dissipation == 2 || c->phys.ip_coef > 0.0 || c->setup.bounded != 0 || c->d_src || c->d_nsurf;
}

template <int N>
cudaError_t prepare_n(const esdc_ctx* c) {
    const int vf = c->setup.volume_flux;
    return extra_face_terms(c) ? prepare_xf<N, true>(vf) : prepare_xf<N, false>(vf);
}

template <int N, bool XF>
cudaError_t launch_vf_xf(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev) {
    switch (c->setup.volume_flux) {
        case kFluxESC: return launch_rhs_n<N, kFluxESC, XF>(c, q, dqdt, s, ev);
        case kFluxKG: return launch_rhs_n<N, kFluxKG, XF>(c, q, dqdt, s, ev);
        case kFluxDC: return launch_rhs_n<N, kFluxDC, XF>(c, q, dqdt, s, ev);
        default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t launch_vf(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev) {
    return extra_face_terms(c) ? launch_vf_xf<N, true>(c, q, dqdt, s, ev) : launch_vf_xf<N, false>(c, q, dqdt, s, ev);
}

}  // namespace

// Opt the fused kernel into more than 48 KB of dynamic shared memory (on the current device).
cudaError_t prepare_rhs_f64(const esdc_ctx* c) {
    switch (c->N) {
        case 2: return prepare_n<2>(c);
        case 3: return prepare_n<3>(c);
        case 4: return prepare_n<4>(c);
        case 5: return prepare_n<5>(c);
        case 6: return prepare_n<6>(c);
        case 7: return prepare_n<7>(c);
        case 8: return prepare_n<8>(c);
        case kLargeN: return prepare_rhs_large(c);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rhs_f64(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev) {
    switch (c->N) {
        case 2: return launch_vf<2>(c, q, dqdt, s, ev);
        case 3: return launch_vf<3>(c, q, dqdt, s, ev);
        case 4: return launch_vf<4>(c, q, dqdt, s, ev);
        case 5: return launch_vf<5>(c, q, dqdt, s, ev);
        case 6: return launch_vf<6>(c, q, dqdt, s, ev);
        case 7: return launch_vf<7>(c, q, dqdt, s, ev);
        case 8: return launch_vf<8>(c, q, dqdt, s, ev);
        case kLargeN: return launch_rhs_large(c, q, dqdt, s, ev);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace esdc
