// FP32 residual kernels of the mixed-precision form: the same ES-C residual as rhs_f64.cu with all
// flux differencing, interface and viscous arithmetic in float32, evaluated on a perturbation
// state so that float32 rounding acts on O(1) quantities rather than on the O(1/(gamma Ma^2))
// pressure and enthalpy.
//
// Input: the shadow state dq = (rho - rho0, rho u, rho E - E0) in float32 (written by a float64
// kernel from the float64 state, or a Runge-Kutta stage state formed from it in float32 by
// launch_stage_f32), float32 geometry, neighbour table.  Reference state rho0 = 1,
// p0 = R (T0 = 1), beta0 = 1/(2R), E0 = p0/(gamma-1).
//
// The Chandrashekar flux is split exactly as f = f_ref + df with
//   f_ref = [rho0 ubar.n, p0 n, gamma p0/(gamma-1) ubar.n]
//   df1 = drho_ln ubar.n,  df_m = f1 ubar_m + dp_t n_m,
//   df5 = ubar.n/(gamma-1) (rho0 dI + drho_ln (RT0 + dI)) + f1 (u_a.u_b)/2 + dp_t ubar.n,
// where drho_ln = rho_ln - rho0, dp_t = p_t - p0 and dI = 1/(2 beta_ln) - RT0 are formed from the
// perturbations (no O(p0) cancellation).  The p0 n part of f_ref contributes -p0 sum_l D_l Ja_l
// (zero by the discrete GCL of the float64 metrics) and is dropped from volume and interface
// terms alike; the ubar.n part is linear and is accumulated separately (one extra accumulator)
// and scaled by rho0 and gamma p0/(gamma-1) at the end.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "fpconv.cuh"
#include "kernels.h"
#include "visc_sat.cuh"
#include "f32_common.cuh"

namespace esdc {
namespace {

using namespace f32;

template <int N, bool KG = false>
struct CfgF {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int LINES = 3 * N2;                       // all three directions at once
    // threads per element: one per node up to N = 5, one per line beyond (measured: N = 6 runs 18%
    // faster with 3N^2 threads than with N^3)
    static constexpr int TE = N <= 5 ? (N3 > LINES ? N3 : LINES) : LINES;
    static constexpr int EPB = TE >= 120 ? 1 : (128 + TE - 1) / TE;
    static constexpr int THREADS = EPB * TE;
    // shared floats per element: prim 2 x float4 | w float4 | geometry 3 x float4 | accumulators 3 x 6
    // (aliased by the 3 x float4 viscous fluxes) | own dq 5 | face w 24 N^2 (rounded to whole float4)
    // (+ 2 N3 for the Kennedy-Gruber pair quantities, half the pressure perturbation and eh, as
    // float2 from an even offset)
    static constexpr int KG_OFF = (8 + 4 + 12 + 18 + 5) * N3 + 24 * N2;
    static constexpr int SM = (KG_OFF + (KG ? (KG_OFF & 1) + 2 * N3 : 0) + 3) / 4 * 4;
    // resident CTAs the registers are sized for (N = 5: one element of 125 threads per CTA, six CTAs
    // per SM measured 10% faster than three CTAs of two elements), capped by the CTAs whose shared
    // memory fits one SM (228 KB, 1 KB reserved per CTA): the SF-KG instances need more of it
    static constexpr int MINB0 = N <= 4 ? 4 : (N == 5 ? 6 : 2);
    static constexpr int BY_SMEM = (228 * 1024) / (EPB * SM * 4 + 1024);
    static constexpr int MINB = BY_SMEM < 1 ? 1 : (BY_SMEM < MINB0 ? BY_SMEM : MINB0);
};

// Kennedy-Gruber two-point flux (the SF-KG variant, Sec. 4) split as above: with arithmetic means
// rho_bar = rho0 + dbar, u_bar, p_bar = p0 + dp_bar and e_bar = e0 + de (e = RT/(gamma-1) + |u|^2/2,
// de = eh_a + eh_b), f = f_ref + df with df1 = dbar ubar.n, df_m = f1 ubar_m + dp_bar n_m and
// df5 = ubar.n (rho0 de + dbar (e0 + de) + dp_bar); the reference part f_ref is that of the ES-C
// split (rho0 e0 + p0 = gamma p0/(gamma-1)).
__device__ __forceinline__ void kg_flux_pert(const PrimF& a, const PrimF& b, float n0, float n1, float n2,
                                             const Ref& r, float df[5], float& un) {
    const float dbar = a.hdr + b.hdr;
    const float ub0 = a.hu0 + b.hu0, ub1 = a.hu1 + b.hu1, ub2 = a.hu2 + b.hu2;
    un = ub0 * n0 + ub1 * n1 + ub2 * n2;
    const float dpb = a.hdp + b.hdp;
    const float de = a.eh + b.eh;
    const float f1 = (r.rho0 + dbar) * un;
    df[0] = dbar * un;
    df[1] = f1 * ub0 + dpb * n0;
    df[2] = f1 * ub1 + dpb * n1;
    df[3] = f1 * ub2 + dpb * n2;
    df[4] = un * (r.rho0 * de + dbar * (r.e0 + de) + dpb);
}

// node primitives stored as two float4 per node: (drho/2, u/2), (dbn, u)
__device__ __forceinline__ void load_prim_f(const float4* sP4, int N3, int idx, PrimF& s) {
    const float4 a = sP4[idx], b = sP4[N3 + idx];
    s.hdr = a.x;
    s.hu0 = a.y;
    s.hu1 = a.z;
    s.hu2 = a.w;
    s.dbn = b.x;
    s.u0 = b.y;
    s.u1 = b.z;
    s.u2 = b.w;
}
// the part the second member of a pair uses (no full velocity)
__device__ __forceinline__ void load_prim_half(const float4* sP4, int N3, int idx, PrimF& s) {
    const float4 a = sP4[idx];
    s.hdr = a.x;
    s.hu0 = a.y;
    s.hu1 = a.z;
    s.hu2 = a.w;
    s.dbn = reinterpret_cast<const float*>(sP4 + N3 + idx)[0];
}

// XF: boundary faces (bounded boxes) and a source term, compiled only into the instantiations that
// need them (a run-time test for them cost 2% on periodic boxes)
template <int N, bool XF, bool KG>
__global__ void __launch_bounds__(CfgF<N>::THREADS, CfgF<N, KG>::MINB)
rhs_main_f32(const StageF in, float* __restrict__ out, const float* __restrict__ geom,
             const int32_t* __restrict__ nbr, float* __restrict__ trace, int64_t K, const OpsF ops, const PhysF ph,
             const Ref ref, const float* __restrict__ nsurf, const double* __restrict__ qext,
             const double* __restrict__ src) {
    using C = CfgF<N, KG>;
    constexpr int N2 = C::N2, N3 = C::N3, TE = C::TE;
    extern __shared__ float smf[];
    const int t = threadIdx.x;
    const int el_loc = t / TE;
    const int tl = t - el_loc * TE;
    const int64_t el = (int64_t)blockIdx.x * C::EPB + el_loc;
    const bool active = el < K;
    float* sP = smf + (size_t)el_loc * C::SM;       // [2][N3] float4 primitives | later [8][N3] floats
    float4* sP4 = reinterpret_cast<float4*>(sP);
    float4* sW4 = reinterpret_cast<float4*>(sP + 8 * N3);   // [N3] (w2, w3, w4, w5 - w5_ref)
    float4* sG4 = sW4 + N3;                          // [3][N3] (Ja_l0, Ja_l1, Ja_l2, 1/J)
    float* sA = sP + 24 * N3;                        // [3][6][N3] per-direction accumulators | float4 [3][N3] Ftilde
    float4* sF4 = reinterpret_cast<float4*>(sA);
    float* sQ = sA + 18 * N3;                        // [5][N3] own dq
    float* sWf = sQ + 5 * N3;                        // [6][4][N2] neighbour entropy variables
    float2* sK2 = reinterpret_cast<float2*>(sP + C::KG_OFF + (C::KG_OFF & 1));   // [N3] (hdp, eh), SF-KG only
    const int64_t eoff = el * 5 * N3;

    if (active) {
        for (int node = tl; node < N3; node += TE) {
            float d[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                d[v] = __ldg(in.base + eoff + v * N3 + node);
                sQ[v * N3 + node] = d[v];
            }
            PrimF s;
            to_prim_f(d, ref, s);
            sP4[node] = make_float4(s.hdr, s.hu0, s.hu1, s.hu2);
            sP4[N3 + node] = make_float4(s.dbn, s.u0, s.u1, s.u2);
            if constexpr (KG) sK2[node] = make_float2(s.hdp, s.eh);
            // w5 - w5_ref = -2 (beta - beta0): the constant has no gradient
            const float tb = two_beta(s, ref);
            sW4[node] = make_float4(tb * s.u0, tb * s.u1, tb * s.u2, -ref.two_beta0 * s.dbn);
            float gv[10];
#pragma unroll
            for (int c = 0; c < 10; ++c) gv[c] = geom[(el * 10 + c) * N3 + node];
            const float Ji = frcp(gv[0]);
#pragma unroll
            for (int l = 0; l < 3; ++l) sG4[l * N3 + node] = make_float4(gv[1 + 3 * l], gv[2 + 3 * l], gv[3 + 3 * l], Ji);
        }
    }
    __syncthreads();

    // ---- volume: all three directions at once, one thread per line, own accumulators per direction
    if (active && tl < 3 * N2) {
        const int l = tl / N2, line = tl - l * N2;
        const int base = line_base_f<N>(l, line % N, line / N);
        const int st = dir_stride_f<N>(l);
        const float4* nl = sG4 + l * N3;
        float acc[N][6];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int v = 0; v < 6; ++v) acc[i][v] = 0.0f;
#pragma unroll
        for (int i = 0; i < N - 1; ++i) {
            const int ii = base + i * st;
            PrimF si;
            load_prim_f(sP4, N3, ii, si);
            if constexpr (KG) {
                const float2 k2 = sK2[ii];
                si.hdp = k2.x;
                si.eh = k2.y;
            }
            const float4 ni = nl[ii];
#pragma unroll
            for (int j = i + 1; j < N; ++j) {
                const int jj = base + j * st;
                PrimF sj;
                load_prim_half(sP4, N3, jj, sj);
                const float4 nj = nl[jj];
                float df[5], un;
                // the flux is linear in n: pass n_i + n_j and take S (half of 2S) as the pair coefficient
                if constexpr (KG) {
                    const float2 k2 = sK2[jj];
                    sj.hdp = k2.x;
                    sj.eh = k2.y;
                    kg_flux_pert(si, sj, ni.x + nj.x, ni.y + nj.y, ni.z + nj.z, ref, df, un);
                } else {
                    ec_flux_pert(si, sj, ni.x + nj.x, ni.y + nj.y, ni.z + nj.z, ref, df, un);
                }
                const float c = ops.S[i][j];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    acc[i][v] -= c * df[v];
                    acc[j][v] += c * df[v];
                }
                acc[i][5] -= c * un;
                acc[j][5] += c * un;
            }
        }
        float* A = sA + l * 6 * N3;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int ii = base + i * st;
#pragma unroll
            for (int v = 0; v < 6; ++v) A[v * N3 + ii] = acc[i][v] * ops.winv[i];
        }
    }
    __syncthreads();

    // ---- interface SAT, all six faces at once: face nodes of direction l add into the direction-l
    // accumulators, so edges and corners shared by several directions never collide
    if (active) {
        for (int fn = tl; fn < 6 * N2; fn += TE) {
            const int l = fn / (2 * N2);
            const int rem = fn - l * 2 * N2;
            const int side = rem / N2, fi = rem - side * N2;
            const int st = dir_stride_f<N>(l);
            const int base = line_base_f<N>(l, fi % N, fi / N);
            const int own = base + (side ? (N - 1) * st : 0);
            const int nbn = base + (side ? 0 : (N - 1) * st);
            const int64_t nb = nbr[el * 6 + 2 * l + side];
            float qn[5];
            if (!XF || nb >= 0) {
#pragma unroll
                for (int v = 0; v < 5; ++v) qn[v] = __ldg(in.base + nb * 5 * N3 + v * N3 + nbn);
            } else {
                // boundary face of a bounded box: the float64 exterior state at the own nodes, less
                // the reference state, rounded once
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const double x = qext[eoff + v * N3 + own];
                    qn[v] = d2f_int(v == 0 ? x - ref.rho0d : (v == 4 ? x - ref.E0d : x));
                }
            }
            PrimF so, sn;
            load_prim_f(sP4, N3, own, so);
            if constexpr (KG) {
                const float2 k2 = sK2[own];
                so.hdp = k2.x;
                so.eh = k2.y;
            }
            to_prim_f(qn, ref, sn);
            const float4 nv = sG4[l * N3 + own];
            float n0 = nv.x, n1 = nv.y, n2 = nv.z;
            if (nsurf) {   // optimized metrics: the interface terms take the surface metrics
                const float* ns = nsurf + (el * 6 + 2 * l + side) * 3 * N2 + fi;
                n0 = ns[0];
                n1 = ns[N2];
                n2 = ns[2 * N2];
            }
            float df[5], un;
            if constexpr (KG) kg_flux_pert(so, sn, n0, n1, n2, ref, df, un);
            else ec_flux_pert(so, sn, n0, n1, n2, ref, df, un);
            const float E = side ? 1.0f : -1.0f;
            float lam = 0.0f;
            if (ph.dissipation) {
                const float nn = fsqrt(n0 * n0 + n1 * n1 + n2 * n2);
                const float lo = fabsf(so.u0 * n0 + so.u1 * n1 + so.u2 * n2) + fsqrt(ref.gamma * node_RT(so.dbn, ref)) * nn;
                const float ln = fabsf(sn.u0 * n0 + sn.u1 * n1 + sn.u2 * n2) + fsqrt(ref.gamma * node_RT(sn.dbn, ref)) * nn;
                lam = 0.5f * fmaxf(lo, ln);
            }
            const float wi = ops.winv[side ? N - 1 : 0];
            float* A = sA + l * 6 * N3;
#pragma unroll
            for (int v = 0; v < 5; ++v) A[v * N3 + own] += (-E * df[v] - lam * (sQ[v * N3 + own] - qn[v])) * wi;
            A[5 * N3 + own] += -E * un * wi;
            float* wf = sWf + (2 * l + side) * 4 * N2 + fi;
            const float tb = two_beta(sn, ref);
            wf[0] = tb * sn.u0;
            wf[N2] = tb * sn.u1;
            wf[2 * N2] = tb * sn.u2;
            wf[3 * N2] = -ref.two_beta0 * sn.dbn;
        }
    }
    __syncthreads();
    // ---- viscous chain
    if (ph.viscous) {
        constexpr int NPT = (N3 + TE - 1) / TE;    // nodes per thread
        float Ft[NPT][3][4];
        if (active) {
#pragma unroll
            for (int r = 0; r < NPT; ++r) {
                const int node = tl + r * TE;
                if (node >= N3) break;
                const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
                const float4 w4 = sW4[node];
                const float wown[4] = {w4.x, w4.y, w4.z, w4.w};
                float th[3][4];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
                    const int st = dir_stride_f<N>(a);
                    const int lb = node - ia * st;
                    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const float d = ops.D[ia][j];
                        const float4 wj = sW4[lb + j * st];
                        s.x += d * wj.x;
                        s.y += d * wj.y;
                        s.z += d * wj.z;
                        s.w += d * wj.w;
                    }
                    th[a][0] = s.x;
                    th[a][1] = s.y;
                    th[a][2] = s.z;
                    th[a][3] = s.w;
                    if (ia == 0 || ia == N - 1) {
                        const int side = ia == N - 1;
                        const int fi = a == 0 ? (i2 + N * i3) : (a == 1 ? (i1 + N * i3) : (i1 + N * i2));
                        const float E = side ? 0.5f : -0.5f;
                        const float* wf = sWf + (2 * a + side) * 4 * N2 + fi;
#pragma unroll
                        for (int k = 0; k < 4; ++k) th[a][k] += E * (wf[k * N2] - wown[k]) * ops.winv[ia];
                    }
                }
                const float4 G0 = sG4[node], G1 = sG4[N3 + node], G2 = sG4[2 * N3 + node];
                const float Jinv = G0.w;
                const float Ja[3][3] = {{G0.x, G0.y, G0.z}, {G1.x, G1.y, G1.z}, {G2.x, G2.y, G2.z}};
                float g[3][4];
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        g[m][k] = Jinv * (Ja[0][m] * th[0][k] + Ja[1][m] * th[1][k] + Ja[2][m] * th[2][k]);
                const float4 P1 = sP4[N3 + node];
                const float RT = node_RT(P1.x, ref);
                const float u[3] = {P1.y, P1.z, P1.w};
                float du[3][3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int m = 0; m < 3; ++m) du[k][m] = RT * (g[m][k] + u[k] * g[m][3]);
                const float div = du[0][0] + du[1][1] + du[2][2];
                const float hc = ph.kappa / ph.R * RT * RT;
                float FV[3][4];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        FV[m][i] = ph.mu * (du[i][m] + du[m][i] - (i == m ? (2.0f / 3.0f) * div : 0.0f));
                    FV[m][3] = FV[m][0] * u[0] + FV[m][1] * u[1] + FV[m][2] * u[2] + hc * g[m][3];
                }
#pragma unroll
                for (int l = 0; l < 3; ++l) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        Ft[r][l][k] = Ja[l][0] * FV[0][k] + Ja[l][1] * FV[1][k] + Ja[l][2] * FV[2][k];
                    const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                    if (il == 0 || il == N - 1) {
                        const int side = il == N - 1;
                        const int fi = l == 0 ? (i2 + N * i3) : (l == 1 ? (i1 + N * i3) : (i1 + N * i2));
                        float* tr = trace + ((el * 6 + 2 * l + side) * 4) * N2 + fi;
#pragma unroll
                        for (int k = 0; k < 4; ++k) tr[k * N2] = Ft[r][l][k];
                    }
                }
                // the node's three directions of volume/interface sums, into the third direction's
                // slots (the viscous fluxes will overwrite the first two)
#pragma unroll
                for (int v = 0; v < 6; ++v)
                    sA[(12 + v) * N3 + node] = sA[v * N3 + node] + (sA[(6 + v) * N3 + node] + sA[(12 + v) * N3 + node]);
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int r = 0; r < NPT; ++r) {
                const int node = tl + r * TE;
                if (node >= N3) break;
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    sF4[l * N3 + node] = make_float4(Ft[r][l][0], Ft[r][l][1], Ft[r][l][2], Ft[r][l][3]);
            }
        }
        __syncthreads();
        if (active) {
            for (int node = tl; node < N3; node += TE) {
                const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
                float vs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                    const int st = dir_stride_f<N>(l);
                    const int lb = node - il * st;
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const float d = ops.D[il][j];
                        const float4 f = sF4[l * N3 + lb + j * st];
                        vs[0] += d * f.x;
                        vs[1] += d * f.y;
                        vs[2] += d * f.z;
                        vs[3] += d * f.w;
                    }
                }
                const float Jinv = sG4[node].w;
                const float* sum = sA + 12 * N3 + node;
                const float lin = sum[5 * N3];
                float sv[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                if (XF && src) {
#pragma unroll
                    for (int v = 0; v < 5; ++v) sv[v] = d2f_int(src[eoff + v * N3 + node]);
                }
                out[eoff + node] = (sum[0] + ref.rho0 * lin) * Jinv + sv[0];
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    out[eoff + (1 + k) * N3 + node] = (sum[(1 + k) * N3] + vs[k]) * Jinv + sv[1 + k];
                out[eoff + 4 * N3 + node] = (sum[4 * N3] + ref.H0 * lin + vs[3]) * Jinv + sv[4];
            }
        }
    } else if (active) {
        for (int node = tl; node < N3; node += TE) {
            float a[6];
#pragma unroll
            for (int v = 0; v < 6; ++v) a[v] = sA[v * N3 + node] + (sA[(6 + v) * N3 + node] + sA[(12 + v) * N3 + node]);
            const float Jinv = sG4[node].w;
            float sv[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (XF && src) {
#pragma unroll
                for (int v = 0; v < 5; ++v) sv[v] = d2f_int(src[eoff + v * N3 + node]);
            }
            out[eoff + node] = (a[0] + ref.rho0 * a[5]) * Jinv + sv[0];
#pragma unroll
            for (int k = 1; k < 4; ++k) out[eoff + k * N3 + node] = a[k] * Jinv + sv[k];
            out[eoff + 4 * N3 + node] = (a[4] + ref.H0 * a[5]) * Jinv + sv[4];
        }
    }
}

template <int N>
cudaError_t launch_f32_n(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev) {
    using C = CfgF<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(float);
    const unsigned grid = (unsigned)((c->K + C::EPB - 1) / C::EPB);
    const PhysF& ph = c->physf;
    const Ref ref = make_ref(c);
    if (in.nk != 0) return cudaErrorInvalidValue;   // stage states are formed by launch_stage_f32
    if (ev) cudaEventRecord(ev[0], s);
    const bool xf = c->setup.bounded != 0 || c->d_src != nullptr;
    const bool kg = c->setup.volume_flux == ESDC_FLUX_KG;
    auto go = [&](auto kern, size_t bytes) {
        kern<<<grid, C::THREADS, bytes, s>>>(in, out, c->d_geomf, c->d_nbr, (float*)c->d_trace, c->K, c->opsf, ph,
                                             ref, c->d_nsurff, c->d_qext, c->d_src);
    };
    const size_t smem_kg = (size_t)C::EPB * CfgF<N, true>::SM * sizeof(float);
    if (kg)
        xf ? go(rhs_main_f32<N, true, true>, smem_kg) : go(rhs_main_f32<N, false, true>, smem_kg);
    else
        xf ? go(rhs_main_f32<N, true, false>, smem) : go(rhs_main_f32<N, false, false>, smem);
    if (ev) cudaEventRecord(ev[1], s);
    if (ev) cudaEventRecord(ev[2], s);
    if (ph.viscous) {
        const cudaError_t e = launch_visc_sat<float, N, false>(out, c->d_geomf, c->d_nbr, (const float*)c->d_trace,
                                                               c->K, c->opsf.winv[0], s);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

template <int N>
cudaError_t prepare_f32_n() {
    using C = CfgF<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(float);
    constexpr cudaFuncAttribute kAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int sk = (int)((size_t)C::EPB * CfgF<N, true>::SM * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(rhs_main_f32<N, false, false>, kAttr, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rhs_main_f32<N, true, false>, kAttr, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rhs_main_f32<N, false, true>, kAttr, sk);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rhs_main_f32<N, true, true>, kAttr, sk);
    return e;
}

}  // namespace

cudaError_t prepare_rhs_f32(const esdc_ctx* c) {
    if (pairs_f32_supported(c)) {
        const cudaError_t e = prepare_rhs_f32_pairs(c);
        if (e != cudaSuccess) return e;
    }
    switch (c->N) {
        case 2: return prepare_f32_n<2>();
        case 3: return prepare_f32_n<3>();
        case 4: return prepare_f32_n<4>();
        case 5: return prepare_f32_n<5>();
        case 6: return prepare_f32_n<6>();
        case 7: return prepare_f32_n<7>();
        case 8: return prepare_f32_n<8>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rhs_f32(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev) {
    if (pairs_f32_supported(c)) return launch_rhs_f32_pairs(c, in, out, s, ev);
    switch (c->N) {
        case 2: return launch_f32_n<2>(c, in, out, s, ev);
        case 3: return launch_f32_n<3>(c, in, out, s, ev);
        case 4: return launch_f32_n<4>(c, in, out, s, ev);
        case 5: return launch_f32_n<5>(c, in, out, s, ev);
        case 6: return launch_f32_n<6>(c, in, out, s, ev);
        case 7: return launch_f32_n<7>(c, in, out, s, ev);
        case 8: return launch_f32_n<8>(c, in, out, s, ev);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace esdc
