// Float64 residual at p = 15 (N = 16 LGL nodes per direction, 4096 nodes per element): the degree
// of the paper's cost comparison above the one-CTA-per-element range of rhs_f64.cu (an element's
// float64 state, primitives and geometry no longer fit one SM's shared memory).  Same discretisation
// (eq. discEL, eq. MacroForm, eq. NSL), built in four passes over the element grid:
//   1. lg_volume, one CTA per (element, direction l, plane of N lines of direction l): the N(N-1)/2
//      distinct pairs of each line are evaluated once each, in N-1 rounds of N/2 disjoint pairs (a
//      round-robin tournament schedule, so every node is updated by one thread per round and the
//      shared-memory accumulators need no atomics); the two line ends add the interface SAT of the
//      faces normal to l and record the neighbour's entropy variables for the gradient lift.  Each
//      direction writes its own residual part r_l (scaled by 1/w_i).
//   2. lg_viscous (mu > 0), one CTA per element: the entropy variables of the element in shared
//      memory, theta_a = D_a w + lift, the physical gradient, tau and the heat flux, and the
//      contravariant viscous fluxes Ftilde_l, written to global memory with their face traces.
//   3. lg_visc_div (mu > 0), one CTA per (element, l, plane): r_l += D_l Ftilde_l along the lines
//      plus the BR1 interface term (E_ii/2)(Ftilde_nbr - Ftilde_own)/w_i at the line ends.
//   4. lg_finish: dq/dt = (r_0 + (r_1 + r_2)) / J, plus the source term if one is set.
// Volume flux variants ES-C, SF-KG and DC and the none / local Lax-Friedrichs interface dissipation
// are supported; the other optional terms of rhs_f64.cu are not built at this degree.
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "flux_f64.cuh"
#include "kernels.h"

namespace esdc {
namespace {

constexpr int LN = kLargeN;
constexpr int LN2 = LN * LN, LN3 = LN2 * LN;
constexpr int LT = LN / 2;               // threads per line in the pair rounds, one pair each
constexpr int LTHREADS = LN * LT;        // one plane: N lines
constexpr int VTHREADS = 256;            // lg_viscous threads per element
static_assert(32 % LT == 0, "the threads of a line must share a warp");

// Pair (i < j) handled by slot s in round r of the circle-method tournament over the N nodes of a
// line: node N-1 meets node r, and r + s meets r - s (mod N-1) for s = 1 .. N/2-1.  Over the N-1
// rounds every pair occurs once, and within a round every node occurs once.
__device__ __forceinline__ void round_pair(int r, int s, int& i, int& j) {
    int a, b;
    if (s == 0) {
        a = r;
        b = LN - 1;
    } else {
        a = r + s;
        if (a >= LN - 1) a -= LN - 1;
        b = r - s;
        if (b < 0) b += LN - 1;
    }
    i = a < b ? a : b;
    j = a < b ? b : a;
}

// Position i along its line and the line index t1 of entry k of a plane, chosen so that consecutive
// k are consecutive in memory (the line itself for l = 0, across lines for l = 1, 2).
__device__ __forceinline__ void plane_entry(int l, int k, int& i, int& t1) {
    if (l == 0) {
        i = k % LN;
        t1 = k / LN;
    } else {
        t1 = k % LN;
        i = k / LN;
    }
}

// shared doubles of lg_volume: primitives 8 (hr, hu0..2, beta, qq, RT, c) | metric row l 3 |
// accumulators 5 | DC: nodal contravariant flux 5, each [.][N^2] with index t1 N + i
template <int VF>
constexpr int vol_smem_doubles() {
    return (VF == kFluxDC ? 21 : 16) * LN2;
}

template <int VF>
__global__ void __launch_bounds__(LTHREADS)
lg_volume(const double* __restrict__ q, const double* __restrict__ geom, const int32_t* __restrict__ nbr,
          const double* __restrict__ fnorm, double* __restrict__ rl, double* __restrict__ wf_out, int64_t K,
          const OpsL ops, const Phys ph) {
    extern __shared__ double sm[];
    double* sPr = sm;
    double* sNm = sPr + 8 * LN2;
    double* sAc = sNm + 3 * LN2;
    [[maybe_unused]] double* sFl = sAc + 5 * LN2;
    const int64_t b = blockIdx.x;
    const int64_t el = b / (3 * LN);
    const int rem = (int)(b - el * 3 * LN);
    const int l = rem / LN, t2 = rem - l * LN;
    const int st = dir_stride<LN>(l);
    const double* qe = q + el * 5 * LN3;

    for (int k = threadIdx.x; k < LN2; k += LTHREADS) {
        int i, t1;
        plane_entry(l, k, i, t1);
        const int node = line_base<LN>(l, t1, t2) + i * st;
        const int si = t1 * LN + i;
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = qe[v * LN3 + node];
        Prim s;
        double RT, cs;
        to_prim(qv, ph, s, RT, cs);
        sPr[si] = s.hr;
        sPr[LN2 + si] = s.hu0;
        sPr[2 * LN2 + si] = s.hu1;
        sPr[3 * LN2 + si] = s.hu2;
        sPr[4 * LN2 + si] = s.beta;
        sPr[5 * LN2 + si] = s.qq;
        sPr[6 * LN2 + si] = RT;
        sPr[7 * LN2 + si] = cs;
        const double n0 = geom[(el * 10 + 1 + 3 * l) * LN3 + node];
        const double n1 = geom[(el * 10 + 2 + 3 * l) * LN3 + node];
        const double n2 = geom[(el * 10 + 3 + 3 * l) * LN3 + node];
        sNm[si] = n0;
        sNm[LN2 + si] = n1;
        sNm[2 * LN2 + si] = n2;
#pragma unroll
        for (int v = 0; v < 5; ++v) sAc[v * LN2 + si] = 0.0;
        if constexpr (VF == kFluxDC) {
            double f[5];
            euler_flux_prim(s, RT, n0, n1, n2, ph, f);
#pragma unroll
            for (int v = 0; v < 5; ++v) sFl[v * LN2 + si] = f[v];
        }
    }
    __syncthreads();

    const int line = threadIdx.x / LT, slot = threadIdx.x - (threadIdx.x / LT) * LT;
    const int lb = line * LN;
    for (int r = 0; r < LN - 1; ++r) {
        int i, j;
        round_pair(r, slot, i, j);
        const int ii = lb + i, jj = lb + j;
        double f[5];
        if constexpr (VF == kFluxDC) {
#pragma unroll
            for (int v = 0; v < 5; ++v) f[v] = sFl[v * LN2 + ii] + sFl[v * LN2 + jj];
        } else {
            Prim si, sj;
            load_prim(sPr, LN2, ii, si);
            load_prim(sPr, LN2, jj, sj);
            const double a0 = sNm[ii] + sNm[jj], a1 = sNm[LN2 + ii] + sNm[LN2 + jj],
                         a2 = sNm[2 * LN2 + ii] + sNm[2 * LN2 + jj];     // 2 x averaged metric
            if constexpr (VF == kFluxESC) ec_flux(si, sj, a0, a1, a2, ph, f);
            else kg_flux(si, sj, sPr[6 * LN2 + ii], sPr[6 * LN2 + jj], a0, a1, a2, ph, f);
        }
        const double c = ops.S[i][j];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            sAc[v * LN2 + ii] = fma(-c, f[v], sAc[v * LN2 + ii]);
            sAc[v * LN2 + jj] = fma(c, f[v], sAc[v * LN2 + jj]);
        }
        __syncwarp();
    }

    // interface SAT of the two faces normal to l at the line ends (slot 0: xi_l = -1, slot 1: +1)
    if (slot < 2) {
        const int side = slot;
        const int i = side ? LN - 1 : 0;
        const int lbase = line_base<LN>(l, line, t2);
        const int own = lbase + i * st;
        const int nbn = lbase + (side ? 0 : (LN - 1) * st);
        const int64_t nb = nbr[el * 6 + 2 * l + side];
        double qo[5], qn[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            qo[v] = qe[v * LN3 + own];
            qn[v] = q[nb * 5 * LN3 + v * LN3 + nbn];
        }
        const int si = lb + i;
        Prim so, sn;
        double RTn, cn;
        load_prim(sPr, LN2, si, so);
        to_prim(qn, ph, sn, RTn, cn);
        const double n0 = sNm[si], n1 = sNm[LN2 + si], n2 = sNm[2 * LN2 + si];
        double f[5];
        if constexpr (VF == kFluxESC) {
            ec_flux(so, sn, n0, n1, n2, ph, f);
        } else if constexpr (VF == kFluxKG) {
            kg_flux(so, sn, sPr[6 * LN2 + si], RTn, n0, n1, n2, ph, f);
        } else {
            double fo[5];
            euler_flux_prim(so, sPr[6 * LN2 + si], n0, n1, n2, ph, fo);
            euler_flux_prim(sn, RTn, n0, n1, n2, ph, f);
#pragma unroll
            for (int v = 0; v < 5; ++v) f[v] = 0.5 * (fo[v] + f[v]);
        }
        const double E = side ? 1.0 : -1.0;
        double lam = 0.0;
        if (ph.dissipation == 1) {
            const double nn = fnorm[(el * 6 + 2 * l + side) * LN2 + line + LN * t2];     // |n_J|
            const double lo = 2.0 * fabs(so.hu0 * n0 + so.hu1 * n1 + so.hu2 * n2) + sPr[7 * LN2 + si] * nn;
            const double ln = 2.0 * fabs(sn.hu0 * n0 + sn.hu1 * n1 + sn.hu2 * n2) + cn * nn;
            lam = 0.5 * fmax(lo, ln);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) sAc[v * LN2 + si] += -E * f[v] - lam * (qo[v] - qn[v]);
        double* wf = wf_out + ((el * 6 + 2 * l + side) * 4) * LN2 + line + LN * t2;
        wf[0] = 4.0 * sn.beta * sn.hu0;
        wf[LN2] = 4.0 * sn.beta * sn.hu1;
        wf[2 * LN2] = 4.0 * sn.beta * sn.hu2;
        wf[3 * LN2] = -2.0 * sn.beta;
    }
    __syncthreads();

    double* out = rl + ((int64_t)l * K + el) * 5 * LN3;
    for (int k = threadIdx.x; k < LN2; k += LTHREADS) {
        int i, t1;
        plane_entry(l, k, i, t1);
        const int node = line_base<LN>(l, t1, t2) + i * st;
        const int si = t1 * LN + i;
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v * LN3 + node] = sAc[v * LN2 + si] * ops.winv[i];
    }
}

// Viscous fluxes of one element: entropy variables w2..w5 = (2 beta u, -2 beta) in shared memory,
// theta_a = D_a w + (E/2)(w_nbr - w)/w_end at the faces normal to a, g_m = J^-1 sum_a Ja_am theta_a,
// then tau, the heat flux and Ftilde_l = sum_m Ja_lm F^V_m (eq. Fv, eq. tau), written to ft and, on
// the faces of direction l, to the trace buffer.
__global__ void __launch_bounds__(VTHREADS, 1)
lg_viscous(const double* __restrict__ q, const double* __restrict__ geom, const double* __restrict__ jinv,
           const double* __restrict__ wf_in, double* __restrict__ ft, double* __restrict__ trace, const OpsL ops,
           const Phys ph) {
    extern __shared__ double sW[];       // [4][N^3]
    const int64_t el = blockIdx.x;
    const double* qe = q + el * 5 * LN3;
    for (int node = threadIdx.x; node < LN3; node += VTHREADS) {
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = qe[v * LN3 + node];
        Prim s;
        double RT, cs;
        to_prim(qv, ph, s, RT, cs);
        sW[node] = 4.0 * s.beta * s.hu0;
        sW[LN3 + node] = 4.0 * s.beta * s.hu1;
        sW[2 * LN3 + node] = 4.0 * s.beta * s.hu2;
        sW[3 * LN3 + node] = -2.0 * s.beta;
    }
    __syncthreads();
    for (int node = threadIdx.x; node < LN3; node += VTHREADS) {
        const int i1 = node % LN, i2 = (node / LN) % LN, i3 = node / LN2;
        const double wown[4] = {sW[node], sW[LN3 + node], sW[2 * LN3 + node], sW[3 * LN3 + node]};
        double th[3][4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ia = a == 0 ? i1 : (a == 1 ? i2 : i3);
            const int st = dir_stride<LN>(a);
            const int lb = node - ia * st;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < LN; ++j) s += ops.D[ia][j] * sW[k * LN3 + lb + j * st];
                th[a][k] = s;
            }
            if (ia == 0 || ia == LN - 1) {
                const int side = ia == LN - 1;
                const int fi = a == 0 ? (i2 + LN * i3) : (a == 1 ? (i1 + LN * i3) : (i1 + LN * i2));
                const double E = side ? 0.5 : -0.5;
                const double* wf = wf_in + ((el * 6 + 2 * a + side) * 4) * LN2 + fi;
#pragma unroll
                for (int k = 0; k < 4; ++k) th[a][k] += E * (wf[k * LN2] - wown[k]) * ops.winv[ia];
            }
        }
        const double* G = geom + el * 10 * LN3 + node;
        double Ja[3][3];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int m = 0; m < 3; ++m) Ja[l][m] = G[(1 + 3 * l + m) * LN3];
        const double Jinv = jinv[el * LN3 + node];
        double g[3][4];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[m][k] = Jinv * (Ja[0][m] * th[0][k] + Ja[1][m] * th[1][k] + Ja[2][m] * th[2][k]);
        double qv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qv[v] = qe[v * LN3 + node];
        Prim s;
        double RT, cs;
        to_prim(qv, ph, s, RT, cs);
        const double u[3] = {2.0 * s.hu0, 2.0 * s.hu1, 2.0 * s.hu2};
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
            for (int i = 0; i < 3; ++i) FV[m][i] = ph.mu * (du[i][m] + du[m][i] - (i == m ? (2.0 / 3.0) * div : 0.0));
            FV[m][3] = FV[m][0] * u[0] + FV[m][1] * u[1] + FV[m][2] * u[2] + hc * g[m][3];
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            double Ft[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) Ft[k] = Ja[l][0] * FV[0][k] + Ja[l][1] * FV[1][k] + Ja[l][2] * FV[2][k];
#pragma unroll
            for (int k = 0; k < 4; ++k) ft[((el * 3 + l) * 4 + k) * LN3 + node] = Ft[k];
            const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
            if (il == 0 || il == LN - 1) {
                const int side = il == LN - 1;
                const int fi = l == 0 ? (i2 + LN * i3) : (l == 1 ? (i1 + LN * i3) : (i1 + LN * i2));
                double* tr = trace + ((el * 6 + 2 * l + side) * 4) * LN2 + fi;
#pragma unroll
                for (int k = 0; k < 4; ++k) tr[k * LN2] = Ft[k];
            }
        }
    }
}

// r_l[1..4] += D_l Ftilde_l + (E_ii/2)(Ftilde_nbr - Ftilde_own)/w_i on the plane's lines.
__global__ void __launch_bounds__(LN2)
lg_visc_div(const double* __restrict__ ft, const double* __restrict__ trace, const int32_t* __restrict__ nbr,
            double* __restrict__ rl, int64_t K, const OpsL ops) {
    __shared__ double sF[4][LN2];
    const int64_t b = blockIdx.x;
    const int64_t el = b / (3 * LN);
    const int rem = (int)(b - el * 3 * LN);
    const int l = rem / LN, t2 = rem - l * LN;
    const int st = dir_stride<LN>(l);
    int i, t1;
    plane_entry(l, threadIdx.x, i, t1);
    const int node = line_base<LN>(l, t1, t2) + i * st;
    const int si = t1 * LN + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) sF[k][si] = ft[((el * 3 + l) * 4 + k) * LN3 + node];
    __syncthreads();
    double vs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < LN; ++j) s += ops.D[i][j] * sF[k][t1 * LN + j];
        vs[k] = s;
    }
    if (i == 0 || i == LN - 1) {
        const int side = i == LN - 1;
        const int64_t nb = nbr[el * 6 + 2 * l + side];
        const double hs = side ? 0.5 : -0.5;
        const double* tn = trace + ((nb * 6 + 2 * l + 1 - side) * 4) * LN2 + t1 + LN * t2;
#pragma unroll
        for (int k = 0; k < 4; ++k) vs[k] += hs * (tn[k * LN2] - sF[k][si]) * ops.winv[i];
    }
    double* out = rl + ((int64_t)l * K + el) * 5 * LN3 + node;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[(1 + k) * LN3] += vs[k];
}

// dq/dt = (r_0 + (r_1 + r_2)) / J, one thread per node.
__global__ void __launch_bounds__(256)
lg_finish(const double* __restrict__ rl, const double* __restrict__ jinv, double* __restrict__ dqdt, int64_t K,
          const double* __restrict__ src) {
    const int64_t n = K * LN3, part = K * 5 * LN3;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const int64_t el = g / LN3;
        const int node = (int)(g - el * LN3);
        const double Jinv = jinv[g];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const int64_t i = (el * 5 + v) * LN3 + node;
            const double r = (rl[i] + (rl[part + i] + rl[2 * part + i])) * Jinv;
            dqdt[i] = src ? r + src[i] : r;
        }
    }
}

template <int VF>
cudaError_t launch_volume(const esdc_ctx* c, const double* q, cudaStream_t s) {
    const size_t smem = (size_t)vol_smem_doubles<VF>() * sizeof(double);
    lg_volume<VF><<<(unsigned)(c->K * 3 * LN), LTHREADS, smem, s>>>(q, c->d_geom, c->d_nbr, c->d_fnorm, c->d_lr,
                                                                    c->d_lwf, c->K, c->opsl, c->phys);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_rhs_large(const esdc_ctx* c) {
    (void)c;
    return cudaFuncSetAttribute(lg_viscous, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(4 * LN3 * sizeof(double)));
}

cudaError_t launch_rhs_large(const esdc_ctx* c, const double* q, double* dqdt, cudaStream_t s, cudaEvent_t* ev) {
    if (c->N != LN || !c->d_lr || !c->d_lwf || !c->d_lft) return cudaErrorInvalidValue;
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e;
    switch (c->setup.volume_flux) {
        case kFluxESC: e = launch_volume<kFluxESC>(c, q, s); break;
        case kFluxKG: e = launch_volume<kFluxKG>(c, q, s); break;
        case kFluxDC: e = launch_volume<kFluxDC>(c, q, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (c->phys.viscous) {
        lg_viscous<<<(unsigned)c->K, VTHREADS, 4 * LN3 * sizeof(double), s>>>(q, c->d_geom, c->d_jinv, c->d_lwf,
                                                                              c->d_lft, (double*)c->d_trace,
                                                                              c->opsl, c->phys);
        lg_visc_div<<<(unsigned)(c->K * 3 * LN), LN2, 0, s>>>(c->d_lft, (const double*)c->d_trace, c->d_nbr, c->d_lr,
                                                             c->K, c->opsl);
    }
    int64_t blocks = (c->n_nodes + 255) / 256;
    if (blocks > grid_cap()) blocks = grid_cap();
    lg_finish<<<(unsigned)blocks, 256, 0, s>>>(c->d_lr, c->d_jinv, dqdt, c->K, c->d_src);
    if (ev) {
        cudaEventRecord(ev[1], s);
        cudaEventRecord(ev[2], s);
        cudaEventRecord(ev[3], s);
    }
    return cudaGetLastError();
}

}  // namespace esdc
