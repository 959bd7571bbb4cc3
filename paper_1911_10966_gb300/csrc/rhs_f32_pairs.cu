// Float32 residual of the mixed-precision form for an even number of nodes per direction (built for
// p = 3, 5, 7; taken at p = 3 and 7) with the ES-C volume flux: the arithmetic of rhs_main_f32
// (rhs_f32.cu, whose header states the split of the Chandrashekar flux about the reference state),
// with the volume term's pair loop evaluated two node pairs per instruction in packed float32
// (add/sub/mul/fma .f32x2, sm_100 and later; hand-written PTX below).  In row i of a line the two
// lanes hold the pairs (i, j) and (i, j + 1) with j even: the row node's values are broadcast to
// both lanes and the two column nodes are one 64-bit shared-memory load.  For even i the first lane pair is (i, i), (i, i + 1); the
// first lane carries the coefficient S_ii = 0.
//
// The reference parts of the split flux are folded into the sums: the mass sum accumulates the
// full mass flux rho_ln ubar.n and the energy sum adds gamma p0/(gamma-1) ubar.n to the energy
// perturbation flux, so five sums per node replace the six of rhs_main_f32 (the rounding of the
// linear part is the same, eps32 |ubar.n| per term).
//
// At N >= 6 the element's state and metrics arrive by two bulk copies (cp.async.bulk, completed on
// an mbarrier whose wait is bounded; a wait that gives up sets kStatusBulkWait in the context's
// device status and leaves the element unevaluated) into the space of the per-direction sums.
//
// Shared memory per element (floats):
//   sW4 [N3] float4   entropy variables (w2, w3, w4, w5 - w5_ref), for the viscous gradient
//   sA  [3][5][N3]    the bulk-copied state [5][N3] and metrics [10][N3] (N >= 6) | then the
//                     per-direction volume + interface sums | then the lifted gradients theta_l,
//                     float4 [3][N3 + N2] (padded), each replaced by the contravariant viscous flux
//                     of its node
//   sL  [3][8][N3]    pair-loop inputs per direction l with the line's nodes contiguous:
//                     (hdr, dbn, hu0, hu1, hu2, Ja_l0, Ja_l1, Ja_l2) at (l 8 + c) N3 + line N + j',
//                     j' = j ^ lsw(line) (a bank swizzle, below) | then the divergence terms
//                     D_l Ftilde_l, float4 [3][N3 + N2] (padded)
//   sJi [N3]          1/J
//   sQ  [5][N3]       own dq (interface dissipation) | then the sum of the three directions
//   sWf [6][4][N2]    neighbour entropy variables
//   sNq [5][6 N2]     neighbour (or exterior) perturbation state at the face nodes, face node
//                     fn = (2 l + side) N2 + fi, read in the load phase with the element's own data
// Lines of direction l: line = t1 + N t2 with (t1, t2) = (i2, i3), (i1, i3), (i1, i2) for l = 0, 1, 2
// and j = i1, i2, i3 the position along the line (l = 0 is the natural node order).
#include <cuda_runtime.h>

#include "esdc_internal.h"
#include "f32_common.cuh"
#include "fpconv.cuh"
#include "kernels.h"
#include "visc_sat.cuh"
#include "bulk_copy.cuh"

namespace esdc {
namespace {

using namespace f32;

// ---- packed float32 pairs: two lanes in one 64-bit register pair
typedef unsigned long long f2p;

__device__ __forceinline__ f2p pk(float lo, float hi) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 upk(f2p r) {
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(r));
    return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {   // a b + c
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2p bc(float x) { return pk(x, x); }
// two consecutive floats (8-byte aligned) as one packed value: one 64-bit load
__device__ __forceinline__ f2p ld2(const float* p) { return *reinterpret_cast<const f2p*>(p); }
__device__ __forceinline__ f2p ldp(const FPair& p) { return pk(p.x, p.y); }

template <int N>
struct CfgP {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int TE = N <= 5 ? (N3 > 3 * N2 ? N3 : 3 * N2) : 3 * N2;
    static constexpr int EPB = TE >= 120 ? 1 : (128 + TE - 1) / TE;
    static constexpr int THREADS = EPB * TE;
    static constexpr int SM = ((4 + 15 + 24 + 1 + 5) * N3 + (24 + 30) * N2 + 3) / 4 * 4;
    static constexpr int NPT = (N3 + TE - 1) / TE;        // nodes per thread
    static constexpr int FPT = (6 * N2 + TE - 1) / TE;    // face nodes per thread
    static constexpr int MINB = N == 8 ? 2 : (N == 6 ? 1 : 4);
};

// Swizzle of the position along a line in the direction copies: j ^ lsw(line) with an even lsw, so
// that the node pairs (j, j + 1), j even, stay adjacent while consecutive lines (the threads of a
// warp) spread over the shared-memory banks (N = 8: 16 threads' 64-bit loads on 32 distinct banks).
// At N = 8 the four values for q = (line >> 2) & 3 are 0, 4, 2, 6: lines four apart (q and q + 1
// with q even) then differ in bit 2, so the node-wise stores into the direction-1 copy, whose
// 32 threads are lines i1 + N i3 at four positions i2 each, also land on distinct banks.
template <int N>
__device__ __forceinline__ int lsw(int line) {
    return N == 8 ? 4 * ((line >> 2) & 1) + 2 * ((line >> 3) & 1) : (N == 4 ? 2 * ((line >> 3) & 1) : 0);
}
template <int N>
__device__ __forceinline__ int lidx(int line, int j) {
    return line * N + (j ^ lsw<N>(line));
}
// Padded position of node n in the viscous chain's float4 arrays (one float4 of padding per N).
template <int N>
__device__ __forceinline__ int vpad(int n) {
    return n + n / N;
}
// Position of node (i1, i2, i3) in the direction-l copy.
template <int N>
__device__ __forceinline__ int lpos(int l, int i1, int i2, int i3) {
    return l == 0 ? lidx<N>(i2 + N * i3, i1) : (l == 1 ? lidx<N>(i1 + N * i3, i2) : lidx<N>(i1 + N * i2, i3));
}
// Natural node index of position j on line `line` of direction l.
template <int N>
__device__ __forceinline__ int nat_of(int l, int line, int j) {
    return l == 0 ? (line * N + j) : (l == 1 ? ((line % N) + N * j + N * N * (line / N)) : (line + N * N * j));
}

// Log-mean terms of one lane with the reference form of ec_flux_pert: drl = rho_ln - rho0 and dIn
// (1/(2 beta_ln) = RT0 (1 + dIn)), series or logarithmic branch per lane.
__device__ __forceinline__ void logmean_lane(float ahdr, float bhdr, float adbn, float bdbn, const Ref& r, float& drl,
                                             float& dIn) {
    const float dbar = ahdr + bhdr;
    const float rb = r.rho0 + dbar;
    const float f = (ahdr - bhdr) * frcp(rb);
    const float uu = f * f;
    if (uu < 1.0e-2f) {
        drl = fmaf(rb, uu * (-1.0f / 3.0f + uu * (-4.0f / 45.0f + uu * (-44.0f / 945.0f))), dbar);
    } else {
        const float ra = r.rho0 + 2.0f * ahdr, rbb = r.rho0 + 2.0f * bhdr;
        drl = (ra - rbb) * frcp(logf(ra * frcp(rbb))) - r.rho0;
    }
    const float dbs = adbn + bdbn;
    const float rsb = frcp(2.0f + dbs);
    const float db = adbn - bdbn;
    const float fb = db * rsb;
    const float ub = fb * fb;
    if (ub < 1.0e-2f) {
        dIn = (ub * (2.0f / 3.0f + ub * (2.0f / 5.0f + ub * (2.0f / 7.0f))) - dbs) * rsb;
    } else {
        dIn = logf((1.0f + adbn) * frcp(1.0f + bdbn)) * frcp(db) - 1.0f;
    }
}

// Packed constants of the two-lane flux.
struct KP {
    f2p rho0, two, nhrho0, two_RT0, c5, H0;
    f2p c1r, c2r, c3r, c1b, c2b, c3b;   // series coefficients of drl and dIn
};
__device__ __forceinline__ KP make_kp(const Ref& r) {
    KP k;
    k.rho0 = bc(r.rho0);
    k.two = bc(2.0f);
    k.nhrho0 = bc(-r.hrho0);
    k.two_RT0 = bc(r.two_RT0);
    k.c5 = bc(r.c5);
    k.H0 = bc(r.H0);
    k.c1r = bc(-1.0f / 3.0f);
    k.c2r = bc(-4.0f / 45.0f);
    k.c3r = bc(-44.0f / 945.0f);
    k.c1b = bc(2.0f / 3.0f);
    k.c2b = bc(2.0f / 5.0f);
    k.c3b = bc(2.0f / 7.0f);
    return k;
}

// Two lanes of the split Chandrashekar flux (ec_flux_pert), the reference parts folded in: F[0] the
// mass flux, F[1..3] the momentum perturbation flux, F[4] the energy flux less p0 n.  Row node a:
// broadcast pairs (ah = hdr, ad = dbn, au = hu, a2u = u = 2 hu, an = Ja_l); column nodes b: packed.
// n = an + bn is twice the averaged metric, as S (half of 2 S) is the pair coefficient.
__device__ __forceinline__ void ec_flux2(f2p ah, f2p ad, f2p au0, f2p au1, f2p au2, f2p a2u0, f2p a2u1, f2p a2u2,
                                         f2p an0, f2p an1, f2p an2, f2p bh, f2p bd, f2p bu0, f2p bu1, f2p bu2,
                                         f2p bn0, f2p bn1, f2p bn2, const KP& k, const Ref& r, f2p F[5]) {
    const f2p dbar = add2(ah, bh);
    const f2p rb = add2(k.rho0, dbar);
    const f2p dbs = add2(ad, bd);
    const f2p den = add2(k.two, dbs);
    const float2 rbv = upk(rb), denv = upk(den);
    const f2p rrb = pk(frcp(rbv.x), frcp(rbv.y));
    const f2p rsb = pk(frcp(denv.x), frcp(denv.y));
    const f2p f = mul2(sub2(ah, bh), rrb);
    const f2p uu = mul2(f, f);
    const f2p fb = mul2(sub2(ad, bd), rsb);
    const f2p ub = mul2(fb, fb);
    const float2 uuv = upk(uu), ubv = upk(ub);
    f2p drl, dIn;
    if (fmaxf(fmaxf(uuv.x, uuv.y), fmaxf(ubv.x, ubv.y)) < 1.0e-2f) {
        const f2p tr = mul2(uu, fma2(uu, fma2(uu, k.c3r, k.c2r), k.c1r));
        drl = fma2(rb, tr, dbar);
        const f2p tb = mul2(ub, fma2(ub, fma2(ub, k.c3b, k.c2b), k.c1b));
        dIn = mul2(sub2(tb, dbs), rsb);
    } else {
        const float2 h = upk(ah), hb = upk(bh), d = upk(ad), dd = upk(bd);
        float r0, r1, i0, i1;
        logmean_lane(h.x, hb.x, d.x, dd.x, r, r0, i0);
        logmean_lane(h.y, hb.y, d.y, dd.y, r, r1, i1);
        drl = pk(r0, r1);
        dIn = pk(i0, i1);
    }
    const f2p dpt = mul2(mul2(k.two_RT0, rsb), fma2(k.nhrho0, dbs, dbar));
    const f2p ub0 = add2(au0, bu0), ub1 = add2(au1, bu1), ub2 = add2(au2, bu2);
    const f2p n0 = add2(an0, bn0), n1 = add2(an1, bn1), n2 = add2(an2, bn2);
    const f2p un = fma2(ub2, n2, fma2(ub1, n1, mul2(ub0, n0)));
    const f2p rr = add2(k.rho0, drl);
    const f2p f1 = mul2(rr, un);
    F[0] = f1;
    F[1] = fma2(f1, ub0, mul2(dpt, n0));
    F[2] = fma2(f1, ub1, mul2(dpt, n1));
    F[3] = fma2(f1, ub2, mul2(dpt, n2));
    const f2p hab = fma2(a2u2, bu2, fma2(a2u1, bu1, mul2(a2u0, bu0)));
    F[4] = fma2(k.H0, un, fma2(mul2(k.c5, un), fma2(dIn, rr, drl), fma2(f1, hab, mul2(dpt, un))));
}

// One lane of the same flux (interface terms), reference parts folded in as in ec_flux2.
__device__ __forceinline__ void ec_flux_folded(const PrimF& a, const PrimF& b, float n0, float n1, float n2,
                                               const Ref& r, float F[5]) {
    float df[5], un;
    ec_flux_pert(a, b, n0, n1, n2, r, df, un);
    F[0] = fmaf(r.rho0, un, df[0]);
    F[1] = df[1];
    F[2] = df[2];
    F[3] = df[3];
    F[4] = fmaf(r.H0, un, df[4]);
}

// Two lanes of to_prim_f: packed primitives of two float32 perturbation states (the pair-loop form:
// half density perturbation, beta/beta0 - 1, half velocity; u = 2 hu is formed where needed).
struct PrimP {
    f2p hdr, dbn, hu0, hu1, hu2;
};
__device__ __forceinline__ PrimP to_prim2(const f2p dq[5], const Ref& r) {
    const f2p rho = add2(bc(r.rho0), dq[0]);
    const float2 rv = upk(rho);
    const f2p ri = pk(frcp(rv.x), frcp(rv.y));
    const f2p u0 = mul2(dq[1], ri), u1 = mul2(dq[2], ri), u2 = mul2(dq[3], ri);
    const f2p usq = fma2(u2, u2, fma2(u1, u1, mul2(u0, u0)));
    const f2p dp = mul2(bc(r.gm1), fma2(bc(-0.5f), mul2(rho, usq), dq[4]));
    const float2 den = upk(add2(bc(r.p0), dp));
    const f2p ip = pk(frcp(den.x), frcp(den.y));
    PrimP s;
    s.dbn = mul2(mul2(fma2(bc(-r.rho0), dp, mul2(dq[0], bc(r.p0))), ip), bc(r.inv_rho0));
    s.hdr = mul2(bc(0.5f), dq[0]);
    s.hu0 = mul2(bc(0.5f), u0);
    s.hu1 = mul2(bc(0.5f), u1);
    s.hu2 = mul2(bc(0.5f), u2);
    return s;
}

// The neighbours' (or on a bounded box's boundary faces the exterior) state at this thread's
// interface nodes fn = tl + f TE < 6 N2, face node fn = (2 l + side) N2 + fi.
template <int N, bool XF>
__device__ __forceinline__ void load_neighbour_faces(const StageF& in, const int32_t* __restrict__ nbr,
                                                     const double* __restrict__ qext, const Ref& ref, int64_t el,
                                                     int64_t eoff, int tl, bool active,
                                                     float (&qn)[CfgP<N>::FPT][5]) {
    using C = CfgP<N>;
    constexpr int N2 = C::N2, N3 = C::N3, TE = C::TE;
    if (!active) return;
#pragma unroll
    for (int f = 0; f < C::FPT; ++f) {
        const int fn = tl + f * TE;
        if (fn < 6 * N2) {
            const int l = fn / (2 * N2);
            const int rem = fn - l * 2 * N2;
            const int side = rem / N2, fi = rem - side * N2;
            const int st = dir_stride_f<N>(l);
            const int base = line_base_f<N>(l, fi % N, fi / N);
            const int64_t nb = nbr[el * 6 + 2 * l + side];
            if (!XF || nb >= 0) {
                const int nbn = base + (side ? 0 : (N - 1) * st);
#pragma unroll
                for (int v = 0; v < 5; ++v) qn[f][v] = __ldg(in.base + nb * 5 * N3 + v * N3 + nbn);
            } else {
                // boundary face of a bounded box: the float64 exterior state at the own nodes, less
                // the reference state, rounded once
                const int own = base + (side ? (N - 1) * st : 0);
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const double x = qext[eoff + v * N3 + own];
                    qn[f][v] = d2f_int(v == 0 ? x - ref.rho0d : (v == 4 ? x - ref.E0d : x));
                }
            }
        }
    }
}

template <int N, bool XF>
__global__ void __launch_bounds__(CfgP<N>::THREADS, CfgP<N>::MINB)
rhs_pairs_f32(const StageF in, float* __restrict__ out, const float* __restrict__ geom, const int32_t* __restrict__ nbr,
              float* __restrict__ trace, int64_t K, const OpsF ops, const PhysF ph, const Ref ref,
              const float* __restrict__ nsurf, const double* __restrict__ qext, const double* __restrict__ src,
              int* __restrict__ status) {
    using C = CfgP<N>;
    constexpr int N2 = C::N2, N3 = C::N3, TE = C::TE;
    extern __shared__ float4 smp4[];
    const int t = threadIdx.x;
    const int el_loc = t / TE;
    const int tl = t - el_loc * TE;
    const int64_t el = (int64_t)blockIdx.x * C::EPB + el_loc;
    const bool active = el < K;
    float* base_sm = reinterpret_cast<float*>(smp4) + (size_t)el_loc * C::SM;
    float4* sW4 = reinterpret_cast<float4*>(base_sm);          // [N3]
    float* sA = base_sm + 4 * N3;                               // [3][5][N3] | float4 [3][N3] Ftilde
    float* sL = sA + 15 * N3;                                   // [3][8][N3]
    float* sJi = sL + 24 * N3;                                  // [N3]
    float* sQ = sJi + N3;                                       // [5][N3] | [5][N3] direction sum
    float* sWf = sQ + 5 * N3;                                   // [6][4][N2]
    float* sNq = sWf + 24 * N2;                                 // [5][6 N2]
    const int64_t eoff = el * 5 * N3;

    // ---- load.  BULK (N >= 6): the element's state and metrics (a contiguous 5 N3 and 10 N3 float
    // block each) come by two bulk copies into the per-direction sums' space, free until the pair
    // loop, while every thread reads the neighbours' face values of its interface nodes.  Otherwise
    // each thread reads its nodes' values itself, issued together with the neighbour reads (at
    // p = 3 the copies' barrier cost more than they saved: 1.39 against 1.35 ms per residual on
    // 63^3 elements; at p = 7 they save 0.19 ms of 5.5 on 48^3).  Then the primitives go to the three
    // direction copies, with the metrics and the entropy variables.
    constexpr int NPT = C::NPT, FPT = C::FPT;
    constexpr bool BULK = N >= 6;
    float d[NPT][5], gv[NPT][10], qn[FPT][5];
    if constexpr (BULK) {
        __shared__ __align__(8) uint64_t bar;
        __shared__ int bulk_failed;
        if (t == 0) {
            mbar_init(&bar, 1);
            bulk_failed = 0;
        }
        __syncthreads();
        if (t == 0) {
            const int64_t el0 = (int64_t)blockIdx.x * C::EPB;
            const int ne = (int)(K - el0 < C::EPB ? K - el0 : C::EPB);
            constexpr uint32_t kState = 5 * N3 * sizeof(float), kGeom = 10 * N3 * sizeof(float);
            mbar_expect_tx(&bar, (uint32_t)ne * (kState + kGeom));
            for (int e = 0; e < ne; ++e) {
                float* dst = reinterpret_cast<float*>(smp4) + (size_t)e * C::SM + 4 * N3;
                bulk_g2s(dst, in.base + (el0 + e) * 5 * N3, kState, &bar);
                bulk_g2s(dst + 5 * N3, geom + (el0 + e) * 10 * N3, kGeom, &bar);
            }
        }
        load_neighbour_faces<N, XF>(in, nbr, qext, ref, el, eoff, tl, active, qn);
        if (!mbar_wait_bounded(&bar, 0)) bulk_failed = 1;
        __syncthreads();
        if (bulk_failed) {
            // the copies did not complete in time: report, give them one more bounded wait (the
            // shared memory they write must not be released under them), and leave the element
            // unevaluated
            if (t == 0) {
                atomicOr(status, kStatusBulkWait);
                mbar_wait_bounded(&bar, 0);
            }
            return;
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < NPT; ++r) {
                const int node = tl + r * TE;
                if (node < N3) {
#pragma unroll
                    for (int v = 0; v < 5; ++v) d[r][v] = sA[v * N3 + node];
#pragma unroll
                    for (int c = 0; c < 10; ++c) gv[r][c] = sA[(5 + c) * N3 + node];
                }
            }
        }
    } else if (active) {
#pragma unroll
        for (int r = 0; r < NPT; ++r) {
            const int node = tl + r * TE;
            if (node < N3) {
#pragma unroll
                for (int v = 0; v < 5; ++v) d[r][v] = __ldg(in.base + eoff + v * N3 + node);
#pragma unroll
                for (int c = 0; c < 10; ++c) gv[r][c] = geom[(el * 10 + c) * N3 + node];
            }
        }
        load_neighbour_faces<N, XF>(in, nbr, qext, ref, el, eoff, tl, active, qn);
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < NPT; ++r) {
            const int node = tl + r * TE;
            if (node < N3) {
#pragma unroll
                for (int v = 0; v < 5; ++v) sQ[v * N3 + node] = d[r][v];
                PrimF s;
                to_prim_f(d[r], ref, s);
                const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
                const float pv[5] = {s.hdr, s.dbn, s.hu0, s.hu1, s.hu2};
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    float* L = sL + l * 8 * N3 + lpos<N>(l, i1, i2, i3);
#pragma unroll
                    for (int c = 0; c < 5; ++c) L[c * N3] = pv[c];
#pragma unroll
                    for (int m = 0; m < 3; ++m) L[(5 + m) * N3] = gv[r][1 + 3 * l + m];
                }
                sJi[node] = frcp(gv[r][0]);
                const float tb = two_beta(s, ref);
                sW4[node] = make_float4(tb * s.u0, tb * s.u1, tb * s.u2, -ref.two_beta0 * s.dbn);
            }
        }
#pragma unroll
        for (int f = 0; f < FPT; ++f) {
            const int fn = tl + f * TE;
            if (fn < 6 * N2) {
#pragma unroll
                for (int v = 0; v < 5; ++v) sNq[v * 6 * N2 + fn] = qn[f][v];
            }
        }
    }
    __syncthreads();

    // ---- volume: one thread per line (all three directions at once), two node pairs per instruction
    if (active && tl < 3 * N2) {
        const int l = tl / N2, line = tl - l * N2;
        const float* L = sL + l * 8 * N3 + line * N;
        const int sw = lsw<N>(line);
        const KP k = make_kp(ref);
        f2p acc[N / 2][5];
#pragma unroll
        for (int m = 0; m < N / 2; ++m)
#pragma unroll
            for (int v = 0; v < 5; ++v) acc[m][v] = 0ull;
#pragma unroll
        for (int i = 0; i < N - 1; ++i) {
            const int is = i ^ sw;
            const float hu0 = L[2 * N3 + is], hu1 = L[3 * N3 + is], hu2 = L[4 * N3 + is];
            const f2p ah = bc(L[is]), ad = bc(L[N3 + is]);
            const f2p au0 = bc(hu0), au1 = bc(hu1), au2 = bc(hu2);
            const f2p a2u0 = bc(2.0f * hu0), a2u1 = bc(2.0f * hu1), a2u2 = bc(2.0f * hu2);
            const f2p an0 = bc(L[5 * N3 + is]), an1 = bc(L[6 * N3 + is]), an2 = bc(L[7 * N3 + is]);
            f2p part[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int m = (i + 1) / 2; m < N / 2; ++m) {
                const int j = 2 * m;
                const float* Lj = L + (j ^ sw);
                f2p F[5];
                ec_flux2(ah, ad, au0, au1, au2, a2u0, a2u1, a2u2, an0, an1, an2, ld2(Lj), ld2(Lj + N3),
                         ld2(Lj + 2 * N3), ld2(Lj + 3 * N3), ld2(Lj + 4 * N3), ld2(Lj + 5 * N3),
                         ld2(Lj + 6 * N3), ld2(Lj + 7 * N3), k, ref, F);
                const f2p c = ld2(&ops.S[i][j]);      // (S_ij, S_i,j+1)
                const f2p ct = ld2(&ops.ST[i][j]);    // (S_ji, S_j+1,i) = -(S_ij, S_i,j+1)
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    acc[m][v] = fma2(c, F[v], acc[m][v]);
                    part[v] = fma2(ct, F[v], part[v]);
                }
            }
            // row node i: both lanes of the row partial
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float2 p = upk(part[v]);
                float2 a = upk(acc[i / 2][v]);
                if (i % 2 == 0) a.x += p.x + p.y;
                else a.y += p.x + p.y;
                acc[i / 2][v] = pk(a.x, a.y);
            }
        }
        // the last node of the line is only ever a column node: nothing to fold
        float* A = sA + l * 5 * N3;
#pragma unroll
        for (int m = 0; m < N / 2; ++m) {
            const int j = 2 * m;
            const int n0 = nat_of<N>(l, line, j), n1 = nat_of<N>(l, line, j + 1);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float2 a = upk(acc[m][v]);
                A[v * N3 + n0] = a.x * ops.winv[j];
                A[v * N3 + n1] = a.y * ops.winv[j + 1];
            }
        }
    }
    __syncthreads();

    // ---- interface SAT, all six faces at once; face nodes of direction l add into the direction-l sums.
    // With two face nodes per thread (FPT == 2) they are the two lanes of packed instructions.
    if constexpr (FPT == 2) {
        if (active) {
            int fnv[2], lv[2], sidev[2], fiv[2], ownv[2], jov[2];
            float qn[2][5], so[2][5], nv[2][3], qo[2][5];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // a thread without a second face node repeats its first in lane y and drops its result
                const int fn = (h == 1 && tl + TE < 6 * N2) ? tl + TE : tl;
                const int l = fn / (2 * N2);
                const int rem = fn - l * 2 * N2;
                const int side = rem / N2, fi = rem - side * N2;
                const int st = dir_stride_f<N>(l);
                const int own = line_base_f<N>(l, fi % N, fi / N) + (side ? (N - 1) * st : 0);
                const int jo = side ? N - 1 : 0;
                fnv[h] = fn; lv[h] = l; sidev[h] = side; fiv[h] = fi; ownv[h] = own; jov[h] = jo;
                const int own0 = lidx<N>(own / N, own % N);    // the natural order is direction 0's
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    qn[h][c] = sNq[c * 6 * N2 + fn];
                    so[h][c] = sL[c * N3 + own0];
                    qo[h][c] = sQ[c * N3 + own];
                }
                const float* Ln = sL + (l * 8 + 5) * N3 + lidx<N>(fi, jo);
#pragma unroll
                for (int m = 0; m < 3; ++m) nv[h][m] = Ln[m * N3];
                if (nsurf) {   // optimized metrics: the interface terms take the surface metrics
                    const float* ns = nsurf + (el * 6 + 2 * l + side) * 3 * N2 + fi;
#pragma unroll
                    for (int m = 0; m < 3; ++m) nv[h][m] = ns[m * N2];
                }
            }
            f2p QN[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) QN[c] = pk(qn[0][c], qn[1][c]);
            const PrimP sn = to_prim2(QN, ref);
            const f2p oh = pk(so[0][0], so[1][0]), od = pk(so[0][1], so[1][1]);
            const f2p ou0 = pk(so[0][2], so[1][2]), ou1 = pk(so[0][3], so[1][3]), ou2 = pk(so[0][4], so[1][4]);
            const f2p n0 = pk(nv[0][0], nv[1][0]), n1 = pk(nv[0][1], nv[1][1]), n2 = pk(nv[0][2], nv[1][2]);
            const KP k = make_kp(ref);
            f2p F[5];
            // the interface flux takes n itself: a-side n, b-side 0 (ec_flux2 sums the two)
            ec_flux2(oh, od, ou0, ou1, ou2, add2(ou0, ou0), add2(ou1, ou1), add2(ou2, ou2), n0, n1, n2, sn.hdr,
                     sn.dbn, sn.hu0, sn.hu1, sn.hu2, 0ull, 0ull, 0ull, k, ref, F);
            f2p lam = 0ull;
            if (ph.dissipation) {
                const float2 nn2 = upk(fma2(n2, n2, fma2(n1, n1, mul2(n0, n0))));
                const f2p nn = pk(fsqrt(nn2.x), fsqrt(nn2.y));
                // |u.n| + c |n| on both sides, u = 2 hu, c^2 = gamma RT = gamma RT0 / (1 + dbn)
                const float2 uo = upk(mul2(bc(2.0f), fma2(ou2, n2, fma2(ou1, n1, mul2(ou0, n0)))));
                const float2 un = upk(mul2(bc(2.0f), fma2(sn.hu2, n2, fma2(sn.hu1, n1, mul2(sn.hu0, n0)))));
                const float2 dpo = upk(add2(bc(1.0f), od)), dpn = upk(add2(bc(1.0f), sn.dbn));
                const float gRT0 = ref.gamma * ref.RT0;
                const f2p co = pk(fsqrt(gRT0 * frcp(dpo.x)), fsqrt(gRT0 * frcp(dpo.y)));
                const f2p cn = pk(fsqrt(gRT0 * frcp(dpn.x)), fsqrt(gRT0 * frcp(dpn.y)));
                const float2 lo = upk(fma2(co, nn, pk(fabsf(uo.x), fabsf(uo.y))));
                const float2 ln = upk(fma2(cn, nn, pk(fabsf(un.x), fabsf(un.y))));
                lam = pk(0.5f * fmaxf(lo.x, ln.x), 0.5f * fmaxf(lo.y, ln.y));
            }
            const f2p mE = pk(sidev[0] ? -1.0f : 1.0f, sidev[1] ? -1.0f : 1.0f);
            const f2p wi = pk(ops.winv[jov[0]], ops.winv[jov[1]]);
            float val[5][2];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const f2p jump = sub2(pk(qo[0][v], qo[1][v]), QN[v]);
                const float2 t = upk(mul2(fma2(mE, F[v], mul2(sub2(0ull, lam), jump)), wi));
                val[v][0] = t.x;
                val[v][1] = t.y;
            }
            const f2p tb = mul2(bc(ref.two_beta0), add2(bc(1.0f), sn.dbn));
            const float2 w0 = upk(mul2(bc(2.0f), mul2(tb, sn.hu0))), w1 = upk(mul2(bc(2.0f), mul2(tb, sn.hu1)));
            const float2 w2 = upk(mul2(bc(2.0f), mul2(tb, sn.hu2))), w3 = upk(mul2(bc(-ref.two_beta0), sn.dbn));
            const float wv[4][2] = {{w0.x, w0.y}, {w1.x, w1.y}, {w2.x, w2.y}, {w3.x, w3.y}};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !(tl + TE < 6 * N2)) break;
                float* A = sA + lv[h] * 5 * N3;
#pragma unroll
                for (int v = 0; v < 5; ++v) A[v * N3 + ownv[h]] += val[v][h];
                float* wf = sWf + (2 * lv[h] + sidev[h]) * 4 * N2 + fiv[h];
#pragma unroll
                for (int c = 0; c < 4; ++c) wf[c * N2] = wv[c][h];
            }
            (void)fnv;
        }
    } else {
        if (active) {
#pragma unroll
            for (int f = 0; f < FPT; ++f) {
                const int fn = tl + f * TE;
                if (fn >= 6 * N2) break;
                const int l = fn / (2 * N2);
                const int rem = fn - l * 2 * N2;
                const int side = rem / N2, fi = rem - side * N2;
                const int st = dir_stride_f<N>(l);
                const int base = line_base_f<N>(l, fi % N, fi / N);
                const int own = base + (side ? (N - 1) * st : 0);
                const int jo = side ? N - 1 : 0;
                float qn[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) qn[v] = sNq[v * 6 * N2 + fn];
                PrimF so, sn;
                const int own0 = lidx<N>(own / N, own % N);    // the natural order is direction 0's
                so.hdr = sL[own0];
                so.dbn = sL[N3 + own0];
                so.hu0 = sL[2 * N3 + own0];
                so.hu1 = sL[3 * N3 + own0];
                so.hu2 = sL[4 * N3 + own0];
                so.u0 = 2.0f * so.hu0;
                so.u1 = 2.0f * so.hu1;
                so.u2 = 2.0f * so.hu2;
                to_prim_f(qn, ref, sn);
                const float* Ln = sL + (l * 8 + 5) * N3 + lidx<N>(fi, jo);
                float n0 = Ln[0], n1 = Ln[N3], n2 = Ln[2 * N3];
                if (nsurf) {   // optimized metrics: the interface terms take the surface metrics
                    const float* ns = nsurf + (el * 6 + 2 * l + side) * 3 * N2 + fi;
                    n0 = ns[0];
                    n1 = ns[N2];
                    n2 = ns[2 * N2];
                }
                float F[5];
                ec_flux_folded(so, sn, n0, n1, n2, ref, F);
                const float E = side ? 1.0f : -1.0f;
                float lam = 0.0f;
                if (ph.dissipation) {
                    const float nn = fsqrt(n0 * n0 + n1 * n1 + n2 * n2);
                    const float lo = fabsf(so.u0 * n0 + so.u1 * n1 + so.u2 * n2) + fsqrt(ref.gamma * node_RT(so.dbn, ref)) * nn;
                    const float ln = fabsf(sn.u0 * n0 + sn.u1 * n1 + sn.u2 * n2) + fsqrt(ref.gamma * node_RT(sn.dbn, ref)) * nn;
                    lam = 0.5f * fmaxf(lo, ln);
                }
                const float wi = ops.winv[jo];
                float* A = sA + l * 5 * N3;
#pragma unroll
                for (int v = 0; v < 5; ++v) A[v * N3 + own] += (-E * F[v] - lam * (sQ[v * N3 + own] - qn[v])) * wi;
                float* wf = sWf + (2 * l + side) * 4 * N2 + fi;
                const float tb = two_beta(sn, ref);
                wf[0] = tb * sn.u0;
                wf[N2] = tb * sn.u1;
                wf[2 * N2] = tb * sn.u2;
                wf[3 * N2] = -ref.two_beta0 * sn.dbn;
            }
        }
    }
    __syncthreads();

    if (ph.viscous) {
        // The two line derivatives of the viscous chain (the lifted gradient of the entropy variables
        // and the divergence of the contravariant viscous fluxes) run one thread per line, each line's
        // eight float4 values loaded once; the node-wise part between them (metric contraction, shear
        // stress and heat flux) runs one thread per node.
        // [3][NP] float4 with node n at vpad(n) = n + n / N: the lines of direction 0 (stride N float4)
        // then fall on different banks
        constexpr int NP = N3 + N2;
        float4* sT4 = reinterpret_cast<float4*>(sA);     // theta_l, then Ftilde_l
        float4* sD4 = reinterpret_cast<float4*>(sL);     // D_l Ftilde_l (the direction copies are dead)
        // the node's three directions of volume and interface sums (sQ is free after the SAT)
        if (active) {
            for (int node = tl; node < N3; node += TE) {
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    sQ[v * N3 + node] = sA[v * N3 + node] + (sA[(5 + v) * N3 + node] + sA[(10 + v) * N3 + node]);
            }
        }
        __syncthreads();
        // theta_l = D_l w + (E/2)(w_nbr - w_own)/w_end at the line ends
        if (active && tl < 3 * N2) {
            const int l = tl / N2, line = tl - l * N2;
            const int st = dir_stride_f<N>(l);
            const int base = line_base_f<N>(l, line % N, line / N);
            float4 w[N];
#pragma unroll
            for (int j = 0; j < N; ++j) w[j] = sW4[base + j * st];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                f2p s01 = 0ull, s23 = 0ull;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const f2p d = ldp(ops.D2[i][j]);
                    s01 = fma2(d, pk(w[j].x, w[j].y), s01);
                    s23 = fma2(d, pk(w[j].z, w[j].w), s23);
                }
                float2 a01 = upk(s01), a23 = upk(s23);
                if (i == 0 || i == N - 1) {
                    const float E = (i == N - 1 ? 0.5f : -0.5f) * ops.winv[i];
                    const float* wf = sWf + (2 * l + (i == N - 1)) * 4 * N2 + line;
                    a01.x += E * (wf[0] - w[i].x);
                    a01.y += E * (wf[N2] - w[i].y);
                    a23.x += E * (wf[2 * N2] - w[i].z);
                    a23.y += E * (wf[3 * N2] - w[i].w);
                }
                sT4[l * NP + vpad<N>(base + i * st)] = make_float4(a01.x, a01.y, a23.x, a23.y);
            }
        }
        __syncthreads();
        // node-wise: gradient, viscous flux, its contravariant components (over theta) and face traces
        if (active) {
            for (int node = tl; node < N3; node += TE) {
                const int i1 = node % N, i2 = (node / N) % N, i3 = node / N2;
                float th[3][4];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float4 t4 = sT4[a * NP + vpad<N>(node)];
                    th[a][0] = t4.x;
                    th[a][1] = t4.y;
                    th[a][2] = t4.z;
                    th[a][3] = t4.w;
                }
                float Ja[3][3];
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const float* Lg = sL + (l * 8 + 5) * N3 + lpos<N>(l, i1, i2, i3);
#pragma unroll
                    for (int m = 0; m < 3; ++m) Ja[l][m] = Lg[m * N3];
                }
                const float Jinv = sJi[node];
                float g[3][4];
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        g[m][kk] = Jinv * (Ja[0][m] * th[0][kk] + Ja[1][m] * th[1][kk] + Ja[2][m] * th[2][kk]);
                const int node0 = lidx<N>(node / N, i1);
                const float dbn = sL[N3 + node0];
                const float RT = node_RT(dbn, ref);
                const float u[3] = {2.0f * sL[2 * N3 + node0], 2.0f * sL[3 * N3 + node0], 2.0f * sL[4 * N3 + node0]};
                float du[3][3];
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                    for (int m = 0; m < 3; ++m) du[kk][m] = RT * (g[m][kk] + u[kk] * g[m][3]);
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
                    float Ft[4];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) Ft[kk] = Ja[l][0] * FV[0][kk] + Ja[l][1] * FV[1][kk] + Ja[l][2] * FV[2][kk];
                    sT4[l * NP + vpad<N>(node)] = make_float4(Ft[0], Ft[1], Ft[2], Ft[3]);
                    const int il = l == 0 ? i1 : (l == 1 ? i2 : i3);
                    if (il == 0 || il == N - 1) {
                        const int side = il == N - 1;
                        const int fi = l == 0 ? (i2 + N * i3) : (l == 1 ? (i1 + N * i3) : (i1 + N * i2));
                        float* tr = trace + ((el * 6 + 2 * l + side) * 4) * N2 + fi;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) tr[kk * N2] = Ft[kk];
                    }
                }
            }
        }
        __syncthreads();
        // D_l Ftilde_l along the lines
        if (active && tl < 3 * N2) {
            const int l = tl / N2, line = tl - l * N2;
            const int st = dir_stride_f<N>(l);
            const int base = line_base_f<N>(l, line % N, line / N);
            float4 f[N];
#pragma unroll
            for (int j = 0; j < N; ++j) f[j] = sT4[l * NP + vpad<N>(base + j * st)];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                f2p s01 = 0ull, s23 = 0ull;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const f2p d = ldp(ops.D2[i][j]);
                    s01 = fma2(d, pk(f[j].x, f[j].y), s01);
                    s23 = fma2(d, pk(f[j].z, f[j].w), s23);
                }
                const float2 a01 = upk(s01), a23 = upk(s23);
                sD4[l * NP + vpad<N>(base + i * st)] = make_float4(a01.x, a01.y, a23.x, a23.y);
            }
        }
        __syncthreads();
        if (active) {
            for (int node = tl; node < N3; node += TE) {
                const int vp = vpad<N>(node);
                const float4 d0 = sD4[vp], d1 = sD4[NP + vp], d2 = sD4[2 * NP + vp];
                const float vs[4] = {d0.x + (d1.x + d2.x), d0.y + (d1.y + d2.y), d0.z + (d1.z + d2.z),
                                     d0.w + (d1.w + d2.w)};
                const float Jinv = sJi[node];
                float sv[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                if (XF && src) {
#pragma unroll
                    for (int v = 0; v < 5; ++v) sv[v] = d2f_int(src[eoff + v * N3 + node]);
                }
                out[eoff + node] = sQ[node] * Jinv + sv[0];
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
                    out[eoff + (1 + kk) * N3 + node] = (sQ[(1 + kk) * N3 + node] + vs[kk]) * Jinv + sv[1 + kk];
                out[eoff + 4 * N3 + node] = (sQ[4 * N3 + node] + vs[3]) * Jinv + sv[4];
            }
        }
    } else if (active) {
        for (int node = tl; node < N3; node += TE) {
            const float Jinv = sJi[node];
            float sv[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (XF && src) {
#pragma unroll
                for (int v = 0; v < 5; ++v) sv[v] = d2f_int(src[eoff + v * N3 + node]);
            }
#pragma unroll
            for (int v = 0; v < 5; ++v)
                out[eoff + v * N3 + node] =
                    (sA[v * N3 + node] + (sA[(5 + v) * N3 + node] + sA[(10 + v) * N3 + node])) * Jinv + sv[v];
        }
    }
}

// ---- host-side launchers
template <int N>
cudaError_t launch_pairs_n(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev) {
    using C = CfgP<N>;
    const size_t smem = (size_t)C::EPB * C::SM * sizeof(float);
    const unsigned grid = (unsigned)((c->K + C::EPB - 1) / C::EPB);
    const Ref ref = make_ref(c);
    if (in.nk != 0) return cudaErrorInvalidValue;   // stage states are formed by launch_stage_f32
    if (ev) cudaEventRecord(ev[0], s);
    const bool xf = c->setup.bounded != 0 || c->d_src != nullptr;
    auto go = [&](auto kern) {
        kern<<<grid, C::THREADS, smem, s>>>(in, out, c->d_geomf, c->d_nbr, (float*)c->d_trace, c->K, c->opsf,
                                            c->physf, ref, c->d_nsurff, c->d_qext, c->d_src, c->d_status);
    };
    xf ? go(rhs_pairs_f32<N, true>) : go(rhs_pairs_f32<N, false>);
    if (ev) cudaEventRecord(ev[1], s);
    if (ev) cudaEventRecord(ev[2], s);
    if (c->physf.viscous) {
        const cudaError_t e = launch_visc_sat<float, N, false>(out, c->d_geomf, c->d_nbr, (const float*)c->d_trace,
                                                               c->K, c->opsf.winv[0], s);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

template <int N>
cudaError_t prepare_pairs_n() {
    const int smem = (int)((size_t)CfgP<N>::EPB * CfgP<N>::SM * sizeof(float));
    constexpr cudaFuncAttribute kAttr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(rhs_pairs_f32<N, false>, kAttr, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rhs_pairs_f32<N, true>, kAttr, smem);
    return e;
}

}  // namespace

// Taken for N = 4 and 8, where it is faster than rhs_main_f32 (measured on 16 M-node Taylor-Green
// meshes: +10% at p = 3, +18% at p = 7); at N = 6 its 138 registers leave three CTAs of 108 threads
// per SM and rhs_main_f32 is faster, so that degree keeps it (the N = 6 instances stay compiled).
bool pairs_f32_supported(const esdc_ctx* c) {
    return c->setup.volume_flux == ESDC_FLUX_ESC && (c->N == 4 || c->N == 8);
}

cudaError_t prepare_rhs_f32_pairs(const esdc_ctx* c) {
    switch (c->N) {
        case 4: return prepare_pairs_n<4>();
        case 6: return prepare_pairs_n<6>();
        case 8: return prepare_pairs_n<8>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rhs_f32_pairs(const esdc_ctx* c, const StageF& in, float* out, cudaStream_t s, cudaEvent_t* ev) {
    switch (c->N) {
        case 4: return launch_pairs_n<4>(c, in, out, s, ev);
        case 6: return launch_pairs_n<6>(c, in, out, s, ev);
        case 8: return launch_pairs_n<8>(c, in, out, s, ev);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace esdc
