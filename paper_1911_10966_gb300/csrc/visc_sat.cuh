// Viscous interface SAT of the BR1 discretisation (SAT^V, Sec. 4): on every face node of an element,
//   dq/dt[m] += (n_side / 2) P_end^-1 (Ftilde.n of the neighbour - Ftilde.n of the element) / J,
// m = 1..4 (the viscous flux has no mass component), n_side = -1 on the low face and +1 on the high
// face of a direction.  It runs after the element kernel because it reads the neighbours' face
// traces of the contravariant viscous flux, written there as trace[el][face][4][N^2].
//
// One thread per boundary node (N^3 - (N-2)^3 of them per element), summing the faces the node lies
// on (one, two on an edge, three at a corner) in direction order before a single update of dq/dt, so
// threads never share an output and no barrier is needed.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace esdc {

template <int N>
struct VSat {
    static constexpr int N2 = N * N, N3 = N * N * N;
    static constexpr int NB = N3 - (N - 2) * (N - 2) * (N - 2);   // boundary nodes per element
    static constexpr int EPB = (128 + NB - 1) / NB;               // elements per block
    static constexpr int THREADS = EPB * NB;
};

// Boundary node r (0 <= r < NB) -> (i1, i2, i3): the two full faces i3 = 0 and i3 = N-1 first, then
// the perimeter of each inner layer i3 = 1..N-2 (rows i2 = 0 and i2 = N-1, then columns i1 = 0 and
// i1 = N-1 without their corners).
template <int N>
__device__ __forceinline__ void boundary_node(int r, int& i1, int& i2, int& i3) {
    constexpr int N2 = N * N;
    if (r < 2 * N2) {
        i3 = r < N2 ? 0 : N - 1;
        const int f = r < N2 ? r : r - N2;
        i1 = f % N;
        i2 = f / N;
        return;
    }
    constexpr int RING = 4 * (N - 1);
    const int rr = r - 2 * N2;
    i3 = 1 + rr / RING;
    const int k = rr % RING;
    if (k < 2 * N) {
        i1 = k % N;
        i2 = k < N ? 0 : N - 1;
    } else {
        const int c = k - 2 * N;                  // 0 .. 2N-5
        i1 = c < N - 2 ? 0 : N - 1;
        i2 = 1 + (c < N - 2 ? c : c - (N - 2));
    }
}

// out and trace in the residual's precision T; w_end is the inverse LGL end weight
// 1/w_0 = 1/w_{N-1}.  jac: with JINV, 1/J as [K][N3]; otherwise the geometry [K][10][N3] with J at
// component 0 (the float64 path passes the reciprocal to keep a division off its float64 pipe).
template <typename T, int N, bool JINV>
__global__ void __launch_bounds__(VSat<N>::THREADS)
visc_sat_kernel(T* __restrict__ out, const T* __restrict__ jac, const int32_t* __restrict__ nbr,
                const T* __restrict__ trace, int64_t K, T w_end) {
    using C = VSat<N>;
    constexpr int N2 = C::N2, N3 = C::N3;
    const int t = threadIdx.x;
    const int el_loc = t / C::NB;
    const int r = t - el_loc * C::NB;
    const int64_t el = (int64_t)blockIdx.x * C::EPB + el_loc;
    if (el >= K) return;
    int ix[3];
    boundary_node<N>(r, ix[0], ix[1], ix[2]);
    const int node = ix[0] + N * ix[1] + N2 * ix[2];
    // issue every independent load first: the neighbour indices, this element's traces, the
    // Jacobian and the residual being updated; only the neighbour traces wait on a load
    bool on[3];
    int side[3], fi[3];
    int32_t nb[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        on[l] = ix[l] == 0 || ix[l] == N - 1;
        side[l] = ix[l] == N - 1;
        fi[l] = l == 0 ? ix[1] + N * ix[2] : (l == 1 ? ix[0] + N * ix[2] : ix[0] + N * ix[1]);
        nb[l] = on[l] ? nbr[el * 6 + 2 * l + side[l]] : 0;
        // a boundary face (neighbour -1) reads the exterior viscous flux as the interior one: no term
        on[l] = on[l] && nb[l] >= 0;
    }
    T own[3][4];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const T* to = trace + ((el * 6 + 2 * l + side[l]) * 4) * N2 + fi[l];
#pragma unroll
        for (int k = 0; k < 4; ++k) own[l][k] = on[l] ? to[k * N2] : T(0);
    }
    const T Jf = JINV ? jac[el * N3 + node] : jac[el * 10 * N3 + node];
    T* o = out + el * 5 * N3 + node;
    T res[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) res[k] = o[(1 + k) * N3];
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (!on[l]) continue;
        const T* tn = trace + (((int64_t)nb[l] * 6 + 2 * l + 1 - side[l]) * 4) * N2 + fi[l];
        const T hs = side[l] ? T(0.5) : T(-0.5);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += hs * (tn[k * N2] - own[l][k]);
    }
    const T c = JINV ? w_end * Jf : w_end / Jf;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[(1 + k) * N3] = res[k] + c * acc[k];
}

template <typename T, int N, bool JINV>
cudaError_t launch_visc_sat(T* out, const T* jac, const int32_t* nbr, const T* trace, int64_t K, T w_end,
                            cudaStream_t s) {
    using C = VSat<N>;
    const unsigned grid = (unsigned)((K + C::EPB - 1) / C::EPB);
    visc_sat_kernel<T, N, JINV><<<grid, C::THREADS, 0, s>>>(out, jac, nbr, trace, K, w_end);
    return cudaGetLastError();
}

}  // namespace esdc
