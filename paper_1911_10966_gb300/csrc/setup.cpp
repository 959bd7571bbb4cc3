// Host setup: LGL nodes and weights, SBP operators, curvilinear metric terms, connectivity.
// Everything here runs once per context in float64 (long double for the node iteration).
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "esdc_internal.h"

namespace esdc {

// Legendre P_n, P_n' and P_n'' at x (long double); P'' from Legendre's differential equation.
static void legendre3(int n, long double x, long double& P, long double& dP, long double& d2P) {
    long double p0 = 1.0L, p1 = x;
    if (n == 0) { P = 1.0L; dP = 0.0L; d2P = 0.0L; return; }
    for (int k = 1; k < n; ++k) {
        long double p2 = ((2.0L * k + 1.0L) * x * p1 - k * p0) / (k + 1.0L);
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    // P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), valid for |x| < 1
    dP = n * (x * p1 - p0) / (x * x - 1.0L);
    d2P = (2.0L * x * dP - n * (n + 1.0L) * P) / (1.0L - x * x);
}

// LGL nodes: +-1 and the zeros of P_p', found by Newton on P_p' with P_p'' from Legendre's
// equation, in long double.  Weights 2/(p(p+1) P_p(x)^2) (Sec. 2, diagonal-norm SBP on LGL nodes).
int lgl(int p, double* xi, double* w) {
    if (p < 1 || p > kLargeN - 1 || !xi || !w) return ESDC_ERR_ARG;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<long double> x(p + 1);
    x[0] = -1.0L;
    x[p] = 1.0L;
    for (int i = 1; i < p; ++i) {
        long double g = -std::cos(pi * i / (long double)p);   // Chebyshev-Gauss-Lobatto guess
        for (int it = 0; it < 60; ++it) {
            long double P, dP, d2P;
            legendre3(p, g, P, dP, d2P);
            long double step = dP / d2P;
            g -= step;
            if (std::fabs((double)step) < 1e-19) break;
        }
        x[i] = g;
    }
    // enforce exact symmetry of the node set
    for (int i = 0; i <= p / 2; ++i) {
        long double m = 0.5L * (x[p - i] - x[i]);
        x[i] = -m;
        x[p - i] = m;
    }
    if (p % 2 == 0) x[p / 2] = 0.0L;
    for (int i = 0; i <= p; ++i) {
        long double P, dP, d2P;
        if (i == 0 || i == p) {
            P = (i == 0 && (p % 2 == 1)) ? -1.0L : 1.0L;
        } else {
            legendre3(p, x[i], P, dP, d2P);
        }
        xi[i] = (double)x[i];
        w[i] = (double)(2.0L / (p * (p + 1.0L) * P * P));
    }
    return ESDC_OK;
}

// D_ij = P_p(x_i)/(P_p(x_j)(x_i - x_j)) for i != j, D_00 = -p(p+1)/4, D_pp = p(p+1)/4, else 0
// (the closed form of the LGL collocation derivative).  S = (Q - Q^T)/2 with Q = diag(w) D, so
// S is skew by construction and Q = S + E/2 (Definition 1, item 3).
int build_operators(int p, HostSetup& hs) {
    const int N = p + 1;
    hs.p = p;
    hs.N = N;
    hs.xi.assign(N, 0.0);
    hs.w.assign(N, 0.0);
    int st = lgl(p, hs.xi.data(), hs.w.data());
    if (st) return st;
    std::vector<long double> P(N);
    for (int i = 0; i < N; ++i) {
        long double a, b, c;
        if (i == 0) P[i] = (p % 2 == 1) ? -1.0L : 1.0L;
        else if (i == p) P[i] = 1.0L;
        else { legendre3(p, hs.xi[i], a, b, c); P[i] = a; }
    }
    hs.D.assign(N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            long double v;
            if (i != j) v = P[i] / (P[j] * ((long double)hs.xi[i] - (long double)hs.xi[j]));
            else if (i == 0) v = -p * (p + 1.0L) / 4.0L;
            else if (i == p) v = p * (p + 1.0L) / 4.0L;
            else v = 0.0L;
            hs.D[i * N + j] = (double)v;
        }
    hs.S.assign(N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            hs.S[i * N + j] = 0.5 * (hs.w[i] * hs.D[i * N + j] - hs.w[j] * hs.D[j * N + i]);
    return ESDC_OK;
}

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
// the state advances by the golden-ratio increment and is scrambled by two xor-shift-multiplies.
static uint64_t splitmix64(uint64_t& state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int generate_box_coords(const esdc_setup_t& s, const std::vector<double>& xi, std::vector<double>& xyz) {
    const int N = (int)xi.size(), N3 = N * N * N;
    const int k[3] = {s.kx, s.ky, s.kz};
    double L[3], h[3];
    for (int d = 0; d < 3; ++d) {
        L[d] = s.hi[d] - s.lo[d];
        if (!(L[d] > 0.0) || !std::isfinite(L[d])) return ESDC_ERR_ARG;
        h[d] = L[d] / k[d];
    }
    if (!(s.warp_amp >= 0.0) || !std::isfinite(s.warp_amp)) return ESDC_ERR_ARG;
    const double two_pi = 6.283185307179586476925286766559;
    double phi[3][3];
    uint64_t st = s.warp_seed;
    for (int i = 0; i < 3; ++i)
        for (int kk = 0; kk < 3; ++kk) phi[i][kk] = (double)(splitmix64(st) >> 11) * 0x1.0p-53 * two_pi;
    const int64_t K = (int64_t)s.kx * s.ky * s.kz;
    xyz.assign((size_t)K * 3 * N3, 0.0);
    for (int64_t e = 0; e < K; ++e) {
        const int64_t ei[3] = {e % s.kx, (e / s.kx) % s.ky, e / ((int64_t)s.kx * s.ky)};
        for (int n = 0; n < N3; ++n) {
            const int ix[3] = {n % N, (n / N) % N, n / (N * N)};
            double X[3];
            for (int d = 0; d < 3; ++d) X[d] = s.lo[d] + ((double)ei[d] + (xi[ix[d]] + 1.0) * 0.5) * h[d];
            for (int i = 0; i < 3; ++i) {
                double y = X[i];
                if (s.warp_amp != 0.0) {
                    double prod = 1.0;
                    for (int kk = 0; kk < 3; ++kk) prod *= std::sin(two_pi * (X[kk] - s.lo[kk]) / L[kk] + phi[i][kk]);
                    y = X[i] + s.warp_amp * h[i] * prod;
                }
                xyz[((size_t)e * 3 + i) * N3 + n] = y;
            }
        }
    }
    return ESDC_OK;
}

// bounded: bit l set -> the outer faces of direction l are boundaries (neighbour -1)
void build_box_neighbours(int kx, int ky, int kz, int bounded, std::vector<int32_t>& nbr) {
    const int64_t K = (int64_t)kx * ky * kz;
    nbr.assign(K * 6, 0);
    auto id = [&](int a, int b, int c) {
        a = (a % kx + kx) % kx;
        b = (b % ky + ky) % ky;
        c = (c % kz + kz) % kz;
        return (int32_t)(a + (int64_t)kx * (b + (int64_t)ky * c));
    };
    for (int64_t e = 0; e < K; ++e) {
        int ex = (int)(e % kx), ey = (int)((e / kx) % ky), ez = (int)(e / ((int64_t)kx * ky));
        int32_t* n = &nbr[e * 6];
        n[0] = id(ex - 1, ey, ez);
        n[1] = id(ex + 1, ey, ez);
        n[2] = id(ex, ey - 1, ez);
        n[3] = id(ex, ey + 1, ez);
        n[4] = id(ex, ey, ez - 1);
        n[5] = id(ex, ey, ez + 1);
        const int c[3] = {ex, ey, ez}, k[3] = {kx, ky, kz};
        for (int l = 0; l < 3; ++l)
            if (bounded & (1 << l)) {
                if (c[l] == 0) n[2 * l] = -1;
                if (c[l] == k[l] - 1) n[2 * l + 1] = -1;
            }
    }
}

namespace {

// Apply the N x N matrix M (row-major) along direction a (0: xi1 fastest) to a nodal field of one
// element: out_i = sum_j M_ij u_j on every line of direction a.
void apply_mat(const double* M, int N, int a, const double* u, double* out) {
    const int stride = (a == 0) ? 1 : (a == 1 ? N : N * N);
    for (int i3 = 0; i3 < N; ++i3)
        for (int i2 = 0; i2 < N; ++i2)
            for (int i1 = 0; i1 < N; ++i1) {
                const int node = (i3 * N + i2) * N + i1;
                const int ia = (a == 0) ? i1 : (a == 1 ? i2 : i3);
                const int base = node - ia * stride;
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += M[ia * N + j] * u[base + j * stride];
                out[node] = s;
            }
}

void apply_d(const std::vector<double>& D, int N, int a, const double* u, double* out) {
    apply_mat(D.data(), N, a, u, out);
}

// Geometry of one element: J and Ja_lm = J dxi_l/dx_m in conservative curl form,
// Ja[l][m] = -(curl_xi v)_l with v_j = X_{m+2} dX_{m+1}/dxi_j, (m, m+1, m+2) cyclic.
// Coordinates are taken relative to the element's first node (the curl form is invariant under
// translation; relative coordinates keep the products small).
bool element_geometry(const std::vector<double>& D, int N, const double* xyz, double* g) {
    const int N3 = N * N * N;
    std::vector<double> X(3 * N3), dX(9 * N3), v(3 * N3), t1(N3), t2(N3);
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < N3; ++n) X[m * N3 + n] = xyz[m * N3 + n] - xyz[m * N3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a) apply_d(D, N, a, &X[m * N3], &dX[(m * 3 + a) * N3]);
    bool ok = true;
    for (int n = 0; n < N3; ++n) {
        auto F = [&](int m, int a) { return dX[(m * 3 + a) * N3 + n]; };
        double J = F(0, 0) * (F(1, 1) * F(2, 2) - F(1, 2) * F(2, 1))
                 - F(0, 1) * (F(1, 0) * F(2, 2) - F(1, 2) * F(2, 0))
                 + F(0, 2) * (F(1, 0) * F(2, 1) - F(1, 1) * F(2, 0));
        g[n] = J;
        if (!(J > 0.0) || !std::isfinite(J)) ok = false;
    }
    for (int m = 0; m < 3; ++m) {
        const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
        for (int j = 0; j < 3; ++j)
            for (int n = 0; n < N3; ++n) v[j * N3 + n] = X[m2 * N3 + n] * dX[(m1 * 3 + j) * N3 + n];
        // l = 0: D_2 v_3 - D_3 v_2 ; l = 1: D_3 v_1 - D_1 v_3 ; l = 2: D_1 v_2 - D_2 v_1 (1-based)
        const int pa[3][2] = {{1, 2}, {2, 0}, {0, 1}};   // (derivative dir of first term, of second term)
        const int pv[3][2] = {{2, 1}, {0, 2}, {1, 0}};   // (component of first term, of second term)
        for (int l = 0; l < 3; ++l) {
            apply_d(D, N, pa[l][0], &v[pv[l][0] * N3], t1.data());
            apply_d(D, N, pa[l][1], &v[pv[l][1] * N3], t2.data());
            double* dst = g + (1 + l * 3 + m) * N3;
            for (int n = 0; n < N3; ++n) {
                dst[n] = -(t1[n] - t2[n]);
                if (!std::isfinite(dst[n])) ok = false;
            }
        }
    }
    return ok;
}

// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic Jacobi rotations (Golub and
// Van Loan, Matrix Computations, Sec. 8.5): A = U diag(lam) U^T with U orthogonal, eigenvectors in
// its columns.
void sym_eigen(int n, std::vector<double> A, std::vector<double>& U, std::vector<double>& lam) {
    U.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) U[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) (i == j ? diag : off) += A[i * n + j] * A[i * n + j];
        if (off <= 1e-34 * (diag + off)) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                // rotation angle phi with cot(2 phi) = theta zeroes A_pq
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = std::fabs(theta) > 1e150
                                     ? 0.5 / theta
                                     : std::copysign(1.0, theta) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {     // A <- A J
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {     // A <- J^T A
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {     // U <- U J
                    const double ukp = U[k * n + p], ukq = U[k * n + q];
                    U[k * n + p] = c * ukp - sn * ukq;
                    U[k * n + q] = sn * ukp + c * ukq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

// Fast diagonalisation (Lynch, Rice and Thomas, Numer. Math. 6, 1964) of the Gram matrix
// G = sum_l Q_l^T Q_l of the tensor-product SBP matrices Q_l = P (x) P (x) Q along xi_l: with
// A = Q^T Q and the generalised eigenvectors A V = P^2 V diag(lam), V^T P^2 V = I, the matrix
// W = V (x) V (x) V gives W^T G W = diag(lam_k1 + lam_k2 + lam_k3).  G is singular (G 1 = 0; the
// mode k1 = k2 = k3 = k0 of the zero eigenvalue lam_k0, whose eigenvector is constant); for r
// orthogonal to 1 the solution y = W diag(1/(lam_k1 + lam_k2 + lam_k3), 0 at the null mode) W^T r
// satisfies G y = r.
struct FastDiag {
    int N = 0, k0 = 0;
    std::vector<double> V, Vt, lam;   // V[i][k], its transpose, eigenvalues
};

FastDiag make_fast_diag(const HostSetup& hs) {
    const int N = hs.N;
    std::vector<double> Q(N * N), B(N * N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) Q[i * N + j] = hs.w[i] * hs.D[i * N + j];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double a = 0.0;
            for (int k = 0; k < N; ++k) a += Q[k * N + i] * Q[k * N + j];
            B[i * N + j] = a / (hs.w[i] * hs.w[j]);          // P^-1 A P^-1, symmetric
        }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < i; ++j) B[i * N + j] = B[j * N + i] = 0.5 * (B[i * N + j] + B[j * N + i]);
    FastDiag fd;
    fd.N = N;
    std::vector<double> U;
    sym_eigen(N, B, U, fd.lam);
    fd.V.resize(N * N);
    fd.Vt.resize(N * N);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < N; ++k) {
            fd.V[i * N + k] = U[i * N + k] / hs.w[i];
            fd.Vt[k * N + i] = fd.V[i * N + k];
        }
    fd.k0 = (int)(std::min_element(fd.lam.begin(), fd.lam.end()) - fd.lam.begin());
    return fd;
}

// Optimized metrics of one element (Sec. 3).  t_lm = (dx/dxi_a x dx/dxi_b)_m, (l, a, b) cyclic, are
// the analytic (cofactor) metrics of the interpolated mapping; their face values are the surface
// metrics, written to ns[6][3][N^2].  For each m the volume metrics are the Euclidean-nearest a_m to
// t_m with M a_m = b_m, M = [Q_1^T Q_2^T Q_3^T], b_m = sum_l E_l t_lm.  The minimiser is
// a_m = t_m + M^T y with G y = b_m - M t_m, G = M M^T; since Q_l + Q_l^T = E_l the right-hand side is
// sum_l Q_l t_lm = P3 sum_l D_l t_lm (P3 the tensor weights), and (M^T y)_l = Q_l y = P3 D_l y.
// g: [10][N^3] as element_geometry (J, then a_lm l-major).
bool element_geometry_optimized(const HostSetup& hs, const FastDiag& fd, const double* xyz, double* g, double* ns) {
    const int N = hs.N, N2 = N * N, N3 = N2 * N;
    const std::vector<double>& D = hs.D;
    std::vector<double> X(3 * N3), dX(9 * N3), t(9 * N3), r(N3), z(N3), y(N3), tmp(N3), W3(N3);
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < N3; ++n) X[m * N3 + n] = xyz[m * N3 + n] - xyz[m * N3];
    for (int m = 0; m < 3; ++m)
        for (int a = 0; a < 3; ++a) apply_d(D, N, a, &X[m * N3], &dX[(m * 3 + a) * N3]);
    for (int n = 0; n < N3; ++n) W3[n] = hs.w[n % N] * hs.w[(n / N) % N] * hs.w[n / N2];
    bool ok = true;
    auto F = [&](int m, int a, int n) { return dX[(m * 3 + a) * N3 + n]; };
    for (int n = 0; n < N3; ++n) {
        const double J = F(0, 0, n) * (F(1, 1, n) * F(2, 2, n) - F(1, 2, n) * F(2, 1, n))
                       - F(0, 1, n) * (F(1, 0, n) * F(2, 2, n) - F(1, 2, n) * F(2, 0, n))
                       + F(0, 2, n) * (F(1, 0, n) * F(2, 1, n) - F(1, 1, n) * F(2, 0, n));
        g[n] = J;
        if (!(J > 0.0) || !std::isfinite(J)) ok = false;
    }
    for (int l = 0; l < 3; ++l) {
        const int a = (l + 1) % 3, b = (l + 2) % 3;
        for (int m = 0; m < 3; ++m) {
            const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
            for (int n = 0; n < N3; ++n)
                t[(l * 3 + m) * N3 + n] = F(m1, a, n) * F(m2, b, n) - F(m2, a, n) * F(m1, b, n);
        }
    }
    // surface metrics: row l of t on the two faces of direction l
    for (int l = 0; l < 3; ++l)
        for (int side = 0; side < 2; ++side) {
            const int fix = side ? N - 1 : 0;
            for (int t2 = 0; t2 < N; ++t2)
                for (int t1 = 0; t1 < N; ++t1) {
                    const int node = l == 0 ? fix + N * t1 + N2 * t2 : (l == 1 ? t1 + N * fix + N2 * t2 : t1 + N * t2 + N2 * fix);
                    for (int m = 0; m < 3; ++m) ns[((2 * l + side) * 3 + m) * N2 + t1 + N * t2] = t[(l * 3 + m) * N3 + node];
                }
        }
    for (int m = 0; m < 3; ++m) {
        std::fill(r.begin(), r.end(), 0.0);
        for (int l = 0; l < 3; ++l) {
            apply_d(D, N, l, &t[(l * 3 + m) * N3], tmp.data());
            for (int n = 0; n < N3; ++n) r[n] += tmp[n];
        }
        for (int n = 0; n < N3; ++n) r[n] *= W3[n];
        // y = W diag(1/Lambda) W^T r
        apply_mat(fd.Vt.data(), N, 0, r.data(), z.data());
        apply_mat(fd.Vt.data(), N, 1, z.data(), tmp.data());
        apply_mat(fd.Vt.data(), N, 2, tmp.data(), z.data());
        for (int k3 = 0; k3 < N; ++k3)
            for (int k2 = 0; k2 < N; ++k2)
                for (int k1 = 0; k1 < N; ++k1) {
                    const int k = (k3 * N + k2) * N + k1;
                    if (k1 == fd.k0 && k2 == fd.k0 && k3 == fd.k0) z[k] = 0.0;
                    else z[k] /= fd.lam[k1] + fd.lam[k2] + fd.lam[k3];
                }
        apply_mat(fd.V.data(), N, 0, z.data(), tmp.data());
        apply_mat(fd.V.data(), N, 1, tmp.data(), z.data());
        apply_mat(fd.V.data(), N, 2, z.data(), y.data());
        for (int l = 0; l < 3; ++l) {
            apply_d(D, N, l, y.data(), tmp.data());
            double* dst = g + (1 + l * 3 + m) * N3;
            for (int n = 0; n < N3; ++n) {
                dst[n] = t[(l * 3 + m) * N3 + n] + W3[n] * tmp[n];
                if (!std::isfinite(dst[n])) ok = false;
            }
        }
    }
    return ok;
}

double element_min_edge(int N, const double* xyz) {
    const int N3 = N * N * N;
    auto corner = [&](int i3, int i2, int i1, int m) { return xyz[m * N3 + (i3 * N + i2) * N + i1]; };
    const int e[2] = {0, N - 1};
    double best = 1e300;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int A = e[a], B = e[b];
            const int ends[3][2][3] = {{{A, B, 0}, {A, B, N - 1}}, {{A, 0, B}, {A, N - 1, B}}, {{0, A, B}, {N - 1, A, B}}};
            for (int d = 0; d < 3; ++d) {
                double s = 0.0;
                for (int m = 0; m < 3; ++m) {
                    double diff = corner(ends[d][0][0], ends[d][0][1], ends[d][0][2], m)
                                - corner(ends[d][1][0], ends[d][1][1], ends[d][1][2], m);
                    s += diff * diff;
                }
                best = std::min(best, std::sqrt(s));
            }
        }
    return best;
}

}  // namespace

int build_geometry(const esdc_setup_t& s, const double* xyz, HostSetup& hs, std::string& err) {
    const int N = hs.N, N3 = N * N * N, N2 = N * N;
    const int64_t K = (int64_t)s.kx * s.ky * s.kz;
    hs.geom.assign((size_t)K * 10 * N3, 0.0);
    const bool opt = s.metrics == ESDC_METRICS_OPTIMIZED;
    FastDiag fd;
    if (opt) {
        hs.nsurf.assign((size_t)K * 6 * 3 * N2, 0.0);
        fd = make_fast_diag(hs);
    } else {
        hs.nsurf.clear();
    }
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (K < 64) nt = 1;
    std::vector<int> bad(nt, 0);
    std::vector<double> hmin(nt, 1e300);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            for (int64_t e = t; e < K; e += nt) {
                const double* x = xyz + (size_t)e * 3 * N3;
                const bool good = opt ? element_geometry_optimized(hs, fd, x, &hs.geom[(size_t)e * 10 * N3],
                                                                   &hs.nsurf[(size_t)e * 6 * 3 * N2])
                                      : element_geometry(hs.D, N, x, &hs.geom[(size_t)e * 10 * N3]);
                if (!good) bad[t] = 1;
                hmin[t] = std::min(hmin[t], element_min_edge(N, x));
            }
        });
    }
    for (auto& x : th) x.join();
    for (unsigned t = 0; t < nt; ++t)
        if (bad[t]) {
            err = "metric Jacobian J <= 0 or non-finite geometry in the node coordinates";
            return ESDC_ERR_MESH;
        }
    hs.h_min = *std::min_element(hmin.begin(), hmin.end());
    if (!(hs.h_min > 0.0)) {
        err = "degenerate element edge";
        return ESDC_ERR_MESH;
    }
    build_box_neighbours(s.kx, s.ky, s.kz, s.bounded, hs.nbr);
    return ESDC_OK;
}

// Manufactured solution of Sec. 5.1 (eq. mms) and its source div(F^I - F^V).  Every field is
// phi0 + sum_k A_k trig_k(c_k x_k) with c_k = alpha_k pi / L, so all first and second derivatives are
// analytic and the mixed second derivatives vanish; the divergence of tau_ij then reduces to
// mu (sum_j d_jj u_i + d_ii u_i / 3).
void mms_fields(double gamma, double Ma, double Re, double Pr, double L, const double* table, int64_t n,
                const double* x, double* q, double* src) {
    static const int kind[5][3] = {{0, 1, 0}, {0, 1, 1}, {1, 0, 0}, {0, 0, 1}, {0, 0, 1}};   // 0 sin, 1 cos
    const double R = 1.0 / (gamma * Ma * Ma);
    const double mu = Re > 0.0 ? 1.0 / Re : 0.0;
    const double kappa = mu * gamma * R / ((gamma - 1.0) * Pr);
    const double pi = 3.14159265358979323846;
    for (int64_t i = 0; i < n; ++i) {
        double val[5], d[5][3], dd[5][3];
        for (int f = 0; f < 5; ++f) {
            const double* row = table + 7 * f;
            val[f] = row[0];
            for (int k = 0; k < 3; ++k) {
                const double c = row[4 + k] * pi / L;
                const double arg = c * x[3 * i + k];
                const double sn = std::sin(arg), cs = std::cos(arg);
                const double A = row[1 + k];
                if (kind[f][k] == 0) {
                    val[f] += A * sn;
                    d[f][k] = A * c * cs;
                    dd[f][k] = -A * c * c * sn;
                } else {
                    val[f] += A * cs;
                    d[f][k] = -A * c * sn;
                    dd[f][k] = -A * c * c * cs;
                }
            }
        }
        const double rho = val[0], u[3] = {val[1], val[2], val[3]}, p = val[4];
        const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double rE = p / (gamma - 1.0) + 0.5 * rho * usq;
        if (q) {
            double* o = q + 5 * i;
            o[0] = rho;
            for (int k = 0; k < 3; ++k) o[1 + k] = rho * u[k];
            o[4] = rE;
        }
        if (!src) continue;
        // du[a][m] = d u_a / d x_m
        double du[3][3], div = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int m = 0; m < 3; ++m) du[a][m] = d[1 + a][m];
        for (int m = 0; m < 3; ++m) div += du[m][m];
        // inviscid divergence
        double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int m = 0; m < 3; ++m) {
            s[0] += d[0][m] * u[m] + rho * du[m][m];
            const double dH = gamma / (gamma - 1.0) * d[4][m] + 0.5 * d[0][m] * usq +
                              rho * (u[0] * du[0][m] + u[1] * du[1][m] + u[2] * du[2][m]);
            s[4] += du[m][m] * (rE + p) + u[m] * dH;
        }
        for (int a = 0; a < 3; ++a) {
            double t = d[4][a];
            for (int m = 0; m < 3; ++m) t += d[0][m] * u[m] * u[a] + rho * du[m][m] * u[a] + rho * u[m] * du[a][m];
            s[1 + a] = t;
        }
        // viscous divergence
        double tau[3][3], dtau[3];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) tau[a][b] = mu * (du[a][b] + du[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
            dtau[a] = mu * (dd[1 + a][0] + dd[1 + a][1] + dd[1 + a][2] + dd[1 + a][a] / 3.0);
        }
        double ven = 0.0, lapT = 0.0;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) ven += du[a][b] * tau[a][b];
            ven += u[a] * dtau[a];
        }
        for (int m = 0; m < 3; ++m)
            lapT += (dd[4][m] / rho - 2.0 * d[4][m] * d[0][m] / (rho * rho) - p * dd[0][m] / (rho * rho) +
                     2.0 * p * d[0][m] * d[0][m] / (rho * rho * rho)) / R;
        ven += kappa * lapT;
        double* o = src + 5 * i;
        o[0] = s[0];
        for (int a = 0; a < 3; ++a) o[1 + a] = s[1 + a] - dtau[a];
        o[4] = s[4] - ven;
    }
}

}  // namespace esdc
