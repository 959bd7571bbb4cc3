// Internal declarations shared by the host setup, the kernels and the C ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/esdc.h"

namespace esdc {

constexpr int kMaxN = 8;     // p <= 7: one element per CTA (rhs_f64.cu, rhs_f32.cu, the adjoint)
constexpr int kLargeN = 16;  // p = 15: the multi-pass float64 residual (rhs_large_f64.cu)

// Per-degree operators passed by value to kernels (lands in the constant bank).
struct Ops {
    int N;
    double D[kMaxN][kMaxN];    // collocation derivative D = P^-1 Q (Sec. 2, Definition 1)
    double SW[kMaxN][kMaxN];   // S_ij / w_j with S = Q - E/2 skew-symmetric (the adjoint's pair weights)
    double S[kMaxN][kMaxN];    // S itself (the pair coefficient of the forward kernels)
    double w[kLargeN];         // LGL weights (diagonal of P), every supported degree
    double winv[kLargeN];      // 1/w
};

// The same operators for N = kLargeN (the p = 15 residual passes).
struct OpsL {
    int N;
    double D[kLargeN][kLargeN];
    double S[kLargeN][kLargeN];
    double w[kLargeN];
    double winv[kLargeN];
};

struct Phys {
    double gamma, R, mu, kappa;
    double inv_gm1;            // 1/(gamma-1)
    double ip_coef;            // interior-penalty coefficient (0: off)
    int dissipation;           // 0 none, 1 local Lax-Friedrichs, 2 matrix
    int viscous;               // mu > 0
};

// A float32 pair, 8-byte aligned: one 64-bit operand of the packed (f32x2) instructions.
struct alignas(8) FPair {
    float x, y;
};

// FP32 copies used by the mixed-precision kernels.
struct OpsF {
    int N;
    float D[kMaxN][kMaxN];
    float S[kMaxN][kMaxN];
    float w[kMaxN];
    float winv[kMaxN];
    float ST[kMaxN][kMaxN];    // S transposed: ST[i][j] = S[j][i] = -S[i][j]
    FPair D2[kMaxN][kMaxN];    // (D[i][j], D[i][j]): D as a packed operand of both lanes
};

struct PhysF {
    float gamma, R, mu, kappa, inv_gm1;
    float rho0, p0;            // reference state subtracted in the FP32 kernels
    int dissipation, viscous;
};

// Host-side results of setup (float64).
struct HostSetup {
    int p = 0, N = 0;
    std::vector<double> xi, w;           // LGL nodes / weights
    std::vector<double> D;               // N*N row-major
    std::vector<double> S;               // N*N row-major, exactly skew
    std::vector<double> geom;            // [K][10][N^3]: J, Ja_lm (l-major)
    std::vector<double> nsurf;           // [K][6][3][N^2] surface metrics (optimized metrics only)
    std::vector<int32_t> nbr;            // [K][6]
    double h_min = 0.0;
};

int lgl(int p, double* xi, double* w);
int build_operators(int p, HostSetup& hs);
int build_geometry(const esdc_setup_t& s, const double* xyz, HostSetup& hs, std::string& err);
void build_box_neighbours(int kx, int ky, int kz, int bounded, std::vector<int32_t>& nbr);
// node coordinates of the box mesh generator (setup lo, hi, warp_amp, warp_seed) on the LGL nodes xi
int generate_box_coords(const esdc_setup_t& s, const std::vector<double>& xi, std::vector<double>& xyz);
// manufactured solution (q, nullable) and its source div(F^I - F^V) (src, nullable) at n points (host)
void mms_fields(double gamma, double Ma, double Re, double Pr, double L, const double* table, int64_t n,
                const double* x, double* q, double* src);
void set_last_error(const std::string& msg);   // message returned by esdc_last_error on this thread
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, looked up once per
// device); grid-stride launches are capped at grid_cap() = 16 CTAs per SM.
int sm_count();
inline long long grid_cap() { return 16LL * sm_count(); }

}  // namespace esdc

struct esdc_ctx {
    esdc_setup_t setup;
    int device = 0;
    int N = 0, N3 = 0;
    int64_t K = 0, n_nodes = 0;
    esdc::Ops ops;
    esdc::OpsL opsl;                 // filled for N = kLargeN only
    esdc::OpsF opsf;
    esdc::Phys phys;
    esdc::PhysF physf;
    double h_min = 0.0;
    // device buffers owned by the library
    double* d_geom = nullptr;        // [K][10][N3]
    double* d_jinv = nullptr;        // [K][N3] 1/J
    double* d_xyz = nullptr;         // [K][3][N3] node coordinates (initial states)
    double* d_fnorm = nullptr;       // [K][6][N2] |n_J| of the interface metric at the face nodes
    double* d_nsurf = nullptr;       // [K][6][3][N2] surface metrics of the optimized metrics (else null)
    // p = 15 residual passes (N = kLargeN only)
    double* d_lr = nullptr;          // [3][K][5][N3] per-direction residual parts
    double* d_lwf = nullptr;         // [K][6][4][N2] neighbour entropy variables at the faces
    double* d_lft = nullptr;         // [K][3][4][N3] contravariant viscous fluxes
    const double* d_qext = nullptr;  // caller-owned exterior (Dirichlet) state, [K][5][N3] (bounded boxes)
    const double* d_src = nullptr;   // caller-owned source term added to dq/dt, [K][5][N3]
    float* d_geomf = nullptr;        // [K][10][N3] float32 copy (mixed precision)
    float* d_nsurff = nullptr;       // [K][6][3][N2] float32 copy of the surface metrics (mixed precision)
    int32_t* d_nbr = nullptr;        // [K][6]
    void* d_trace = nullptr;         // [K][6][4][N2] viscous normal-flux traces (f64 or f32)
    float* d_shadow = nullptr;       // [K][5][N3] float32 perturbation state (mixed precision)
    double* d_red = nullptr;         // reduction partials
    double* d_red_out = nullptr;     // reduction results
    double* d_lntab = nullptr;       // [128][3] logarithm table of the budgets (T_k, -ln T_k head, tail)
    int* d_status = nullptr;         // device status bits (kStatusBulkWait), read by esdc_device_status
    int red_blocks = 0;
    // adjoint buffers, allocated on the first vector-Jacobian product
    double* d_adj_g = nullptr;       // [K][6][5][N2] interface cotangents for the neighbour
    double* d_adj_t = nullptr;       // [K][6][4][N2] lifted-gradient cotangents for the neighbour
    double* d_adj_mu = nullptr;      // per-block partial sums of lambda . R_visc
    double* d_adj_acc = nullptr;     // accumulated d/dmu
    // one DP5 step captured as a CUDA graph, replayed by multi-step esdc_rk_step calls; valid for
    // the recorded state, workspace, step size and optional-term pointers
    void* graph_exec = nullptr;      // cudaGraphExec_t
    void* capture_stream = nullptr;  // cudaStream_t (private, non-blocking) used only for capture
    const void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double graph_dt = 0.0;
    // CUDA-event profiling of the residual kernels (esdc_profile)
    int profiling = 0;
    std::vector<void*> prof_events;  // cudaEvent_t quadruples: main start/stop, face start/stop
    size_t prof_used = 0;
    // staging for esdc_rhs_host
    double* d_stage_q = nullptr;
    void* d_stage_r = nullptr;
};
