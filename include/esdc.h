/*
 * esdc.h -- C ABI of the GB300 entropy-stable discontinuous collocation (ES-C) residual library.
 *
 * The library evaluates the semi-discrete residual of the compressible Navier-Stokes equations on
 * conforming hexahedral meshes with Legendre-Gauss-Lobatto (LGL) collocation (arXiv 1911.10966,
 * Sec. 4, eq. NSL): Chandrashekar flux differencing (eq. discEL), entropy-variable BR1 viscous
 * terms (eq. MacroForm), entropy-stable interface SATs and curvilinear metric terms (Sec. 3), and
 * advances it with the Dormand-Prince 5(4) explicit Runge-Kutta scheme (Sec. 5), at a fixed step or
 * with an adaptive step (esdc_rk_adaptive).
 *
 * Conventions for every entry point:
 *   - Return value: ESDC_OK (0) or a negative ESDC_ERR_* code; esdc_last_error() gives a message
 *     for the calling thread.  No C++ exception crosses this boundary and no kernel traps.
 *   - "dev" pointers are CUDA device pointers owned by the CALLER; "host" pointers are ordinary
 *     host memory owned by the caller.  The library owns its context, operators, geometry, face
 *     trace buffers and small reduction scratch (allocated in esdc_create, freed in esdc_destroy).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls enqueue work
 *     asynchronously on it unless stated otherwise.
 *   - State layout: q[K][5][N][N][N] float64, variable order (rho, rho u1, rho u2, rho u3, rho E),
 *     node index (i3*N + i2)*N + i1 (xi1 fastest).  N = p + 1.  One element is one contiguous
 *     5*N^3 block.  Element e of a kx*ky*kz box is e = ex + kx*(ey + ky*ez).
 *   - Nondimensionalisation: rho_inf = T_inf = 1, R = 1/(gamma Ma^2), mu = 1/Re, kappa = mu cp/Pr.
 */
#ifndef ESDC_H
#define ESDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESDC_OK 0
#define ESDC_ERR_ARG (-1)         /* bad argument, shape, null pointer or size                  */
#define ESDC_ERR_MESH (-2)        /* non-positive or non-finite metric Jacobian at setup        */
#define ESDC_ERR_CUDA (-3)        /* a CUDA runtime call failed                                 */
#define ESDC_ERR_STATE (-4)       /* non-finite or non-physical state found by a reduction      */
#define ESDC_ERR_UNSUPPORTED (-5) /* valid request this build does not implement                */

#define ESDC_PREC_FP64 0          /* whole residual in float64                                  */
#define ESDC_PREC_FP32 1          /* residual arithmetic in float32, state/RK/budgets float64   */

/* Volume-flux variants (Sec. 4).  ESDC_FLUX_ESC: the entropy-stable collocation of the paper
 * (Chandrashekar two-point flux, eq. discEL).  ESDC_FLUX_KG: the same Hadamard flux differencing with
 * the Kennedy-Gruber two-point flux (the paper's SF-KG).  ESDC_FLUX_DC: standard collocation, D
 * applied to the nodal contravariant Euler fluxes (the paper's DC), with the central interface flux.
 * All three use the same interface dissipation, viscous terms and metrics; ESC and KG also run in
 * the float32-mixed form, DC is float64 only (ESDC_ERR_UNSUPPORTED); all three have an adjoint. */
/* Interface dissipation of SAT^(I) (the paper defers the SAT to its references).  ESDC_DISS_NONE:
 * entropy conservative.  ESDC_DISS_LLF: local Lax-Friedrichs, lambda/2 (q_own - q_nbr) with
 * lambda = max over both sides of |u.n_J| + c |n_J|.  ESDC_DISS_MATRIX: Roe-type entropy-stable
 * matrix dissipation D (w_own - w_nbr)/2, D = R |Lambda| R^T at the averaged state (log-mean
 * density, mean velocity, p = rho_bar/(2 beta_bar)) with eigenvectors scaled so that R R^T = dq/dw;
 * float64 only (ESDC_ERR_UNSUPPORTED for float32); the adjoint supports it. */
#define ESDC_DISS_NONE 0
#define ESDC_DISS_LLF 1
#define ESDC_DISS_MATRIX 2

#define ESDC_FLUX_ESC 0
#define ESDC_FLUX_KG 1
#define ESDC_FLUX_DC 2

typedef struct esdc_ctx esdc_ctx; /* opaque, library owned */

/* Problem description: a kx*ky*kz structured box of hexahedra, periodic in every direction except
 * those flagged in `bounded` (Dirichlet data on their outer faces). */
typedef struct esdc_setup {
    int p;                  /* polynomial degree, 1 <= p <= 7 or p = 15 (N = p + 1 LGL nodes per
                               direction; p = 15 below)                                             */
    int kx, ky, kz;         /* elements per direction, each >= 1                                  */
    double gamma;           /* ratio of specific heats (> 1)                                      */
    double Pr;              /* Prandtl number (> 0)                                               */
    double Ma;              /* reference Mach number (> 0): sets R = 1/(gamma Ma^2)                */
    double Re;              /* Reynolds number; Re <= 0 means inviscid (mu = 0)                   */
    int dissipation;        /* ESDC_DISS_NONE, ESDC_DISS_LLF or ESDC_DISS_MATRIX (below)          */
    int precision;          /* ESDC_PREC_FP64 or ESDC_PREC_FP32                                   */
    int volume_flux;        /* ESDC_FLUX_ESC (the method), ESDC_FLUX_KG or ESDC_FLUX_DC           */
    double ip_coef;         /* interior-penalty coefficient sigma >= 0 (0: off; below)             */
    int bounded;            /* bit l (l = 0, 1, 2) set: the outer faces normal to xi_l are
                               boundaries with Dirichlet data (esdc_set_exterior); 0: periodic      */
    int metrics;            /* ESDC_METRICS_CURL (0) or ESDC_METRICS_OPTIMIZED (1), below          */
    /* box mesh generator, used when esdc_create / esdc_host_* get node_xyz = NULL (below) */
    double lo[3], hi[3];    /* box corners, hi > lo                                               */
    double warp_amp;        /* sinusoidal warp amplitude as a fraction of the element size (>= 0) */
    uint64_t warp_seed;     /* seed of the nine warp phases                                        */
} esdc_setup_t;

/* Box mesh generator (node_xyz = NULL): element e = ex + kx (ey + ky ez) spans
 * [lo + (ex, ey, ez) h, lo + (ex + 1, ey + 1, ez + 1) h], h = (hi - lo)/(kx, ky, kz), with the tensor
 * LGL nodes mapped affinely, then displaced in component i by
 *   warp_amp h_i prod_k sin(2 pi (X_k - lo_k)/L_k + phi_ik),   L = hi - lo,
 * which is L-periodic in every direction, so shared and periodic faces keep identical nodes.  The
 * phases phi_ik (i-major) are successive outputs of splitmix64 (Steele, Lea and Flood, OOPSLA 2014)
 * started from warp_seed, each mapped to [0, 2 pi) as (z >> 11) 2^-53 2 pi.  With warp_amp = 0 the
 * mesh is affine and the seed is unused. */

/* Metric terms (Sec. 3).  ESDC_METRICS_CURL: the conservative curl form of the degree-p interpolant
 * of the mapping at every node; it satisfies the discrete GCL sum_l D_l Ja_lm = 0 exactly and the
 * interface terms use its face values.  ESDC_METRICS_OPTIMIZED: the paper's optimized metrics.  The
 * surface metrics are analytic: row l of the cofactor matrix of dx/dxi of the interpolated mapping
 * (dx/dxi_a x dx/dxi_b with (l, a, b) cyclic) at the face nodes of direction l, which depends only on
 * the face's nodes and so is the same from both sides.  The volume metrics are, for each m, the
 * Euclidean-nearest values to the cofactor metrics at all nodes that satisfy the discrete GCL with
 * those surface metrics, sum_l Q_l^T Ja_lm = sum_l E_l Ja^surf_lm (Q_l, E_l the tensor-product SBP
 * matrices; the condition under which the skew flux differencing keeps a uniform flow).  The
 * interface SAT (two-point flux, dissipation, interior penalty) then reads the surface metrics; the
 * volume and viscous terms read the volume metrics.  Float64 and float32-mixed; the adjoint
 * supports them. */
#define ESDC_METRICS_CURL 0
#define ESDC_METRICS_OPTIMIZED 1

/* Degree p = 15 (the top degree of the paper's cost comparison, Sec. 5.2): the float64 residual is
 * built in several passes instead of one CTA per element.  Built for periodic boxes with the curl-form
 * metrics, the three volume fluxes and ESDC_DISS_NONE or ESDC_DISS_LLF, viscous or inviscid; float32,
 * matrix dissipation, interior penalty, boundaries, optimized metrics, the adjoint and
 * esdc_budgets_noalloc are refused (ESDC_ERR_UNSUPPORTED, or ESDC_ERR_ARG for the last).  Degrees
 * 8 to 14 are refused with ESDC_ERR_UNSUPPORTED. */

/* Interior penalty (the IP term of eq. NSL; its constants are in the paper's references).  With
 * ip_coef = sigma > 0 and mu > 0, every face node adds -(1/P_ii) sigma mu |n_J| / h dq/dw (w_own -
 * w_nbr), with dq/dw at the averaged state of ESDC_DISS_MATRIX and h = (J_own + J_nbr)/|n_J|; the
 * term is symmetric in the two sides, conserves, and produces entropy.  Float64 only; the adjoint
 * supports it (the term is linear in mu, so it enters lambda . dR/dmu). */

/*
 * esdc_lgl -- the N = p+1 LGL nodes xi[N] (ascending on [-1, 1]) and quadrature weights w[N]
 * (Sec. 2, Definition 1: the norm matrix P = diag(w) of the SBP operator).  Host only, no GPU.
 * xi, w: host arrays of N doubles, caller owned.  Errors: ESDC_ERR_ARG for p outside [1, 15] or NULL.
 */
int esdc_lgl(int p, double* xi_host, double* w_host);

/*
 * esdc_operators -- host copies of the library's degree-p SBP operator (Sec. 2, Definition 1):
 * D[N*N] = P^-1 Q (row-major, D[i*N+j]) and S[N*N] = (Q - Q^T)/2, the skew part with Q = S + E/2.
 * Host only, no GPU.  Either output may be NULL.  Errors: ESDC_ERR_ARG.
 */
int esdc_operators(int p, double* D_host, double* S_host);

/*
 * esdc_host_geometry -- the metric terms esdc_create would build, computed on the host without a
 * GPU: J_host[K][N^3], Ja_host[K][9][N^3] (entry l*3 + m = J dxi_l/dx_m: the volume metrics of
 * setup->metrics, Sec. 3) and the smallest element edge h_min.  Any output may be NULL.
 * Errors: ESDC_ERR_ARG, ESDC_ERR_MESH (J <= 0 or non-finite).
 */
int esdc_host_geometry(const esdc_setup_t* setup, const double* node_xyz_host, double* J_host,
                       double* Ja_host, double* h_min);

/*
 * esdc_host_surface_metrics -- the metrics the interface terms read at the face nodes, computed on
 * the host without a GPU (Sec. 3): nsurf_host[K][6][3][N^2], face f = 2 l + side (side 0: xi_l = -1),
 * component m = 0..2 of Ja_l. at face node t1 + N t2, where (t1, t2) are the node's indices in the
 * two other directions in increasing direction order.  ESDC_METRICS_OPTIMIZED: the analytic
 * (cofactor) surface metrics; ESDC_METRICS_CURL: the face values of the curl-form volume metrics.
 * Errors: ESDC_ERR_ARG (NULL pointers), ESDC_ERR_MESH.
 */
int esdc_host_surface_metrics(const esdc_setup_t* setup, const double* node_xyz_host, double* nsurf_host);

/*
 * esdc_host_coordinates -- the node coordinates of the box mesh generator (node_xyz = NULL) for
 * setup, xyz_host[K][3][N][N][N], computed on the host without a GPU.  esdc_host_geometry and
 * esdc_host_surface_metrics also accept node_xyz_host = NULL for the same mesh.
 * Errors: ESDC_ERR_ARG (NULL output, hi <= lo, negative or non-finite warp_amp).
 */
int esdc_host_coordinates(const esdc_setup_t* setup, double* xyz_host);

/*
 * esdc_create -- build operators and geometry and allocate library buffers on the current device.
 * node_xyz_host: [K][3][N][N][N] float64 node coordinates (component-major per element), the
 *   degree-p mapping X of every element (Sec. 2, eq. 3d_mapping) sampled at the tensor LGL nodes;
 *   faces shared by neighbours (including periodic images) must hold the same nodes (Assumption 1).
 *   NULL: the box mesh generator above (setup->lo, hi, warp_amp, warp_seed).
 * Metric terms J dxi_l/dx_m are built on the host in float64 in conservative curl form, which
 * meets the discrete GCL (Sec. 3, eq. discGCLconvection), and J = det(dx/dxi).
 * Synchronous.  Errors: ESDC_ERR_ARG, ESDC_ERR_MESH (J <= 0 or non-finite), ESDC_ERR_CUDA.
 */
int esdc_create(const esdc_setup_t* setup, const double* node_xyz_host, esdc_ctx** out);

/* esdc_destroy -- free everything the context owns (synchronises the device).  NULL is a no-op. */
int esdc_destroy(esdc_ctx* ctx);

/* esdc_layout -- K elements, N nodes per direction, n_nodes = K*N^3.  Any output may be NULL. */
int esdc_layout(const esdc_ctx* ctx, int64_t* K, int* N, int64_t* n_nodes);

/*
 * esdc_geometry -- copy the float64 geometry to host arrays: J_host[K][N^3] and
 * Ja_host[K][9][N^3] with entry (l*3 + m) = J dxi_l/dx_m (Sec. 3).  Either may be NULL.  Synchronous.
 */
int esdc_geometry(const esdc_ctx* ctx, double* J_host, double* Ja_host);

/*
 * esdc_init_state -- write an initial state at the node coordinates given to esdc_create into
 * q_dev[K][5][N^3] (float64 device memory, caller owned), in the library's nondimensionalisation
 * (rho_inf = T_inf = 1, R = 1/(gamma Ma^2), gamma and Ma of the setup).  Asynchronous on stream.
 *   ESDC_IC_TGV: the Taylor-Green vortex of Sec. 5.2 with T = 1:
 *     rho = 1 + gamma Ma^2/16 (cos 2x1 + cos 2x2)(cos 2x3 + 2), u = (sin x1 cos x2 cos x3,
 *     -cos x1 sin x2 cos x3, 0), p = rho R.  params_host: NULL.
 *   ESDC_IC_VORTEX: the isentropic vortex of Sec. 5.1.1 (eq. iv_sol) about an axis, plus a uniform
 *     drift: with r the distance to the axis, T = 1 - (gamma-1) Ma^2 beta^2/(8 pi^2) exp(1 - r^2),
 *     rho = T^(1/(gamma-1)), u = u_inf + beta/(2 pi) exp((1 - r^2)/2) (a x r_vec), p = rho R T.
 *     params_host[10] = beta, centre[3], axis[3] (any length > 0), u_inf[3]; NULL: 5, 0, (1, 1, 1), 0.
 *   ESDC_IC_FREESTREAM: uniform state; params_host[5] = rho, u[3], p; NULL: 1, (0.3, 0.2, 0.1), R.
 * Errors: ESDC_ERR_ARG (unknown ic, NULL q_dev, zero axis, non-positive rho or p).
 */
#define ESDC_IC_TGV 0
#define ESDC_IC_VORTEX 1
#define ESDC_IC_FREESTREAM 2
int esdc_init_state(esdc_ctx* ctx, int ic, const double* params_host, double* q_dev, void* stream);

/*
 * esdc_rhs -- dq/dt = J^-1 [ -I^(E) + SAT^(I) + sum_la D_l Chat_la theta_a + SAT^(V) ] (eq. NSL),
 * with I^(E) the Hadamard flux differencing of eq. discEL using the Chandrashekar two-point flux.
 * q_dev: [K][5][N^3] float64 device state (read only).
 * dqdt_dev: [K][5][N^3] device output; float64 for ESDC_PREC_FP64, float32 for ESDC_PREC_FP32.
 * ESDC_PREC_FP32: q is first rounded to the float32 perturbation (rho - 1, rho u, rho E - E0) in a
 * library buffer (the subtraction in float64), and the whole residual is then float32 arithmetic
 * with the reference state rho = 1, p = R split off exactly (see csrc/rhs_f32.cu).
 * q_dev and dqdt_dev must not overlap.  Asynchronous on stream.
 */
int esdc_rhs(esdc_ctx* ctx, const double* q_dev, void* dqdt_dev, void* stream);

/*
 * esdc_rhs_host -- esdc_rhs on HOST buffers: copies q_host to library-owned device staging memory,
 * evaluates the residual and copies dq/dt back (float64 or float32 as for esdc_rhs).  The staging
 * buffers are allocated on the first call and kept until esdc_destroy.  Synchronous on stream.
 */
int esdc_rhs_host(esdc_ctx* ctx, const double* q_host, void* dqdt_host, void* stream);

/*
 * esdc_workspace_bytes -- device workspace needed by esdc_rk_step (what = 0): for ESDC_PREC_FP64
 * six stage derivatives and one stage state, each K*5*N^3 float64; for ESDC_PREC_FP32 six float32
 * stage derivatives and two float32 perturbation states, the step's base and the current stage
 * state (each sub-buffer 256-byte aligned).
 * what = 1: esdc_rk_adaptive's workspace: for ESDC_PREC_FP64 nine K*5*N^3 float64 buffers; for
 * ESDC_PREC_FP32 ten K*5*N^3 float32 buffers and one float64 buffer.
 */
int esdc_workspace_bytes(const esdc_ctx* ctx, int what, size_t* bytes);

/*
 * esdc_rk_adaptive -- integrate q from t0 to t_end with the Dormand-Prince 5(4) pair and adaptive
 * step sizes (Sec. 5: DP5 with "adaptive time-stepping based on signal processing", Soderlind 2003,
 * Soderlind & Wang 2006; the paper states neither the filter nor the norm, so the library's choice
 * is fixed here):
 *   error estimate  e = dt sum_j (b_j - bhat_j) k_j with the embedded 4th-order weights and the
 *                   seventh stage evaluated at the new solution (first same as last);
 *   error norm      err = sqrt(mean over all K*5*N^3 values of (e / (atol + rtol max(|q_n|,
 *                   |q_n+1|)))^2), accepted when err <= 1;
 *   step control    H211b filter, b = 4: dt_n+1 = dt_n L(rho_n), rho_n = (0.8/err_n)^(1/20)
 *                   (0.8/err_n-1)^(1/20) (dt_n/dt_n-1)^(-1/4) over accepted steps (first step:
 *                   err_n-1 = err_n, ratio 1); a rejected step is retried with dt L((0.8/err)^(1/5)),
 *                   or dt L(0) when err is not finite (an unphysical stage state);
 *                   limiter L(rho) = 1 + atan(rho - 1); the last step lands on t_end.
 * q_dev: [K][5][N^3] float64, advanced in place.  dt_inout: first trial step on entry (> 0), the
 * proposed next step on exit.  rtol, atol > 0.  max_steps: bound on attempted (accepted + rejected)
 * steps; the call returns ESDC_OK when it is reached, with stats_host[3] < t_end.  workspace_dev:
 * esdc_workspace_bytes(ctx, 1) bytes, 256-byte aligned.  stats_host[4] (nullable): accepted steps,
 * rejected steps, residual evaluations, time reached.  dt_history_host (nullable): the first
 * history_capacity accepted step sizes.  The accept/reject decision runs on the host: the call
 * synchronises stream once per attempted step.  Float64 and float32-mixed contexts: in the latter
 * the seven stage derivatives are float32 residuals of float32 perturbation stage states, and the
 * candidate solution, the error estimate and the controller are float64 (tolerances well above
 * float32 rounding of the residual, ~1e-6 relative, are meaningful).  A bounded box without an
 * exterior state fails with ESDC_ERR_ARG.
 */
int esdc_rk_adaptive(esdc_ctx* ctx, double* q_dev, double t0, double t_end, double* dt_inout, double rtol,
                     double atol, int max_steps, void* workspace_dev, size_t workspace_bytes, double* stats_host,
                     double* dt_history_host, int history_capacity, void* stream);

/*
 * esdc_rk_step -- nsteps fixed steps of size dt of the 5th-order Dormand-Prince solution
 * (six residual evaluations per step; Sec. 5 uses this integrator with adaptive steps).
 * q_dev: [K][5][N^3] float64, updated in place.  workspace_dev: caller-owned device memory of at
 * least esdc_workspace_bytes(ctx, 0) bytes, 256-byte aligned.  The solution q and its update
 * q += dt sum_j b_j k_j are float64 in both precision modes; in ESDC_PREC_FP32 the stage states that
 * feed the float32 residual are float32 perturbations (rho - 1, rho u, rho E - E0) formed from the
 * float64 state.  With nsteps >= 2 (and profiling off) one step is captured once as a CUDA graph and
 * replayed nsteps times; the graph is rebuilt when q, the workspace, dt or the exterior/source arrays
 * change.  Results are identical to nsteps single-step calls.  Asynchronous on stream.
 */
int esdc_rk_step(esdc_ctx* ctx, double* q_dev, double dt, int nsteps, void* workspace_dev,
                 size_t workspace_bytes, void* stream);

/*
 * esdc_budgets -- float64 reductions over all nodes with the quadrature weights P J (Sec. 5.3
 * kinetic energy; entropy S = -rho s/(gamma-1), s = log(p rho^-gamma)):
 *   out[0] = sum P J S(q),  out[1] = sum P J rho|u|^2/2,
 *   out[2] = sum P J w(q).dq/dt,  out[3] = sum P J (dKE/dq).dq/dt   (out[2..3] = 0 if dqdt NULL).
 * dqdt_dev: float64 for ESDC_PREC_FP64 contexts, float32 for ESDC_PREC_FP32 (same as esdc_rhs).
 * Deterministic order (bitwise reproducible run to run).  Synchronises stream.
 * Returns ESDC_ERR_STATE (out still written) if any node has non-finite values, rho <= 0 or p <= 0.
 */
int esdc_budgets(esdc_ctx* ctx, const double* q_dev, const void* dqdt_dev, double out_host[4],
                 void* stream);

/*
 * esdc_budgets_async -- the same reductions as esdc_budgets, written to device memory without
 * synchronising, so that a time loop can record the budgets of every step and read them back
 * later: out_dev[5] (caller-owned float64 device memory) receives (sum P J S, sum P J rho|u|^2/2,
 * sum P J w.dq/dt, sum P J (dKE/dq).dq/dt, number of non-finite or non-physical nodes); out_dev[2..3]
 * are 0 when dqdt_dev is NULL.  A non-physical state is reported only through out_dev[4].  Uses the
 * context's reduction scratch: calls on one context must not overlap on the GPU (same stream, or
 * ordered).  Errors: ESDC_ERR_ARG, ESDC_ERR_CUDA (launch).
 */
int esdc_budgets_async(esdc_ctx* ctx, const double* q_dev, const void* dqdt_dev, double* out_dev, void* stream);

/*
 * esdc_set_exterior -- the exterior state of the boundary faces of a bounded box (setup.bounded != 0):
 * a [K][5][N^3] float64 device array in the layout of q, read only at the boundary face nodes of
 * each element, where it is the state on the far side of the face.  With it the interface SAT of a
 * boundary face is the interior one with that state as the neighbour: the two-point flux and the
 * dissipation of Sec. 3-4 impose the Dirichlet data weakly, the gradient lift (SAT^theta) uses its
 * entropy variables, and the viscous interface term SAT^(V) is zero (the exterior viscous flux is
 * read as the interior one; the paper's boundary SATs are in its references).  The pointer is
 * kept, not copied: the array must stay valid while the context evaluates residuals.  NULL clears
 * it.  A residual or adjoint of a bounded box without an exterior state fails with ESDC_ERR_ARG.
 * Float64 and float32-mixed contexts; the float32 residual rounds the exterior state, less the
 * reference state, to float32 as it does the state.
 */
int esdc_set_exterior(esdc_ctx* ctx, const double* q_ext_dev);

/*
 * esdc_set_source -- a source term added to dq/dt by every residual of the context, e.g. the
 * manufactured-solution source of Sec. 5.1 (esdc_mms_fields).  [K][5][N^3] float64 device array,
 * kept (not copied) until replaced; NULL clears it.  Every context (p = 15 included); the float32
 * residual adds it rounded to float32.
 */
int esdc_set_source(esdc_ctx* ctx, const double* source_dev);

/*
 * esdc_mms_fields -- the manufactured solution of the paper's viscous error-vs-cost study (Sec. 5.1,
 * eq. mms) and its source term, on the host.  Each of rho, u1, u2, u3, p is
 * phi0 + sum_k phi_k trig_k(alpha_k pi x_k / L) with trig_k = sin or cos as in eq. mms, from
 * table[5][7] = (phi0, phi_x1, phi_x2, phi_x3, alpha_x1, alpha_x2, alpha_x3) per row (already in the
 * library's units: rho_inf = T_inf = 1, R = 1/(gamma Ma^2)).  At n points x_host[n][3] it writes the
 * conserved state q_host[n][5] and the source s_host[n][5] = div(F^I - F^V) of that field (analytic
 * derivatives; mu = 1/Re, kappa = mu gamma R/((gamma - 1) Pr)), either output nullable.  Host only,
 * no GPU.  Errors: ESDC_ERR_ARG.
 */
int esdc_mms_fields(double gamma, double Ma, double Re, double Pr, double L, const double* table, int64_t n,
                    const double* x_host, double* q_host, double* s_host);

/*
 * esdc_dt_cfl -- dt = cfl * min(h/(N^2 max(|u|+c)), h^2/(N^4 nu)), nu = max(4/3, gamma/Pr) mu/rho_min,
 * h = smallest element edge (the paper integrates adaptively; this fixed-step rule is the
 * library's).  Synchronises stream.  ESDC_ERR_STATE on a non-physical state.
 */
int esdc_dt_cfl(esdc_ctx* ctx, const double* q_dev, double cfl, double* dt_host, void* stream);

/*
 * esdc_rhs_vjp -- the adjoint of esdc_rhs (no counterpart in the paper, whose method this
 * differentiates): grad = (dR/dq)^T lambda for the float64 residual R(q) = dq/dt of eq. NSL,
 * through the Chandrashekar flux and its log means, the interface dissipation, the BR1 viscous
 * chain and the metric terms.  At non-smooth points it uses d|x| = sign(x), sign(0) = 0, and splits
 * the cotangent of max(a, b) in half at a tie.  If grad_mu_host is not NULL it also returns
 * lambda . dR/dmu (R is linear in mu through mu, kappa = mu cp/Pr and the interior penalty) and
 * synchronises stream.  q_dev, lambda_dev, grad_dev: [K][5][N^3] float64 device arrays (grad_dev
 * must not alias the others).  ESDC_PREC_FP64 contexts with p <= 7 (ESDC_ERR_UNSUPPORTED
 * otherwise): any volume flux, any interface dissipation, the interior penalty, either metric
 * option, periodic or bounded boxes.  On a bounded box the exterior state (esdc_set_exterior, ESDC_ERR_ARG
 * if absent) is constant in q: a boundary face passes its cotangent to the own nodes only.  A source
 * term (esdc_set_source) is constant in q too and leaves the product unchanged.
 * The first call allocates the adjoint face buffers (K*6*9*N^2 float64), kept until esdc_destroy.
 */
int esdc_rhs_vjp(esdc_ctx* ctx, const double* q_dev, const double* lambda_dev, double* grad_dev,
                 double* grad_mu_host, void* stream);

/*
 * esdc_ke_gradient -- grad = d/dq of the integrated kinetic energy sum P J rho|u|^2/2
 * (= P J (-|u|^2/2, u, 0) per node): the seed of the kinetic-energy adjoint.  Asynchronous.
 */
int esdc_ke_gradient(esdc_ctx* ctx, const double* q_dev, double* grad_dev, void* stream);

/*
 * esdc_rk_step_ckpt -- esdc_rk_step that first stores the state of every step, the checkpoints of
 * esdc_rk_adjoint (no counterpart in the paper, whose method this differentiates).
 * store_k1 = 0: ckpt_dev[n] = q before step n, n = 0..nsteps-1 (nsteps*K*5*N^3 float64).
 * store_k1 = 1: ckpt_dev[2n] = q before step n and ckpt_dev[2n+1] = its residual f(q), the step's
 * first stage derivative, which the step writes there directly (2*nsteps*K*5*N^3 float64; float64
 * contexts only, ESDC_ERR_UNSUPPORTED otherwise; steps launched one by one, no graph replay).  The
 * reverse sweep then recomputes four residuals per step instead of five.
 * ckpt_dev: caller owned, 16-byte aligned.  Asynchronous.
 */
int esdc_rk_step_ckpt(esdc_ctx* ctx, double* q_dev, double dt, int nsteps, double* ckpt_dev, int store_k1,
                      void* workspace_dev, size_t workspace_bytes, void* stream);

/* esdc_rk_adjoint_workspace_bytes -- workspace of esdc_rk_adjoint: 12 state-sized float64 buffers. */
int esdc_rk_adjoint_workspace_bytes(const esdc_ctx* ctx, size_t* bytes);

/*
 * esdc_rk_adjoint -- discrete adjoint of nsteps DP5 steps (reverse sweep with stage
 * recomputation from the checkpoints of esdc_rk_step_ckpt, store_k1 as given there).  On entry
 * lambda_dev holds dL/dq_N; on exit dL/dq_0.  grad_mu_host (nullable) receives dL/dmu.  Per step:
 * five residuals (four with store_k1) rebuild the stage states Y_1..Y_6 from the checkpoint, then
 * for t = 6..1 psi_t = J(Y_t)^T kappa_t with kappa_t = dt b_t lambda_{n+1} + sum_{s>t} dt a_st psi_s,
 * and lambda_n = lambda_{n+1} + sum_t psi_t.  ESDC_PREC_FP64 contexts only.  Synchronises stream
 * when grad_mu_host is not NULL.
 */
int esdc_rk_adjoint(esdc_ctx* ctx, const double* ckpt_dev, int store_k1, double dt, int nsteps, double* lambda_dev,
                    double* grad_mu_host, void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * esdc_rk_step_stages -- esdc_rk_step that stores the six stage states of every step, the stage
 * checkpoints of the adjoint (no counterpart in the paper, whose method this differentiates):
 * stages_dev[(n*6 + t)] = Y_t of step n, each K*5*N^3 float64 (Y_0 = q before step n; Y_t the
 * state at which the t-th residual of the step is evaluated).  stages_dev: nsteps*6*K*5*N^3 float64,
 * caller owned, 16-byte aligned.  The stage combinations write there directly, so storing costs one
 * copy of q per step.  ESDC_PREC_FP64 contexts only (ESDC_ERR_UNSUPPORTED otherwise).  Asynchronous.
 */
int esdc_rk_step_stages(esdc_ctx* ctx, double* q_dev, double dt, int nsteps, double* stages_dev,
                        void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * esdc_rk_adjoint_stages -- the reverse sweep of esdc_rk_adjoint from stored stage states
 * (esdc_rk_step_stages): per step six vector-Jacobian products and no residual recomputation.
 * The arguments of esdc_rk_adjoint but store_k1, and the same workspace (esdc_rk_adjoint_workspace_bytes)
 * and results.
 */
int esdc_rk_adjoint_stages(esdc_ctx* ctx, const double* stages_dev, double dt, int nsteps, double* lambda_dev,
                           double* grad_mu_host, void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * esdc_device_status -- status bits the context's kernels recorded on the device since the last
 * clear: 1 (ESDC_STATUS_BULK_WAIT) = a kernel's bounded wait for its bulk shared-memory copies gave
 * up (no longer than about a second), and it left its elements' results unwritten.  0 when all
 * waits completed.  clear = 1 resets the bits.  Synchronises stream (the read is ordered after the
 * work already on it).
 */
#define ESDC_STATUS_BULK_WAIT 1
int esdc_device_status(esdc_ctx* ctx, int* status_host, int clear, void* stream);

/*
 * esdc_profile -- enable (on = 1) or disable CUDA-event timing of the residual kernels of this
 * context: every esdc_rhs (also inside esdc_rk_step) then records an event pair around the fused
 * element kernel and another around the viscous interface kernel on the call's stream.
 * esdc_profile_read synchronises, returns the summed milliseconds of each kernel and the number of
 * residual evaluations timed since profiling was enabled, and resets the sums.  Not part of the
 * method (a measurement aid).
 */
int esdc_profile(esdc_ctx* ctx, int on);
int esdc_profile_read(esdc_ctx* ctx, double* ms_element_kernel, double* ms_face_kernel, int64_t* count);

/*
 * esdc_probe_fma -- measured FMA throughput of the current device in FLOP/s (2 per FMA): kind 0
 * float64, kind 1 float32; eight independent chains per thread, 8 CTAs of 256 threads per SM,
 * best of three timed launches.  Allocates and frees a small scratch buffer.  Synchronous.
 * Not part of the method: it supplies the arithmetic roofline denominators.
 */
int esdc_probe_fma(int kind, double* flops_per_s, void* stream);

/*
 * esdc_budgets_noalloc -- the four float64 budgets of esdc_budgets for callers that cannot
 * allocate device memory: code running where cudaMalloc is forbidden or unsafe (while another
 * component captures the stream into a graph, inside a fixed device-memory budget handed out once
 * at start-up, or in hosts whose allocator owns all device memory).  It needs no context and
 * performs no cudaMalloc, cudaFree or other allocating call.  The paper has no counterpart: it is
 * a deployment variant of the budget reduction, not part of the method.
 *   N: nodes per direction (2..8); K: elements; gamma: ratio of specific heats;
 *   w_host[N]: the LGL weights (esdc_lgl); q_dev, dqdt_dev (nullable), J_dev: float64 device
 *   arrays in the esdc_rhs layouts, J_dev[K][N^3] the metric Jacobian (esdc_geometry);
 *   out_dev[5]: caller-owned device memory receiving (sum PJ S, KE, sum PJ w.dq/dt, dKE/dt, number
 *   of non-finite or non-physical nodes); out_dev[2..3] are 0 when dqdt_dev is NULL.
 * Scratch: a static device array of 65536 x 5 doubles (2.6 MB) in every process that loads the
 * library, held on each GPU until exit; inputs above 268,435,456 nodes are rejected with
 * ESDC_ERR_ARG.  A call on a stream that is not being captured looks the array's device address up
 * (cudaGetSymbolAddress with the current device), so the address stays valid after a device reset;
 * a call during stream capture reuses the address of the last uncaptured call on that device, so
 * make one call on each device before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race and give wrong sums.
 * Asynchronous on stream; deterministic order.  Errors: ESDC_ERR_ARG, ESDC_ERR_CUDA.
 */
int esdc_budgets_noalloc(int N, int64_t K, double gamma, const double* w_host, const double* q_dev,
                         const double* dqdt_dev, const double* J_dev, double* out_dev, void* stream);

/* esdc_strerror -- static description of a status code. */
const char* esdc_strerror(int status);

/* esdc_last_error -- message of the last failing call on this thread ("" if none). */
const char* esdc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ESDC_H */
