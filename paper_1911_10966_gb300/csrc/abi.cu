// extern "C" entry points declared in include/esdc.h: argument checks, buffer ownership and the
// sequencing of kernels.  No arithmetic of the method lives here.
#include <cuda_runtime.h>

#include <cmath>
#include <utility>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "esdc_internal.h"
#include "kernels.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(ESDC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                   \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, #expr); \
    } while (0)

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Dormand-Prince 5(4) coefficients (Dormand & Prince 1980): stage matrix rows 2..6 and the
// 5th-order weights (the 7th, FSAL stage only feeds the embedded error estimate, unused here).
const double kA[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0}};
const double kB[6] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0};
// embedded 4th-order weights of the pair (Dormand & Prince 1980); stage 7 is the residual at the new
// solution (its row of A is b)
const double kBhat[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                         187.0 / 2100.0, 1.0 / 40.0};
// digital-filter step control: H211b (Soderlind 2003) with b = 4 on an O(dt^5) estimate, setpoint
// 0.8, ratio limiter 1 + atan(rho - 1) (Soderlind & Wang 2006)
const double kCtrlB = 4.0, kCtrlK = 5.0, kCtrlTheta = 0.8;

// Four profiling events for the next residual evaluation (NULL when profiling is off).
cudaEvent_t* next_events(esdc_ctx* c) {
    if (!c->profiling) return nullptr;
    if (c->prof_used + 4 > c->prof_events.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
            c->prof_events.push_back((void*)ev);
        }
    }
    cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(&c->prof_events[c->prof_used]);
    c->prof_used += 4;
    return ev;
}

int rhs_impl(esdc_ctx* c, const double* q, void* dqdt, cudaStream_t s) {
    if (c->setup.bounded != 0 && !c->d_qext)
        return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    cudaError_t e;
    if (c->setup.precision == ESDC_PREC_FP64) {
        e = esdc::launch_rhs_f64(c, q, (double*)dqdt, s, next_events(c));
    } else {
        e = esdc::launch_shadow(c, q, c->d_shadow, s);
        esdc::StageF in{};
        in.base = c->d_shadow;
        if (e == cudaSuccess) e = esdc::launch_rhs_f32(c, in, (float*)dqdt, s, next_events(c));
    }
    if (e != cudaSuccess) return cuda_fail(e, "esdc_rhs launch");
    return ESDC_OK;
}

// Mixed precision: nsteps DP5 steps with float32 residuals on float32 perturbation stage states
// (formed by a streaming kernel from the step's shadow state and the earlier stage derivatives) and
// the float64 solution update q += dt sum_j b_j k_j (accumulated in float64).
// Stage st of a float32-mixed DP5 step of size h: the stage state base + h sum_j a_st,j k_j (into y;
// the base itself for st = 0), then its residual into out.
cudaError_t stage_then_rhs_f32(esdc_ctx* c, const float* base, float* const k[], int st, double h, float* y,
                               float* out, cudaStream_t s) {
    esdc::StageF in{};
    in.base = base;
    for (int j = 0; j < st; ++j) {
        if (kA[st][j] == 0.0) continue;
        in.k[in.nk] = k[j];
        in.c[in.nk] = (float)(h * kA[st][j]);
        ++in.nk;
    }
    if (in.nk > 0) {
        const cudaError_t e = esdc::launch_stage_f32(c, in, y, s);
        if (e != cudaSuccess) return e;
        in = esdc::StageF{};
        in.base = y;
    }
    return esdc::launch_rhs_f32(c, in, out, s, next_events(c));
}

// the float32 shadow of q in the workspace (the base state of the first step)
int rk_shadow_f32(esdc_ctx* c, const double* q, void* ws, cudaStream_t s) {
    const size_t sub = round256((size_t)c->n_nodes * 5 * sizeof(float));
    cudaError_t e = esdc::launch_shadow(c, q, (float*)((char*)ws + 6 * sub), s);
    if (e != cudaSuccess) return cuda_fail(e, "shadow");
    return ESDC_OK;
}

// nsteps float32-mixed DP5 steps from the shadow already in the workspace (each step's update
// writes the next shadow)
int rk_steps_f32(esdc_ctx* c, double* q, double dt, int nsteps, void* ws, cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(float));
    float* k[6];
    for (int j = 0; j < 6; ++j) k[j] = (float*)((char*)ws + j * sub);
    float* base = (float*)((char*)ws + 6 * sub);
    float* ystage = (float*)((char*)ws + 7 * sub);
    cudaError_t e;
    for (int step = 0; step < nsteps; ++step) {
        for (int st = 0; st < 6; ++st) {
            e = stage_then_rhs_f32(c, base, k, st, dt, ystage, k[st], s);
            if (e != cudaSuccess) return cuda_fail(e, "stage residual (float32)");
        }
        esdc::Combine64F cb{};
        for (int j = 0; j < 6; ++j)
            if (kB[j] != 0.0) {
                cb.k[cb.nk] = k[j];
                cb.coef[cb.nk] = dt * kB[j];
                ++cb.nk;
            }
        e = esdc::launch_final_f32(c, q, base, cb, s);
        if (e != cudaSuccess) return cuda_fail(e, "step update (float64)");
    }
    return ESDC_OK;
}

int rk_step_f32(esdc_ctx* c, double* q, double dt, int nsteps, void* ws, cudaStream_t s) {
    const int r = rk_shadow_f32(c, q, ws, s);
    return r ? r : rk_steps_f32(c, q, dt, nsteps, ws, s);
}

// nsteps float64 DP5 steps.  stages (nullable): the six stage states of every step are written to
// stages + (step * 6 + t) * K*5*N^3, t = 0 being the state at the start of the step; the stage
// combinations then write there instead of the workspace buffer, so storing them costs one copy of q
// per step.
int rk_step_f64(esdc_ctx* c, double* q, double dt, int nsteps, void* ws, cudaStream_t s, double* stages,
                double* k1_out) {
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(double));
    double* k[6];
    for (int j = 0; j < 6; ++j) k[j] = (double*)((char*)ws + j * sub);
    double* stage_ws = (double*)((char*)ws + 6 * sub);
    for (int step = 0; step < nsteps; ++step) {
        if (k1_out) k[0] = k1_out + (size_t)step * n;   // the first stage derivative written out directly
        for (int st = 0; st < 6; ++st) {
            double* dst = stages ? stages + ((size_t)step * 6 + st) * n : stage_ws;
            const double* qs = q;
            if (st == 0) {
                if (stages) CUDA_TRY(cudaMemcpyAsync(dst, q, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            } else {
                esdc::Combine cb{};
                cb.nk = st;
                for (int j = 0; j < st; ++j) {
                    cb.k[j] = k[j];
                    cb.coef[j] = dt * kA[st][j];
                }
                cudaError_t e = esdc::launch_combine(dst, q, cb, n, s);
                if (e != cudaSuccess) return cuda_fail(e, "stage combine");
                qs = dst;
            }
            int r = rhs_impl(c, qs, k[st], s);
            if (r) return r;
        }
        esdc::Combine cb{};
        cb.nk = 0;
        for (int j = 0; j < 6; ++j)
            if (kB[j] != 0.0) {
                cb.k[cb.nk] = k[j];
                cb.coef[cb.nk] = dt * kB[j];
                ++cb.nk;
            }
        cudaError_t e = esdc::launch_combine(q, q, cb, n, s);
        if (e != cudaSuccess) return cuda_fail(e, "step combine");
    }
    return ESDC_OK;
}

// Multi-step esdc_rk_step: one step is captured once as a CUDA graph on a private stream and replayed
// nsteps times on the caller's stream, so the ~20 launches of a step cost one graph launch.  The
// graph bakes in the state, workspace, step size and optional-term pointers; any change recaptures.
// While esdc_profile is on, no graph is used: a replayed graph would repeat the event records of
// its capture without the counts that esdc_profile_read reports, so profiled steps launch directly.
// Returns ESDC_OK, or 1 when the graph could not be built or is not used (the caller then launches
// directly).
int rk_steps_graph(esdc_ctx* c, double* q, double dt, int nsteps, void* ws, cudaStream_t s) {
    if (c->profiling) return 1;
    const void* key[5] = {q, ws, c->d_qext, c->d_src, (const void*)(intptr_t)c->setup.precision};
    bool valid = c->graph_exec != nullptr && c->graph_dt == dt;
    for (int i = 0; i < 5 && valid; ++i) valid = key[i] == c->graph_key[i];
    if (!valid) {
        if (c->graph_exec) {
            cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
            c->graph_exec = nullptr;
        }
        if (!c->capture_stream) {
            cudaStream_t cs;
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return 1;
            }
            c->capture_stream = cs;
        }
        cudaStream_t cs = (cudaStream_t)c->capture_stream;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        const int r = c->setup.precision == ESDC_PREC_FP32 ? rk_steps_f32(c, q, dt, 1, ws, cs)
                                                            : rk_step_f64(c, q, dt, 1, ws, cs, nullptr, nullptr);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaGraphExec_t exec = nullptr;
        const bool ok = r == ESDC_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            return r ? r : 1;
        }
        c->graph_exec = exec;
        c->graph_dt = dt;
        for (int i = 0; i < 5; ++i) c->graph_key[i] = key[i];
    }
    for (int i = 0; i < nsteps; ++i) CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)c->graph_exec, s));
    return ESDC_OK;
}

// Reverse sweep over one DP5 step from its six stage states Y[0..5] (float64 contexts).  On entry
// lam = dL/dq_{n+1}; on exit dL/dq_n.  For t = 5..0:
//   kappa_t = dt b_t lam + sum_{s>t} dt a_st psi_s,   psi_t = J(Y_t)^T kappa_t,
// then lam += sum_t psi_t; lambda . dR/dmu of every VJP accumulates into d_adj_acc.  psi[6] and kappa
// are state-sized buffers; psi may alias buffers whose contents are no longer needed.
int adjoint_step(esdc_ctx* c, const double* const Y[6], double dt, double* lam, double* const psi[6], double* kappa,
                 cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    for (int t = 5; t >= 0; --t) {
        esdc::LinComb lc{};
        if (kB[t] != 0.0) {
            lc.x[lc.n] = lam;
            lc.c[lc.n++] = dt * kB[t];
        }
        for (int u = 5; u > t; --u)
            if (kA[u][t] != 0.0) {
                lc.x[lc.n] = psi[u];
                lc.c[lc.n++] = dt * kA[u][t];
            }
        cudaError_t e = esdc::launch_lincomb(kappa, lc, n, s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint stage cotangent");
        e = esdc::launch_rhs_vjp(c, Y[t], kappa, psi[t], c->d_adj_acc, s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint vjp");
    }
    esdc::LinComb lc{};
    lc.x[lc.n] = lam;
    lc.c[lc.n++] = 1.0;
    for (int t = 5; t >= 0; --t) {
        lc.x[lc.n] = psi[t];
        lc.c[lc.n++] = 1.0;
    }
    cudaError_t e = esdc::launch_lincomb(lam, lc, n, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint accumulate");
    return ESDC_OK;
}

double step_limiter(double rho) { return 1.0 + std::atan(rho - 1.0); }

double h211b_ratio(double err, double err_prev, double rho_prev) {
    const double e = 1.0 / (kCtrlB * kCtrlK);
    return std::pow(kCtrlTheta / err, e) * std::pow(kCtrlTheta / err_prev, e) * std::pow(rho_prev, -1.0 / kCtrlB);
}

// Adaptive DP5(4) on a float64 context; see esdc_rk_adaptive.  Workspace: 7 stage derivatives, one
// stage state, one candidate solution.
int rk_adaptive_f64(esdc_ctx* c, double* q, double t0, double t_end, double* dt_io, double rtol, double atol,
                    int max_steps, void* ws, double* stats, double* hist, int hist_cap, cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(double));
    double* k[7];
    for (int j = 0; j < 7; ++j) k[j] = (double*)((char*)ws + j * sub);
    double* stage = (double*)((char*)ws + 7 * sub);
    double* qn = (double*)((char*)ws + 8 * sub);
    double t = t0, dt = *dt_io;
    int acc = 0, rej = 0;
    int64_t nrhs = 0;
    double err_prev = -1.0, h_prev = -1.0;
    int r;
    if (t < t_end) {
        r = rhs_impl(c, q, k[0], s);
        if (r) return r;
        ++nrhs;
    }
    while (t < t_end && acc + rej < max_steps) {
        const bool last = t + dt >= t_end;
        const double h = last ? t_end - t : dt;
        for (int st = 1; st < 6; ++st) {
            esdc::Combine cb{};
            cb.nk = st;
            for (int j = 0; j < st; ++j) {
                cb.k[j] = k[j];
                cb.coef[j] = h * kA[st][j];
            }
            cudaError_t e = esdc::launch_combine(stage, q, cb, n, s);
            if (e != cudaSuccess) return cuda_fail(e, "stage combine");
            r = rhs_impl(c, stage, k[st], s);
            if (r) return r;
        }
        esdc::Combine cb{};
        for (int j = 0; j < 6; ++j)
            if (kB[j] != 0.0) {
                cb.k[cb.nk] = k[j];
                cb.coef[cb.nk] = h * kB[j];
                ++cb.nk;
            }
        cudaError_t e = esdc::launch_combine(qn, q, cb, n, s);
        if (e != cudaSuccess) return cuda_fail(e, "candidate solution");
        r = rhs_impl(c, qn, k[6], s);
        if (r) return r;
        nrhs += 6;
        esdc::LinComb lc{};
        for (int j = 0; j < 7; ++j) {
            const double d = (j < 6 ? kB[j] : 0.0) - kBhat[j];
            if (d != 0.0) {
                lc.x[lc.n] = k[j];
                lc.c[lc.n++] = h * d;
            }
        }
        e = esdc::launch_dp54_error(c, q, qn, lc, rtol, atol, s);
        if (e != cudaSuccess) return cuda_fail(e, "error estimate");
        double sum = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&sum, c->d_red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double err = std::sqrt(sum / (double)n);
        if (err <= 1.0) {
            const double rho = h211b_ratio(err, err_prev < 0.0 ? err : err_prev, h_prev < 0.0 ? 1.0 : h / h_prev);
            CUDA_TRY(cudaMemcpyAsync(q, qn, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            std::swap(k[0], k[6]);          // first same as last
            t = last ? t_end : t + h;
            if (hist && acc < hist_cap) hist[acc] = h;
            ++acc;
            err_prev = err;
            h_prev = h;
            dt = h * step_limiter(rho);
        } else {
            // a non-finite estimate (a stage state gone unphysical) counts as rho = 0
            ++rej;
            dt = h * step_limiter(std::isfinite(err) ? std::pow(kCtrlTheta / err, 1.0 / kCtrlK) : 0.0);
        }
    }
    *dt_io = dt;
    if (stats) {
        stats[0] = acc;
        stats[1] = rej;
        stats[2] = (double)nrhs;
        stats[3] = t;
    }
    return ESDC_OK;
}

// Adaptive DP5(4) on a float32-mixed context: the same controller as rk_adaptive_f64; the stage
// derivatives are float32 residuals of float32 perturbation stage states formed on load from the
// step's shadow state, the candidate solution q + h sum_j b_j k_j and the error estimate are float64.
// Workspace: 7 float32 stage derivatives, the shadows of q and of the candidate, the float64
// candidate.
int rk_adaptive_f32(esdc_ctx* c, double* q, double t0, double t_end, double* dt_io, double rtol, double atol,
                    int max_steps, void* ws, double* stats, double* hist, int hist_cap, cudaStream_t s) {
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(float));
    float* k[7];
    for (int j = 0; j < 7; ++j) k[j] = (float*)((char*)ws + j * sub);
    float* base = (float*)((char*)ws + 7 * sub);
    float* base_n = (float*)((char*)ws + 8 * sub);
    float* ystage = (float*)((char*)ws + 9 * sub);
    double* qn = (double*)((char*)ws + 10 * sub);
    double t = t0, dt = *dt_io;
    int acc = 0, rej = 0;
    int64_t nrhs = 0;
    double err_prev = -1.0, h_prev = -1.0;
    cudaError_t e;
    if (t < t_end) {
        e = esdc::launch_shadow(c, q, base, s);
        if (e != cudaSuccess) return cuda_fail(e, "shadow");
        esdc::StageF in{};
        in.base = base;
        e = esdc::launch_rhs_f32(c, in, k[0], s, next_events(c));
        if (e != cudaSuccess) return cuda_fail(e, "residual (float32)");
        ++nrhs;
    }
    while (t < t_end && acc + rej < max_steps) {
        const bool last = t + dt >= t_end;
        const double h = last ? t_end - t : dt;
        for (int st = 1; st < 6; ++st) {
            e = stage_then_rhs_f32(c, base, k, st, h, ystage, k[st], s);
            if (e != cudaSuccess) return cuda_fail(e, "stage residual (float32)");
        }
        // candidate: qn = q + h sum_j b_j k_j in float64, and its shadow
        CUDA_TRY(cudaMemcpyAsync(qn, q, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        esdc::Combine64F cb{};
        for (int j = 0; j < 6; ++j)
            if (kB[j] != 0.0) {
                cb.k[cb.nk] = k[j];
                cb.coef[cb.nk] = h * kB[j];
                ++cb.nk;
            }
        e = esdc::launch_final_f32(c, qn, base_n, cb, s);
        if (e != cudaSuccess) return cuda_fail(e, "candidate solution");
        esdc::StageF in{};
        in.base = base_n;
        e = esdc::launch_rhs_f32(c, in, k[6], s, next_events(c));
        if (e != cudaSuccess) return cuda_fail(e, "residual (float32)");
        nrhs += 6;
        esdc::LinCombF lc{};
        for (int j = 0; j < 7; ++j) {
            const double d = (j < 6 ? kB[j] : 0.0) - kBhat[j];
            if (d != 0.0) {
                lc.x[lc.n] = k[j];
                lc.c[lc.n++] = h * d;
            }
        }
        e = esdc::launch_dp54_error_f32(c, q, qn, lc, rtol, atol, s);
        if (e != cudaSuccess) return cuda_fail(e, "error estimate");
        double sum = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&sum, c->d_red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double err = std::sqrt(sum / (double)n);
        if (err <= 1.0) {
            const double rho = h211b_ratio(err, err_prev < 0.0 ? err : err_prev, h_prev < 0.0 ? 1.0 : h / h_prev);
            CUDA_TRY(cudaMemcpyAsync(q, qn, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            std::swap(k[0], k[6]);          // first same as last
            std::swap(base, base_n);        // the candidate's shadow is the next step's base
            t = last ? t_end : t + h;
            if (hist && acc < hist_cap) hist[acc] = h;
            ++acc;
            err_prev = err;
            h_prev = h;
            dt = h * step_limiter(rho);
        } else {
            ++rej;
            dt = h * step_limiter(std::isfinite(err) ? std::pow(kCtrlTheta / err, 1.0 / kCtrlK) : 0.0);
        }
    }
    *dt_io = dt;
    if (stats) {
        stats[0] = acc;
        stats[1] = rej;
        stats[2] = (double)nrhs;
        stats[3] = t;
    }
    return ESDC_OK;
}

// The element kernel instantiation depends on the optional face terms; opt the one in use into its
// shared-memory size.
int prepare_variant(esdc_ctx* c) {
    if (c->setup.precision != ESDC_PREC_FP64) return ESDC_OK;
    const cudaError_t e = esdc::prepare_rhs_f64(c);
    if (e != cudaSuccess) return cuda_fail(e, "kernel set-up");
    return ESDC_OK;
}

int ensure_adjoint(esdc_ctx* c) {
    if (c->setup.precision != ESDC_PREC_FP64 || c->N > esdc::kMaxN)
        return fail(ESDC_ERR_UNSUPPORTED, "the adjoint is built for float64 contexts with p <= 7");
    if (c->setup.bounded != 0 && !c->d_qext)
        return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    if (c->d_adj_g) return ESDC_OK;
    const size_t N2 = (size_t)c->N * c->N;
    CUDA_TRY(cudaMalloc(&c->d_adj_g, (size_t)c->K * 6 * 5 * N2 * sizeof(double)));
    CUDA_TRY(cudaMalloc(&c->d_adj_t, (size_t)c->K * 6 * 4 * N2 * sizeof(double)));
    CUDA_TRY(cudaMalloc(&c->d_adj_mu, esdc::adjoint_mu_blocks(c) * sizeof(double)));
    CUDA_TRY(cudaMalloc(&c->d_adj_acc, 8 * sizeof(double)));
    CUDA_TRY(esdc::prepare_adjoint(c));
    return ESDC_OK;
}

int adjoint_checks(esdc_ctx* c, const double* ckpt, double dt, int nsteps, double* lam, void* ws, size_t ws_bytes) {
    if (!c || !ckpt || !lam || !ws) return fail(ESDC_ERR_ARG, "null argument");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(ESDC_ERR_ARG, "nsteps >= 0 and finite dt required");
    const size_t need = 12 * round256((size_t)c->n_nodes * 5 * sizeof(double));
    if (ws_bytes < need) return fail(ESDC_ERR_ARG, "adjoint workspace too small");
    if (!aligned(ws, 256) || !aligned(lam, 16) || !aligned(ckpt, 16))
        return fail(ESDC_ERR_ARG, "lam/ckpt must be 16-byte and workspace 256-byte aligned");
    return ensure_adjoint(c);
}

int adjoint_finish(esdc_ctx* c, double* grad_mu, cudaStream_t s) {
    if (grad_mu) {
        CUDA_TRY(cudaMemcpyAsync(grad_mu, c->d_adj_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return ESDC_OK;
}

void free_ctx(esdc_ctx* c) {
    if (!c) return;
    if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
    if (c->capture_stream) cudaStreamDestroy((cudaStream_t)c->capture_stream);
    for (void* ev : c->prof_events) cudaEventDestroy((cudaEvent_t)ev);
    cudaFree(c->d_geom);
    cudaFree(c->d_jinv);
    cudaFree(c->d_xyz);
    cudaFree(c->d_fnorm);
    cudaFree(c->d_nsurf);
    cudaFree(c->d_lr);
    cudaFree(c->d_lwf);
    cudaFree(c->d_lft);
    cudaFree(c->d_geomf);
    cudaFree(c->d_nsurff);
    cudaFree(c->d_nbr);
    cudaFree(c->d_trace);
    cudaFree(c->d_shadow);
    cudaFree(c->d_red);
    cudaFree(c->d_red_out);
    cudaFree(c->d_status);
    cudaFree(c->d_lntab);
    cudaFree(c->d_stage_q);
    cudaFree(c->d_adj_g);
    cudaFree(c->d_adj_t);
    cudaFree(c->d_adj_mu);
    cudaFree(c->d_adj_acc);
    cudaFree(c->d_stage_r);
    delete c;
}

}  // namespace

namespace esdc {
void set_last_error(const std::string& msg) { g_err = msg; }

int sm_count() {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 148;
        cache[dev] = n;
    }
    return cache[dev];
}
}  // namespace esdc

extern "C" {

const char* esdc_last_error(void) { return g_err.c_str(); }

const char* esdc_strerror(int status) {
    switch (status) {
        case ESDC_OK: return "ok";
        case ESDC_ERR_ARG: return "invalid argument";
        case ESDC_ERR_MESH: return "invalid mesh geometry";
        case ESDC_ERR_CUDA: return "CUDA runtime error";
        case ESDC_ERR_STATE: return "non-finite or non-physical state";
        case ESDC_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

int esdc_lgl(int p, double* xi_host, double* w_host) {
    if (p < 1 || p > esdc::kLargeN - 1) return fail(ESDC_ERR_ARG, "p must be in [1, 15]");
    if (!xi_host || !w_host) return fail(ESDC_ERR_ARG, "null output pointer");
    return esdc::lgl(p, xi_host, w_host);
}

int esdc_operators(int p, double* D, double* S) {
    if (p < 1 || p > esdc::kLargeN - 1) return fail(ESDC_ERR_ARG, "p must be in [1, 15]");
    esdc::HostSetup hs;
    int st = esdc::build_operators(p, hs);
    if (st) return fail(st, "operator construction failed");
    if (D) std::memcpy(D, hs.D.data(), hs.D.size() * sizeof(double));
    if (S) std::memcpy(S, hs.S.data(), hs.S.size() * sizeof(double));
    return ESDC_OK;
}

static int check_setup(const esdc_setup_t& s) {
    if (s.p < 1 || s.p > esdc::kLargeN - 1) return fail(ESDC_ERR_ARG, "p must be in [1, 7] or 15");
    if (s.p > esdc::kMaxN - 1 && s.p != esdc::kLargeN - 1)
        return fail(ESDC_ERR_UNSUPPORTED, "degrees 8 to 14 are not built (p in [1, 7] or 15)");
    if (s.kx < 1 || s.ky < 1 || s.kz < 1) return fail(ESDC_ERR_ARG, "element counts must be >= 1");
    if ((int64_t)s.kx * s.ky * s.kz > (int64_t)INT32_MAX / 6) return fail(ESDC_ERR_ARG, "too many elements");
    if (!(s.gamma > 1.0) || !(s.Pr > 0.0) || !(s.Ma > 0.0) || !std::isfinite(s.Re))
        return fail(ESDC_ERR_ARG, "gamma > 1, Pr > 0, Ma > 0 and finite Re required");
    if (s.dissipation != ESDC_DISS_NONE && s.dissipation != ESDC_DISS_LLF && s.dissipation != ESDC_DISS_MATRIX)
        return fail(ESDC_ERR_ARG, "dissipation must be ESDC_DISS_NONE, ESDC_DISS_LLF or ESDC_DISS_MATRIX");
    if (s.dissipation == ESDC_DISS_MATRIX && s.precision != ESDC_PREC_FP64)
        return fail(ESDC_ERR_UNSUPPORTED, "the matrix dissipation is built for float64 only");
    if (!(s.ip_coef >= 0.0) || !std::isfinite(s.ip_coef)) return fail(ESDC_ERR_ARG, "ip_coef must be finite and >= 0");
    if (s.bounded < 0 || s.bounded > 7) return fail(ESDC_ERR_ARG, "bounded must be a bit mask in [0, 7]");
    if (s.ip_coef > 0.0 && s.precision != ESDC_PREC_FP64)
        return fail(ESDC_ERR_UNSUPPORTED, "the interior penalty is built for float64 only");
    if (s.precision != ESDC_PREC_FP64 && s.precision != ESDC_PREC_FP32)
        return fail(ESDC_ERR_ARG, "precision must be ESDC_PREC_FP64 or ESDC_PREC_FP32");
    if (s.volume_flux != ESDC_FLUX_ESC && s.volume_flux != ESDC_FLUX_KG && s.volume_flux != ESDC_FLUX_DC)
        return fail(ESDC_ERR_ARG, "volume_flux must be ESDC_FLUX_ESC, ESDC_FLUX_KG or ESDC_FLUX_DC");
    if (s.volume_flux == ESDC_FLUX_DC && s.precision != ESDC_PREC_FP64)
        return fail(ESDC_ERR_UNSUPPORTED, "the DC volume flux is built for float64 only");
    if (s.metrics != ESDC_METRICS_CURL && s.metrics != ESDC_METRICS_OPTIMIZED)
        return fail(ESDC_ERR_ARG, "metrics must be ESDC_METRICS_CURL or ESDC_METRICS_OPTIMIZED");
    if (s.p == esdc::kLargeN - 1 &&
        (s.precision != ESDC_PREC_FP64 || s.dissipation == ESDC_DISS_MATRIX || s.ip_coef > 0.0 || s.bounded != 0 ||
         s.metrics != ESDC_METRICS_CURL))
        return fail(ESDC_ERR_UNSUPPORTED, "p = 15 is built for float64 periodic boxes with curl-form metrics and "
                                          "no or local Lax-Friedrichs dissipation, without interior penalty");
    return ESDC_OK;
}

// The node coordinates for setup: the caller's, or the box mesh generator's when xyz is NULL (held
// in gen).  Operators must be built (hs.xi) first.
static int resolve_coords(const esdc_setup_t& s, const esdc::HostSetup& hs, const double*& xyz,
                          std::vector<double>& gen) {
    if (xyz) return ESDC_OK;
    if (esdc::generate_box_coords(s, hs.xi, gen) != ESDC_OK)
        return fail(ESDC_ERR_ARG, "box generator: hi > lo and a finite warp_amp >= 0 required");
    xyz = gen.data();
    return ESDC_OK;
}

int esdc_host_coordinates(const esdc_setup_t* setup, double* out) {
    if (!setup || !out) return fail(ESDC_ERR_ARG, "null argument");
    int st = check_setup(*setup);
    if (st) return st;
    esdc::HostSetup hs;
    st = esdc::build_operators(setup->p, hs);
    if (st) return fail(st, "operator construction failed");
    const double* xyz = nullptr;
    std::vector<double> gen;
    st = resolve_coords(*setup, hs, xyz, gen);
    if (st) return st;
    std::memcpy(out, gen.data(), gen.size() * sizeof(double));
    return ESDC_OK;
}

int esdc_host_geometry(const esdc_setup_t* setup, const double* xyz, double* J, double* Ja, double* h_min) {
    if (!setup) return fail(ESDC_ERR_ARG, "null argument");
    int st = check_setup(*setup);
    if (st) return st;
    esdc::HostSetup hs;
    st = esdc::build_operators(setup->p, hs);
    if (st) return fail(st, "operator construction failed");
    std::vector<double> gen;
    st = resolve_coords(*setup, hs, xyz, gen);
    if (st) return st;
    std::string err;
    st = esdc::build_geometry(*setup, xyz, hs, err);
    if (st) return fail(st, err);
    const int64_t K = (int64_t)setup->kx * setup->ky * setup->kz;
    const size_t N3 = (size_t)hs.N * hs.N * hs.N;
    for (int64_t e = 0; e < K; ++e) {
        if (J) std::memcpy(J + e * N3, &hs.geom[e * 10 * N3], N3 * sizeof(double));
        if (Ja) std::memcpy(Ja + e * 9 * N3, &hs.geom[(e * 10 + 1) * N3], 9 * N3 * sizeof(double));
    }
    if (h_min) *h_min = hs.h_min;
    return ESDC_OK;
}

int esdc_host_surface_metrics(const esdc_setup_t* setup, const double* xyz, double* nsurf) {
    if (!setup || !nsurf) return fail(ESDC_ERR_ARG, "null argument");
    int st = check_setup(*setup);
    if (st) return st;
    esdc::HostSetup hs;
    st = esdc::build_operators(setup->p, hs);
    if (st) return fail(st, "operator construction failed");
    std::vector<double> gen;
    st = resolve_coords(*setup, hs, xyz, gen);
    if (st) return st;
    std::string err;
    st = esdc::build_geometry(*setup, xyz, hs, err);
    if (st) return fail(st, err);
    const int64_t K = (int64_t)setup->kx * setup->ky * setup->kz;
    const int N = hs.N, N2 = N * N, N3 = N2 * N;
    if (!hs.nsurf.empty()) {
        std::memcpy(nsurf, hs.nsurf.data(), hs.nsurf.size() * sizeof(double));
        return ESDC_OK;
    }
    for (int64_t e = 0; e < K; ++e)
        for (int l = 0; l < 3; ++l)
            for (int side = 0; side < 2; ++side) {
                const int fix = side ? N - 1 : 0;
                for (int t2 = 0; t2 < N; ++t2)
                    for (int t1 = 0; t1 < N; ++t1) {
                        const int node = l == 0 ? fix + N * t1 + N2 * t2
                                                : (l == 1 ? t1 + N * fix + N2 * t2 : t1 + N * t2 + N2 * fix);
                        for (int m = 0; m < 3; ++m)
                            nsurf[((e * 6 + 2 * l + side) * 3 + m) * N2 + t1 + N * t2] =
                                hs.geom[(e * 10 + 1 + 3 * l + m) * N3 + node];
                    }
            }
    return ESDC_OK;
}

int esdc_create(const esdc_setup_t* setup, const double* xyz, esdc_ctx** out) {
    if (!setup || !out) return fail(ESDC_ERR_ARG, "null argument");
    *out = nullptr;
    const esdc_setup_t& s = *setup;
    int st0 = check_setup(s);
    if (st0) return st0;

    esdc::HostSetup hs;
    int st = esdc::build_operators(s.p, hs);
    if (st) return fail(st, "operator construction failed");
    std::vector<double> gen;
    st = resolve_coords(s, hs, xyz, gen);
    if (st) return st;
    std::string err;
    st = esdc::build_geometry(s, xyz, hs, err);
    if (st) return fail(st, err);

    esdc_ctx* c = new (std::nothrow) esdc_ctx();
    if (!c) return fail(ESDC_ERR_ARG, "out of host memory");
    c->setup = s;
    c->N = hs.N;
    c->N3 = hs.N * hs.N * hs.N;
    c->K = (int64_t)s.kx * s.ky * s.kz;
    c->n_nodes = c->K * c->N3;
    c->h_min = hs.h_min;
    std::memset(&c->ops, 0, sizeof(c->ops));
    std::memset(&c->opsf, 0, sizeof(c->opsf));
    std::memset(&c->opsl, 0, sizeof(c->opsl));
    c->ops.N = c->opsf.N = c->opsl.N = hs.N;
    for (int i = 0; i < hs.N; ++i) {
        c->ops.w[i] = c->opsl.w[i] = hs.w[i];
        c->ops.winv[i] = c->opsl.winv[i] = 1.0 / hs.w[i];
        for (int j = 0; j < hs.N; ++j) {
            c->opsl.D[i][j] = hs.D[i * hs.N + j];
            c->opsl.S[i][j] = hs.S[i * hs.N + j];
        }
        if (hs.N > esdc::kMaxN) continue;           // the per-element kernels' operators (p <= 7)
        c->opsf.w[i] = (float)hs.w[i];
        c->opsf.winv[i] = (float)(1.0 / hs.w[i]);
        for (int j = 0; j < hs.N; ++j) {
            c->ops.D[i][j] = hs.D[i * hs.N + j];
            c->ops.SW[i][j] = hs.S[i * hs.N + j] / hs.w[j];
            c->ops.S[i][j] = hs.S[i * hs.N + j];
            c->opsf.D[i][j] = (float)hs.D[i * hs.N + j];
            c->opsf.S[i][j] = (float)hs.S[i * hs.N + j];
            c->opsf.ST[i][j] = (float)hs.S[j * hs.N + i];
            c->opsf.D2[i][j].x = c->opsf.D2[i][j].y = (float)hs.D[i * hs.N + j];
        }
    }
    const double R = 1.0 / (s.gamma * s.Ma * s.Ma);
    const double mu = s.Re > 0.0 ? 1.0 / s.Re : 0.0;
    const double cp = s.gamma * R / (s.gamma - 1.0);
    c->phys.gamma = s.gamma;
    c->phys.R = R;
    c->phys.mu = mu;
    c->phys.kappa = mu * cp / s.Pr;
    c->phys.inv_gm1 = 1.0 / (s.gamma - 1.0);
    c->phys.dissipation = s.dissipation;
    c->phys.viscous = mu > 0.0;
    c->phys.ip_coef = mu > 0.0 ? s.ip_coef : 0.0;
    c->physf.gamma = (float)s.gamma;
    c->physf.R = (float)R;
    c->physf.mu = (float)mu;
    c->physf.kappa = (float)c->phys.kappa;
    c->physf.inv_gm1 = (float)c->phys.inv_gm1;
    c->physf.rho0 = 1.0f;
    c->physf.p0 = (float)R;
    c->physf.dissipation = s.dissipation;
    c->physf.viscous = c->phys.viscous;

    cudaError_t e = cudaGetDevice(&c->device);
    const size_t N2 = (size_t)hs.N * hs.N;
    const size_t geom_bytes = (size_t)c->K * 10 * c->N3 * sizeof(double);
    c->red_blocks = 4 * esdc::sm_count();  // 4 blocks of 256 threads per SM, fixed per context (the order of
                                     // the reduction, so its result, depends only on the device)
    if (e == cudaSuccess) e = cudaMalloc(&c->d_geom, geom_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_nbr, (size_t)c->K * 6 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_trace, (size_t)c->K * 6 * 4 * N2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_red, (size_t)c->red_blocks * 5 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_red_out, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_lntab, esdc::kLnTab * 3 * sizeof(double));
    if (e == cudaSuccess) {
        std::vector<double> tab(esdc::kLnTab * 3);
        esdc::fill_ln_table(tab.data());
        e = cudaMemcpy(c->d_lntab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(c->d_geom, hs.geom.data(), geom_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<double> jinv((size_t)c->K * c->N3);
        for (int64_t el = 0; el < c->K; ++el)
            for (int i = 0; i < c->N3; ++i) jinv[el * c->N3 + i] = 1.0 / hs.geom[(el * 10) * c->N3 + i];
        e = cudaMalloc(&c->d_jinv, jinv.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_jinv, jinv.data(), jinv.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_nbr, hs.nbr.data(), hs.nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const size_t xyz_bytes = (size_t)c->K * 3 * c->N3 * sizeof(double);
        e = cudaMalloc(&c->d_xyz, xyz_bytes);
        if (e == cudaSuccess) e = cudaMemcpy(c->d_xyz, xyz, xyz_bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && hs.N == esdc::kLargeN) {
        e = cudaMalloc(&c->d_lr, (size_t)3 * c->n_nodes * 5 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_lwf, (size_t)c->K * 6 * 4 * N2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->d_lft, (size_t)c->K * 3 * 4 * c->N3 * sizeof(double));
    }
    if (e == cudaSuccess) {
        // |n_J| of the metric the interface terms use (surface metrics of the optimized metrics,
        // else the face values of the volume metrics), per face node in the kernels' face order
        const int N = hs.N, NN = N * N, N3 = NN * N;
        std::vector<double> fn((size_t)c->K * 6 * NN);
        for (int64_t el = 0; el < c->K; ++el)
            for (int l = 0; l < 3; ++l)
                for (int side = 0; side < 2; ++side) {
                    const int fix = side ? N - 1 : 0;
                    for (int t2 = 0; t2 < N; ++t2)
                        for (int t1 = 0; t1 < N; ++t1) {
                            const int fi = t1 + N * t2;
                            const int node = l == 0 ? fix + N * t1 + NN * t2
                                                    : (l == 1 ? t1 + N * fix + NN * t2 : t1 + N * t2 + NN * fix);
                            double n[3];
                            for (int m = 0; m < 3; ++m)
                                n[m] = hs.nsurf.empty()
                                           ? hs.geom[((size_t)el * 10 + 1 + 3 * l + m) * N3 + node]
                                           : hs.nsurf[(((size_t)el * 6 + 2 * l + side) * 3 + m) * NN + fi];
                            fn[((size_t)el * 6 + 2 * l + side) * NN + fi] = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                        }
                }
        e = cudaMalloc(&c->d_fnorm, fn.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_fnorm, fn.data(), fn.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !hs.nsurf.empty()) {
        e = cudaMalloc(&c->d_nsurf, hs.nsurf.size() * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_nsurf, hs.nsurf.data(), hs.nsurf.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = esdc::prepare_rhs_f64(c);
    if (e == cudaSuccess && s.precision == ESDC_PREC_FP32) {
        std::vector<float> gf(hs.geom.size());
        for (size_t i = 0; i < gf.size(); ++i) gf[i] = (float)hs.geom[i];
        e = cudaMalloc(&c->d_geomf, gf.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(c->d_geomf, gf.data(), gf.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_shadow, (size_t)c->n_nodes * 5 * sizeof(float));
        if (e == cudaSuccess && !hs.nsurf.empty()) {
            std::vector<float> nf(hs.nsurf.size());
            for (size_t i = 0; i < nf.size(); ++i) nf[i] = (float)hs.nsurf[i];
            e = cudaMalloc(&c->d_nsurff, nf.size() * sizeof(float));
            if (e == cudaSuccess) e = cudaMemcpy(c->d_nsurff, nf.data(), nf.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = esdc::prepare_rhs_f32(c);
    }
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "esdc_create");
    }
    *out = c;
    return ESDC_OK;
}

int esdc_destroy(esdc_ctx* ctx) {
    if (!ctx) return ESDC_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    free_ctx(ctx);
    cudaSetDevice(prev);
    return ESDC_OK;
}

int esdc_layout(const esdc_ctx* c, int64_t* K, int* N, int64_t* n_nodes) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    if (K) *K = c->K;
    if (N) *N = c->N;
    if (n_nodes) *n_nodes = c->n_nodes;
    return ESDC_OK;
}

int esdc_init_state(esdc_ctx* c, int ic, const double* params, double* q, void* stream) {
    if (!c || !q) return fail(ESDC_ERR_ARG, "null argument");
    esdc::InitParams prm{};
    const double R = c->phys.R;
    if (ic == ESDC_IC_TGV) {
    } else if (ic == ESDC_IC_VORTEX) {
        const double def[10] = {5.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < 10; ++i) prm.v[i] = params ? params[i] : def[i];
        const double na = std::sqrt(prm.v[4] * prm.v[4] + prm.v[5] * prm.v[5] + prm.v[6] * prm.v[6]);
        if (!(na > 0.0) || !std::isfinite(na)) return fail(ESDC_ERR_ARG, "the vortex axis must be a nonzero vector");
        for (int i = 4; i < 7; ++i) prm.v[i] /= na;
    } else if (ic == ESDC_IC_FREESTREAM) {
        const double def[5] = {1.0, 0.3, 0.2, 0.1, R};
        for (int i = 0; i < 5; ++i) prm.v[i] = params ? params[i] : def[i];
        if (!(prm.v[0] > 0.0) || !(prm.v[4] > 0.0)) return fail(ESDC_ERR_ARG, "rho and p must be positive");
    } else {
        return fail(ESDC_ERR_ARG, "ic must be ESDC_IC_TGV, ESDC_IC_VORTEX or ESDC_IC_FREESTREAM");
    }
    CUDA_TRY(esdc::launch_init_state(c, ic, prm, q, (cudaStream_t)stream));
    return ESDC_OK;
}

int esdc_geometry(const esdc_ctx* c, double* J, double* Ja) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    const size_t N3 = c->N3;
    for (int64_t e = 0; e < c->K; ++e) {
        if (J) CUDA_TRY(cudaMemcpy(J + e * N3, c->d_geom + e * 10 * N3, N3 * sizeof(double), cudaMemcpyDeviceToHost));
        if (Ja)
            CUDA_TRY(cudaMemcpy(Ja + e * 9 * N3, c->d_geom + (e * 10 + 1) * N3, 9 * N3 * sizeof(double),
                                cudaMemcpyDeviceToHost));
    }
    return ESDC_OK;
}

int esdc_rhs(esdc_ctx* c, const double* q, void* dqdt, void* stream) {
    if (!c || !q || !dqdt) return fail(ESDC_ERR_ARG, "null argument");
    const size_t elt = c->setup.precision == ESDC_PREC_FP64 ? sizeof(double) : sizeof(float);
    const uintptr_t a = (uintptr_t)q, b = (uintptr_t)dqdt;
    const uintptr_t na = c->n_nodes * 5 * sizeof(double), nb = c->n_nodes * 5 * elt;
    if (a < b + nb && b < a + na) return fail(ESDC_ERR_ARG, "q and dqdt overlap");
    return rhs_impl(c, q, dqdt, (cudaStream_t)stream);
}

int esdc_rhs_host(esdc_ctx* c, const double* q_host, void* dqdt_host, void* stream) {
    if (!c || !q_host || !dqdt_host) return fail(ESDC_ERR_ARG, "null argument");
    const size_t elt = c->setup.precision == ESDC_PREC_FP64 ? sizeof(double) : sizeof(float);
    const size_t qb = (size_t)c->n_nodes * 5 * sizeof(double), rb = (size_t)c->n_nodes * 5 * elt;
    if (!c->d_stage_q) {
        CUDA_TRY(cudaMalloc(&c->d_stage_q, qb));
        CUDA_TRY(cudaMalloc(&c->d_stage_r, rb));
    }
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(c->d_stage_q, q_host, qb, cudaMemcpyHostToDevice, s));
    int st = rhs_impl(c, c->d_stage_q, c->d_stage_r, s);
    if (st) return st;
    CUDA_TRY(cudaMemcpyAsync(dqdt_host, c->d_stage_r, rb, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ESDC_OK;
}

int esdc_workspace_bytes(const esdc_ctx* c, int what, size_t* bytes) {
    if (!c || !bytes) return fail(ESDC_ERR_ARG, "null argument");
    if (what != 0 && what != 1) return fail(ESDC_ERR_ARG, "unknown workspace kind");
    if (what == 1 && c->setup.precision == ESDC_PREC_FP32)
        *bytes = 10 * round256((size_t)c->n_nodes * 5 * sizeof(float)) + round256((size_t)c->n_nodes * 5 * sizeof(double));
    else if (what == 1) *bytes = 9 * round256((size_t)c->n_nodes * 5 * sizeof(double));
    else if (c->setup.precision == ESDC_PREC_FP64) *bytes = 7 * round256((size_t)c->n_nodes * 5 * sizeof(double));
    else *bytes = 8 * round256((size_t)c->n_nodes * 5 * sizeof(float));
    return ESDC_OK;
}

int esdc_rk_step(esdc_ctx* c, double* q, double dt, int nsteps, void* ws, size_t ws_bytes, void* stream) {
    if (!c || !q || !ws) return fail(ESDC_ERR_ARG, "null argument");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(ESDC_ERR_ARG, "nsteps >= 0 and finite dt required");
    size_t need = 0;
    esdc_workspace_bytes(c, 0, &need);
    if (ws_bytes < need) return fail(ESDC_ERR_ARG, "workspace too small");
    if (!aligned(ws, 256) || !aligned(q, 16)) return fail(ESDC_ERR_ARG, "q must be 16-byte and workspace 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->setup.bounded != 0 && !c->d_qext)
        return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    if (nsteps >= 2 && !c->profiling) {
        // graph replay; the float32 shadow of q is formed once, before the first step
        if (c->setup.precision == ESDC_PREC_FP32) {
            const int r = rk_shadow_f32(c, q, ws, s);
            if (r) return r;
        }
        const int r = rk_steps_graph(c, q, dt, nsteps, ws, s);
        if (r <= 0) return r;
        // graph unavailable: direct launches (the shadow is already in place)
        if (c->setup.precision == ESDC_PREC_FP32) return rk_steps_f32(c, q, dt, nsteps, ws, s);
        return rk_step_f64(c, q, dt, nsteps, ws, s, nullptr, nullptr);
    }
    if (c->setup.precision == ESDC_PREC_FP32) return rk_step_f32(c, q, dt, nsteps, ws, s);
    return rk_step_f64(c, q, dt, nsteps, ws, s, nullptr, nullptr);
}

int esdc_budgets(esdc_ctx* c, const double* q, const void* dqdt, double out[4], void* stream) {
    if (!c || !q || !out) return fail(ESDC_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = esdc::launch_budgets(c, q, dqdt, c->setup.precision == ESDC_PREC_FP32, nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "budgets launch");
    double r[5];
    CUDA_TRY(cudaMemcpyAsync(r, c->d_red_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < 4; ++i) out[i] = r[i];
    if (!dqdt) out[2] = out[3] = 0.0;
    if (r[4] > 0.0) return fail(ESDC_ERR_STATE, "non-finite or non-physical values at " + std::to_string((long long)r[4]) + " nodes");
    return ESDC_OK;
}

int esdc_budgets_async(esdc_ctx* c, const double* q, const void* dqdt, double* out_dev, void* stream) {
    if (!c || !q || !out_dev) return fail(ESDC_ERR_ARG, "null argument");
    cudaError_t e = esdc::launch_budgets(c, q, dqdt, c->setup.precision == ESDC_PREC_FP32, out_dev,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "budgets launch");
    return ESDC_OK;
}

int esdc_set_exterior(esdc_ctx* c, const double* q_ext) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    if (q_ext && !aligned(q_ext, 16)) return fail(ESDC_ERR_ARG, "q_ext must be 16-byte aligned");
    c->d_qext = q_ext;
    return prepare_variant(c);
}

int esdc_set_source(esdc_ctx* c, const double* src) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    if (src && !aligned(src, 16)) return fail(ESDC_ERR_ARG, "source must be 16-byte aligned");
    c->d_src = src;
    return prepare_variant(c);
}

int esdc_mms_fields(double gamma, double Ma, double Re, double Pr, double L, const double* table, int64_t n,
                    const double* x, double* q, double* src) {
    if (!table || !x || n < 0) return fail(ESDC_ERR_ARG, "null argument or negative count");
    if (!(gamma > 1.0) || !(Ma > 0.0) || !(Pr > 0.0) || !(L > 0.0) || !std::isfinite(Re))
        return fail(ESDC_ERR_ARG, "gamma > 1, Ma > 0, Pr > 0, L > 0 and finite Re required");
    esdc::mms_fields(gamma, Ma, Re, Pr, L, table, n, x, q, src);
    return ESDC_OK;
}

int esdc_dt_cfl(esdc_ctx* c, const double* q, double cfl, double* dt, void* stream) {
    if (!c || !q || !dt) return fail(ESDC_ERR_ARG, "null argument");
    if (!(cfl > 0.0)) return fail(ESDC_ERR_ARG, "cfl must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = esdc::launch_cfl(c, q, s);
    if (e != cudaSuccess) return cuda_fail(e, "cfl launch");
    double r[3];
    CUDA_TRY(cudaMemcpyAsync(r, c->d_red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (r[2] > 0.0 || !(r[0] > 0.0)) return fail(ESDC_ERR_STATE, "non-physical state in esdc_dt_cfl");
    const double N2 = (double)c->N * c->N;
    double d = c->h_min / (N2 * r[0]);
    if (c->phys.viscous) {
        const double rho_min = -r[1];
        const double nu = std::fmax(4.0 / 3.0, c->setup.gamma / c->setup.Pr) * c->phys.mu / rho_min;
        d = std::fmin(d, c->h_min * c->h_min / (N2 * N2 * nu));
    }
    *dt = cfl * d;
    return ESDC_OK;
}

int esdc_rhs_vjp(esdc_ctx* c, const double* q, const double* lam, double* grad, double* grad_mu, void* stream) {
    if (!c || !q || !lam || !grad) return fail(ESDC_ERR_ARG, "null argument");
    int st = ensure_adjoint(c);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (grad_mu) CUDA_TRY(cudaMemsetAsync(c->d_adj_acc, 0, sizeof(double), s));
    cudaError_t e = esdc::launch_rhs_vjp(c, q, lam, grad, grad_mu ? c->d_adj_acc : nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "esdc_rhs_vjp launch");
    if (grad_mu) {
        CUDA_TRY(cudaMemcpyAsync(grad_mu, c->d_adj_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return ESDC_OK;
}

int esdc_ke_gradient(esdc_ctx* c, const double* q, double* grad, void* stream) {
    if (!c || !q || !grad) return fail(ESDC_ERR_ARG, "null argument");
    cudaError_t e = esdc::launch_ke_gradient(c, q, grad, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "esdc_ke_gradient");
    return ESDC_OK;
}

int esdc_rk_adaptive(esdc_ctx* c, double* q, double t0, double t_end, double* dt_inout, double rtol, double atol,
                     int max_steps, void* ws, size_t ws_bytes, double* stats, double* dt_history, int history_capacity,
                     void* stream) {
    if (!c || !q || !ws || !dt_inout) return fail(ESDC_ERR_ARG, "null argument");
    if (!std::isfinite(t0) || !std::isfinite(t_end) || t_end < t0 || !(*dt_inout > 0.0) ||
        !std::isfinite(*dt_inout) || !(rtol > 0.0) || !(atol > 0.0) || max_steps < 0 || history_capacity < 0)
        return fail(ESDC_ERR_ARG, "need t0 <= t_end, dt > 0, rtol > 0, atol > 0, max_steps >= 0");
    size_t need = 0;
    esdc_workspace_bytes(c, 1, &need);
    if (ws_bytes < need) return fail(ESDC_ERR_ARG, "workspace too small");
    if (!aligned(ws, 256) || !aligned(q, 16))
        return fail(ESDC_ERR_ARG, "q must be 16-byte and workspace 256-byte aligned");
    if (c->setup.bounded != 0 && !c->d_qext)
        return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    if (c->setup.precision == ESDC_PREC_FP32)
        return rk_adaptive_f32(c, q, t0, t_end, dt_inout, rtol, atol, max_steps, ws, stats, dt_history,
                               history_capacity, (cudaStream_t)stream);
    return rk_adaptive_f64(c, q, t0, t_end, dt_inout, rtol, atol, max_steps, ws, stats, dt_history, history_capacity,
                           (cudaStream_t)stream);
}

int esdc_rk_step_ckpt(esdc_ctx* c, double* q, double dt, int nsteps, double* ckpt, int store_k1, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!c || !q || !ckpt) return fail(ESDC_ERR_ARG, "null argument");
    const size_t n5 = (size_t)c->n_nodes * 5;
    cudaStream_t s = (cudaStream_t)stream;
    if (store_k1) {
        // direct launches of the float64 step, the first residual written into the checkpoint
        if (c->setup.precision != ESDC_PREC_FP64) return fail(ESDC_ERR_UNSUPPORTED, "store_k1 needs a float64 context");
        if (!ws) return fail(ESDC_ERR_ARG, "null argument");
        if (nsteps < 0 || !std::isfinite(dt)) return fail(ESDC_ERR_ARG, "nsteps >= 0 and finite dt required");
        size_t need = 0;
        esdc_workspace_bytes(c, 0, &need);
        if (ws_bytes < need) return fail(ESDC_ERR_ARG, "workspace too small");
        if (!aligned(ws, 256) || !aligned(q, 16) || !aligned(ckpt, 16))
            return fail(ESDC_ERR_ARG, "q/ckpt must be 16-byte and workspace 256-byte aligned");
        if (c->setup.bounded != 0 && !c->d_qext)
            return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    }
    for (int step = 0; step < nsteps; ++step) {
        double* qs = ckpt + (store_k1 ? 2 * (size_t)step : (size_t)step) * n5;
        CUDA_TRY(cudaMemcpyAsync(qs, q, n5 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const int st = store_k1 ? rk_step_f64(c, q, dt, 1, ws, s, nullptr, qs + n5)
                                : esdc_rk_step(c, q, dt, 1, ws, ws_bytes, stream);
        if (st) return st;
    }
    return ESDC_OK;
}

int esdc_rk_adjoint_workspace_bytes(const esdc_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(ESDC_ERR_ARG, "null argument");
    *bytes = 12 * round256((size_t)c->n_nodes * 5 * sizeof(double));
    return ESDC_OK;
}

int esdc_rk_adjoint(esdc_ctx* c, const double* ckpt, int store_k1, double dt, int nsteps, double* lam,
                    double* grad_mu, void* ws, size_t ws_bytes, void* stream) {
    int st = adjoint_checks(c, ckpt, dt, nsteps, lam, ws, ws_bytes);
    if (st) return st;
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(double));
    double* K6[6];            // stage derivatives of the recomputation, then the stage cotangents psi_t
    double* Qs[6];
    for (int j = 0; j < 6; ++j) K6[j] = (double*)((char*)ws + j * sub);
    Qs[0] = nullptr;
    for (int j = 1; j < 6; ++j) Qs[j] = (double*)((char*)ws + (5 + j) * sub);
    double* kappa = (double*)((char*)ws + 11 * sub);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(c->d_adj_acc, 0, sizeof(double), s));
    for (int step = nsteps - 1; step >= 0; --step) {
        const double* qn = ckpt + (store_k1 ? 2 * (size_t)step : (size_t)step) * n;
        // recompute the stage states of this step from its checkpoint: Y_1 = q_n and Y_t from the
        // stage derivatives k_1 .. k_(t-1), so five residuals (k_6 = f(Y_6) is not needed), four when
        // the checkpoint holds k_1 = f(q_n)
        const double* kin[6] = {K6[0], K6[1], K6[2], K6[3], K6[4], K6[5]};
        if (store_k1) kin[0] = qn + n;
        for (int t = 0; t < 6; ++t) {
            const double* qs = qn;
            if (t > 0) {
                esdc::Combine cb{};
                cb.nk = t;
                for (int j = 0; j < t; ++j) {
                    cb.k[j] = kin[j];
                    cb.coef[j] = dt * kA[t][j];
                }
                cudaError_t e = esdc::launch_combine(Qs[t], qn, cb, n, s);
                if (e != cudaSuccess) return cuda_fail(e, "adjoint stage recompute");
                qs = Qs[t];
            }
            if (t == 5) break;
            if (t == 0 && store_k1) continue;
            st = rhs_impl(c, qs, K6[t], s);
            if (st) return st;
        }
        const double* Y[6] = {qn, Qs[1], Qs[2], Qs[3], Qs[4], Qs[5]};
        st = adjoint_step(c, Y, dt, lam, K6, kappa, s);
        if (st) return st;
    }
    return adjoint_finish(c, grad_mu, s);
}

int esdc_rk_step_stages(esdc_ctx* c, double* q, double dt, int nsteps, double* stages, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!c || !q || !ws || !stages) return fail(ESDC_ERR_ARG, "null argument");
    if (c->setup.precision != ESDC_PREC_FP64) return fail(ESDC_ERR_UNSUPPORTED, "stage storage needs a float64 context");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(ESDC_ERR_ARG, "nsteps >= 0 and finite dt required");
    size_t need = 0;
    esdc_workspace_bytes(c, 0, &need);
    if (ws_bytes < need) return fail(ESDC_ERR_ARG, "workspace too small");
    if (!aligned(ws, 256) || !aligned(q, 16) || !aligned(stages, 16))
        return fail(ESDC_ERR_ARG, "q/stages must be 16-byte and workspace 256-byte aligned");
    if (c->setup.bounded != 0 && !c->d_qext)
        return fail(ESDC_ERR_ARG, "a bounded box needs an exterior state (esdc_set_exterior)");
    return rk_step_f64(c, q, dt, nsteps, ws, (cudaStream_t)stream, stages, nullptr);
}

int esdc_rk_adjoint_stages(esdc_ctx* c, const double* stages, double dt, int nsteps, double* lam, double* grad_mu,
                           void* ws, size_t ws_bytes, void* stream) {
    int st = adjoint_checks(c, stages, dt, nsteps, lam, ws, ws_bytes);
    if (st) return st;
    const int64_t n = c->n_nodes * 5;
    const size_t sub = round256((size_t)n * sizeof(double));
    double* psi[6];
    for (int j = 0; j < 6; ++j) psi[j] = (double*)((char*)ws + j * sub);
    double* kappa = (double*)((char*)ws + 6 * sub);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(c->d_adj_acc, 0, sizeof(double), s));
    for (int step = nsteps - 1; step >= 0; --step) {
        const double* Y[6];
        for (int t = 0; t < 6; ++t) Y[t] = stages + ((size_t)step * 6 + t) * n;
        st = adjoint_step(c, Y, dt, lam, psi, kappa, s);
        if (st) return st;
    }
    return adjoint_finish(c, grad_mu, s);
}

int esdc_device_status(esdc_ctx* c, int* status, int clear, void* stream) {
    if (!c || !status) return fail(ESDC_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (clear) CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ESDC_OK;
}

int esdc_profile(esdc_ctx* c, int on) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    c->profiling = on ? 1 : 0;
    c->prof_used = 0;
    return ESDC_OK;
}

int esdc_profile_read(esdc_ctx* c, double* ms_main, double* ms_face, int64_t* count) {
    if (!c) return fail(ESDC_ERR_ARG, "null context");
    double a = 0.0, b = 0.0;
    const size_t n = c->prof_used / 4;
    for (size_t i = 0; i < n; ++i) {
        cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(&c->prof_events[4 * i]);
        CUDA_TRY(cudaEventSynchronize(ev[3]));
        float x = 0.f, y = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&x, ev[0], ev[1]));
        CUDA_TRY(cudaEventElapsedTime(&y, ev[2], ev[3]));
        a += x;
        b += y;
    }
    if (ms_main) *ms_main = a;
    if (ms_face) *ms_face = b;
    if (count) *count = (int64_t)n;
    c->prof_used = 0;
    return ESDC_OK;
}

int esdc_probe_fma(int kind, double* flops_per_s, void* stream) {
    if (!flops_per_s || (kind != 0 && kind != 1)) return fail(ESDC_ERR_ARG, "kind 0 or 1 and an output pointer");
    cudaError_t e = esdc::probe_fma(kind, flops_per_s, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "esdc_probe_fma");
    return ESDC_OK;
}

}  // extern "C"
