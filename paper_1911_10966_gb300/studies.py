"""Workload studies on one GPU (each prints JSON lines):

  python -m paper_1911_10966_gb300.studies precision   # TGV 48^3 p=7, 200 DP5 steps, fp32-mixed vs fp64
  python -m paper_1911_10966_gb300.studies psweep      # p = 2..7 at ~16M nodes (+ the 256^3-node meshes
                                                        #   of the paper's cost study, Sec. 5.2, p = 1, 3, 7)
  python -m paper_1911_10966_gb300.studies hconv       # isentropic vortex L2 error, p = 3, 4, 5, 4^3..32^3
  python -m paper_1911_10966_gb300.studies variants    # ES-C / SF-KG / DC DP5 step time, 256^3 nodes, p = 1, 3, 7
  python -m paper_1911_10966_gb300.studies mms         # manufactured solution, Dirichlet boundaries: error vs cost

All arithmetic runs in libesdc.so; this module only sets up meshes and states, times calls with CUDA
events and computes error norms of the returned fields.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np
import torch

from . import inputs as I
from .solver import Solver, lgl


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_rhs(s: Solver, q, reps=5):
    r = s.rhs(q)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(reps):
        s.rhs(q, out=r)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time_step(s: Solver, q, dt, reps=3):
    s.rk_step(q, dt, 1)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    s.rk_step(q, dt, reps)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def precision(steps=200, sample_every=20, k=48, p=7):
    """Taylor-Green vortex, Re 1600, Ma 0.1, k^3 affine hexahedra on [-pi, pi]^3, p = 7: the same
    fixed-step DP5 trajectory with the float64 residual and with the float32-mixed residual; the
    kinetic-energy and entropy dissipation rates (float64 budgets of each state) are compared."""
    t0 = time.time()
    s64 = Solver.box(p, k, k, k, Re=1600.0)
    s32 = Solver(p, k, k, k, s64.coords, Re=1600.0, precision="fp32")
    q0 = I.taylor_green(s64.coords)
    n = s64.n_nodes
    q64 = s64.to_device(q0)
    del q0
    q32 = q64.clone()
    dt = s64.dt_cfl(q64, 0.5)
    setup_s = time.time() - t0
    vol = (2 * math.pi) ** 3
    hist = []
    ms64 = ms32 = 0.0
    for it in range(0, steps + 1, sample_every):
        r64 = s64.rhs(q64)
        b64 = s64.budgets(q64, r64)
        del r64
        r32 = s32.rhs(q32)
        b32 = s32.budgets(q32, r32)
        del r32
        hist.append({"step": it, "t": it * dt, "ke64": b64[1] / vol, "ke32": b32[1] / vol,
                     "dke64": b64[3] / vol, "dke32": b32[3] / vol, "ds64": b64[2] / vol, "ds32": b32[2] / vol})
        if it == steps:
            break
        a, b = _events()
        a.record()
        s64.rk_step(q64, dt, sample_every)
        b.record()
        torch.cuda.synchronize()
        ms64 += a.elapsed_time(b)
        a.record()
        s32.rk_step(q32, dt, sample_every)
        b.record()
        torch.cuda.synchronize()
        ms32 += a.elapsed_time(b)
    rel = lambda a, b: abs(a - b) / abs(b)
    out = {"study": "precision", "workload": f"TGV Re1600 Ma0.1 {k}^3 affine p={p}", "nodes": n, "steps": steps,
           "dt": dt, "setup_s": setup_s,
           "f64": {"ms_per_step": ms64 / steps, "node_rhs_per_s": n * 6 / (ms64 / steps * 1e-3)},
           "f32_mixed": {"ms_per_step": ms32 / steps, "node_rhs_per_s": n * 6 / (ms32 / steps * 1e-3)},
           "dke_rel_err_final": rel(hist[-1]["dke32"], hist[-1]["dke64"]),
           "dke_rel_err_max": max(rel(h["dke32"], h["dke64"]) for h in hist),
           "ds_rel_err_final": rel(hist[-1]["ds32"], hist[-1]["ds64"]),
           "ds_rel_err_max": max(rel(h["ds32"], h["ds64"]) for h in hist),
           "ke_rel_err_final": rel(hist[-1]["ke32"], hist[-1]["ke64"]),
           "history": hist}
    print(json.dumps(out), flush=True)
    return out


# elements per direction giving ~16M nodes per degree (N^3 K ~ 16.0M)
PSWEEP = {2: 84, 3: 63, 4: 50, 5: 42, 6: 36, 7: 32}
# the paper's cost study: 256 DOF per direction (16,777,216 nodes) at p = 1, 3, 7 (Sec. 5.2), and
# p = 15 (float64 only: the multi-pass residual)
PAPER_E3 = {1: 128, 3: 64, 7: 32}
PAPER_E3_P15 = {15: 16}


def psweep():
    """Residual throughput (nodes x RHS / s) per polynomial degree at ~16M nodes, Taylor-Green
    Re = 1600 and inviscid, float64 and float32-mixed; plus the DP5 step time on the paper's
    256^3-node cost-study meshes."""
    rows = []
    for p, k in PSWEEP.items():
        for Re in (1600.0, 0.0):
            for prec in ("fp64", "fp32"):
                s = Solver.box(p, k, k, k, Re=Re, precision=prec)
                q = s.to_device(I.taylor_green(s.coords))
                ms = _time_rhs(s, q)
                row = {"study": "psweep", "p": p, "k": k, "nodes": s.n_nodes, "Re": Re, "precision": prec,
                       "rhs_ms": ms, "node_rhs_per_s": s.n_nodes / (ms * 1e-3)}
                print(json.dumps(row), flush=True)
                rows.append(row)
                del q, s
                torch.cuda.empty_cache()
    for p, k in PAPER_E3.items():
        for prec in ("fp64", "fp32"):
            s = Solver.box(p, k, k, k, Re=1600.0, Ma=0.05, precision=prec)
            q = s.to_device(I.taylor_green(s.coords, Ma=0.05))
            dt = s.dt_cfl(q, 0.5)
            ms = _time_step(s, q, dt)
            row = {"study": "paper_cost_mesh", "p": p, "k": k, "nodes": s.n_nodes, "Ma": 0.05, "Re": 1600.0,
                   "precision": prec, "dp5_step_ms": ms, "node_rhs_per_s": s.n_nodes * 6 / (ms * 1e-3)}
            print(json.dumps(row), flush=True)
            rows.append(row)
            del q, s
            torch.cuda.empty_cache()
    return rows


def variants():
    """The paper's cost comparison (Sec. 5.2, "Error vs. cost" figure): Taylor-Green at Ma 0.05,
    Re 1600, 256^3 nodes at p = 1, 3, 7, 15, time per fixed DP5 step (six residuals) with the ES-C,
    SF-KG and DC volume fluxes in float64."""
    rows = []
    for p, k in {**PAPER_E3, **PAPER_E3_P15}.items():
        for vf in ("esc", "kg", "dc"):
            s = Solver.box(p, k, k, k, Re=1600.0, Ma=0.05, volume_flux=vf)
            q = s.to_device(I.taylor_green(s.coords, Ma=0.05))
            dt = s.dt_cfl(q, 0.5)
            ms = _time_step(s, q, dt)
            row = {"study": "variants", "p": p, "k": k, "nodes": s.n_nodes, "volume_flux": vf, "dp5_step_ms": ms,
                   "node_rhs_per_s": s.n_nodes * 6 / (ms * 1e-3), "rhs_ms": _time_rhs(s, q)}
            print(json.dumps(row), flush=True)
            rows.append(row)
            del q, s
            torch.cuda.empty_cache()
    return rows


def mms(t_end=1.5):
    """The paper's viscous error-vs-cost study (Sec. 5.1): the supersonic manufactured solution on
    [0, 1]^3 with exact Dirichlet data on every boundary, Re = 4e6, marched from the exact field with
    fixed DP5 steps at CFL 0.5 for t_end = 1.5 flow-through times (the supersonic flow carries
    every perturbation out of the box), ES-C and DC, p = 1..4.  Reports the P-norm L2 error of rho
    against the exact field and the wall time."""
    from .solver import mms_fields
    rows = []
    for vf in ("esc", "dc"):
        for p, ks in ((1, (4, 8, 16, 32)), (2, (4, 8, 16)), (3, (4, 8, 16)), (4, (4, 8, 16))):
            prev = None
            for k in ks:
                s = Solver.box(p, k, k, k, lo=(0.0,) * 3, hi=(1.0,) * 3, Ma=I.MMS_MA, Re=I.MMS_RE,
                               bounded=(True, True, True), volume_flux=vf)
                qx, src = mms_fields(s.coords, I.manufactured_table(), gamma=1.4, Ma=I.MMS_MA, Re=I.MMS_RE,
                                     Pr=0.72, L=1.0)
                exact = s.to_device(qx)
                sd = s.to_device(src)
                s.set_exterior(exact)
                s.set_source(sd)
                q = exact.clone()
                dt0 = s.dt_cfl(q, 0.5)
                nsteps = max(1, int(math.ceil(t_end / dt0)))
                dt = t_end / nsteps
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.rk_step(q, dt, nsteps)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
                J, _ = s.geometry()
                _, wq = lgl(p)
                P = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
                err = ((q[:, 0] - exact[:, 0]).cpu().numpy()) ** 2
                l2 = float(np.sqrt((P[None] * J * err).sum()))
                row = {"study": "mms", "volume_flux": vf, "p": p, "k": k, "nodes": s.n_nodes, "steps": nsteps,
                       "l2_rho": l2, "wall_s": wall,
                       "order": (math.log(prev / l2) / math.log(2.0)) if prev else None}
                prev = l2
                print(json.dumps(row), flush=True)
                rows.append(row)
                del q, exact, sd, s
    return rows


def _vortex(x, t, u_inf, Ma=0.5):
    """Exact translating isentropic vortex (axis along x3) at time t, periodic images ignored."""
    c = (u_inf[0] * t, u_inf[1] * t, 0.0)
    return I.isentropic_vortex(x, Ma=Ma, beta=5.0, center=c, axis=(0.0, 0.0, 1.0), u_inf=u_inf)


def hconv(t_final=0.5):
    """Isentropic vortex (strength 5, Ma 0.5, axis x3, drift (1, -1, 0)/sqrt(2)) on [-5,5]^3,
    inviscid, advanced to t_final with DP5 at CFL 0.25; P-norm L2 error of rho against the exact
    translated vortex, p = 3, 4, 5 on 4^3 .. 32^3 (the axis along x3 keeps the periodic-image floor
    near 2e-5, see the study notes)."""
    u_inf = (1 / math.sqrt(2), -1 / math.sqrt(2), 0.0)
    rows = []
    for p in (3, 4, 5):
        prev = None
        for k in (4, 8, 16, 32):
            s = Solver.box(p, k, k, k, lo=(-5.0,) * 3, hi=(5.0,) * 3, Ma=0.5, Re=0.0)
            q = s.to_device(_vortex(s.coords, 0.0, u_inf))
            dt0 = s.dt_cfl(q, 0.25)
            nsteps = max(1, int(math.ceil(t_final / dt0)))
            dt = t_final / nsteps
            s.rk_step(q, dt, nsteps)
            ex = _vortex(s.coords, t_final, u_inf)
            J, _ = s.geometry()
            _, wq = lgl(p)
            P = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
            err = (q[:, 0].cpu().numpy() - ex[:, 0]) ** 2
            l2 = float(np.sqrt((P[None] * J * err).sum()))
            row = {"study": "hconv", "p": p, "k": k, "h": 10.0 / k, "steps": nsteps, "l2_rho": l2,
                   "order": (math.log(prev / l2) / math.log(2.0)) if prev else None}
            prev = l2
            print(json.dumps(row), flush=True)
            rows.append(row)
            del q, s
    return rows


def rhs(p=4, k=16, volume_flux="esc", Re=1600.0, precision="fp64", warp=0.1, reps=5):
    """Residual time of one configuration (Taylor-Green on the warped periodic box), `reps` timed
    calls after one warm-up: the command the kernel profiles are taken on."""
    s = Solver.box(p, k, k, k, warp=warp, Re=Re, precision=precision, volume_flux=volume_flux)
    q = s.to_device(I.taylor_green(s.coords))
    ms = _time_rhs(s, q, reps=reps)
    row = {"study": "rhs", "p": p, "k": k, "nodes": s.n_nodes, "Re": Re, "precision": precision,
           "volume_flux": volume_flux, "rhs_ms": ms, "node_rhs_per_s": s.n_nodes / (ms * 1e-3)}
    print(json.dumps(row), flush=True)
    return [row]


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "psweep"
    if which == "rhs":
        kw = dict(a.split("=", 1) for a in sys.argv[2:])
        conv = {"p": int, "k": int, "Re": float, "warp": float, "reps": int}
        rhs(**{key: conv.get(key, str)(val) for key, val in kw.items()})
    else:
        {"precision": precision, "psweep": psweep, "hconv": hconv, "variants": variants, "mms": mms}[which]()
