"""Helpers shared by the GPU tests: build the CUDA solver and the oracle on the same seeded workload.

Each side computes its own LGL nodes and feeds them to the shared input module (node placement and
initial states only); nothing computed by one side is handed to the other.
"""
import math

import numpy as np
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

TWO_PI_BOX = ([-math.pi] * 3, [math.pi] * 3)


def make_pair(p, k, *, warp=0.0, seed=0, Ma=0.1, Re=1600.0, dissipation=True, box=TWO_PI_BOX,
              state="tgv", noise=0.0, noise_seed=1, precision="fp64", oracle_elems=None, volume_flux="esc",
              metrics="curl"):
    """GPU solver + state and the oracle's mesh + state for the same workload.  With oracle_elems
    the oracle side is the two-ring submesh around those elements (returned mesh/state are the
    submesh's; the residual rows of oracle_elems are returned as mesh.rows)."""
    from paper_1911_10966_gb300.solver import Solver, lgl
    kx, ky, kz = k
    lo, hi = box
    xi_gpu, _ = lgl(p)
    x_gpu = I.box_coords(xi_gpu, kx, ky, kz, lo, hi, warp=warp, seed=seed)
    solver = Solver(p, kx, ky, kz, x_gpu, Ma=Ma, Re=Re, dissipation=dissipation, precision=precision,
                    volume_flux=volume_flux, metrics=metrics)
    s = O.sbp_operator(p)
    x_ora = I.box_coords(s.xi.numpy(), kx, ky, kz, lo, hi, warp=warp, seed=seed)
    gas = O.Gas.from_mach(Ma, Re)
    if oracle_elems is not None:
        mesh, E2, rows = O.make_submesh(p, x_ora, O.box_neighbours(kx, ky, kz), oracle_elems, metrics=metrics)
        mesh.rows = rows
        x_ora = x_ora[E2.numpy()]
    else:
        mesh = O.make_mesh(p, x_ora, kx, ky, kz, metrics=metrics)

    def st(x):
        if state == "tgv":
            q = I.taylor_green(x, Ma=Ma)
        elif state == "freestream":
            q = I.freestream(x, Ma=Ma)
        elif state == "vortex":
            q = I.isentropic_vortex(x, Ma=Ma, u_inf=(1 / math.sqrt(2), -1 / math.sqrt(2), 0.0))
        else:
            raise ValueError(state)
        return I.perturb(q, seed=noise_seed, rel=noise) if noise > 0 else q

    return solver, solver.to_device(st(x_gpu)), mesh, gas, torch.tensor(st(x_ora))


EPS64 = 2.220446049250313e-16


def term_scale(q, mesh, gas, elems=None):
    """T_v = max over nodes of sum_l sum_j |2 D_ij| |f_v(q_i, q_j)| / J: the magnitude of the terms
    whose sum is the residual.  Rounding in any float64 evaluation of the residual (the oracle's
    included) is of order eps * T_v, which exceeds 1e-12 ||R_v|| for smooth low-Mach states where
    the pressure flux (~1/(gamma Ma^2)) cancels to O(1)."""
    import dataclasses
    q = torch.as_tensor(q, dtype=torch.float64)
    E = torch.arange(q.shape[0]) if elems is None else torch.as_tensor(elems)
    sabs = dataclasses.replace(mesh.sbp, D=mesh.sbp.D.abs())
    t = O.volume_term(q[E], mesh.Ja[E], sabs, gas, flux=lambda a, b, n, g: O.ec_flux_n(a, b, n, g).abs())
    t = t.abs() / mesh.J[E].unsqueeze(1)
    return [float(t[:, v].max()) for v in range(5)]


def geometry_rounding(p):
    """Relative round-off of a float64 curl-form metric construction at degree p beyond 7: D is
    applied twice, so the two sides' independent constructions differ by ~eps |D|^2 with
    |D| = p(p+1)/4 (measured 2 eps |D|^2 at p = 15 against each other, each within a few ulps of a
    40-digit D); 16 eps |D|^2 bounds it.  Up to p = 7 the c_round term below already covers it."""
    return 0.0 if p <= 7 else 16 * EPS64 * (p * (p + 1) / 4.0) ** 2


def assert_parity(r_gpu, r_ora, q_ora, mesh, gas, elems=None, tol=1e-12, c_round=8.0, geo_rel=0.0):
    """Per variable: ||R_gpu - R_ora||_inf <= max(tol ||R_ora||_inf, c_round eps T_v, geo_rel T_v).
    c_round = 8: the two evaluation orders of the oracle itself differ by about 1 eps T_v, and at
    p = 7 the two independent float64 constructions of the curl-form metrics (which differ by ~4e-13
    relative) add up to 4.5 eps T_v in the momentum residual of the 48^3 Taylor-Green mesh.
    geo_rel: the metric round-off of geometry_rounding(p) for degrees above 7."""
    a = r_gpu.detach().double().cpu()
    b = torch.as_tensor(r_ora).double()
    T = term_scale(q_ora, mesh, gas, elems)
    rep = []
    for v in range(5):
        err = float((a[:, v] - b[:, v]).abs().max())
        R = float(b[:, v].abs().max())
        bound = max(tol * R, c_round * EPS64 * T[v], geo_rel * T[v])
        rep.append((v, err / R if R > 0 else err, EPS64 * T[v] / R if R > 0 else float("inf")))
        assert err <= bound, f"variable {v}: |dR| = {err:.3e}, ||R|| = {R:.3e}, eps*T = {EPS64 * T[v]:.3e}"
    print("parity (v, normwise, eps*kappa):", " ".join(f"{v}:{e:.1e}/{k:.1e}" for v, e, k in rep))
    return rep


def normwise_errors(r_gpu, r_ora, abs_floor=0.0):
    """Per-variable ||R_gpu - R_ora||_inf / max(||R_ora||_inf, abs_floor)."""
    a = r_gpu.detach().double().cpu()
    b = torch.as_tensor(r_ora).double()
    out = []
    for v in range(5):
        den = max(float(b[:, v].abs().max()), abs_floor)
        out.append(float((a[:, v] - b[:, v]).abs().max()) / den)
    return out
