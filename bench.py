"""Benchmark of the ES-C residual + DP5 step on one GB300 (prints one JSON line).

Headline workload: Taylor-Green vortex, Re = 1600, Ma = 0.1, on a 48^3 periodic box of affine
hexahedra on [-pi, pi]^3, p = 7 (512 nodes per element, 56,623,104 nodes, 2.26 GB of float64 state),
float64 residual.  One step = one fixed Dormand-Prince 5 step at CFL 0.5 (six residual evaluations,
stage combinations) plus the float64 budget reduction of the new state.
Metric: residual DOF/s = nodes x residual evaluations / s.

The same line carries, on the same mesh, the float32-mixed form (step rate, residual error per
variable, and the kinetic-energy and entropy dissipation-rate errors after 200 DP5 steps against the
float64 trajectory), and as secondary objects: the 16^3 warped p = 4 Taylor-Green workload, the
adjoint cost on it and on the 8^3 warped p = 4 isentropic vortex (50 steps), the polynomial-degree
sweep at ~16 M nodes (p = 2..7, float64 and float32-mixed, viscous and inviscid), the volume-flux
variants, the adaptive integrator and, from the CPU-baseline leg, the oracle's timings and the
parity of the GPU residuals against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --study ipsweep|mms|hconv|variants|rhs [key=value ...]   (extra studies, JSON lines)

N > 1 (under torchrun): every rank advances an independent replica of the workload (no data-path
collective); value = all ranks' node-residuals / max-over-ranks time ("weak" scaling).
--impl reference times the CPU oracle (plain float64 torch) on the host cores instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PI_BOX = ((-math.pi,) * 3, (math.pi,) * 3)
HEADLINE = dict(name="tgv_48cubed_p7_affine", p=7, k=48, warp=0.0, seed=0, Ma=0.1, Re=1600.0, cfl=0.5)
TGV_SMALL = dict(name="tgv_4cubed_p3_affine", p=3, k=4, warp=0.0, seed=0, Ma=0.1, Re=1600.0, cfl=0.5)
TGV_WARPED = dict(name="tgv_16cubed_p4_warped", p=4, k=16, warp=0.1, seed=0, Ma=0.1, Re=1600.0, cfl=0.5)
VORTEX = dict(name="vortex_8cubed_p4_warped", p=4, k=8, warp=0.1, seed=1, Ma=0.5, Re=1000.0, cfl=0.5,
              lo=(-5.0,) * 3, hi=(5.0,) * 3, steps=50)
# isentropic vortex of the adjoint workload: strength 5, centre 0, axis (1,1,1), drift (1,-1,0)/sqrt 2
VORTEX_PARAMS = [5.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 1 / math.sqrt(2), -1 / math.sqrt(2), 0.0]
# elements per direction giving ~16M nodes per degree (the polynomial-degree sweep meshes)
PSWEEP_K = {2: 84, 3: 63, 4: 50, 5: 42, 6: 36, 7: 32}
PRECISION_STEPS = 200
RHS_PER_STEP = 6
L2_BYTES = 129 * 2 ** 20
# the oracle's sample of the headline mesh: a contiguous block of SAMPLE_BLOCK^3 elements (with the
# two rings of neighbours whose face states and gradients its residual reads)
SAMPLE_BLOCK = 8
CPU_BASELINE_SECONDS = 10.0
FP64_NOMINAL_TFLOPS = 1.25       # GB300 float64 (non-tensor) rate at the 2070 MHz maximum SM clock
HBM_FALLBACK_GBS = 6800.0


def nodes_of(w) -> int:
    return w["k"] ** 3 * (w["p"] + 1) ** 3


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of the GB300s, else the fallback."""
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(f))["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "of fallback"


# ------------------------------------------------------------------------------------------------
# Algorithmic work per node per residual evaluation (convention: +, -, * = 1 flop; fma = 2;
# division, square root and logarithm = 1 each).  Counted from the operations the method needs on
# a curvilinear mesh with the viscous terms on and the log means on their series branch.
# ------------------------------------------------------------------------------------------------
FLOPS_PAIR = 82          # one two-point flux contracted with the averaged metric + pair accumulation
FLOPS_LINE_NODE = 30     # per node: three directions x (5 mul + 5 add) scaling by 1/w
FLOPS_NODE_PRE = 22      # primitives, beta and entropy variables
FLOPS_SAT_NODE = 140     # per face node: neighbour primitives, EC flux, LLF dissipation, lift
FLOPS_VISC_NODE = 211    # physical gradient, tau, heat flux, contravariant fluxes (plus 24N + 96/N)
FLOPS_DIV_NODE = 12      # (plus 24N) divergence of the contravariant viscous fluxes
FLOPS_SCALE_NODE = 5
FLOPS_VSAT_NODE = 15     # per face node: BR1 viscous interface term


def element_kernel_flops_per_node(p: int, viscous: bool = True) -> float:
    N = p + 1
    f = FLOPS_PAIR * 3 * (N - 1) / 2 + FLOPS_LINE_NODE + FLOPS_NODE_PRE + FLOPS_SAT_NODE * 6 / N + FLOPS_SCALE_NODE
    if viscous:
        f += FLOPS_VISC_NODE + 24 * N + 96 / N + FLOPS_DIV_NODE + 24 * N
    return f


def residual_flops_per_node(p: int, viscous: bool = True) -> float:
    return element_kernel_flops_per_node(p, viscous) + (FLOPS_VSAT_NODE * 6 / (p + 1) if viscous else 0.0)


def element_kernel_bytes_per_node(p: int) -> float:
    """Compulsory HBM bytes of the element kernel: read q (40) and geometry (80), write dq/dt (40)
    and the viscous face traces (6 N^2 x 32 per element).  Neighbour face states are L2 hits."""
    N = p + 1
    return 40 + 80 + 40 + 6 * 32 / N


def element_kernel_bytes_per_node_f32(p: int) -> float:
    """float32 form: read the float32 perturbation state (20) and float32 geometry (40), write
    dq/dt (20) and the float32 viscous traces (6 N^2 x 16 per element)."""
    N = p + 1
    return 20 + 40 + 20 + 6 * 16 / N


LAUNCHER_MARK = b"// ---- host-side launchers"


def _sha(path):
    """Hash of a kernel source file up to its host-side launcher section (the device code), followed
    by the local device headers it includes (recursively, each once)."""
    import re
    data = open(path, "rb").read()
    cut = data.find(LAUNCHER_MARK)
    data = data[:cut] if cut >= 0 else data
    seen = set()

    def add(buf):
        out = b""
        for name in re.findall(rb'#include "([A-Za-z0-9_]+\.cuh)"', buf):
            f = os.path.join(os.path.dirname(path), name.decode())
            if name in seen or not os.path.exists(f):
                continue
            seen.add(name)
            inc = open(f, "rb").read()
            out += inc + add(inc)
        return out

    data += add(data)
    return hashlib.sha256(data).hexdigest()[:16]


def _ncu_traffic(profile, kernel_src, n_nodes):
    """DRAM bytes per launch of a kernel at n_nodes, from the committed ncu summary `profile` if it
    was taken on the current source: the captured launch's bytes scaled by the nodes it processed
    (the element kernels' traffic is per element, so it grows in proportion)."""
    f = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(f):
        return None
    sha = val = nodes = None
    for line in open(f).read().splitlines():
        if line.startswith("source_sha256_16:"):
            sha = line.split(":", 1)[1].strip()
        elif line.startswith("dram_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].strip())
        elif line.startswith("nodes_per_launch:"):
            nodes = float(line.split(":", 1)[1].strip())
    if sha != _sha(kernel_src) or val is None or not nodes:
        return None
    return val * n_nodes / nodes


def _src(name):
    return os.path.join(ROOT, "paper_1911_10966_gb300", "csrc", name)


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"esdc_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """Max of a per-rank time over all ranks (the only collective of the replica runs)."""
    if dist is None:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def replica_throughput(n_nodes: int, world: int, ms_max: float, rhs_per_step: int = RHS_PER_STEP) -> float:
    """Whole-job node-residuals per second: every rank advances its own replica of n_nodes."""
    return world * n_nodes * rhs_per_step / (ms_max * 1e-3)


def _config(args):
    W = HEADLINE
    return {"workload": W["name"], "mesh": f"{W['k']}^3 affine hexahedra on [-pi, pi]^3, periodic",
            "p": W["p"], "nodes": nodes_of(W), "Re": W["Re"], "Ma": W["Ma"], "cfl": W["cfl"],
            "step": "DP5 step (6 residuals) + float64 budgets recorded on the device",
            "replicas": args.gpus, "l2": "inputs larger than L2 (2.26 GB state, 4.5 GB geometry per residual)"}


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ------------------------------------------------------------------------------------------------
# The oracle side (CPU-baseline leg and the reference arm only)
# ------------------------------------------------------------------------------------------------
def block_elements(k: int, b: int) -> np.ndarray:
    """Ids of the contiguous b^3 block of elements at the low corner of a k^3 box."""
    e = np.arange(b)
    return (e[None, None, :] + k * (e[None, :, None] + k * e[:, None, None])).reshape(-1)


def oracle_sample(w=HEADLINE, block=SAMPLE_BLOCK):
    """The oracle's problem on a sample of workload w: the block of block^3 elements with its two
    rings of neighbours (all that its residual reads).  Returns (O, submesh, gas, q, E, rows)."""
    from oracle import esdc_oracle as O
    from paper_1911_10966_gb300 import inputs as I
    p, k = w["p"], w["k"]
    lo, hi = w.get("lo", PI_BOX[0]), w.get("hi", PI_BOX[1])
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, lo, hi, warp=w["warp"], seed=w["seed"])
    E = torch.tensor(block_elements(k, block))
    sub, E2, rows = O.make_submesh(p, x, O.box_neighbours(k, k, k), E)
    q = torch.tensor(I.taylor_green(x[E2.numpy()], Ma=w["Ma"]))
    del x
    return O, sub, O.Gas.from_mach(w["Ma"], w["Re"]), q, E, rows


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores, on the headline workload.  Each step: the six
    residual evaluations of a DP5 step on the 8^3-element block sample (with the two rings of
    neighbours its residual reads), so that the whole run stays within minutes."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    O, sub, gas, q, E, rows = oracle_sample()
    for _ in range(args.warmup):
        O.rhs(q, sub, gas, elems=rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(RHS_PER_STEP):
            O.rhs(q, sub, gas, elems=rows)
    el = time.perf_counter() - t0
    n = E.numel() * (HEADLINE["p"] + 1) ** 3
    val = n * RHS_PER_STEP * args.steps / el
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": "residual DOF/s (nodes x RHS / s), FP64", "value": val,
            "unit": "node-RHS/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": val, "unit": "node-RHS/s", "cores": cores, "kind": "oracle",
                             "sample": _sample_text(E.numel(), sub.J.shape[0], cores)},
            "e2e": {"value": val, "unit": "node-RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _sample_text(n_elems, n_closure, cores):
    W = HEADLINE
    return (f"per step the six residuals of a DP5 step on the contiguous {SAMPLE_BLOCK}^3 block ({n_elems} elements, "
            f"{n_elems * (W['p'] + 1) ** 3} nodes) of the {W['k']}^3 p={W['p']} mesh; the oracle also builds the "
            f"metrics and face states of the {n_closure - n_elems} neighbour elements its residual reads (counted as "
            f"cost, not as nodes); {cores} threads")


def _term_scale(O, q, mesh, gas, rows):
    """T_v = max over nodes of sum_l sum_j |2 D_ij| |f_v(q_i, q_j)| / J, the magnitude of the terms
    whose sum is the residual (float64 rounding of any evaluation is of order eps T_v)."""
    sabs = dataclasses.replace(mesh.sbp, D=mesh.sbp.D.abs())
    t = O.volume_term(q[rows], mesh.Ja[rows], sabs, gas, flux=lambda a, b, n, g: O.ec_flux_n(a, b, n, g).abs())
    t = t.abs() / mesh.J[rows].unsqueeze(1)
    return [float(t[:, v].max()) for v in range(5)]


def _normwise(a, b):
    a, b = torch.as_tensor(a).double(), torch.as_tensor(b).double()
    return [float((a[:, v] - b[:, v]).abs().max() / b[:, v].abs().max()) for v in range(5)]


def cpu_baseline_and_parity(gpu_rows):
    """The oracle (as it stands, float64 torch on the host cores) timed on the headline workload's
    block sample: residual evaluations repeated for about CPU_BASELINE_SECONDS.  From the same oracle
    residual: the parity of the GPU float64 and float32-mixed residuals on the block (gpu_rows), and
    the oracle on the other workload shapes with the GPU's parity there."""
    O, sub, gas, q, E, rows = oracle_sample()
    p = HEADLINE["p"]
    n = E.numel() * (p + 1) ** 3
    cores = torch.get_num_threads()
    t0 = time.perf_counter()
    r = O.rhs(q, sub, gas, elems=rows)
    count = 1
    while time.perf_counter() - t0 < CPU_BASELINE_SECONDS or count < RHS_PER_STEP:
        O.rhs(q, sub, gas, elems=rows)
        count += 1
    el = time.perf_counter() - t0
    base = {"value": n * count / el, "unit": "node-RHS/s", "cores": cores, "kind": "oracle",
            "sample": _sample_text(E.numel(), sub.J.shape[0], cores).replace(
                "per step the six residuals of a DP5 step", f"{count} residual evaluations ({el:.1f} s)")}
    T = _term_scale(O, q, sub, gas, rows)
    parity = {}
    if gpu_rows is not None:
        r64, r32 = gpu_rows
        R = [float(r[:, v].abs().max()) for v in range(5)]
        e64 = _normwise(r64, r)
        parity[HEADLINE["name"]] = {
            "sample": f"the {SAMPLE_BLOCK}^3 element block, Taylor-Green initial state",
            "f64_normwise": e64, "f64_eps_kappa": [2.220446049250313e-16 * T[v] / R[v] for v in range(5)],
            "f64_err_over_eps_T": [e64[v] * R[v] / (2.220446049250313e-16 * T[v]) for v in range(5)]}
        if r32 is not None:
            e32 = _normwise(r32, r)
            parity[HEADLINE["name"]].update({
                "f32_normwise": e32,
                "f32_c_v": [e32[v] * R[v] / (5.960464477539063e-08 * T[v]) for v in range(5)]})
    base["configs"], more = oracle_config_timings()
    parity.update(more)
    return base, parity


def oracle_config_timings():
    """The oracle (as it stands) on the other workload shapes, in node-RHS/s, and where a GPU is
    present the parity of the GPU float64 residual with it (per-variable normwise error): the 4^3
    affine p=3 Taylor-Green box (one residual and ten DP5 steps, whole mesh), the 16^3 warped p=4
    Taylor-Green box (24 seeded elements), the 8^3 warped p=4 isentropic vortex (one residual, whole
    mesh), and one residual of each ~16M-node p-sweep mesh restricted to a seeded sample of 256
    elements (the count is of the sampled nodes, although the oracle also evaluates the entropy-
    variable gradients of their face neighbours)."""
    from oracle import esdc_oracle as O
    from paper_1911_10966_gb300 import inputs as I
    gpu = torch.cuda.is_available()
    out, parity = {}, {}

    def timed(fn):
        t0 = time.perf_counter()
        res = fn()
        return time.perf_counter() - t0, res

    def gpu_rhs(w, x_fn, q_fn, elems=None):
        from paper_1911_10966_gb300.solver import Solver, lgl
        xi, _ = lgl(w["p"])
        x = x_fn(xi)
        s = Solver(w["p"], w["k"], w["k"], w["k"], x, Ma=w["Ma"], Re=w["Re"])
        r = s.rhs(s.to_device(q_fn(x)))
        r = (r if elems is None else r[torch.as_tensor(elems, device=r.device)]).cpu()
        s.close()
        return r

    w = TGV_SMALL
    s = O.sbp_operator(3)
    xf = lambda xi: I.box_coords(xi, 4, 4, 4, *PI_BOX)
    x = xf(s.xi.numpy())
    mesh = O.make_mesh(3, x, 4, 4, 4)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.taylor_green(x, Ma=0.1))
    n = q.shape[0] * 64
    t1, r = timed(lambda: O.rhs(q, mesh, gas))
    dt = O.cfl_dt(q, mesh, gas, 0.5)
    t10, _ = timed(lambda: O.rk_step(q, lambda st: O.rhs(st, mesh, gas), dt, 10))
    out[w["name"]] = {"rhs_node_rhs_per_s": n / t1, "dp5_10_steps_s": t10, "dp5_node_rhs_per_s": n * 60 / t10}
    if gpu:
        parity[w["name"]] = {"sample": "whole mesh", "f64_normwise": _normwise(
            gpu_rhs(w, xf, lambda x: I.taylor_green(x, Ma=0.1)), r)}

    w = TGV_WARPED
    E = torch.tensor(np.random.default_rng(7).choice(16 ** 3, 24, replace=False))
    s = O.sbp_operator(4)
    xf = lambda xi: I.box_coords(xi, 16, 16, 16, *PI_BOX, warp=0.1, seed=0)
    x = xf(s.xi.numpy())
    sub, E2, rows = O.make_submesh(4, x, O.box_neighbours(16, 16, 16), E)
    q = torch.tensor(I.taylor_green(x[E2.numpy()], Ma=0.1))
    t1, r = timed(lambda: O.rhs(q, sub, gas, elems=rows))
    out[w["name"]] = {"rhs_node_rhs_per_s": E.numel() * 125 / t1, "sample_elements": E.numel()}
    if gpu:
        parity[w["name"]] = {"sample": "24 seeded elements", "f64_normwise": _normwise(
            gpu_rhs(w, xf, lambda x: I.taylor_green(x, Ma=0.1), E), r)}

    w = VORTEX
    s = O.sbp_operator(4)
    xf = lambda xi: I.box_coords(xi, 8, 8, 8, w["lo"], w["hi"], warp=0.1, seed=1)
    x = xf(s.xi.numpy())
    mesh = O.make_mesh(4, x, 8, 8, 8)
    gasv = O.Gas.from_mach(0.5, 1000.0)
    qf = lambda x: I.isentropic_vortex(x, Ma=0.5, u_inf=(1 / math.sqrt(2), -1 / math.sqrt(2), 0.0))
    q = torch.tensor(qf(x))
    t1, r = timed(lambda: O.rhs(q, mesh, gasv))
    out[w["name"]] = {"rhs_node_rhs_per_s": q.shape[0] * 125 / t1}
    if gpu:
        parity[w["name"]] = {"sample": "whole mesh", "f64_normwise": _normwise(gpu_rhs(w, xf, qf), r)}

    for p, k in PSWEEP_K.items():
        s = O.sbp_operator(p)
        x = I.box_coords(s.xi.numpy(), k, k, k, *PI_BOX)
        E = torch.tensor(np.sort(np.random.default_rng(p).choice(k ** 3, 256, replace=False)))
        sub, E2, rows = O.make_submesh(p, x, O.box_neighbours(k, k, k), E)
        q = torch.tensor(I.taylor_green(x[E2.numpy()], Ma=0.1))
        el, _ = timed(lambda: O.rhs(q, sub, gas, elems=rows))
        out[f"tgv_psweep_p{p}_{k}cubed"] = {"rhs_node_rhs_per_s": 256 * (p + 1) ** 3 / el, "sample_elements": 256}
    return out, parity


# ------------------------------------------------------------------------------------------------
# The GPU side
# ------------------------------------------------------------------------------------------------
def _check_budgets(hist):
    """The per-step budgets recorded on the device: every state physical, every sum finite."""
    h = hist.cpu()
    if float(h[:, 4].abs().sum()) != 0.0 or not bool(torch.isfinite(h).all()):
        raise RuntimeError("non-physical state during the timed steps")


def timed_steps(solver, q, dt, steps, barrier, flush=None):
    """`steps` DP5 steps, each followed by the float64 budgets written into device memory, timed with
    CUDA events on the launching stream; the library's own events time its residual kernels.
    Returns (ms per step, ms in the element kernel, ms in the face kernel, residual evaluations)."""
    stream = torch.cuda.current_stream()
    evs = [_events() for _ in range(steps)]
    hist = torch.zeros((steps, 5), dtype=torch.float64, device=q.device)
    solver.profile(True)
    barrier()
    for i in range(steps):
        if flush is not None:
            flush.fill_(float(i))
        evs[i][0].record(stream)
        solver.rk_step(q, dt, 1)
        solver.budgets_async(q, hist[i])
        evs[i][1].record(stream)
    barrier()
    ms_main, ms_face, nres = solver.profile_read()
    solver.profile(False)
    _check_budgets(hist)
    return sum(a.elapsed_time(b) for a, b in evs) / steps, ms_main, ms_face, nres


def _time_rhs_ms(s, q, reps=3):
    r = s.rhs(q)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(reps):
        s.rhs(q, out=r)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _rates(solver, q):
    """(KE, dS/dt, dKE/dt) per unit volume from the float64 budgets of q and its residual."""
    b = solver.budgets(q, solver.rhs(q))
    return b[1], b[2], b[3]


def run_ours(args):
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1911_10966_gb300.solver import Solver, probe_fma

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    W = HEADLINE
    p, k = W["p"], W["k"]
    t_setup = time.perf_counter()
    s64 = Solver(p, k, k, k, None, Ma=W["Ma"], Re=W["Re"], lo=PI_BOX[0], hi=PI_BOX[1])
    q = s64.init_state("tgv")
    q0 = q.clone()
    dt = s64.dt_cfl(q, W["cfl"])
    setup_s = time.perf_counter() - t_setup
    n = s64.n_nodes
    for _ in range(args.warmup):
        s64.rk_step(q, dt, 1)
        s64.budgets(q)
    peak_f64 = probe_fma("f64")

    # ---- device-timed region: inputs resident in HBM (and larger than L2)
    with ClockSampler(local) as clk:
        time.sleep(0.6)          # let the sampler start before the timed region
        ms_step, ms_main, ms_face, nres = timed_steps(s64, q, dt, args.steps, barrier)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms_step, dist, q.device)
    value = replica_throughput(n, ws, ms_max)
    kernel_ms = ms_main / max(nres, 1)

    # ---- the float32-mixed form on the same mesh, the same number of steps from the same state
    fp32 = None
    r_rows = None
    E_blk = torch.as_tensor(block_elements(k, SAMPLE_BLOCK), device=q.device)
    r64 = s64.rhs(q0)
    rows64 = r64[E_blk].cpu()
    rows32 = None
    q32 = None
    if not args.no_fp32:
        s32 = Solver(p, k, k, k, s64.coords, Ma=W["Ma"], Re=W["Re"], precision="fp32")
        r32 = s32.rhs(q0)
        rows32 = r32[E_blk].cpu()
        e_v = [float((r32[:, v].double() - r64[:, v]).abs().max() / r64[:, v].abs().max()) for v in range(5)]
        del r32
        q32 = q0.clone()
        for _ in range(args.warmup):
            s32.rk_step(q32, dt, 1)
            s32.budgets(q32)
        peak32 = probe_fma("f32")
        ms32, m32, f32ms, nres32 = timed_steps(s32, q32, dt, args.steps, barrier)
        k32 = m32 / max(nres32, 1)
        fp32 = _fp32_object(p, n, ms32, k32, f32ms / max(nres32, 1), peak32, e_v, ws, dist, q.device)
        fp32["speedup_vs_f64_step"] = ms_step / ms32
        fp32["speedup_vs_f64_rhs"] = kernel_ms / k32
    del r64
    r_rows = (rows64, rows32)

    # ---- 200-step trajectory in both precisions: dissipation-rate errors of the float32-mixed form
    done = args.warmup + args.steps
    if fp32 is not None:
        if args.precision_steps > 0:
            fp32["trajectory"] = _precision_run(s64, s32, q, q32, dt, done, args.precision_steps)
        # every bounded wait of the element kernel's bulk copies completed during the whole leg
        fp32["device_status"] = s32.device_status()
        if fp32["device_status"] != 0:
            raise RuntimeError("a bounded wait for bulk shared-memory copies gave up: results invalid")
        s32.close()
        del q32
        torch.cuda.empty_cache()

    # ---- end to end through the public API with host buffers
    e2e_val, e2e_info = _e2e(s64, q0, dt, max(3, min(args.steps, 6)), barrier, dist, ws, n)
    del q0

    ms_rhs = _time_rhs_ms(s64, q, reps=3)
    s64.close()
    del q
    torch.cuda.empty_cache()

    secondary = {}
    if not args.headline_only:
        secondary["tgv_16cubed_p4_warped"] = _small_workload_leg(args, barrier)
        secondary["adjoint_vortex_8cubed_p4_warped"] = _adjoint_vortex_leg()
        secondary["psweep_16M_nodes"] = _psweep_leg()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    src = _src("rhs_f64.cu")
    fl = element_kernel_flops_per_node(p) * n
    achieved = fl / (kernel_ms * 1e-3) / 1e12
    peak = peak_f64 / 1e12
    hbm, hbm_src = hbm_peak()
    cpu_base, parity = (None, None)
    if ws == 1 and not args.no_cpu_baseline:
        cpu_base, parity = cpu_baseline_and_parity(r_rows)
    line = {
        "metric": "residual DOF/s (nodes x RHS / s), FP64", "value": value, "unit": "node-RHS/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args),
        "roofline": {"bound": "alu", "kernel": "rhs_main_f64<8>", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": _ncu_traffic("rhs_main_f64_tgv_p7.md", src, n),
                     "peak_source": "of measured: float64 FMA throughput (esdc_probe_fma) in this run",
                     "peak_nominal": FP64_NOMINAL_TFLOPS, "frac_nominal": achieved / FP64_NOMINAL_TFLOPS,
                     "flops_per_launch": fl, "kernel_ms": kernel_ms,
                     "hbm_frac": element_kernel_bytes_per_node(p) * n / (kernel_ms * 1e-3) / (hbm * 1e9),
                     "hbm_peak_source": hbm_src},
        "cpu_baseline": cpu_base,
        "e2e": {"value": e2e_val, "unit": "node-RHS/s", "h2d_bytes_per_step": n * 40,
                "d2h_bytes_per_step": n * 40, **e2e_info},
        # per step: element + viscous face kernel per residual, five stage combinations and the
        # solution update, budgets + final sum
        "gpu_launches": args.steps * (RHS_PER_STEP * 2 + RHS_PER_STEP + 2),
        "clocks": clocks,
        "setup_s": setup_s,
        "rhs_only": {"value": n / (ms_rhs * 1e-3), "unit": "node-RHS/s", "ms": ms_rhs,
                     "element_kernel_ms": kernel_ms, "face_kernel_ms": ms_face / max(nres, 1)},
        "fp32_mixed": fp32,
        "parity": parity,
    }
    line.update(secondary)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _e2e(solver, q0, dt, steps, barrier, dist, ws, n):
    """End-to-end DP5 steps through the public API with host buffers: every step copies its input
    state from pinned host memory to the device, advances it one DP5 step with the float64 budgets
    recorded on the device, and copies the new state back to pinned host memory.  The copies run on
    a copy stream with two device buffers, so step i's device-to-host copy and step i+1's
    host-to-device copy overlap step i+1's and step i's compute (the copy engines work beside the
    SMs); the budgets of every step are read back at the end.  Returns (node-RHS/s over the wall
    time of all steps, info)."""
    comp = torch.cuda.current_stream()
    cp = torch.cuda.Stream(device=q0.device)
    q_host = q0.cpu().pin_memory()
    outs = [torch.empty_like(q_host).pin_memory() for _ in range(2)]
    bufs = [torch.empty_like(q0) for _ in range(2)]
    hist = torch.zeros((steps, 5), dtype=torch.float64, device=q0.device)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for e in ev_out:
        e.record(cp)
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(cp):
        bufs[0].copy_(q_host, non_blocking=True)
    ev_in[0].record(cp)
    for i in range(steps):
        b = i % 2
        comp.wait_event(ev_in[b])
        solver.rk_step(bufs[b], dt, 1)
        solver.budgets_async(bufs[b], hist[i])
        ev_done[b].record(comp)
        with torch.cuda.stream(cp):
            if i + 1 < steps:
                nb = (i + 1) % 2
                cp.wait_event(ev_done[nb])          # buffer nb's previous step is computed ...
                cp.wait_event(ev_out[nb])           # ... and copied out
                bufs[nb].copy_(q_host, non_blocking=True)
                ev_in[nb].record(cp)
            cp.wait_event(ev_done[b])
            outs[b].copy_(bufs[b], non_blocking=True)
            ev_out[b].record(cp)
    cp.synchronize()
    comp.synchronize()
    h = hist.cpu()
    barrier()
    el = (time.perf_counter() - t0) / steps
    _check_budgets(h)
    val = replica_throughput(n, ws, max_over_ranks(el * 1e3, dist, q0.device))
    return val, {"steps": steps, "ms_per_step": el * 1e3,
                 "what": "state copied host -> device and back every step on a copy stream overlapping the "
                         "compute (two device buffers), budgets recorded on the device and read at the end"}


def _fp32_object(p, n, ms_step, kernel_ms, face_ms, peak32, e_v, ws, dist, device):
    fl = element_kernel_flops_per_node(p) * n
    by = element_kernel_bytes_per_node_f32(p) * n
    hbm, hbm_src = hbm_peak()
    t_alu = fl / peak32
    t_hbm = by / (hbm * 1e9)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": fl / (kernel_ms * 1e-3) / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s",
                "peak_source": "of measured: float32 FMA throughput (esdc_probe_fma) in this run"}
    else:
        roof = {"bound": "hbm", "achieved": by / (kernel_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": hbm_src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"kernel": f"rhs_pairs_f32<{p + 1}>", "kernel_ms": kernel_ms, "face_kernel_ms": face_ms,
                 "flops_per_launch": fl, "bytes_per_launch": by,
                 "traffic": _ncu_traffic("rhs_pairs_f32_tgv_p7.md", _src("rhs_f32_pairs.cu"), n),
                 "alu_frac": fl / (kernel_ms * 1e-3) / peak32, "hbm_frac": by / (kernel_ms * 1e-3) / (hbm * 1e9)})
    ms_max = max_over_ranks(ms_step, dist, device)
    return {"value": replica_throughput(n, ws, ms_max), "unit": "node-RHS/s", "ms_per_step": ms_max,
            "dtype": "f32 residual, f64 state/update/budgets", "roofline": roof,
            "residual_error_vs_f64": {"per_variable": e_v, "variables": ["rho", "rho u1", "rho u2", "rho u3", "rho E"],
                                      "state": "Taylor-Green initial state, whole mesh, normwise"},
            # per step: shadow state, element + viscous face kernel per residual, the float32 stage
            # states of the five later stages, the float64 update, budgets + final sum
            "gpu_launches_per_step": 1 + RHS_PER_STEP * 2 + (RHS_PER_STEP - 1) + 1 + 2}


def _precision_run(s64, s32, q64, q32, dt, done, total):
    """Continue both trajectories (already `done` steps from the same initial state) to `total` DP5
    steps with multi-step calls, and compare the float64 budgets of the two states and of their
    residuals: kinetic energy, its dissipation rate -dKE/dt and the entropy rate dS/dt."""
    vol = (2 * math.pi) ** 3
    rel = lambda a, b: abs(a - b) / abs(b)
    hist = []
    marks = sorted({done} | set(range(50 * math.ceil(done / 50), total + 1, 50)) | {max(done, total)})
    step = done
    ms64 = ms32 = 0.0
    for m in marks:
        if m > step:
            a, b = _events()
            a.record()
            s64.rk_step(q64, dt, m - step)
            b.record()
            torch.cuda.synchronize()
            ms64 += a.elapsed_time(b)
            a.record()
            s32.rk_step(q32, dt, m - step)
            b.record()
            torch.cuda.synchronize()
            ms32 += a.elapsed_time(b)
            step = m
        k64, s64r, d64 = _rates(s64, q64)
        k32, s32r, d32 = _rates(s32, q32)
        hist.append({"step": step, "t": step * dt, "ke": k64 / vol, "ke_rate_f64": -d64 / vol,
                     "ke_rate_f32": -d32 / vol, "ds_f64": s64r / vol, "ds_f32": s32r / vol,
                     "ke_rate_rel_err": rel(d32, d64), "ds_rel_err": rel(s32r, s64r), "ke_rel_err": rel(k32, k64)})
    moved = step - done
    return {"steps": step, "dt": dt, "history": hist,
            "ke_rate_rel_err_final": hist[-1]["ke_rate_rel_err"],
            "ke_rate_rel_err_max": max(h["ke_rate_rel_err"] for h in hist),
            "ds_rate_rel_err_final": hist[-1]["ds_rel_err"],
            "ds_rate_rel_err_max": max(h["ds_rel_err"] for h in hist),
            "ke_rel_err_final": hist[-1]["ke_rel_err"],
            "ms_per_step_graph_f64": ms64 / moved if moved else None,
            "ms_per_step_graph_f32": ms32 / moved if moved else None,
            "what": "both precisions advanced from the same initial state with fixed DP5 steps (CUDA-graph "
                    "replay after the timed steps); float64 budgets of each state and its own residual"}


def _small_workload_leg(args, barrier):
    """The 16^3 warped p = 4 Taylor-Green workload: float64 and float32-mixed step rates, the
    multi-step (graph replay) rate, the adjoint cost, the volume-flux variants and the adaptive
    integrator."""
    from paper_1911_10966_gb300.solver import Solver
    W = TGV_WARPED
    s = Solver.box(W["p"], W["k"], W["k"], W["k"], warp=W["warp"], seed=W["seed"], Ma=W["Ma"], Re=W["Re"])
    q0 = s.init_state("tgv")     # same formula as the input module, at the same nodes
    dt = s.dt_cfl(q0, W["cfl"])
    n = s.n_nodes
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=q0.device)
    steps = 10
    out = {"nodes": n, "l2": "flushed between timed steps (256 MiB write)"}
    q = q0.clone()
    for _ in range(3):
        s.rk_step(q, dt, 1)
    ms, mm, mf, nr = timed_steps(s, q, dt, steps, barrier, flush)
    out["f64"] = {"ms_per_step": ms, "node_rhs_per_s": n * 6 / (ms * 1e-3), "element_kernel_ms": mm / max(nr, 1),
                  "face_kernel_ms": mf / max(nr, 1)}
    out["f64"]["multi_step"] = _multi_step_ms(s, q0.clone(), dt, 10, flush)
    ms_rhs = _time_rhs_ms(s, q0, reps=10)
    out["f64"]["rhs_ms"] = ms_rhs
    if not args.no_fp32:
        s32 = Solver(W["p"], W["k"], W["k"], W["k"], s.coords, Ma=W["Ma"], Re=W["Re"], precision="fp32")
        q = q0.clone()
        for _ in range(3):
            s32.rk_step(q, dt, 1)
        ms, mm, mf, nr = timed_steps(s32, q, dt, steps, barrier, flush)
        r64, r32 = s.rhs(q0), s32.rhs(q0)
        out["f32_mixed"] = {"ms_per_step": ms, "node_rhs_per_s": n * 6 / (ms * 1e-3),
                            "element_kernel_ms": mm / max(nr, 1), "face_kernel_ms": mf / max(nr, 1),
                            "multi_step": _multi_step_ms(s32, q0.clone(), dt, 50, flush),
                            "residual_error_vs_f64": [float((r32[:, v].double() - r64[:, v]).abs().max()
                                                            / r64[:, v].abs().max()) for v in range(5)]}
        s32.close()
    out["adjoint"] = _adjoint_leg(s, q0, dt, ms_rhs, 5, flush)
    out["volume_flux_variants"] = _variants_leg(s, q0, ms_rhs)
    out["adaptive_dp54"] = _adaptive_leg(s, q0, dt)
    # freestream preservation on the warped mesh
    qf = s.init_state("freestream")
    rf = s.rhs(qf)
    out["freestream_max_abs_residual_over_pressure_scale"] = float(rf.abs().max()) / (1.0 / (1.4 * W["Ma"] ** 2))
    s.close()
    return out


def _multi_step_ms(solver, q, dt, steps, flush):
    """DP5 steps without budgets, (a) one call per step (direct launches) and (b) one call for all
    steps (one step captured as a CUDA graph and replayed): ms per step each."""
    stream = torch.cuda.current_stream()
    a, b = _events()
    solver.rk_step(q, dt, 2)                  # capture outside the timed region
    out = {}
    for name in ("direct", "graph"):
        flush.fill_(4.0)
        a.record(stream)
        if name == "direct":
            for _ in range(steps):
                solver.rk_step(q, dt, 1)
        else:
            solver.rk_step(q, dt, steps)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b) / steps
    return {"ms_per_step_direct": out["direct"], "ms_per_step_graph": out["graph"], "steps": steps}


def _adjoint_leg(solver, q, dt, ms_rhs, nsteps, flush=None):
    """Cost of the hand-written adjoint: one vector-Jacobian product against one residual, and the
    gradient of the final kinetic energy through nsteps DP5 steps against the forward steps alone,
    with stage checkpoints (the six stage states of every step stored by the forward pass) and with
    per-step checkpoints plus stage recomputation in the reverse sweep."""
    stream = torch.cuda.current_stream()
    lam = torch.randn(q.shape, dtype=torch.float64, device=q.device, generator=torch.Generator(q.device).manual_seed(3))
    g = solver.rhs_vjp(q, lam)
    reps = 10
    a, b = _events()

    def fl(v):
        if flush is not None:
            flush.fill_(v)

    fl(1.0)
    a.record(stream)
    for _ in range(reps):
        g = solver.rhs_vjp(q, lam)
    b.record(stream)
    torch.cuda.synchronize()
    ms_vjp = a.elapsed_time(b) / reps
    qa = q.clone()
    solver.rk_step(qa, dt, nsteps)            # warm-up (graph capture)
    qa = q.clone()
    fl(2.0)
    a.record(stream)
    solver.rk_step(qa, dt, nsteps)
    b.record(stream)
    torch.cuda.synchronize()
    ms_fwd = a.elapsed_time(b)

    def gradient(kind):
        qb = q.clone()
        ck = solver.rk_step_ckpt(qb, dt, nsteps, stages=kind == "stages", k1=kind == "k1")
        lamN = solver.ke_gradient(qb)
        return solver.rk_adjoint(ck, dt, lamN)

    out = {}
    for kind in ("stages", "k1", "state"):
        gradient(kind)                        # warm-up: workspaces and checkpoint memory
        fl(3.0)
        a.record(stream)
        _, gmu = gradient(kind)
        b.record(stream)
        torch.cuda.synchronize()
        out[kind] = (a.elapsed_time(b), gmu)
        torch.cuda.empty_cache()
    ms_grad, gmu = out["stages"]
    ms_grad_rc, gmu_rc = out["k1"]
    ms_grad_st, gmu_st = out["state"]
    return {"vjp_ms": ms_vjp, "rhs_ms": ms_rhs, "vjp_over_rhs": ms_vjp / ms_rhs,
            "trajectory_steps": nsteps, "forward_ms": ms_fwd, "gradient_ms": ms_grad,
            "gradient_over_forward": ms_grad / ms_fwd,
            "gradient_recompute_ms": ms_grad_rc, "gradient_recompute_over_forward": ms_grad_rc / ms_fwd,
            "gradient_recompute_state_only_ms": ms_grad_st,
            "gradient_recompute_state_only_over_forward": ms_grad_st / ms_fwd,
            "dke_dmu": gmu, "dke_dmu_recompute_rel_diff": max(abs(gmu - gmu_rc), abs(gmu - gmu_st)) / abs(gmu),
            "dtype": "f64",
            "what": "d KE(q_N)/d(q_0, mu): forward storing the stage states (6 per step) + reverse sweep "
                    "(6 VJPs per step); recompute variant: per-step checkpoints of the state and its "
                    "residual (2 per step), 4 residual recomputations + 6 VJPs per step; state-only "
                    "variant: the state alone (1 per step), 5 recomputations; forward = the N steps alone "
                    "(one multi-step call)"}


def _adjoint_vortex_leg():
    """The differentiation workload: isentropic vortex (strength 5, centre 0, axis (1,1,1), drift
    (1,-1,0)/sqrt 2, Ma 0.5) on 8^3 warped hexahedra of [-5, 5]^3, p = 4, Re = 1000; gradient of the
    kinetic energy after 50 DP5 steps at CFL 0.5 with respect to the initial state and mu."""
    from paper_1911_10966_gb300.solver import Solver
    W = VORTEX
    s = Solver.box(W["p"], W["k"], W["k"], W["k"], lo=W["lo"], hi=W["hi"], warp=W["warp"], seed=W["seed"],
                   Ma=W["Ma"], Re=W["Re"])
    q = s.init_state("vortex", VORTEX_PARAMS)
    dt = s.dt_cfl(q, W["cfl"])
    ms_rhs = _time_rhs_ms(s, q, reps=20)
    out = _adjoint_leg(s, q, dt, ms_rhs, W["steps"])
    out["nodes"] = s.n_nodes
    s.close()
    return out


def _variants_leg(solver, q0, ms_rhs):
    """Residual cost of the paper's comparison discretisations on the same workload (float64): the
    Kennedy-Gruber split form (SF-KG) and standard collocation (DC) beside ES-C, and ES-C with the
    Roe-type matrix interface dissipation instead of local Lax-Friedrichs."""
    from paper_1911_10966_gb300.solver import Solver
    W = TGV_WARPED
    out = {"esc": {"rhs_ms": ms_rhs, "node_rhs_per_s": solver.n_nodes / (ms_rhs * 1e-3)}}
    for vf, diss in (("kg", True), ("dc", True), ("esc", "matrix")):
        s = Solver(W["p"], W["k"], W["k"], W["k"], solver.coords, Ma=W["Ma"], Re=W["Re"], volume_flux=vf,
                   dissipation=diss)
        ms = _time_rhs_ms(s, q0, reps=10)
        out[vf if diss is True else "esc_matrix_dissipation"] = {"rhs_ms": ms,
                                                                 "node_rhs_per_s": s.n_nodes / (ms * 1e-3)}
        s.close()
    return out


def _adaptive_leg(solver, q0, dt):
    """Adaptive DP5(4) (esdc_rk_adaptive) over 200 CFL steps of physical time, rtol = atol = 1e-8,
    first trial step 4 CFL steps: residual throughput including the error estimate and the per-step
    host decision."""
    tol, span = 1e-8, 200.0
    q = q0.clone()
    solver.rk_adaptive(q, 0.0, 2.0 * dt, dt, rtol=tol, atol=tol)        # warm-up: workspace
    q = q0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solver.rk_adaptive(q, 0.0, span * dt, 4.0 * dt, rtol=tol, atol=tol)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"t_end_over_cfl_dt": span, "rtol": tol, "atol": tol, "accepted": st["accepted"],
            "rejected": st["rejected"], "rhs": st["rhs"], "wall_ms": wall * 1e3,
            "node_rhs_per_s": solver.n_nodes * st["rhs"] / wall, "mean_dt_over_cfl_dt": span / st["accepted"]}


def _psweep_leg(reps=3):
    """Residual throughput per polynomial degree at ~16 M nodes (affine Taylor-Green boxes, Ma 0.1),
    Re = 1600 and inviscid, float64 and float32-mixed: nodes / residual time, `reps` timed residuals
    after one warm-up, each precision's element-kernel time from the library's own events."""
    from paper_1911_10966_gb300.solver import Solver
    rows = []
    for p, k in PSWEEP_K.items():
        coords = None
        for Re in (1600.0, 0.0):
            for prec in ("fp64", "fp32"):
                s = Solver(p, k, k, k, coords, Ma=0.1, Re=Re, precision=prec, lo=PI_BOX[0], hi=PI_BOX[1])
                coords = s.coords
                q = s.init_state("tgv")
                s.rhs(q)
                s.profile(True)
                ms = _time_rhs_ms(s, q, reps)
                mm, _, nr = s.profile_read()
                s.profile(False)
                kms = mm / max(nr, 1)
                fl = element_kernel_flops_per_node(p, Re > 0) * s.n_nodes
                rows.append({"p": p, "k": k, "nodes": s.n_nodes, "Re": Re, "precision": prec, "rhs_ms": ms,
                             "node_rhs_per_s": s.n_nodes / (ms * 1e-3), "element_kernel_ms": kms,
                             "element_kernel_tflops": fl / (kms * 1e-3) / 1e12})
                s.close()
                del q
                torch.cuda.empty_cache()
    return {"rows": rows, "what": "one residual = element kernel + viscous face kernel; algorithmic flops "
                                  "per node as in the roofline (float32 rows count the same flops)"}


# ------------------------------------------------------------------------------------------------
# Extra studies (not the bench line): python bench.py --study <name> [key=value ...]; each prints
# JSON lines.  All arithmetic runs in libesdc.so; these only set up meshes and states, time calls
# and compute error norms of the returned fields.
# ------------------------------------------------------------------------------------------------
# the paper's cost study (Sec. 5.2): 256 nodes per direction (16,777,216 nodes) at p = 1, 3, 7, 15
PAPER_COST_K = {1: 128, 3: 64, 7: 32, 15: 16}


def _p_norm_l2(s, a, b):
    """P-norm L2 difference of the density of two device states on solver s's mesh."""
    from paper_1911_10966_gb300.solver import lgl
    J, _ = s.geometry()
    _, wq = lgl(s.p)
    P = wq[:, None, None] * wq[None, :, None] * wq[None, None, :]
    err = ((a[:, 0] - b[:, 0]).cpu().numpy()) ** 2
    return float(np.sqrt((P[None] * J * err).sum()))


def study_rhs(p=4, k=16, volume_flux="esc", Re=1600.0, precision="fp64", warp=0.1, reps=5, vjp=0):
    """Residual (or with vjp=1 vector-Jacobian product) time of one configuration, Taylor-Green on
    the periodic [-pi, pi]^3 box with warp amplitude `warp`: `reps` timed calls after one warm-up.
    This is the command the kernel profiles are taken on."""
    from paper_1911_10966_gb300.solver import Solver
    p, k, reps, vjp = int(p), int(k), int(reps), int(vjp)
    s = Solver.box(p, k, k, k, warp=float(warp), Re=float(Re), precision=precision, volume_flux=volume_flux)
    q = s.init_state("tgv")
    if vjp:
        lam = torch.ones_like(q)
        s.rhs_vjp(q, lam)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        for _ in range(reps):
            s.rhs_vjp(q, lam)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
    else:
        ms = _time_rhs_ms(s, q, reps)
    row = {"study": "rhs", "p": p, "k": k, "nodes": s.n_nodes, "Re": float(Re), "precision": precision,
           "volume_flux": volume_flux, "vjp": vjp, "ms": ms, "node_rhs_per_s": s.n_nodes / (ms * 1e-3)}
    print(json.dumps(row), flush=True)
    s.close()


def study_steps(p=7, k=20, precision="fp32", warp=0.0, Re=1600.0, steps=3, warmup=1):
    """DP5 steps of the bench's step form (one step per call, the float64 budgets of every step into
    device memory) on the Taylor-Green box of k^3 elements at degree p: the command the kernel
    profiles of the step's other kernels (stage states, update, budgets) are taken on."""
    from paper_1911_10966_gb300.solver import Solver
    p, k, steps, warmup = int(p), int(k), int(steps), int(warmup)
    s = Solver.box(p, k, k, k, warp=float(warp), Re=float(Re), precision=precision)
    q = s.init_state("tgv")
    dt = s.dt_cfl(q, 0.5)
    for _ in range(warmup):
        s.rk_step(q, dt, 1)
        s.budgets(q)
    ms, ms_main, ms_face, nres = timed_steps(s, q, dt, steps, lambda: None)
    print(json.dumps({"study": "steps", "p": p, "k": k, "nodes": s.n_nodes, "precision": precision, "steps": steps,
                      "ms_per_step": ms, "element_kernel_ms": ms_main / max(nres, 1),
                      "face_kernel_ms": ms_face / max(nres, 1), "device_status": s.device_status()}), flush=True)
    s.close()


def study_variants(degrees="1,3,7,15"):
    """The paper's cost comparison (Sec. 5.2, "Error vs. cost" figure): Taylor-Green at Ma 0.05,
    Re 1600, 256^3 nodes at p = 1, 3, 7, 15, time per fixed DP5 step (six residuals) with the ES-C,
    SF-KG and DC volume fluxes in float64, and ES-C in the float32-mixed form (p <= 7)."""
    from paper_1911_10966_gb300.solver import Solver
    for p in [int(x) for x in str(degrees).split(",")]:
        k = PAPER_COST_K[p]
        coords = None
        for vf, prec in (("esc", "fp64"), ("kg", "fp64"), ("dc", "fp64"), ("esc", "fp32")):
            if prec == "fp32" and p > 7:
                continue
            s = Solver(p, k, k, k, coords, Re=1600.0, Ma=0.05, volume_flux=vf, precision=prec,
                       lo=PI_BOX[0], hi=PI_BOX[1])
            coords = s.coords
            q = s.init_state("tgv")
            dt = s.dt_cfl(q, 0.5)
            s.rk_step(q, dt, 1)
            torch.cuda.synchronize()
            a, b = _events()
            a.record()
            s.rk_step(q, dt, 3)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 3
            row = {"study": "variants", "p": p, "k": k, "nodes": s.n_nodes, "volume_flux": vf, "precision": prec,
                   "dp5_step_ms": ms, "node_rhs_per_s": s.n_nodes * 6 / (ms * 1e-3),
                   "rhs_ms": _time_rhs_ms(s, q)}
            print(json.dumps(row), flush=True)
            s.close()
            del q
            torch.cuda.empty_cache()


def _mms_run(p, k, vf="esc", ip_coef=0.0, t_end=1.5, cfl=0.5):
    """The supersonic manufactured solution on [0, 1]^3 with exact Dirichlet data on every face,
    marched from the exact field with fixed DP5 steps to t_end: (P-norm L2 error of rho, wall s,
    steps, dt)."""
    from paper_1911_10966_gb300 import inputs as I
    from paper_1911_10966_gb300.solver import Solver, mms_fields
    s = Solver.box(p, k, k, k, lo=(0.0,) * 3, hi=(1.0,) * 3, Ma=I.MMS_MA, Re=I.MMS_RE,
                   bounded=(True, True, True), volume_flux=vf, ip_coef=ip_coef)
    qx, src = mms_fields(s.coords, I.manufactured_table(), gamma=1.4, Ma=I.MMS_MA, Re=I.MMS_RE, Pr=0.72, L=1.0)
    exact = s.to_device(qx)
    sd = s.to_device(src)
    s.set_exterior(exact)
    s.set_source(sd)
    q = exact.clone()
    dt0 = s.dt_cfl(q, cfl)
    nsteps = max(1, int(math.ceil(t_end / dt0)))
    dt = t_end / nsteps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.rk_step(q, dt, nsteps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    l2 = _p_norm_l2(s, q, exact)
    s.close()
    return l2, wall, nsteps, dt


def study_mms(t_end=1.5):
    """The paper's viscous error-vs-cost study (Sec. 5.1): the supersonic manufactured solution on
    [0, 1]^3, Re = 4e6, ES-C and DC, p = 1..4, P-norm L2 error of rho after t_end flow-through times
    against the exact field, and the wall time of the run."""
    for vf in ("esc", "dc"):
        for p, ks in ((1, (4, 8, 16, 32)), (2, (4, 8, 16)), (3, (4, 8, 16)), (4, (4, 8, 16))):
            prev = None
            for k in ks:
                l2, wall, nsteps, _ = _mms_run(p, k, vf, t_end=float(t_end))
                print(json.dumps({"study": "mms", "volume_flux": vf, "p": p, "k": k, "nodes": k ** 3 * (p + 1) ** 3,
                                  "steps": nsteps, "l2_rho": l2, "wall_s": wall,
                                  "order": (math.log(prev / l2) / math.log(2.0)) if prev else None}), flush=True)
                prev = l2


def study_hconv(t_final=0.5):
    """Isentropic vortex (strength 5, Ma 0.5, axis x3, drift (1, -1, 0)/sqrt(2)) on [-5,5]^3,
    inviscid, advanced to t_final with DP5 at CFL 0.25; P-norm L2 error of rho against the exact
    translated vortex (its periodic images ignored), p = 3, 4, 5 on 4^3 .. 32^3."""
    from paper_1911_10966_gb300.solver import Solver
    t_final = float(t_final)
    u_inf = (1 / math.sqrt(2), -1 / math.sqrt(2), 0.0)
    for p in (3, 4, 5):
        prev = None
        for k in (4, 8, 16, 32):
            s = Solver.box(p, k, k, k, lo=(-5.0,) * 3, hi=(5.0,) * 3, Ma=0.5, Re=0.0)
            vortex = lambda t: s.init_state("vortex", [5.0, u_inf[0] * t, u_inf[1] * t, 0.0, 0.0, 0.0, 1.0, *u_inf])
            q = vortex(0.0)
            dt0 = s.dt_cfl(q, 0.25)
            nsteps = max(1, int(math.ceil(t_final / dt0)))
            s.rk_step(q, t_final / nsteps, nsteps)
            l2 = _p_norm_l2(s, q, vortex(t_final))
            print(json.dumps({"study": "hconv", "p": p, "k": k, "h": 10.0 / k, "steps": nsteps, "l2_rho": l2,
                              "order": (math.log(prev / l2) / math.log(2.0)) if prev else None}), flush=True)
            prev = l2
            s.close()


IP_SIGMAS = (0.0, 0.5, 1.0, 2.0, 4.0)


def _stable_cfl(s, q0, steps=100, lo=0.25, hi=4.0, tol=0.02):
    """Largest CFL number (dt = CFL dt_cfl(0.5)/0.5) at which `steps` fixed DP5 steps from q0 keep every
    state physical and the kinetic energy within 1.5 times its initial value, by bisection."""
    dt1 = s.dt_cfl(q0, 1.0)
    ke0 = s.budgets(q0)[1]

    def ok(c):
        q = q0.clone()
        s.rk_step(q, c * dt1, steps)
        b = s.budgets(q, check=False)
        return all(math.isfinite(x) for x in b) and b[1] <= 1.5 * ke0 and bool(torch.isfinite(q).all()) \
            and float(q[:, 0].min()) > 0.0

    if not ok(lo):
        return None
    while hi - lo > tol * lo:
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo


def study_ipsweep(Re_jump=100.0, steps_jump=200):
    """The interior-penalty coefficient sweep (the IP term of eq. NSL), sigma in IP_SIGMAS.  The term
    acts only on jumps of the entropy variables across element faces.
    (1) Manufactured solution (Re 4e6, exact Dirichlet data), p = 3, 4 on 8^3 elements: P-norm L2
        error of rho after 1.5 flow-through times.
    (2) The 16^3 warped p = 4 Taylor-Green workload (Re 1600): entropy and kinetic-energy rates of the
        state after 100 DP5 steps at CFL 0.5 (the initial state is continuous, so the term is zero
        there), and the largest stable CFL number over 100 DP5 steps.
    (3) Element-wise jumps: a uniform flow (Ma 0.1, u = (0.3, 0.2, 0.1)) on the 8^3 warped p = 4 box
        with a density perturbation of +-1e-3 alternating from element to element (pressure uniform),
        at Re_jump, with the local Lax-Friedrichs interface dissipation and without it (EC): the
        entropy rate of that state, the P-norm L2 norm of the perturbation after steps_jump DP5 steps
        at CFL 0.5 relative to its initial norm, and the largest stable CFL."""
    from paper_1911_10966_gb300 import inputs as I
    from paper_1911_10966_gb300.solver import Solver
    for p in (3, 4):
        for sig in IP_SIGMAS:
            l2, wall, nsteps, dt = _mms_run(p, 8, "esc", ip_coef=sig)
            print(json.dumps({"study": "ipsweep", "case": "mms_8cubed", "p": p, "sigma": sig, "l2_rho": l2,
                              "steps": nsteps, "dt": dt, "wall_s": wall}), flush=True)
    W = TGV_WARPED
    x = I.box_coords(_lgl_nodes(W["p"]), W["k"], W["k"], W["k"], *PI_BOX, warp=W["warp"], seed=W["seed"])
    for sig in IP_SIGMAS:
        s = Solver(W["p"], W["k"], W["k"], W["k"], x, Ma=W["Ma"], Re=W["Re"], ip_coef=sig)
        q0 = s.init_state("tgv")
        q = q0.clone()
        s.rk_step(q, s.dt_cfl(q0, 0.5), 100)
        b = s.budgets(q, s.rhs(q))
        print(json.dumps({"study": "ipsweep", "case": "tgv_16cubed_p4_warped", "sigma": sig,
                          "entropy_rate_after_100_steps": b[2], "ke_rate_after_100_steps": b[3],
                          "stable_cfl_100_steps": _stable_cfl(s, q0)}), flush=True)
        s.close()
    k, p, Ma = 8, 4, 0.1
    x = I.box_coords(_lgl_nodes(p), k, k, k, *PI_BOX, warp=0.1, seed=0)
    N = p + 1
    e = np.arange(k ** 3)
    parity = (-1.0) ** ((e % k) + (e // k) % k + e // (k * k))
    R = 1.0 / (1.4 * Ma * Ma)
    rho = np.broadcast_to((1.0 + 1e-3 * parity)[:, None, None, None], (k ** 3, N, N, N)).copy()
    u = (0.3, 0.2, 0.1)
    q_np = I.primitive_to_conserved(rho, [np.full_like(rho, c) for c in u], np.full_like(rho, R), 1.4)
    base = I.freestream(x, u=u, Ma=Ma)
    for diss, sig in [(d, g) for d in (True, False) for g in IP_SIGMAS]:
        s = Solver(p, k, k, k, x, Ma=Ma, Re=float(Re_jump), ip_coef=sig, dissipation=diss)
        q0 = s.to_device(q_np)
        qb = s.to_device(base)
        n0 = _p_norm_l2(s, q0, qb)
        b = s.budgets(q0, s.rhs(q0))
        q = q0.clone()
        dt = s.dt_cfl(q0, 0.5)
        s.rk_step(q, dt, int(steps_jump))
        print(json.dumps({"study": "ipsweep", "case": "element_jumps_8cubed_p4_warped", "Re": float(Re_jump),
                          "interface_dissipation": "llf" if diss else "none", "sigma": sig,
                          "entropy_rate": b[2], "steps": int(steps_jump), "dt": dt,
                          "perturbation_rel_norm": _p_norm_l2(s, q, qb) / n0,
                          "stable_cfl_100_steps": _stable_cfl(s, q0)}), flush=True)
        s.close()


def _lgl_nodes(p):
    from paper_1911_10966_gb300.solver import lgl
    return lgl(p)[0]


STUDIES = {"rhs": study_rhs, "steps": study_steps, "variants": study_variants, "mms": study_mms,
           "hconv": study_hconv, "ipsweep": study_ipsweep}


def _study(name, kw):
    if name not in STUDIES:
        raise SystemExit(f"unknown study {name!r}; one of {sorted(STUDIES)}")
    torch.cuda.set_device(0)
    STUDIES[name](**kw)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--precision-steps", type=int, default=PRECISION_STEPS,
                    help="length of the float32-mixed vs float64 trajectory (0: skip)")
    ap.add_argument("--headline-only", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--study", default=None, help="run an extra study instead of the bench line")
    ap.add_argument("kv", nargs="*", help="key=value arguments of --study")
    args = ap.parse_args()
    if args.study:
        _study(args.study, dict(a.split("=", 1) for a in args.kv))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
