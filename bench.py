"""Benchmark of the ES-C residual + DP5 step on one GB300 (prints one JSON line).

Workload (default): Taylor-Green vortex, Re = 1600, Ma = 0.1, on a 16^3 periodic box of hexahedra with
smooth sinusoidal node warping (amplitude 0.1 h, phases from seed 0), p = 4 (125 nodes per element,
512,000 nodes), float64 residual.  One step = one fixed Dormand-Prince 5 step (six residual
evaluations, stage combinations) plus the float64 budget reduction of the new state.
Metric: residual DOF/s = nodes x residual evaluations / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): every rank advances an independent replica of the workload (no data-path
collective); value = all ranks' node-residuals / max-over-ranks time ("weak" scaling).
--impl reference times the CPU oracle (plain float64 torch) on the host cores instead.
"""
from __future__ import annotations

import argparse
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

WORKLOAD = dict(name="tgv_16cubed_p4_warped", p=4, k=16, warp=0.1, seed=0, Ma=0.1, Re=1600.0, cfl=0.5)
RHS_PER_STEP = 6
L2_BYTES = 129 * 2 ** 20


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
    by the float64 device functions it includes (flux_f64.cuh) when they sit beside it."""
    data = open(path, "rb").read()
    cut = data.find(LAUNCHER_MARK)
    data = data[:cut] if cut >= 0 else data
    inc = os.path.join(os.path.dirname(path), "flux_f64.cuh")
    if b'#include "flux_f64.cuh"' in data and os.path.exists(inc):
        data += open(inc, "rb").read()
    return hashlib.sha256(data).hexdigest()[:16]


def _ncu_traffic(kernel_src):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current source."""
    f = os.path.join(ROOT, "profiles", "rhs_main_f64_tgv_16cubed_p4.md")
    if not os.path.exists(f):
        return None
    txt = open(f).read()
    sha = None
    val = None
    for line in txt.splitlines():
        if line.startswith("source_sha256_16:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].strip())
    return val if (sha == _sha(kernel_src) and val is not None) else None


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"esdc_clocks_{os.getpid()}.csv")

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


def _config(args, extra=None):
    c = {"workload": WORKLOAD["name"], "mesh": f"{WORKLOAD['k']}^3 hexahedra, sinusoidal warp 0.1h",
         "p": WORKLOAD["p"], "nodes": WORKLOAD["k"] ** 3 * (WORKLOAD["p"] + 1) ** 3, "Re": WORKLOAD["Re"],
         "Ma": WORKLOAD["Ma"], "step": "DP5 step (6 residuals) + float64 budgets recorded on the device",
         "replicas": args.gpus, "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


REF_SAMPLE_ELEMENTS = 512


def _oracle_problem():
    from oracle import esdc_oracle as O
    from paper_1911_10966_gb300 import inputs as I
    p, k = WORKLOAD["p"], WORKLOAD["k"]
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [-math.pi] * 3, [math.pi] * 3, warp=WORKLOAD["warp"], seed=WORKLOAD["seed"])
    mesh = O.make_mesh(p, x, k, k, k)
    gas = O.Gas.from_mach(WORKLOAD["Ma"], WORKLOAD["Re"])
    q = torch.tensor(I.taylor_green(x, Ma=WORKLOAD["Ma"]))
    return O, mesh, gas, q


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores.  Each step: the six residual evaluations of a
    DP5 step restricted to a fixed seeded sample of 512 of the 4096 elements (each with its
    neighbour closure), so that the whole run stays within minutes."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    O, mesh, gas, q = _oracle_problem()
    E = torch.tensor(np.sort(np.random.default_rng(0).choice(mesh.J.shape[0], REF_SAMPLE_ELEMENTS, replace=False)))
    for _ in range(args.warmup):
        O.rhs(q, mesh, gas, elems=E)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(RHS_PER_STEP):
            O.rhs(q, mesh, gas, elems=E)
    el = time.perf_counter() - t0
    n = REF_SAMPLE_ELEMENTS * (WORKLOAD["p"] + 1) ** 3
    val = n * RHS_PER_STEP * args.steps / el
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": "residual DOF/s (nodes x RHS / s), FP64", "value": val,
            "unit": "node-RHS/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": val, "unit": "node-RHS/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step 6 oracle residuals on {REF_SAMPLE_ELEMENTS} of 4096 elements, "
                                       f"{cores} threads"},
            "e2e": {"value": val, "unit": "node-RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    """Oracle timed on the host cores: one DP5 step (6 residuals) of the full workload, plus the
    oracle on the other workload shapes (oracle_config_timings)."""
    O, mesh, gas, q = _oracle_problem()
    p, k = WORKLOAD["p"], WORKLOAD["k"]
    dt = O.cfl_dt(q, mesh, gas, WORKLOAD["cfl"])
    t0 = time.perf_counter()
    O.rk_step(q, lambda st: O.rhs(st, mesh, gas), dt, 1)
    el = time.perf_counter() - t0
    cores = torch.get_num_threads()
    return {"value": k ** 3 * (p + 1) ** 3 * RHS_PER_STEP / el, "unit": "node-RHS/s", "cores": cores, "kind": "oracle",
            "sample": f"one DP5 step (6 residuals) of the full 16^3 p=4 workload, {el:.1f} s on {cores} threads",
            "configs": oracle_config_timings()}


ORACLE_SAMPLE_ELEMENTS = 256
# elements per direction giving ~16M nodes per degree (the p-sweep meshes)
PSWEEP_K = {2: 84, 3: 63, 4: 50, 5: 42, 6: 36, 7: 32}


def oracle_config_timings():
    """The oracle (as it stands, float64 torch on the host cores) on the other workload shapes, in
    node-RHS/s: the 4^3 affine p=3 Taylor-Green box (one residual and ten DP5 steps, whole mesh), the
    8^3 warped p=4 isentropic vortex (one residual, whole mesh), and one residual of each ~16M-node
    p-sweep mesh (p = 2..7) restricted to a seeded sample of 256 elements (the whole mesh would take
    minutes per degree; the count is of the sampled nodes, although the oracle also evaluates the
    entropy-variable gradients of their face neighbours)."""
    from oracle import esdc_oracle as O
    from paper_1911_10966_gb300 import inputs as I
    out = {}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    s = O.sbp_operator(3)
    x = I.box_coords(s.xi.numpy(), 4, 4, 4, [-math.pi] * 3, [math.pi] * 3)
    mesh = O.make_mesh(3, x, 4, 4, 4)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.taylor_green(x, Ma=0.1))
    n = q.shape[0] * 64
    t1 = timed(lambda: O.rhs(q, mesh, gas))
    dt = O.cfl_dt(q, mesh, gas, 0.5)
    t10 = timed(lambda: O.rk_step(q, lambda st: O.rhs(st, mesh, gas), dt, 10))
    out["tgv_4cubed_p3"] = {"rhs_node_rhs_per_s": n / t1, "dp5_10_steps_s": t10,
                            "dp5_node_rhs_per_s": n * 60 / t10}
    s = O.sbp_operator(4)
    x = I.box_coords(s.xi.numpy(), 8, 8, 8, [-5.0] * 3, [5.0] * 3, warp=0.1, seed=1)
    mesh = O.make_mesh(4, x, 8, 8, 8)
    gas = O.Gas.from_mach(0.5, 1000.0)
    q = torch.tensor(I.isentropic_vortex(x, Ma=0.5, u_inf=(1 / math.sqrt(2), -1 / math.sqrt(2), 0.0)))
    out["vortex_8cubed_p4_warped"] = {"rhs_node_rhs_per_s": q.shape[0] * 125 / timed(lambda: O.rhs(q, mesh, gas))}
    gas = O.Gas.from_mach(0.1, 1600.0)
    for p, k in PSWEEP_K.items():
        s = O.sbp_operator(p)
        x = I.box_coords(s.xi.numpy(), k, k, k, [-math.pi] * 3, [math.pi] * 3)
        E = torch.tensor(np.sort(np.random.default_rng(p).choice(k ** 3, ORACLE_SAMPLE_ELEMENTS, replace=False)))
        sub, E2, rows = O.make_submesh(p, x, O.box_neighbours(k, k, k), E)
        q = torch.tensor(I.taylor_green(x[E2.numpy()], Ma=0.1))
        el = timed(lambda: O.rhs(q, sub, gas, elems=rows))
        out[f"tgv_psweep_p{p}_{k}cubed"] = {"rhs_node_rhs_per_s": ORACLE_SAMPLE_ELEMENTS * (p + 1) ** 3 / el,
                                            "sample_elements": ORACLE_SAMPLE_ELEMENTS}
    return out


def run_ours(args):
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1911_10966_gb300 import inputs as I
    from paper_1911_10966_gb300.solver import Solver, probe_fma

    W = WORKLOAD
    solver = Solver.box(W["p"], W["k"], W["k"], W["k"], warp=W["warp"], seed=W["seed"], Ma=W["Ma"], Re=W["Re"])
    q_init = I.taylor_green(solver.coords, Ma=W["Ma"])
    q = solver.to_device(q_init)
    dt = solver.dt_cfl(q, W["cfl"])
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=q.device)
    n = solver.n_nodes
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        solver.rk_step(q, dt, 1)
        solver.budgets(q)
    peak_f64 = probe_fma("f64")

    # ---- device-timed region: inputs resident in HBM
    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # float64 budgets of every step, recorded on the device and read back after the timed region
    hist = torch.zeros((args.steps, 5), dtype=torch.float64, device=q.device)
    solver.profile(True)
    with ClockSampler(local) as clk:
        time.sleep(0.6)          # let the sampler start before the timed region
        barrier()
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            solver.rk_step(q, dt, 1)
            solver.budgets_async(q, hist[i])
            evs[i][1].record(stream)
        barrier()
    ms_main, ms_face, nres = solver.profile_read()
    solver.profile(False)
    _check_budgets(hist)
    ms_step = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ms_max = max_over_ranks(ms_step, dist, q.device)
    value = replica_throughput(n, ws, ms_max)

    # ---- end to end through the public API with host buffers
    q_host = torch.from_numpy(np.ascontiguousarray(q_init)).pin_memory()
    q_back = torch.empty_like(q_host).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        qd = q.copy_(q_host, non_blocking=True)
        solver.rk_step(qd, dt, 1)
        solver.budgets(qd)
        q_back.copy_(qd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_val = replica_throughput(n, ws, max_over_ranks(e2e_s * 1e3, dist, q.device))

    # ---- residual-only throughput (the metric's unit operation), same stream and inputs
    r = torch.empty_like(q)
    solver.rhs(q, out=r)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    flush.fill_(0.0)
    a.record(stream)
    for _ in range(reps):
        solver.rhs(q, out=r)
    b.record(stream)
    torch.cuda.synchronize()
    ms_rhs = a.elapsed_time(b) / reps

    multi64 = _multi_step_ms(solver, solver.to_device(q_init), dt, 10, flush)
    adj = _adjoint_leg(solver, solver.to_device(q_init), dt, ms_rhs, flush)
    ada = _adaptive_leg(solver, q_init, dt)
    var = _variants_leg(solver, q_init, ms_rhs)
    fp32 = _fp32_leg(args, solver, q_init, dt, flush, barrier, dist, ws) if not args.no_fp32 else None
    if fp32 is not None:
        fp32["speedup_vs_f64_rhs"] = (ms_main / max(nres, 1)) / fp32["roofline"]["kernel_ms"]

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    src = os.path.join(ROOT, "paper_1911_10966_gb300", "csrc", "rhs_f64.cu")
    fl = element_kernel_flops_per_node(W["p"]) * n
    kernel_ms = ms_main / max(nres, 1)
    achieved = fl / (kernel_ms * 1e-3) / 1e12
    peak = peak_f64 / 1e12
    clocks = clk.summary()
    line = {
        "metric": "residual DOF/s (nodes x RHS / s), FP64", "value": value, "unit": "node-RHS/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(args),
        "roofline": {"bound": "alu", "kernel": "rhs_main_f64<5>", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": _ncu_traffic(src),
                     "peak_source": "measured float64 FMA throughput (esdc_probe_fma) in this run",
                     "flops_per_launch": fl, "kernel_ms": kernel_ms,
                     "hbm_frac": element_kernel_bytes_per_node(W["p"]) * n / (kernel_ms * 1e-3) / 6690.1e9},
        "cpu_baseline": cpu_baseline_sample() if (ws == 1 and not args.no_cpu_baseline) else None,
        "e2e": {"value": e2e_val, "unit": "node-RHS/s", "h2d_bytes_per_step": n * 40,
                "d2h_bytes_per_step": n * 40 + 40},
        # per step: element + viscous face kernel per residual, five stage combinations and the
        # solution update, budgets + final sum
        "gpu_launches": args.steps * (RHS_PER_STEP * 2 + RHS_PER_STEP + 2),
        "clocks": clocks,
        "rhs_only": {"value": n / (ms_rhs * 1e-3), "unit": "node-RHS/s", "ms": ms_rhs,
                     "face_kernel_ms": ms_face / max(nres, 1)},
        "fp32_mixed": fp32,
        "multi_step": multi64,
        "adjoint": adj,
        "adaptive_dp54": ada,
        "volume_flux_variants": var,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _multi_step_ms(solver, q, dt, steps, flush):
    """DP5 steps without budgets, (a) one call per step (direct launches) and (b) one call for all
    steps (one step captured as a CUDA graph and replayed): ms per step each."""
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    return {"ms_per_step_direct": out["direct"], "ms_per_step_graph": out["graph"], "steps": steps,
            "what": "DP5 steps without budgets: one call per step vs one multi-step call (CUDA-graph replay)"}


def _check_budgets(hist):
    """The per-step budgets recorded on the device: every state physical, every sum finite."""
    h = hist.cpu()
    if float(h[:, 4].abs().sum()) != 0.0 or not bool(torch.isfinite(h).all()):
        raise RuntimeError("non-physical state during the timed steps")


def _fp32_leg(args, s64, q_init, dt, flush, barrier, dist, ws):
    """The mixed-precision form on the same workload: float32 residual, float64 state and budgets."""
    from paper_1911_10966_gb300.solver import Solver, probe_fma
    W = WORKLOAD
    s32 = Solver(W["p"], W["k"], W["k"], W["k"], s64.coords, Ma=W["Ma"], Re=W["Re"], precision="fp32")
    n = s32.n_nodes
    q = s32.to_device(q_init)
    # error of the float32 residual against the float64 path (itself parity-checked against the oracle)
    r64 = s64.rhs(q)
    r32 = s32.rhs(q)
    e_v = [float((r32[:, v].double() - r64[:, v]).abs().max() / r64[:, v].abs().max()) for v in range(5)]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        s32.rk_step(q, dt, 1)
        s32.budgets(q)
    peak32 = probe_fma("f32")
    steps = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    hist = torch.zeros((steps, 5), dtype=torch.float64, device=q.device)
    s32.profile(True)
    barrier()
    for i in range(steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        s32.rk_step(q, dt, 1)
        s32.budgets_async(q, hist[i])
        evs[i][1].record(stream)
    barrier()
    ms_main, ms_face, nres = s32.profile_read()
    s32.profile(False)
    _check_budgets(hist)
    ms_step = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / steps, dist, q.device)
    multi = _multi_step_ms(s32, q, dt, 50, flush)
    # kinetic-energy dissipation rate after the same number of steps in both precisions
    qa = s64.to_device(q_init)
    qb = s32.to_device(q_init)
    s64.rk_step(qa, dt, 5)
    s32.rk_step(qb, dt, 5)
    k64 = s64.budgets(qa, s64.rhs(qa))[3]
    k32 = s32.budgets(qb, s32.rhs(qb))[3]
    kernel_ms = ms_main / max(nres, 1)
    fl = element_kernel_flops_per_node(W["p"]) * n
    by = element_kernel_bytes_per_node_f32(W["p"]) * n
    t_alu = fl / peak32
    t_hbm = by / 6690.1e9
    bound = "alu" if t_alu >= t_hbm else "hbm"
    if bound == "alu":
        roof = {"bound": "alu", "achieved": fl / (kernel_ms * 1e-3) / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": by / (kernel_ms * 1e-3) / 1e9, "peak": 6690.1, "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"kernel": "rhs_main_f32<5>", "kernel_ms": kernel_ms, "flops_per_launch": fl, "bytes_per_launch": by,
                 "alu_frac": fl / (kernel_ms * 1e-3) / peak32, "hbm_frac": by / (kernel_ms * 1e-3) / 6690.1e9,
                 "peak_source": "measured float32 FMA throughput (esdc_probe_fma) / MEASURED_PEAKS hbm_gbs"})
    return {"value": replica_throughput(n, ws, ms_step), "unit": "node-RHS/s", "ms_per_step": ms_step,
            "dtype": "f32 residual, f64 state/update/budgets", "roofline": roof,
            "residual_error_vs_f64": {"per_variable": e_v, "variables": ["rho", "rho u1", "rho u2", "rho u3", "rho E"]},
            "ke_rate_rel_error_5_steps": abs(k32 - k64) / abs(k64),
            "multi_step": multi,
            # per step: shadow state, element + viscous face kernel per residual (stage states are
            # formed inside the element kernel), the float64 update, budgets + final sum
            "gpu_launches": steps * (1 + RHS_PER_STEP * 2 + 1 + 2),
            "speedup_vs_f64_rhs": None}


def _adjoint_leg(solver, q, dt, ms_rhs, flush):
    """Cost of the hand-written adjoint on the same workload: one vector-Jacobian product against one
    residual, and the gradient of the final kinetic energy through 5 DP5 steps against the 5 forward
    steps alone, with stage checkpoints (the six stage states of every step stored by the forward
    pass) and with per-step checkpoints plus stage recomputation in the reverse sweep."""
    stream = torch.cuda.current_stream()
    lam = torch.randn(q.shape, dtype=torch.float64, device=q.device, generator=torch.Generator(q.device).manual_seed(3))
    g = solver.rhs_vjp(q, lam)
    reps = 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1.0)
    a.record(stream)
    for _ in range(reps):
        g = solver.rhs_vjp(q, lam)
    b.record(stream)
    torch.cuda.synchronize()
    ms_vjp = a.elapsed_time(b) / reps
    nsteps = 5
    qa = q.clone()
    flush.fill_(2.0)
    a.record(stream)
    solver.rk_step(qa, dt, nsteps)
    b.record(stream)
    torch.cuda.synchronize()
    ms_fwd = a.elapsed_time(b)

    def gradient(stages):
        qb = q.clone()
        ck = solver.rk_step_ckpt(qb, dt, nsteps, stages=stages)
        lamN = solver.ke_gradient(qb)
        return solver.rk_adjoint(ck, dt, lamN)

    out = {}
    for stages in (True, False):
        gradient(stages)                      # warm-up: workspaces and checkpoint memory
        flush.fill_(3.0)
        a.record(stream)
        _, gmu = gradient(stages)
        b.record(stream)
        torch.cuda.synchronize()
        out[stages] = (a.elapsed_time(b), gmu)
    ms_grad, gmu = out[True]
    ms_grad_rc, gmu_rc = out[False]
    return {"vjp_ms": ms_vjp, "rhs_ms": ms_rhs, "vjp_over_rhs": ms_vjp / ms_rhs,
            "trajectory_steps": nsteps, "forward_ms": ms_fwd, "gradient_ms": ms_grad,
            "gradient_over_forward": ms_grad / ms_fwd,
            "gradient_recompute_ms": ms_grad_rc, "gradient_recompute_over_forward": ms_grad_rc / ms_fwd,
            "dke_dmu": gmu, "dke_dmu_recompute_rel_diff": abs(gmu - gmu_rc) / abs(gmu), "dtype": "f64",
            "what": "d KE(q_5)/d(q_0, mu): forward storing the stage states + reverse sweep (6 VJPs per "
                    "step); recompute variant: per-step checkpoints, 6 residual recomputations + 6 VJPs "
                    "per step"}


def _variants_leg(solver, q_init, ms_rhs):
    """Residual cost of the paper's comparison discretisations on the same workload (float64): the
    Kennedy-Gruber split form (SF-KG) and standard collocation (DC) beside ES-C, and ES-C with the
    Roe-type matrix interface dissipation instead of local Lax-Friedrichs."""
    from paper_1911_10966_gb300.solver import Solver
    W = WORKLOAD
    out = {"esc": {"rhs_ms": ms_rhs, "node_rhs_per_s": solver.n_nodes / (ms_rhs * 1e-3)}}
    for vf, diss in (("kg", True), ("dc", True), ("esc", "matrix")):
        s = Solver(W["p"], W["k"], W["k"], W["k"], solver.coords, Ma=W["Ma"], Re=W["Re"], volume_flux=vf,
                   dissipation=diss)
        ms = _time_rhs_ms(s, q_init)
        out[vf if diss is True else "esc_matrix_dissipation"] = {"rhs_ms": ms,
                                                                 "node_rhs_per_s": s.n_nodes / (ms * 1e-3)}
        s.close()
    return out


def _time_rhs_ms(s, q_init, reps=10):
    q = s.to_device(q_init)
    r = s.rhs(q)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        s.rhs(q, out=r)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _adaptive_leg(solver, q_init, dt):
    """Adaptive DP5(4) (esdc_rk_adaptive) on the same workload over 200 CFL steps of physical time,
    rtol = atol = 1e-8, first trial step 4 CFL steps: residual throughput including the error
    estimate and the per-step host decision."""
    tol, span = 1e-8, 200.0
    q = solver.to_device(q_init)
    solver.rk_adaptive(q, 0.0, 2.0 * dt, dt, rtol=tol, atol=tol)        # warm-up: workspace
    q = solver.to_device(q_init)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solver.rk_adaptive(q, 0.0, span * dt, 4.0 * dt, rtol=tol, atol=tol)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"t_end_over_cfl_dt": span, "rtol": tol, "atol": tol, "accepted": st["accepted"],
            "rejected": st["rejected"], "rhs": st["rhs"], "wall_ms": wall * 1e3,
            "node_rhs_per_s": solver.n_nodes * st["rhs"] / wall, "mean_dt_over_cfl_dt": span / st["accepted"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the mixed-precision leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
