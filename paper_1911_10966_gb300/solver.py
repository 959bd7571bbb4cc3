"""Python front end: a thin owner of one library context plus torch tensors for device memory.

Every computation (residual, Runge-Kutta stages, budgets, CFL reduction) is a call into
libesdc.so; this module only checks shapes/dtypes and passes pointers and the current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as nat
from . import inputs


def lgl(p: int):
    """The library's LGL nodes and weights (Sec. 2, Definition 1)."""
    xi = np.zeros(p + 1)
    w = np.zeros(p + 1)
    nat.check(nat.lib().esdc_lgl(p, xi.ctypes.data, w.ctypes.data), "esdc_lgl")
    return xi, w


def probe_fma(kind: str = "f64") -> float:
    """Measured FMA throughput of the current GPU in FLOP/s (library microbenchmark)."""
    out = ctypes.c_double()
    nat.check(nat.lib().esdc_probe_fma(0 if kind == "f64" else 1, ctypes.byref(out), _stream_ptr()),
              "esdc_probe_fma")
    return out.value


def mms_fields(x, table, gamma=1.4, Ma=1.0, Re=0.0, Pr=0.72, L=1.0):
    """The library's manufactured solution and its source term (esdc_mms_fields) at node coordinates
    x [K, 3, N, N, N] (numpy): returns (q, source), each [K, 5, N, N, N]."""
    x = np.ascontiguousarray(np.moveaxis(np.asarray(x, dtype=np.float64), 1, -1))
    n = x.size // 3
    tab = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(5, 7))
    q = np.empty(x.shape[:-1] + (5,))
    s = np.empty(x.shape[:-1] + (5,))
    nat.check(nat.lib().esdc_mms_fields(gamma, Ma, Re, Pr, L, tab.ctypes.data, n, x.ctypes.data, q.ctypes.data,
                                        s.ctypes.data), "esdc_mms_fields")
    return np.ascontiguousarray(np.moveaxis(q, -1, 1)), np.ascontiguousarray(np.moveaxis(s, -1, 1))


def _stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """ES-C residual and DP5 time stepping on one GPU for a periodic kx*ky*kz hexahedral box.

    coords: numpy [K, 3, N, N, N] node coordinates (degree-p mapping at the LGL nodes).
    precision: "fp64" (whole residual in float64) or "fp32" (float32 residual, float64 state).
    dissipation: True (local Lax-Friedrichs), False (entropy conservative) or "matrix" (Roe-type
    entropy-stable matrix dissipation; float64 only).
    volume_flux: "esc" (the paper's ES-C), "kg" (SF-KG) or "dc" (DC); the last two float64 only.
    ip_coef: interior-penalty coefficient (0: off; float64 only).
    bounded: per direction, True for boundary faces with Dirichlet data (set_exterior) instead of
    periodic connectivity (float64 only).
    metrics: "curl" (conservative curl form) or "optimized" (the paper's optimized volume metrics
    with analytic surface metrics in the interface terms; float64 only).
    """

    def __init__(self, p, kx, ky, kz, coords, *, gamma=1.4, Pr=0.72, Ma=0.1, Re=0.0, dissipation=True,
                 precision="fp64", volume_flux="esc", ip_coef=0.0, bounded=(False, False, False), metrics="curl",
                 device=None, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, warp=0.0, seed=0):
        """coords None: the library's box mesh generator on [lo, hi] with warp amplitude `warp` and
        splitmix64 phases from `seed` (esdc_host_coordinates); self.coords then holds its nodes."""
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU implementation exists)")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        self.p, self.N = p, p + 1
        self.kx, self.ky, self.kz = kx, ky, kz
        self.K = kx * ky * kz
        self.gamma, self.Pr, self.Ma, self.Re = gamma, Pr, Ma, Re
        self.precision = precision
        if volume_flux not in nat.FLUX:
            raise ValueError("volume_flux must be 'esc', 'kg' or 'dc'")
        self.volume_flux = volume_flux
        if metrics not in nat.METRICS:
            raise ValueError("metrics must be 'curl' or 'optimized'")
        self.metrics = metrics
        self.dtype_r = torch.float64 if precision == "fp64" else torch.float32
        diss = 2 if dissipation == "matrix" else (1 if dissipation else 0)
        st = nat.Setup(p, kx, ky, kz, gamma, Pr, Ma, Re, diss,
                       nat.PREC_FP64 if precision == "fp64" else nat.PREC_FP32, nat.FLUX[volume_flux],
                       float(ip_coef), sum(1 << l for l in range(3) if bounded[l]), nat.METRICS[metrics],
                       (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi), float(warp), int(seed))
        if coords is None:
            coords = np.empty((self.K, 3, self.N, self.N, self.N))
            nat.check(nat.lib().esdc_host_coordinates(ctypes.byref(st), coords.ctypes.data), "esdc_host_coordinates")
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        if coords.shape != (self.K, 3, self.N, self.N, self.N):
            raise ValueError(f"coords must have shape {(self.K, 3, self.N, self.N, self.N)}, got {coords.shape}")
        self.coords = coords
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_create(ctypes.byref(st), coords.ctypes.data, ctypes.byref(self._ctx)),
                      "esdc_create")
        self._ws = None
        self._adj_ws = None
        self._ada_ws = None
        self._ext = None
        self._src = None

    @classmethod
    def box(cls, p, kx, ky, kz, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, warp=0.0, seed=0, **kw):
        xi, _ = lgl(p)
        return cls(p, kx, ky, kz, inputs.box_coords(xi, kx, ky, kz, lo, hi, warp=warp, seed=seed), **kw)

    # -- lifetime
    def close(self):
        if self._ctx is not None and self._ctx.value:
            nat.lib().esdc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    @property
    def n_nodes(self):
        return self.K * self.N ** 3

    @property
    def state_shape(self):
        return (self.K, 5, self.N, self.N, self.N)

    def _check_state(self, q, dtype=torch.float64):
        if not (isinstance(q, torch.Tensor) and q.is_cuda and q.dtype == dtype and q.is_contiguous()
                and tuple(q.shape) == self.state_shape and q.device == self.device):
            raise ValueError(f"expected a contiguous {dtype} CUDA tensor of shape {self.state_shape} on {self.device}")

    def to_device(self, q_np):
        return torch.as_tensor(np.ascontiguousarray(q_np), dtype=torch.float64, device=self.device)

    def init_state(self, ic="tgv", params=None):
        """A new float64 state tensor holding an initial state computed on the device at the node
        coordinates: "tgv" (Taylor-Green vortex), "vortex" (params: beta, centre[3], axis[3],
        u_inf[3]) or "freestream" (params: rho, u[3], p); see esdc_init_state."""
        if ic not in nat.IC:
            raise ValueError("ic must be 'tgv', 'vortex' or 'freestream'")
        q = torch.empty((self.K, 5, self.N, self.N, self.N), dtype=torch.float64, device=self.device)
        pa = None
        if params is not None:
            pa = np.ascontiguousarray(params, dtype=np.float64)
            if pa.size != {"vortex": 10, "freestream": 5}.get(ic, 0):
                raise ValueError("wrong number of parameters for " + ic)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_init_state(self._ctx, nat.IC[ic], pa.ctypes.data if pa is not None else None,
                                                q.data_ptr(), _stream_ptr()), "esdc_init_state")
        return q

    def geometry(self):
        N3 = self.N ** 3
        J = np.zeros((self.K, N3))
        Ja = np.zeros((self.K, 9, N3))
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_geometry(self._ctx, J.ctypes.data, Ja.ctypes.data), "esdc_geometry")
        return J.reshape(self.K, self.N, self.N, self.N), Ja.reshape(self.K, 3, 3, self.N, self.N, self.N)

    # -- the hot path
    def rhs(self, q, out=None):
        self._check_state(q)
        if out is None:
            out = torch.empty(self.state_shape, dtype=self.dtype_r, device=self.device)
        else:
            self._check_state(out, self.dtype_r)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_rhs(self._ctx, q.data_ptr(), out.data_ptr(), _stream_ptr()), "esdc_rhs")
        return out

    def rhs_host(self, q_host, out_host=None):
        """Residual of a host (CPU, preferably pinned) float64 state; returns a host tensor."""
        if not (isinstance(q_host, torch.Tensor) and not q_host.is_cuda and q_host.dtype == torch.float64
                and q_host.is_contiguous() and tuple(q_host.shape) == self.state_shape):
            raise ValueError("q_host must be a contiguous float64 CPU tensor of the state shape")
        if out_host is None:
            out_host = torch.empty(self.state_shape, dtype=self.dtype_r, pin_memory=True)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_rhs_host(self._ctx, q_host.data_ptr(), out_host.data_ptr(), _stream_ptr()),
                      "esdc_rhs_host")
        return out_host

    def workspace_bytes(self):
        b = ctypes.c_size_t()
        nat.check(nat.lib().esdc_workspace_bytes(self._ctx, 0, ctypes.byref(b)), "esdc_workspace_bytes")
        return b.value

    def rk_step(self, q, dt, nsteps=1):
        """Advance q in place by nsteps fixed Dormand-Prince 5 steps."""
        self._check_state(q)
        nb = self.workspace_bytes()
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_rk_step(self._ctx, q.data_ptr(), float(dt), int(nsteps), self._ws.data_ptr(),
                                             self._ws.numel(), _stream_ptr()), "esdc_rk_step")
        return q

    def budgets(self, q, dqdt=None, check=True):
        """(sum PJ S, KE, sum PJ w.dq/dt, dKE/dt) in float64 (synchronises)."""
        self._check_state(q)
        if dqdt is not None:
            self._check_state(dqdt, self.dtype_r)
        out = (ctypes.c_double * 4)()
        with torch.cuda.device(self.device):
            code = nat.lib().esdc_budgets(self._ctx, q.data_ptr(), dqdt.data_ptr() if dqdt is not None else None,
                                          out, _stream_ptr())
        if check:
            nat.check(code, "esdc_budgets")
        return tuple(out)

    def set_exterior(self, q_ext):
        """Exterior (Dirichlet) state of the boundary faces, a state-shaped float64 CUDA tensor read
        at the boundary face nodes; the solver keeps a reference.  None clears it."""
        if q_ext is not None:
            self._check_state(q_ext)
        nat.check(nat.lib().esdc_set_exterior(self._ctx, q_ext.data_ptr() if q_ext is not None else None),
                  "esdc_set_exterior")
        self._ext = q_ext

    def set_source(self, source):
        """Source term added to dq/dt (state-shaped float64 CUDA tensor, referenced); None clears it."""
        if source is not None:
            self._check_state(source)
        nat.check(nat.lib().esdc_set_source(self._ctx, source.data_ptr() if source is not None else None),
                  "esdc_set_source")
        self._src = source

    def budgets_async(self, q, out, dqdt=None):
        """Write (sum PJ S, KE, sum PJ w.dq/dt, dKE/dt, non-physical node count) into the float64
        CUDA tensor `out` (5 contiguous elements) without synchronising."""
        self._check_state(q)
        if dqdt is not None:
            self._check_state(dqdt, self.dtype_r)
        if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
                and out.numel() >= 5 and out.device == self.device):
            raise ValueError("out must be a contiguous float64 CUDA tensor of at least 5 elements on the solver's device")
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_budgets_async(self._ctx, q.data_ptr(), dqdt.data_ptr() if dqdt is not None else None,
                                                   out.data_ptr(), _stream_ptr()), "esdc_budgets_async")
        return out

    # -- adjoint (float64 contexts)
    def rhs_vjp(self, q, lam, want_mu=False):
        """(dR/dq)^T lam and, if want_mu, lam . dR/dmu."""
        self._check_state(q)
        self._check_state(lam)
        g = torch.empty_like(q)
        gm = ctypes.c_double()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_rhs_vjp(self._ctx, q.data_ptr(), lam.data_ptr(), g.data_ptr(),
                                             ctypes.byref(gm) if want_mu else None, _stream_ptr()), "esdc_rhs_vjp")
        return (g, gm.value) if want_mu else g

    def ke_gradient(self, q):
        self._check_state(q)
        g = torch.empty_like(q)
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_ke_gradient(self._ctx, q.data_ptr(), g.data_ptr(), _stream_ptr()),
                      "esdc_ke_gradient")
        return g

    def rk_adaptive(self, q, t0, t_end, dt0, rtol=1e-6, atol=1e-6, max_steps=100000, history=0):
        """Advance q in place from t0 to t_end with adaptive DP5(4) (float64 or float32-mixed).  Returns a
        dict: accepted, rejected, rhs (residual evaluations), t (time reached), dt_next and, if
        history > 0, dt_history (the first `history` accepted step sizes)."""
        self._check_state(q)
        b = ctypes.c_size_t()
        nat.check(nat.lib().esdc_workspace_bytes(self._ctx, 1, ctypes.byref(b)), "esdc_workspace_bytes")
        if self._ada_ws is None or self._ada_ws.numel() < b.value:
            self._ada_ws = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        dt = ctypes.c_double(float(dt0))
        stats = (ctypes.c_double * 4)()
        hist = (ctypes.c_double * max(int(history), 1))()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_rk_adaptive(self._ctx, q.data_ptr(), float(t0), float(t_end), ctypes.byref(dt),
                                                 float(rtol), float(atol), int(max_steps), self._ada_ws.data_ptr(),
                                                 self._ada_ws.numel(), stats, hist if history else None,
                                                 int(history), _stream_ptr()), "esdc_rk_adaptive")
        out = {"accepted": int(stats[0]), "rejected": int(stats[1]), "rhs": int(stats[2]), "t": stats[3],
               "dt_next": dt.value}
        if history:
            out["dt_history"] = list(hist)[:min(int(history), out["accepted"])]
        return out

    def rk_step_ckpt(self, q, dt, nsteps, stages=False, k1=True):
        """Advance q in place and return the checkpoints of the adjoint: with stages=True the six stage
        states of every step, [nsteps, 6, K, 5, N, N, N] (no recomputation in the reverse sweep);
        otherwise the state before each step with its residual (k1=True, [nsteps, 2, K, 5, N, N, N];
        four residual recomputations per step in the reverse sweep) or alone (k1=False,
        [nsteps, K, 5, N, N, N]; five)."""
        self._check_state(q)
        if stages:
            shape = (nsteps, 6) + self.state_shape
        elif k1:
            shape = (nsteps, 2) + self.state_shape
        else:
            shape = (nsteps,) + self.state_shape
        ck = torch.empty(shape, dtype=torch.float64, device=self.device)
        nb = self.workspace_bytes()
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        L = nat.lib()
        with torch.cuda.device(self.device):
            if stages:
                nat.check(L.esdc_rk_step_stages(self._ctx, q.data_ptr(), float(dt), int(nsteps), ck.data_ptr(),
                                                self._ws.data_ptr(), self._ws.numel(), _stream_ptr()),
                          "esdc_rk_step_stages")
            else:
                nat.check(L.esdc_rk_step_ckpt(self._ctx, q.data_ptr(), float(dt), int(nsteps), ck.data_ptr(),
                                              1 if k1 else 0, self._ws.data_ptr(), self._ws.numel(), _stream_ptr()),
                          "esdc_rk_step_ckpt")
        return ck

    def _checkpoint_kind(self, ckpt):
        """'stages', 'k1' or 'state' for a tensor returned by rk_step_ckpt of this solver."""
        ok = ckpt.is_cuda and ckpt.dtype == torch.float64 and ckpt.is_contiguous() and ckpt.device == self.device
        nd = len(self.state_shape)
        if ok and ckpt.dim() == nd + 2 and tuple(ckpt.shape[2:]) == self.state_shape and ckpt.shape[1] in (2, 6):
            return "stages" if ckpt.shape[1] == 6 else "k1"
        if ok and ckpt.dim() == nd + 1 and tuple(ckpt.shape[1:]) == self.state_shape:
            return "state"
        raise ValueError("ckpt must come from rk_step_ckpt of this solver")

    def rk_adjoint(self, ckpt, dt, lam):
        """Reverse sweep from the checkpoints of rk_step_ckpt (per-step states, with or without their
        residuals: stage recomputation; stage states: none): lam (dL/dq_N) is replaced by dL/dq_0;
        returns (lam, dL/dmu)."""
        self._check_state(lam)
        kind = self._checkpoint_kind(ckpt)
        nsteps = ckpt.shape[0]
        b = ctypes.c_size_t()
        nat.check(nat.lib().esdc_rk_adjoint_workspace_bytes(self._ctx, ctypes.byref(b)), "workspace")
        if self._adj_ws is None or self._adj_ws.numel() < b.value:
            self._adj_ws = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        gm = ctypes.c_double()
        L = nat.lib()
        with torch.cuda.device(self.device):
            if kind == "stages":
                nat.check(L.esdc_rk_adjoint_stages(self._ctx, ckpt.data_ptr(), float(dt), int(nsteps), lam.data_ptr(),
                                                   ctypes.byref(gm), self._adj_ws.data_ptr(), self._adj_ws.numel(),
                                                   _stream_ptr()), "esdc_rk_adjoint_stages")
            else:
                nat.check(L.esdc_rk_adjoint(self._ctx, ckpt.data_ptr(), 1 if kind == "k1" else 0, float(dt),
                                            int(nsteps), lam.data_ptr(), ctypes.byref(gm), self._adj_ws.data_ptr(),
                                            self._adj_ws.numel(), _stream_ptr()), "esdc_rk_adjoint")
        return lam, gm.value

    @property
    def mu(self):
        return 1.0 / self.Re if self.Re > 0 else 0.0

    def device_status(self, clear=True):
        """Status bits the kernels recorded on the device (0: every bounded wait completed; 1: a
        wait for bulk shared-memory copies gave up and its elements were left unevaluated)."""
        st = ctypes.c_int()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_device_status(self._ctx, ctypes.byref(st), 1 if clear else 0, _stream_ptr()),
                      "esdc_device_status")
        return st.value

    def profile(self, on=True):
        """Record CUDA events around the residual kernels of every following evaluation."""
        nat.check(nat.lib().esdc_profile(self._ctx, 1 if on else 0), "esdc_profile")

    def profile_read(self):
        """(ms in the element kernel, ms in the face kernel, evaluations) since profile(True)."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_profile_read(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
                      "esdc_profile_read")
        return a.value, b.value, n.value

    def dt_cfl(self, q, cfl=0.5):
        self._check_state(q)
        dt = ctypes.c_double()
        with torch.cuda.device(self.device):
            nat.check(nat.lib().esdc_dt_cfl(self._ctx, q.data_ptr(), float(cfl), ctypes.byref(dt), _stream_ptr()),
                      "esdc_dt_cfl")
        return dt.value
