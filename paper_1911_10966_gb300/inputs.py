"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no arithmetic of the discretisation: it only places mesh nodes and evaluates
initial conditions.  The 1D collocation nodes are an ARGUMENT (each side passes the Gauss-Lobatto
nodes it computed itself), so the two sides share node placement recipes and nothing else.

Nondimensionalisation used by every workload: rho_inf = T_inf = 1, gas constant R = 1/(gamma Ma^2),
so that p_inf = 1/(gamma Ma^2), c_inf = 1/Ma and velocities are O(1).

Array layouts (numpy, float64):
  coords  [K, 3, N, N, N]   (element, x-component, xi3, xi2, xi1) -- xi1 fastest
  state   [K, 5, N, N, N]   conserved variables (rho, rho u1, rho u2, rho u3, rho E)
Element e of a kx*ky*kz box is e = ex + kx*(ey + ky*ez).
"""
from __future__ import annotations

import math

import numpy as np


def gas_constant(Ma: float, gamma: float) -> float:
    """R = 1/(gamma Ma^2) under rho_inf = T_inf = 1."""
    return 1.0 / (gamma * Ma * Ma)


def warp_phases(seed: int) -> np.ndarray:
    """3x3 phases in [0, 2 pi) for the sinusoidal node warping, from a seeded PCG64 stream."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * math.pi, size=(3, 3))


def splitmix64_phases(seed: int) -> np.ndarray:
    """3x3 phases in [0, 2 pi) (i-major) from successive splitmix64 outputs (Steele, Lea and Flood,
    OOPSLA 2014) started at seed, each mapped as (z >> 11) 2^-53 2 pi: the phases of the library's
    own box mesh generator (esdc_create with no node coordinates)."""
    mask = (1 << 64) - 1
    state = seed & mask
    out = np.empty((3, 3))
    for n in range(9):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        out[n // 3, n % 3] = float(z >> 11) * 2.0 ** -53 * (2.0 * math.pi)
    return out


def box_coords(xi, kx, ky, kz, lo, hi, warp=0.0, seed=0, phases=None) -> np.ndarray:
    """Node coordinates of a kx*ky*kz hexahedral box mesh, optionally warped.

    xi    : the N one-dimensional reference nodes on [-1, 1] (supplied by the caller)
    warp  : amplitude as a fraction of the element size h_i; the displacement of component i is
            warp*h_i*prod_k sin(2 pi (X_k - lo_k)/L_k + phi_ik), L-periodic in every direction, so
            periodic faces and shared faces stay watertight (Sec. 2, Assumption 1).
    phases: the 3x3 phi (default: warp_phases(seed))
    """
    xi = np.asarray(xi, dtype=np.float64)
    N = xi.size
    k = np.array([kx, ky, kz])
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    h = L / k
    K = int(kx * ky * kz)
    e = np.arange(K)
    eidx = [e % kx, (e // kx) % ky, e // (kx * ky)]
    t = (xi + 1.0) * 0.5
    X = np.empty((K, 3, N, N, N))
    # component d varies along xi_{d+1}; array axes are (xi3, xi2, xi1)
    shapes = {0: (1, 1, N), 1: (1, N, 1), 2: (N, 1, 1)}
    for d in range(3):
        base = lo[d] + (eidx[d][:, None] + t[None, :]) * h[d]          # [K, N]
        X[:, d] = base.reshape((K,) + shapes[d])
    if warp != 0.0:
        phi = warp_phases(seed) if phases is None else np.asarray(phases, dtype=np.float64)
        Y = X.copy()
        for i in range(3):
            prod = np.ones((K, N, N, N))
            for kk in range(3):
                prod = prod * np.sin(2.0 * math.pi * (X[:, kk] - lo[kk]) / L[kk] + phi[i, kk])
            Y[:, i] = X[:, i] + warp * h[i] * prod
        X = Y
    return X


def primitive_to_conserved(rho, u, p, gamma) -> np.ndarray:
    """(rho, u[3], p) -> (rho, rho u, rho E) with rho E = p/(gamma-1) + rho |u|^2 / 2."""
    rho = np.asarray(rho, dtype=np.float64)
    q = np.empty((rho.shape[0], 5) + rho.shape[1:])
    q[:, 0] = rho
    for d in range(3):
        q[:, 1 + d] = rho * u[d]
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return q


def taylor_green(x, Ma=0.1, gamma=1.4) -> np.ndarray:
    """Taylor-Green vortex initial state (Sec. 5.2): T = 1, density perturbation of order Ma^2."""
    R = gas_constant(Ma, gamma)
    x1, x2, x3 = x[:, 0], x[:, 1], x[:, 2]
    rho = 1.0 + gamma * Ma * Ma / 16.0 * (np.cos(2 * x1) + np.cos(2 * x2)) * (np.cos(2 * x3) + 2.0)
    u = [np.sin(x1) * np.cos(x2) * np.cos(x3), -np.cos(x1) * np.sin(x2) * np.cos(x3), np.zeros_like(x1)]
    T = np.ones_like(x1)
    return primitive_to_conserved(rho, u, rho * R * T, gamma)


def isentropic_vortex(x, Ma=0.5, gamma=1.4, beta=5.0, center=(0.0, 0.0, 0.0),
                      axis=(1.0, 1.0, 1.0), u_inf=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Isentropic vortex (Sec. 5.1.1, eq. iv_sol) about an arbitrary axis, plus a uniform drift."""
    R = gas_constant(Ma, gamma)
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    c = np.asarray(center, dtype=np.float64)
    d = np.stack([x[:, i] - c[i] for i in range(3)], axis=1)       # offset from centre
    along = sum(d[:, i] * a[i] for i in range(3))
    rvec = [d[:, i] - along * a[i] for i in range(3)]               # radial vector
    r2 = rvec[0] ** 2 + rvec[1] ** 2 + rvec[2] ** 2
    T = 1.0 - (gamma - 1.0) * Ma * Ma * beta * beta / (8.0 * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    # tangential unit direction a x r_hat times u_t = r beta/(2 pi) exp((1-r^2)/2)
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))         # u_t / r
    cr = [a[1] * rvec[2] - a[2] * rvec[1], a[2] * rvec[0] - a[0] * rvec[2], a[0] * rvec[1] - a[1] * rvec[0]]
    u = [u_inf[i] + amp * cr[i] for i in range(3)]
    return primitive_to_conserved(rho, u, rho * R * T, gamma)


def freestream(x, rho=1.0, u=(0.3, 0.2, 0.1), p=None, Ma=0.1, gamma=1.4) -> np.ndarray:
    """Uniform state; p defaults to 1/(gamma Ma^2)."""
    if p is None:
        p = 1.0 / (gamma * Ma * Ma)
    ones = np.ones_like(x[:, 0])
    return primitive_to_conserved(rho * ones, [u[0] * ones, u[1] * ones, u[2] * ones], p * ones, gamma)


def density_wave(x, amp=0.1, u=(1.0, 0.5, 0.25), wavenumber=(1.0, 1.0, 1.0), Ma=0.1, gamma=1.4):
    """rho = 1 + amp sin(k.x), constant u and p: an exact travelling solution of the Euler equations."""
    p = 1.0 / (gamma * Ma * Ma)
    ph = sum(wavenumber[i] * x[:, i] for i in range(3))
    rho = 1.0 + amp * np.sin(ph)
    ones = np.ones_like(rho)
    return primitive_to_conserved(rho, [u[0] * ones, u[1] * ones, u[2] * ones], p * ones, gamma)


def shear_wave(x, amp=1.0, Ma=0.1, gamma=1.4):
    """u1 = amp sin(x2), rho = T = 1 (uniform pressure)."""
    R = gas_constant(Ma, gamma)
    ones = np.ones_like(x[:, 0])
    zero = np.zeros_like(ones)
    return primitive_to_conserved(ones, [amp * np.sin(x[:, 1]), zero, zero], R * ones, gamma)


def temperature_wave(x, amp=0.1, Ma=0.1, gamma=1.4):
    """T = 1 + amp sin(x1), u = 0, uniform pressure p = R (so rho = 1/T)."""
    R = gas_constant(Ma, gamma)
    T = 1.0 + amp * np.sin(x[:, 0])
    zero = np.zeros_like(T)
    return primitive_to_conserved(1.0 / T, [zero, zero, zero], R * np.ones_like(T), gamma)


def perturb(q, seed=1234, rel=1e-3) -> np.ndarray:
    """Multiplicative seeded noise q*(1 + rel*n), n ~ N(0,1), indexed by node (not by coordinate)."""
    rng = np.random.default_rng(seed)
    return q * (1.0 + rel * rng.standard_normal(q.shape))


def random_direction(shape, seed=1234, scale=None) -> np.ndarray:
    """Seeded normal(0,1) test vector; optionally scaled per variable by scale[v]."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape)
    if scale is not None:
        v = v * np.asarray(scale).reshape((1, -1) + (1,) * (len(shape) - 2))
    return v


# Manufactured solution of the paper's viscous error-vs-cost study (Sec. 5.1, eq. mms and its table of
# constants) on [0, L]^3, L = 1.  Rows rho, u1, u2, u3, p; columns phi0, phi_x1, phi_x2, phi_x3,
# alpha_x1, alpha_x2, alpha_x3.  Readings: the table's "U_3^{x3}" in the u1 row is U_1^{x3}; the
# printed p_x3 = 2/3 is used as printed.  The dimensional values (velocity 800, pressure 1e5, rho 1)
# are scaled to this module's units: velocities by 800, pressures by 1e5/R, so that the reference
# Mach number per component is 800 / sqrt(1.4e5) = 2.138 (the paper's Ma ~ 2.14) and T = 1 at the
# reference state.
MMS_TABLE = (
    (1.0, 3.0 / 20.0, -1.0 / 10.0, 1.0 / 5.0, 1.0, 0.5, 1.0),
    (800.0, 50.0, -30.0, 50.0, 1.5, 0.6, 1.0),
    (800.0, -75.0, 40.0, 10.0, 0.5, 1.5, 1.5),
    (800.0, 15.0, -25.0, 20.0, 1.5, 0.5, 1.25),
    (1.0e5, 2.0e4, 5.0e4, 2.0 / 3.0, 1.0, 1.5, 1.0),
)
# trigonometric function of each term (0: sin, 1: cos), per row and direction (eq. mms)
MMS_KIND = ((0, 1, 0), (0, 1, 1), (1, 0, 0), (0, 0, 1), (0, 0, 1))
MMS_MA = 800.0 / math.sqrt(1.4e5)
MMS_RE = 4.0e6


def manufactured_primitives(x1, x2, x3, Ma=MMS_MA, gamma=1.4, L=1.0, sin=np.sin, cos=np.cos):
    """(rho, [u1, u2, u3], p) of the manufactured solution at points (x1, x2, x3) in this module's
    units.  sin/cos may be any elementwise functions (array libraries other than numpy)."""
    R = gas_constant(Ma, gamma)
    scale = (1.0, 1.0 / 800.0, 1.0 / 800.0, 1.0 / 800.0, R / 1.0e5)
    out = []
    for row, kind, sc in zip(MMS_TABLE, MMS_KIND, scale):
        v = row[0]
        for k, xk in enumerate((x1, x2, x3)):
            f = cos if kind[k] else sin
            v = v + row[1 + k] * f(row[4 + k] * math.pi * xk / L)
        out.append(sc * v)
    return out[0], out[1:4], out[4]


def manufactured(x, Ma=MMS_MA, gamma=1.4, L=1.0) -> np.ndarray:
    """Conserved state of the manufactured solution at node coordinates x [K, 3, N, N, N]."""
    rho, u, p = manufactured_primitives(x[:, 0], x[:, 1], x[:, 2], Ma, gamma, L)
    return primitive_to_conserved(rho, u, p, gamma)


def manufactured_table(Ma=MMS_MA, gamma=1.4):
    """MMS_TABLE in this module's units (the rows scaled as in manufactured_primitives), the layout
    esdc_mms_fields takes: 5 rows of (phi0, phi_x1, phi_x2, phi_x3, alpha_x1, alpha_x2, alpha_x3)."""
    R = gas_constant(Ma, gamma)
    scale = (1.0, 1.0 / 800.0, 1.0 / 800.0, 1.0 / 800.0, R / 1.0e5)
    return [[r[0] * sc, r[1] * sc, r[2] * sc, r[3] * sc, r[4], r[5], r[6]] for r, sc in zip(MMS_TABLE, scale)]
