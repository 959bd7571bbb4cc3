"""Plain FP64 CPU oracle of the entropy-stable collocation residual (arXiv 1911.10966).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports or calls this module; only the
tests, the smoke check and the CPU-baseline leg of the benchmark do.  It shares no code with the
CUDA path: it computes its own Gauss-Lobatto nodes, SBP operator and metric terms, evaluates the
volume term over ALL node pairs (including j = i) with the plain D matrix, and applies the
interface terms face by face.  Everything is float64 torch CPU tensors so that autograd gives the
oracle's own vector-Jacobian products.

Layouts: q [K, 5, N, N, N] (element, variable, xi3, xi2, xi1); metric Ja [K, 3, 3, N, N, N] with
Ja[:, l, m] = J dxi_l/dx_m; faces are numbered 2*l + side (side 0 = xi_l = -1, side 1 = +1).

Readings of points the paper leaves open (each one is repeated where it is used):
  * metric terms: conservative curl form of the degree-p interpolant of the mapping; it meets the
    discrete GCL (eq. discGCLconvection) exactly.  The same metrics serve the viscous terms.
    Alternatively the paper's optimized metrics (Sec. 3): analytic (cofactor) metrics of the
    interpolant on the faces and the Euclidean-nearest volume metrics that satisfy the discrete
    GCL with them; the interface terms then use the surface metrics.
  * entropy variables: w = [(gamma - s)/(gamma - 1) - rho|u|^2/(2p), rho u/p, -rho/p] with
    s = log(p rho^-gamma), i.e. S = -rho s/(gamma-1) (a positive rescaling of S = -rho s).
  * inviscid interface term: EC two-point flux plus local Lax-Friedrichs dissipation in the
    conserved variables, lambda = max over both sides of |u.n_J| + c |n_J|.
  * viscous interface terms: BR1 (central) lifting of the entropy-variable jump into the gradient
    and central viscous interface flux; interior penalty optional (default off).
Parity status: every function below is pinned by tests in tests/test_oracle_*.py.  The paper fixes
no constant of its interface terms (it defers them to its references), so the readings above are
pinned as readings: the local Lax-Friedrichs magnitude by the closed-form face sum of its entropy
production (lambda/2 (w_L - w_R).(q_L - q_R) over every interface node, computed from face states
alone), the BR1 viscous interface terms by the exact discrete identity sum P w.visc =
-sum P J g^T C g, the matrix dissipation against an eigendecomposition of the flux Jacobian and the
interior penalty by its linearity, conservation and entropy production.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

F64 = torch.float64


# --------------------------------------------------------------------------------------------
# 1D summation-by-parts operator on Legendre-Gauss-Lobatto nodes (Sec. 2, Definition 1)
# --------------------------------------------------------------------------------------------

def _legendre_and_derivative(p: int, x: float):
    """P_p(x) and P_p'(x) by the three-term recurrence."""
    if p == 0:
        return 1.0, 0.0
    pm1, pc = 1.0, x
    dm1, dc = 0.0, 1.0
    for k in range(1, p):
        pn = ((2 * k + 1) * x * pc - k * pm1) / (k + 1)
        dn = dm1 + (2 * k + 1) * pc           # P'_{k+1} = P'_{k-1} + (2k+1) P_k
        pm1, pc = pc, pn
        dm1, dc = dc, dn
    return pc, dc


def lgl_nodes_weights(p: int):
    """Gauss-Lobatto nodes: +-1 and the roots of P_p'; weights 2/(p(p+1) P_p(x_i)^2).

    Newton on q(x) = (1-x^2) P_p'(x), whose derivative is -p(p+1) P_p(x) by Legendre's equation.
    """
    if p < 1:
        raise ValueError("p >= 1")
    x = [math.cos(math.pi * i / p) for i in range(p + 1)]
    x = [-v for v in x]                     # ascending from -1 to +1
    for i in range(1, p):
        xi = x[i]
        for _ in range(100):
            P, dP = _legendre_and_derivative(p, xi)
            step = (1.0 - xi * xi) * dP / (-p * (p + 1) * P)
            xi -= step
            if abs(step) < 1e-17:
                break
        x[i] = xi
    x[0], x[p] = -1.0, 1.0
    w = [2.0 / (p * (p + 1) * _legendre_and_derivative(p, v)[0] ** 2) for v in x]
    return torch.tensor(x, dtype=F64), torch.tensor(w, dtype=F64)


@dataclass
class SBP:
    p: int
    xi: torch.Tensor     # [N]
    w: torch.Tensor      # [N]   diagonal of the norm P
    D: torch.Tensor      # [N,N] D = P^-1 Q
    Q: torch.Tensor
    E: torch.Tensor      # diag(-1, 0, ..., 0, 1)

    @property
    def N(self):
        return self.p + 1


def sbp_operator(p: int) -> SBP:
    """Collocation derivative by barycentric Lagrange differentiation (Definition 1, item 1)."""
    xi, w = lgl_nodes_weights(p)
    N = p + 1
    lam = torch.ones(N, dtype=F64)
    for j in range(N):
        for k in range(N):
            if k != j:
                lam[j] = lam[j] / (xi[j] - xi[k])
    D = torch.zeros(N, N, dtype=F64)
    for i in range(N):
        for j in range(N):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (xi[i] - xi[j])
        D[i, i] = -sum(D[i, j] for j in range(N) if j != i)
    Q = torch.diag(w) @ D
    E = torch.zeros(N, N, dtype=F64)
    E[0, 0], E[-1, -1] = -1.0, 1.0
    return SBP(p, xi, w, D, Q, E)


def dxi(u: torch.Tensor, l: int, D: torch.Tensor) -> torch.Tensor:
    """Apply D along reference direction l (0 -> xi1 = last axis) of the trailing three axes."""
    a = -1 - l
    ut = u.movedim(a, -1)
    return torch.einsum("ij,...j->...i", D, ut).movedim(-1, a)


def face(u: torch.Tensor, l: int, side: int) -> torch.Tensor:
    """Nodes of the face xi_l = -1 (side 0) or +1 (side 1); remaining axes keep their order."""
    N = u.shape[-1]
    return u.select(-1 - l, 0 if side == 0 else N - 1)


# --------------------------------------------------------------------------------------------
# Mesh geometry: Jacobian and metric terms (Sec. 3, eqs. GCL and discGCLconvection)
# --------------------------------------------------------------------------------------------

@dataclass
class Mesh:
    sbp: SBP
    x: torch.Tensor      # [K,3,N,N,N]
    J: torch.Tensor      # [K,N,N,N]
    Ja: torch.Tensor     # [K,3,3,N,N,N]
    nbr: torch.Tensor    # [K,6] long, face neighbours
    h_min: float
    # metrics the interface terms use at face nodes (the analytic surface metrics of the optimized
    # metrics, [K,3,3,N,N,N] of which only face values are read); None: the volume metrics Ja
    Ja_face: torch.Tensor | None = None


def metric_terms(x: torch.Tensor, D: torch.Tensor):
    """J = det(dx/dxi) and Ja[l][m] = J dxi_l/dx_m in conservative curl form.

    For physical component m with (m, m+1, m+2) cyclic: v_j = X_{m+2} dX_{m+1}/dxi_j and
    Ja[:, :, m] = -curl_xi(v).  Discrete derivatives in different directions commute, so
    sum_l D_l Ja[l][m] = 0 (the discrete GCL) holds to round-off.
    """
    # the curl form is invariant under translation of X; coordinates relative to each element's
    # first node keep the products X_l dX_m/dxi small and the round-off proportional to h, not |x|
    x = x - x[:, :, :1, :1, :1]
    dX = [[dxi(x[:, m], a, D) for a in range(3)] for m in range(3)]     # dX[m][a] = dx_m/dxi_a
    J = (dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1])
         - dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0])
         + dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]))
    K, _, N = x.shape[0], x.shape[1], x.shape[-1]
    Ja = torch.empty((K, 3, 3, N, N, N), dtype=F64)
    for m in range(3):
        mp1, mp2 = (m + 1) % 3, (m + 2) % 3
        v = [x[:, mp2] * dX[mp1][j] for j in range(3)]
        curl = [dxi(v[2], 1, D) - dxi(v[1], 2, D),
                dxi(v[0], 2, D) - dxi(v[2], 0, D),
                dxi(v[1], 0, D) - dxi(v[0], 1, D)]
        for l in range(3):
            Ja[:, l, m] = -curl[l]
    return J, Ja


def cofactor_metrics(x: torch.Tensor, D: torch.Tensor) -> torch.Tensor:
    """Ja[l][m] = (dx/dxi_a x dx/dxi_b)_m with (l, a, b) cyclic: the rows of the cofactor matrix of
    dx/dxi, i.e. the analytic metric terms of the degree-p interpolant of the mapping at the nodes (D
    differentiates the interpolant exactly).  On a face xi_l = +-1 row l involves only derivatives
    along the face, so both elements sharing the face see the same values (to round-off)."""
    x = x - x[:, :, :1, :1, :1]
    dX = [[dxi(x[:, m], a, D) for a in range(3)] for m in range(3)]     # dX[m][a] = dx_m/dxi_a
    K, N = x.shape[0], x.shape[-1]
    Ja = torch.empty((K, 3, 3, N, N, N), dtype=F64)
    for l in range(3):
        a, b = (l + 1) % 3, (l + 2) % 3
        for m in range(3):
            m1, m2 = (m + 1) % 3, (m + 2) % 3
            Ja[:, l, m] = dX[m1][a] * dX[m2][b] - dX[m2][a] * dX[m1][b]
    return Ja


def sbp_3d(sbp: SBP):
    """Dense tensor-product operators Q_l = P (x) P (x) Q and E_l = P (x) P (x) E along xi_l (Sec. 2),
    N^3 x N^3 with the nodes numbered xi1 fastest."""
    P = torch.diag(sbp.w)
    k3 = lambda A3, A2, A1: torch.kron(torch.kron(A3, A2), A1)
    Ql = [k3(P, P, sbp.Q), k3(P, sbp.Q, P), k3(sbp.Q, P, P)]
    El = [k3(P, P, sbp.E), k3(P, sbp.E, P), k3(sbp.E, P, P)]
    return Ql, El


def optimized_metrics(x: torch.Tensor, sbp: SBP):
    """The paper's optimized metrics (Sec. 3): surface metrics analytic (the cofactor metrics t of
    the interpolated mapping, read at face nodes) and, for each physical direction m, the volume
    metrics a_m = (a_1m, a_2m, a_3m) nearest to t_m in the Euclidean norm among those that satisfy
    the discrete GCL with those surface metrics, sum_l Q_l^T a_lm = sum_l E_l t_lm (the condition under
    which the skew-symmetric flux differencing with the surface metrics in the interface terms keeps
    a uniform flow).  With M = [Q_1^T Q_2^T Q_3^T] (N^3 x 3 N^3, rank N^3 - 1) the minimiser is
    a_m = t_m + M^+ (b_m - M t_m), M^+ the Moore-Penrose pseudo-inverse.  Returns (a, t)."""
    t = cofactor_metrics(x, sbp.D)
    Ql, El = sbp_3d(sbp)
    M = torch.cat([Q.T for Q in Ql], dim=1)
    Mp = torch.linalg.pinv(M)
    K, N3 = t.shape[0], sbp.N ** 3
    a = torch.empty_like(t)
    for m in range(3):
        tv = t[:, :, m].reshape(K, 3 * N3)
        b = sum(t[:, l, m].reshape(K, N3) @ El[l] for l in range(3))
        a[:, :, m] = (tv + (b - tv @ M.T) @ Mp.T).reshape(t[:, :, m].shape)
    return a, t


def box_neighbours(kx: int, ky: int, kz: int, bounded=(False, False, False)) -> torch.Tensor:
    """Face neighbours of a structured box, element e = ex + kx*(ey + ky*ez): periodic in every
    direction except those flagged in `bounded`, whose outer faces get neighbour -1 (a boundary)."""
    K = kx * ky * kz
    e = torch.arange(K)
    ex, ey, ez = e % kx, (e // kx) % ky, e // (kx * ky)
    idx = lambda a, b, c: (a % kx) + kx * ((b % ky) + ky * (c % kz))
    nb = torch.stack([idx(ex - 1, ey, ez), idx(ex + 1, ey, ez),
                      idx(ex, ey - 1, ez), idx(ex, ey + 1, ez),
                      idx(ex, ey, ez - 1), idx(ex, ey, ez + 1)], dim=1)
    for l, (c, k) in enumerate(((ex, kx), (ey, ky), (ez, kz))):
        if bounded[l]:
            nb[:, 2 * l] = torch.where(c == 0, -1, nb[:, 2 * l])
            nb[:, 2 * l + 1] = torch.where(c == k - 1, -1, nb[:, 2 * l + 1])
    return nb


def smallest_edge(x: torch.Tensor) -> float:
    """Smallest distance between adjacent element corners along the 12 element edges."""
    N = x.shape[-1]
    c = lambda a, b, d: x[:, :, a, b, d]        # corner (xi3 idx, xi2 idx, xi1 idx)
    e = [0, N - 1]
    lens = []
    for i in e:
        for j in e:
            lens.append((c(i, j, 0) - c(i, j, N - 1)).norm(dim=1))
            lens.append((c(i, 0, j) - c(i, N - 1, j)).norm(dim=1))
            lens.append((c(0, i, j) - c(N - 1, i, j)).norm(dim=1))
    return float(torch.stack(lens).min())


def _metrics(x: torch.Tensor, sbp: SBP, metrics: str):
    J, Ja = metric_terms(x, sbp.D)
    if metrics == "curl":
        return J, Ja, None
    if metrics == "optimized":
        a, t = optimized_metrics(x, sbp)
        return J, a, t
    raise ValueError(metrics)


def make_mesh(p: int, x, kx: int, ky: int, kz: int, bounded=(False, False, False), metrics: str = "curl") -> Mesh:
    """metrics: "curl" (conservative curl form everywhere) or "optimized" (the paper's optimized
    volume metrics, analytic surface metrics in the interface terms)."""
    sbp = sbp_operator(p)
    x = torch.as_tensor(x, dtype=F64)
    J, Ja, Jf = _metrics(x, sbp, metrics)
    return Mesh(sbp, x, J, Ja, box_neighbours(kx, ky, kz, bounded), smallest_edge(x), Jf)


def nbr_face(fn, q: torch.Tensor, mesh: Mesh, E: torch.Tensor, l: int, side: int, q_ext=None) -> torch.Tensor:
    """fn(state) on the neighbour side of face (l, side) of elements E, as seen from E's face nodes.
    On a boundary face (neighbour -1) the neighbour side is the exterior state q_ext at E's own face
    nodes (the Dirichlet data of the boundary SAT)."""
    nb = mesh.nbr[E, 2 * l + side]
    vals = face(fn(q[nb.clamp(min=0)]), l, 1 - side)
    if bool((nb < 0).any()):
        if q_ext is None:
            raise ValueError("boundary faces need an exterior state")
        ext = face(fn(torch.as_tensor(q_ext, dtype=F64)[E]), l, side)
        shape = (-1,) + (1,) * (vals.dim() - 1)
        vals = torch.where((nb < 0).view(shape), ext, vals)
    return vals


def make_submesh(p: int, x, nbr: torch.Tensor, elems, metrics: str = "curl"):
    """The mesh restricted to `elems` and the two rings of face neighbours around them, which is
    all the residual on `elems` reads (the viscous terms need the neighbours' lifted gradients,
    which need their neighbours' face states); metric terms are element-local, so they are the
    same as on the full mesh.  Returns (submesh, closure element ids, rows of `elems`)."""
    E = torch.as_tensor(elems, dtype=torch.long)
    E1 = torch.unique(torch.cat([E, nbr[E].reshape(-1)]))
    E2 = torch.unique(torch.cat([E1, nbr[E1].reshape(-1)]))
    pos = torch.full((nbr.shape[0],), -1, dtype=torch.long)
    pos[E2] = torch.arange(E2.numel())
    sub_nbr = pos[nbr[E2]]
    own = torch.arange(E2.numel()).unsqueeze(1).expand_as(sub_nbr)
    sub_nbr = torch.where(sub_nbr < 0, own, sub_nbr)   # outer ring: links never followed for elems
    sbp = sbp_operator(p)
    xs = torch.as_tensor(x[E2.numpy()], dtype=F64)
    J, Ja, Jf = _metrics(xs, sbp, metrics)
    return Mesh(sbp, xs, J, Ja, sub_nbr, smallest_edge(xs), Jf), E2, pos[E]


# --------------------------------------------------------------------------------------------
# Gas physics (Sec. 4: eq. ns_iflux, constitutive relations, entropy, eq. Fv, eq. tau)
# --------------------------------------------------------------------------------------------

@dataclass
class Gas:
    gamma: float = 1.4
    R: float = 1.0
    mu: float = 0.0
    Pr: float = 0.72

    @property
    def cp(self):
        return self.gamma * self.R / (self.gamma - 1.0)

    @property
    def kappa(self):
        return self.mu * self.cp / self.Pr

    @staticmethod
    def from_mach(Ma, Re=0.0, gamma=1.4, Pr=0.72):
        """rho_inf = T_inf = 1, R = 1/(gamma Ma^2), mu = 1/Re (Re <= 0: inviscid)."""
        return Gas(gamma, 1.0 / (gamma * Ma * Ma), (1.0 / Re) if Re > 0 else 0.0, Pr)


def primitives(q: torch.Tensor, gas: Gas):
    """rho, u (list of 3), p = (gamma-1)(rho E - rho|u|^2/2), T = p/(rho R); variable axis is 1."""
    rho = q[:, 0]
    u = [q[:, 1 + d] / rho for d in range(3)]
    p = (gas.gamma - 1.0) * (q[:, 4] - 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    return rho, u, p, p / (rho * gas.R)


def entropy_function(q: torch.Tensor, gas: Gas) -> torch.Tensor:
    """S = -rho s/(gamma-1) with s = log(p) - gamma log(rho)."""
    rho, _, p, _ = primitives(q, gas)
    return -rho * (torch.log(p) - gas.gamma * torch.log(rho)) / (gas.gamma - 1.0)


def entropy_variables(q: torch.Tensor, gas: Gas) -> torch.Tensor:
    """w = dS/dq = [(gamma - s)/(gamma-1) - rho|u|^2/(2p), rho u/p, -rho/p]."""
    rho, u, p, _ = primitives(q, gas)
    s = torch.log(p) - gas.gamma * torch.log(rho)
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    return torch.stack([(gas.gamma - s) / (gas.gamma - 1.0) - rho * usq / (2.0 * p),
                        rho * u[0] / p, rho * u[1] / p, rho * u[2] / p, -rho / p], dim=1)


def euler_flux_n(q: torch.Tensor, n, gas: Gas) -> torch.Tensor:
    """sum_m n_m F_m(q) with F_m from eq. ns_iflux; n is a list of 3 tensors broadcastable to q[:,0]."""
    rho, u, p, _ = primitives(q, gas)
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    H = (q[:, 4] + p) / rho
    return torch.stack([rho * un, rho * un * u[0] + p * n[0], rho * un * u[1] + p * n[1],
                        rho * un * u[2] + p * n[2], rho * un * H], dim=1)


def _phi(x):
    """x/log(1+x), continuous at x = 0 with value 1."""
    zero = x == 0
    xs = torch.where(zero, torch.ones_like(x), x)
    return torch.where(zero, torch.ones_like(x), xs / torch.log1p(xs))


def _dphi(x):
    """d/dx [x/log(1+x)]: Gregory-coefficient series for |x| < 1e-3, closed form otherwise."""
    small = x.abs() < 1e-3
    xs = torch.where(small, torch.ones_like(x), x)
    lg = torch.log1p(xs)
    closed = (lg - xs / (1.0 + xs)) / (lg * lg)
    series = 0.5 + x * (-1.0 / 6.0 + x * (1.0 / 8.0 + x * (-19.0 / 180.0 + x * (3.0 / 32.0))))
    return torch.where(small, series, closed)


class _LogMean(torch.autograd.Function):
    """Logarithmic mean (a - b)/(log a - log b) written as b*phi(a/b - 1)."""

    @staticmethod
    def forward(ctx, a, b):
        x = (a - b) / b
        ctx.save_for_backward(a, b, x)
        return b * _phi(x)

    @staticmethod
    def backward(ctx, g):
        a, b, x = ctx.saved_tensors
        d = _dphi(x)
        return g * d, g * (_phi(x) - (a / b) * d)


def logmean(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """The logarithmic average of Sec. 4 (definition under the ES-C flux)."""
    return _LogMean.apply(a, b)


def ec_flux_n(qa: torch.Tensor, qb: torch.Tensor, n, gas: Gas) -> torch.Tensor:
    """Chandrashekar two-point entropy-conservative flux contracted with n (ES-C flux, Sec. 4).

    f1 = rho_ln ubar_n, f_{2..4} = f1 ubar + p_tilde n,
    f5 = f1 (1/(2(gamma-1) beta_ln) - avg(|u|^2)/2) + ubar . f_{2..4},
    beta = 1/(2RT), p_tilde = R rho_avg T_a T_b / T_avg; avg(|u|^2) is the arithmetic mean of |u|^2.
    """
    ra, ua, pa, Ta = primitives(qa, gas)
    rb, ub, pb, Tb = primitives(qb, gas)
    ba, bb = 1.0 / (2.0 * gas.R * Ta), 1.0 / (2.0 * gas.R * Tb)
    rho_ln, beta_ln = logmean(ra, rb), logmean(ba, bb)
    ubar = [0.5 * (ua[d] + ub[d]) for d in range(3)]
    ubar_n = ubar[0] * n[0] + ubar[1] * n[1] + ubar[2] * n[2]
    p_t = gas.R * 0.5 * (ra + rb) * Ta * Tb / (0.5 * (Ta + Tb))
    usq_avg = 0.5 * ((ua[0] ** 2 + ua[1] ** 2 + ua[2] ** 2) + (ub[0] ** 2 + ub[1] ** 2 + ub[2] ** 2))
    f1 = rho_ln * ubar_n
    fm = [f1 * ubar[d] + p_t * n[d] for d in range(3)]
    f5 = f1 * (1.0 / (2.0 * (gas.gamma - 1.0) * beta_ln) - 0.5 * usq_avg) \
        + ubar[0] * fm[0] + ubar[1] * fm[1] + ubar[2] * fm[2]
    return torch.stack([f1, fm[0], fm[1], fm[2], f5], dim=1)


def kg_flux_n(qa: torch.Tensor, qb: torch.Tensor, n, gas: Gas) -> torch.Tensor:
    """Kennedy-Gruber two-point flux contracted with n (the SF-KG variant, Sec. 4):
    f1 = rho_bar ubar_n, f_{2..4} = f1 ubar + p_bar n, f5 = f1 e_bar + p_bar ubar_n, with arithmetic
    means of rho, u, p and the specific total energy e = rho E / rho."""
    ra, ua, pa, _ = primitives(qa, gas)
    rb, ub, pb, _ = primitives(qb, gas)
    rbar = 0.5 * (ra + rb)
    ubar = [0.5 * (ua[d] + ub[d]) for d in range(3)]
    pbar = 0.5 * (pa + pb)
    ebar = 0.5 * (qa[:, 4] / ra + qb[:, 4] / rb)
    ubar_n = ubar[0] * n[0] + ubar[1] * n[1] + ubar[2] * n[2]
    f1 = rbar * ubar_n
    return torch.stack([f1, f1 * ubar[0] + pbar * n[0], f1 * ubar[1] + pbar * n[1], f1 * ubar[2] + pbar * n[2],
                        f1 * ebar + pbar * ubar_n], dim=1)


def central_flux_n(qa: torch.Tensor, qb: torch.Tensor, n, gas: Gas) -> torch.Tensor:
    """Arithmetic mean of the two Euler fluxes contracted with n: the interface flux read for the DC
    variant, whose volume term uses no two-point flux."""
    return 0.5 * (euler_flux_n(qa, n, gas) + euler_flux_n(qb, n, gas))


def dq_dw(rho, u, p, gas: Gas) -> torch.Tensor:
    """The symmetric matrix dq/dw (inverse Hessian of the entropy function in conserved variables)
    at the state (rho, u, p), shape [..., 5, 5]: rows (rho, rho u, rho E) differentiated by w."""
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    H = (E + p) / rho
    a2 = gas.gamma * p / rho
    m = [rho * u[d] for d in range(3)]
    rows = [[rho, m[0], m[1], m[2], E]]
    for i in range(3):
        rows.append([m[i]] + [m[i] * u[j] + (p if i == j else torch.zeros_like(p)) for j in range(3)]
                    + [rho * H * u[i]])
    rows.append([E, rho * H * u[0], rho * H * u[1], rho * H * u[2], rho * H * H - a2 * p / (gas.gamma - 1.0)])
    return torch.stack([torch.stack(r, dim=-1) for r in rows], dim=-2)


def matrix_dissipation(rho, u, p, n, gas: Gas) -> torch.Tensor:
    """Roe-type entropy-stable dissipation matrix D = R |Lambda| R^T for the direction n (not
    normalised) at the state (rho, u, p), shape [..., 5, 5].  R are the right eigenvectors of the
    flux Jacobian in n scaled so that R R^T = dq/dw (Barth's scaling); the three eigenvalues u.n share
    one eigenspace, so D = |u.n| dq/dw + s (|u.n - a|n|| - |u.n|) r1 r1^T + s (|u.n + a|n|| - |u.n|)
    r5 r5^T with the acoustic eigenvectors r1,5 = (1, u -+ a nhat, H -+ a u.nhat) and s = rho/(2 gamma)."""
    nn = torch.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    nh = [n[d] / nn for d in range(3)]
    a = torch.sqrt(gas.gamma * p / rho)
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    H = a * a / (gas.gamma - 1.0) + 0.5 * usq
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    unh = un / nn
    l1, l2, l5 = (un - a * nn).abs(), un.abs(), (un + a * nn).abs()
    one = torch.ones_like(rho)
    r1 = torch.stack([one, u[0] - a * nh[0], u[1] - a * nh[1], u[2] - a * nh[2], H - a * unh], dim=-1)
    r5 = torch.stack([one, u[0] + a * nh[0], u[1] + a * nh[1], u[2] + a * nh[2], H + a * unh], dim=-1)
    sc = rho / (2.0 * gas.gamma)
    outer = lambda r: r.unsqueeze(-1) * r.unsqueeze(-2)
    return (l2[..., None, None] * dq_dw(rho, u, p, gas) + (sc * (l1 - l2))[..., None, None] * outer(r1)
            + (sc * (l5 - l2))[..., None, None] * outer(r5))


def sound_speed(q: torch.Tensor, gas: Gas) -> torch.Tensor:
    rho, _, p, _ = primitives(q, gas)
    return torch.sqrt(gas.gamma * p / rho)


def viscous_flux(q: torch.Tensor, g: torch.Tensor, gas: Gas) -> torch.Tensor:
    """F^V_m (eq. Fv, eq. tau) from the physical entropy-variable gradient g[:, m, v] = dw_v/dx_m.

    u_k = -w_{k+1}/w_5 and T = -1/(R w_5), so du_k = -dw_{k+1}/w_5 + w_{k+1} dw_5/w_5^2 and
    dT = dw_5/(R w_5^2).  Returns [K, 3 (m), 5, ...].
    """
    rho, u, p, T = primitives(q, gas)
    w5 = -rho / p
    wk = [rho * u[k] / p for k in range(3)]
    du = [[-g[:, m, 1 + k] / w5 + wk[k] * g[:, m, 4] / (w5 * w5) for m in range(3)] for k in range(3)]
    dT = [g[:, m, 4] / (gas.R * w5 * w5) for m in range(3)]         # du[k][m] = du_k/dx_m
    div = du[0][0] + du[1][1] + du[2][2]
    tau = [[gas.mu * (du[i][j] + du[j][i] - (2.0 / 3.0 if i == j else 0.0) * div) for j in range(3)]
           for i in range(3)]
    out = []
    for m in range(3):
        zero = torch.zeros_like(rho)
        energy = tau[0][m] * u[0] + tau[1][m] * u[1] + tau[2][m] * u[2] + gas.kappa * dT[m]
        out.append(torch.stack([zero, tau[0][m], tau[1][m], tau[2][m], energy], dim=1))
    return torch.stack(out, dim=1)


# --------------------------------------------------------------------------------------------
# Semi-discrete residual (eq. discEL, eq. MacroForm, eq. NSL)
# --------------------------------------------------------------------------------------------

def _on_face(out: torch.Tensor, val: torch.Tensor, l: int, side: int) -> torch.Tensor:
    """out + (val placed on face (l, side)); works under autograd."""
    N = out.shape[-1]
    shape = [1] * out.dim()
    shape[out.dim() - 1 - l] = N
    onehot = torch.zeros(shape, dtype=out.dtype)
    onehot.view(-1)[0 if side == 0 else N - 1] = 1.0
    return out + onehot * val.unsqueeze(out.dim() - 1 - l)


def volume_term(q: torch.Tensor, Ja: torch.Tensor, sbp: SBP, gas: Gas, flux=None) -> torch.Tensor:
    """-sum_l sum_j 2 D_l(i,j) f(q_i, q_j; (Ja_l(i) + Ja_l(j))/2): the Hadamard flux differencing
    of eq. discEL (with A_lm on both sides of D_l), over every pair j of the xi_l line through i."""
    flux = flux or ec_flux_n
    out = torch.zeros_like(q)
    for l in range(3):
        a = -1 - l
        qt = q.movedim(a, -1)
        nt = Ja[:, l].movedim(a, -1)
        qi, qj = qt.unsqueeze(-1), qt.unsqueeze(-2)
        nbar = [0.5 * (nt[:, m].unsqueeze(-1) + nt[:, m].unsqueeze(-2)) for m in range(3)]
        F = flux(qi, qj, nbar, gas)
        out = out + (-2.0 * torch.einsum("ij,...ij->...i", sbp.D, F)).movedim(-1, a)
    return out


def dc_volume_term(q: torch.Tensor, Ja: torch.Tensor, sbp: SBP, gas: Gas) -> torch.Tensor:
    """-sum_l D_l Ftilde_l, Ftilde_l = sum_m Ja_lm F_m(q) at each node: the standard collocation (DC)
    divergence of the inviscid flux (Sec. 4), D applied to the nodal contravariant fluxes."""
    out = torch.zeros_like(q)
    for l in range(3):
        Ft = euler_flux_n(q, [Ja[:, l, m] for m in range(3)], gas)
        out = out - dxi(Ft, l, sbp.D)
    return out


def inviscid_sat(q: torch.Tensor, mesh: Mesh, gas: Gas, E: torch.Tensor, dissipation=True,
                 flux=None, q_ext=None) -> torch.Tensor:
    """SAT^(I) on elements E at every face node: -(1/P_ii) E_ii [f*(own, nbr).n_S - f(own).n_J] minus
    (1/P_ii) lambda/2 (q_own - q_nbr) when dissipation is True (local Lax-Friedrichs reading), or
    minus (1/P_ii) D (w_own - w_nbr)/2 with the Roe-type matrix D when dissipation == "matrix".  n_J is
    the volume metric at the face node, n_S the surface metric (mesh.Ja_face; n_J when it is None);
    lambda and D are taken with n_S."""
    flux = flux or ec_flux_n
    sbp = mesh.sbp
    qE = q[E]
    out = torch.zeros_like(qE)
    wend = float(sbp.w[0])
    for l in range(3):
        for side in (0, 1):
            f = 2 * l + side
            qo = face(qE, l, side)
            qn = nbr_face(lambda x: x, q, mesh, E, l, side, q_ext)
            nJ = face(mesh.Ja[E, l], l, side)
            nv = [nJ[:, m] for m in range(3)]
            n = nv if mesh.Ja_face is None else [face(mesh.Ja_face[E, l], l, side)[:, m] for m in range(3)]
            sgn = -1.0 if side == 0 else 1.0
            # the own flux takes the volume metric (it is the E part of the volume term moved to the
            # face); the two-point flux and the dissipation take the surface metric
            val = -sgn * (flux(qo, qn, n, gas) - euler_flux_n(qo, nv, gas))
            if dissipation == "matrix":
                # reading: D at the averaged state (rho_ln, ubar, p = rho_bar/(2 beta_bar)) applied to
                # the jump of the entropy variables
                ro, uo, po, To = primitives(qo, gas)
                rn, un_, pn, Tn = primitives(qn, gas)
                bo, bn = 1.0 / (2.0 * gas.R * To), 1.0 / (2.0 * gas.R * Tn)
                rh = logmean(ro, rn)
                uh = [0.5 * (uo[d] + un_[d]) for d in range(3)]
                ph = 0.5 * (ro + rn) / (bo + bn)
                Dm = matrix_dissipation(rh, uh, ph, n, gas)
                jw = entropy_variables(qo, gas) - entropy_variables(qn, gas)
                val = val - 0.5 * torch.einsum("k...ij,kj...->ki...", Dm, jw)
            elif dissipation:
                _, uo, _, _ = primitives(qo, gas)
                _, un_, _, _ = primitives(qn, gas)
                nn = torch.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
                lo = (uo[0] * n[0] + uo[1] * n[1] + uo[2] * n[2]).abs() + sound_speed(qo, gas) * nn
                ln = (un_[0] * n[0] + un_[1] * n[1] + un_[2] * n[2]).abs() + sound_speed(qn, gas) * nn
                lam = torch.maximum(lo, ln)
                val = val - 0.5 * lam.unsqueeze(1) * (qo - qn)
            out = _on_face(out, val / wend, l, side)
    return out


def entropy_gradient(q: torch.Tensor, mesh: Mesh, gas: Gas, E: torch.Tensor, q_ext=None) -> torch.Tensor:
    """theta_a = D_a w + SAT^theta (eq. NSL), with the BR1 lift (1/P_ii) E_ii (w_nbr - w_own)/2 on
    the faces normal to a.  Returns [|E|, 3 (a), 5, N, N, N]."""
    sbp = mesh.sbp
    wE = entropy_variables(q[E], gas)
    wend = float(sbp.w[0])
    th = []
    for a in range(3):
        t = dxi(wE, a, sbp.D)
        for side in (0, 1):
            wo = face(wE, a, side)
            wn = nbr_face(lambda x: entropy_variables(x, gas), q, mesh, E, a, side, q_ext)
            sgn = -1.0 if side == 0 else 1.0
            t = _on_face(t, sgn * 0.5 * (wn - wo) / wend, a, side)
        th.append(t)
    return torch.stack(th, dim=1)


def physical_gradient(theta: torch.Tensor, J: torch.Tensor, Ja: torch.Tensor) -> torch.Tensor:
    """g[:, m] = (1/J) sum_a Ja[a][m] theta_a (chain rule, Sec. 3)."""
    return torch.stack([sum(Ja[:, a, m].unsqueeze(1) * theta[:, a] for a in range(3)) / J.unsqueeze(1)
                        for m in range(3)], dim=1)


def contravariant_viscous_flux(q: torch.Tensor, mesh: Mesh, gas: Gas, E: torch.Tensor, q_ext=None):
    """Ftilde_l = sum_m Ja[l][m] F^V_m = sum_a Chat_la theta_a (eq. Chatij): [|E|, 3, 5, N, N, N].
    Also returns the physical gradient g used to build it."""
    th = entropy_gradient(q, mesh, gas, E, q_ext)
    g = physical_gradient(th, mesh.J[E], mesh.Ja[E])
    FV = viscous_flux(q[E], g, gas)
    Ja = mesh.Ja[E]
    Ft = torch.stack([sum(Ja[:, l, m].unsqueeze(1) * FV[:, m] for m in range(3)) for l in range(3)], dim=1)
    return Ft, g


def viscous_term(q: torch.Tensor, mesh: Mesh, gas: Gas, E: torch.Tensor, q_ext=None) -> torch.Tensor:
    """sum_l D_l Ftilde_l + SAT^(V), SAT^(V) = (1/P_ii) E_ii (Ftilde_l,nbr - Ftilde_l,own)/2 on the
    xi_l faces (eq. MacroForm / eq. NSL with the BR1 reading; interior penalty off)."""
    sbp = mesh.sbp
    K = q.shape[0]
    E1 = torch.unique(torch.cat([E, mesh.nbr[E].reshape(-1)]))
    E1 = E1[E1 >= 0]
    pos = torch.full((K,), -1, dtype=torch.long)
    pos[E1] = torch.arange(E1.numel())
    Ft, _ = contravariant_viscous_flux(q, mesh, gas, E1, q_ext)
    own = Ft[pos[E]]
    wend = float(sbp.w[0])
    out = sum(dxi(own[:, l], l, sbp.D) for l in range(3))
    for l in range(3):
        for side in (0, 1):
            fo = face(own[:, l], l, side)
            nb = mesh.nbr[E, 2 * l + side]
            fn = face(Ft[pos[nb.clamp(min=0)], l], l, 1 - side)
            # boundary faces (reading): the exterior viscous flux is the interior one, no SAT^(V)
            fn = torch.where((nb < 0).view((-1,) + (1,) * (fn.dim() - 1)), fo, fn)
            sgn = -1.0 if side == 0 else 1.0
            out = _on_face(out, sgn * 0.5 * (fn - fo) / wend, l, side)
    return out



def interior_penalty(q: torch.Tensor, mesh: Mesh, gas: Gas, E: torch.Tensor, coef: float,
                     q_ext=None) -> torch.Tensor:
    """Interior-penalty term IP (eq. NSL; its constants are in the paper's references).  Reading: at
    every face node -(1/P_ii) coef mu |n_J| / h dq/dw (w_own - w_nbr), with dq/dw at the averaged state
    of the matrix dissipation and h = (J_own + J_nbr)/|n_J| (the sum of the two elements' normal
    half-widths), symmetric in the two sides so that the term conserves and produces entropy."""
    sbp = mesh.sbp
    qE = q[E]
    out = torch.zeros_like(qE)
    wend = float(sbp.w[0])
    for l in range(3):
        for side in (0, 1):
            f = 2 * l + side
            qo = face(qE, l, side)
            qn = nbr_face(lambda x: x, q, mesh, E, l, side, q_ext)
            nJ = face((mesh.Ja if mesh.Ja_face is None else mesh.Ja_face)[E, l], l, side)
            nn = torch.sqrt(nJ[:, 0] ** 2 + nJ[:, 1] ** 2 + nJ[:, 2] ** 2)
            # on a boundary face the exterior Jacobian is read as the interior one
            Jo = face(mesh.J[E].unsqueeze(1), l, side)[:, 0]
            Jn = nbr_face(lambda x: x, mesh.J.unsqueeze(1), mesh, E, l, side, mesh.J.unsqueeze(1))[:, 0]
            h = (Jo + Jn) / nn
            ro, uo, po, To = primitives(qo, gas)
            rn, un_, pn, Tn = primitives(qn, gas)
            bo, bn = 1.0 / (2.0 * gas.R * To), 1.0 / (2.0 * gas.R * Tn)
            M = dq_dw(logmean(ro, rn), [0.5 * (uo[d] + un_[d]) for d in range(3)], 0.5 * (ro + rn) / (bo + bn), gas)
            jw = entropy_variables(qo, gas) - entropy_variables(qn, gas)
            val = -(coef * gas.mu * nn / h).unsqueeze(1) * torch.einsum("k...ij,kj...->ki...", M, jw)
            out = _on_face(out, val / wend, l, side)
    return out


def manufactured_source(prim_fn, x, gas: Gas) -> torch.Tensor:
    """Source of the method of manufactured solutions (Sec. 5.1): S = div(F^I - F^V) of the exact
    field, so that dq/dt = R(q) + S is steady at the exact solution.  prim_fn(x1, x2, x3) returns
    (rho, [u1, u2, u3], p) as differentiable torch functions of the coordinates; the derivatives are
    taken by autograd (first derivatives for the entropy-variable gradient of F^V, second for the
    divergence).  x: [K, 3, N, N, N]; returns [K, 5, N, N, N]."""
    x = torch.as_tensor(x, dtype=F64)
    shape = x[:, 0].shape
    xs = [x[:, d].reshape(-1).clone().requires_grad_(True) for d in range(3)]
    rho, u, p = prim_fn(*xs)
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    q = torch.stack([rho, rho * u[0], rho * u[1], rho * u[2], E], dim=1)
    ones = torch.ones_like(rho)
    zero = torch.zeros_like(rho)
    Fi = torch.stack([euler_flux_n(q, [ones if m == d else zero for d in range(3)], gas) for m in range(3)], dim=1)
    w = entropy_variables(q, gas)
    g = torch.zeros(q.shape[0], 3, 5, dtype=F64)
    for v in range(5):
        gv = torch.autograd.grad(w[:, v].sum(), xs, create_graph=True)
        for m in range(3):
            g[:, m, v] = gv[m]
    F = Fi - viscous_flux(q, g, gas)                      # [M, 3 (m), 5]
    S = torch.zeros(q.shape[0], 5, dtype=F64)
    for v in range(5):
        for m in range(3):
            S[:, v] += torch.autograd.grad(F[:, m, v].sum(), xs[m], retain_graph=True)[0]
    return S.detach().reshape(shape[0], *shape[1:], 5).movedim(-1, 1).contiguous()

SCHEMES = ("esc", "kg", "dc")


def rhs(q, mesh: Mesh, gas: Gas, dissipation=True, elems=None, flux=None, scheme="esc",
        ip_coef: float = 0.0, q_ext=None, source=None) -> torch.Tensor:
    """dq/dt = J^-1 [-volume + SAT^(I) + viscous + SAT^(V)] on elements `elems` (default all).
    scheme: "esc" (Chandrashekar two-point flux, the paper's ES-C), "kg" (Kennedy-Gruber two-point
    flux, SF-KG) or "dc" (nodal fluxes differentiated by D, with the central interface flux).
    ip_coef > 0 adds the interior-penalty term (viscous runs only).  On a mesh with boundary faces,
    q_ext (same layout as q) holds the exterior (Dirichlet) state read at the boundary face nodes; a
    source (same layout) is added to dq/dt."""
    q = torch.as_tensor(q, dtype=F64)
    K = q.shape[0]
    E = torch.arange(K) if elems is None else torch.as_tensor(elems, dtype=torch.long)
    if scheme == "dc":
        r = dc_volume_term(q[E], mesh.Ja[E], mesh.sbp, gas) + inviscid_sat(q, mesh, gas, E, dissipation,
                                                                           central_flux_n, q_ext)
    else:
        if scheme == "kg":
            flux = kg_flux_n
        elif scheme != "esc":
            raise ValueError(scheme)
        r = volume_term(q[E], mesh.Ja[E], mesh.sbp, gas, flux) + inviscid_sat(q, mesh, gas, E, dissipation, flux,
                                                                             q_ext)
    if gas.mu > 0.0:
        r = r + viscous_term(q, mesh, gas, E, q_ext)
        if ip_coef > 0.0:
            r = r + interior_penalty(q, mesh, gas, E, ip_coef, q_ext)
    r = r / mesh.J[E].unsqueeze(1)
    if source is not None:
        r = r + torch.as_tensor(source, dtype=F64)[E]
    return r


# --------------------------------------------------------------------------------------------
# Time integration: Dormand-Prince 5(4) explicit Runge-Kutta, fixed step (Sec. 5)
# --------------------------------------------------------------------------------------------

DP5_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
]
DP5_B = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]
DP5_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0]


def rk_step(q, f, dt: float, nsteps: int = 1):
    """nsteps fixed steps of the 5th-order Dormand-Prince solution: six new stages per step."""
    for _ in range(nsteps):
        k = []
        for s in range(6):
            qs = q
            for j, a in enumerate(DP5_A[s]):
                qs = qs + (dt * a) * k[j]
            k.append(f(qs))
        for j, b in enumerate(DP5_B):
            if b != 0.0:
                q = q + (dt * b) * k[j]
    return q


# Adaptive Dormand-Prince 5(4) with a digital-filter step controller (Sec. 5: the paper integrates
# with DP5 and "adaptive time-stepping based on signal processing", citing Soderlind 2003 and
# Soderlind & Wang 2006, without stating the filter, the error norm or the tolerances).  Readings:
#   * error estimate: the embedded 4th-order solution of Dormand & Prince (1980); the 7th stage is
#     the residual at the new solution (first same as last), err_vec = dt sum_j (b_j - bhat_j) k_j;
#   * error norm: weighted RMS over all nodes and variables (Hairer, Norsett & Wanner, Solving ODEs
#     I, eq. II.4.11): sc = atol + rtol max(|q_n|, |q_n+1|), err = sqrt(mean((err_vec/sc)^2));
#   * filter: H211b with b = 4 (Soderlind 2003): the next step is dt_n rho_n with
#     rho_n = (theta/err_n)^(1/(b k)) (theta/err_n-1)^(1/(b k)) (dt_n/dt_n-1)^(-1/b) over accepted
#     steps, k = 5 (the estimate is O(dt^5)), setpoint theta = 0.8; on the first step
#     err_n-1 = err_n and dt_n-1 = dt_n;
#   * limiter: rho_hat = 1 + atan(rho - 1) (Soderlind & Wang 2006, kappa = 1);
#   * a step is accepted when err <= 1; a rejected step is retried with
#     dt rho_hat((theta/err)^(1/k)) and leaves the filter's history unchanged; a non-finite err (a
#     trial step so large that a stage state is unphysical) counts as rho = 0, i.e. dt rho_hat(0);
#   * the last step is shortened to land on t_end.

DP5_BHAT = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]
DP54_K = 5
H211B_B = 4.0
CTRL_THETA = 0.8


def dp54_error_norm(q0, q1, err_vec, rtol: float, atol: float) -> float:
    """Weighted RMS norm of the embedded error estimate (reading above)."""
    sc = atol + rtol * torch.maximum(q0.abs(), q1.abs())
    return float(torch.sqrt(((err_vec / sc) ** 2).mean()))


def step_limiter(rho: float) -> float:
    """Smooth step-ratio limiter 1 + atan(rho - 1)."""
    return 1.0 + math.atan(rho - 1.0)


def h211b_ratio(err: float, err_prev: float, rho_prev: float) -> float:
    """Unlimited H211b step-size ratio from the current and previous error norms and the previous
    accepted step-size ratio."""
    e = 1.0 / (H211B_B * DP54_K)
    return (CTRL_THETA / err) ** e * (CTRL_THETA / err_prev) ** e * rho_prev ** (-1.0 / H211B_B)


def dp54_step(q, k1, f, dt: float):
    """One Dormand-Prince step from q with first stage k1 = f(q): returns (q_new, k7 = f(q_new),
    err_vec) with the 5th-order solution and the embedded error estimate."""
    k = [k1]
    for s in range(1, 6):
        qs = q
        for j, a in enumerate(DP5_A[s]):
            qs = qs + (dt * a) * k[j]
        k.append(f(qs))
    q_new = q
    for j, b in enumerate(DP5_B):
        if b != 0.0:
            q_new = q_new + (dt * b) * k[j]
    k.append(f(q_new))
    err_vec = torch.zeros_like(q)
    for j in range(7):
        d = (DP5_B[j] if j < 6 else 0.0) - DP5_BHAT[j]
        if d != 0.0:
            err_vec = err_vec + (dt * d) * k[j]
    return q_new, k[6], err_vec


def rk_adaptive(q, f, t0: float, t_end: float, dt0: float, rtol: float, atol: float, max_steps: int = 1000):
    """Integrate q from t0 to t_end with adaptive DP5(4) (readings above).  Returns (q, stats) with
    stats = {"accepted": [dt of each accepted step], "rejected": count, "rhs": evaluations,
    "dt_next": the proposed next step}."""
    t = t0
    dt = dt0
    k1 = f(q) if t < t_end else None
    nrhs = 1 if t < t_end else 0
    err_prev, h_prev = None, None
    accepted, rejected = [], 0
    while t < t_end and len(accepted) + rejected < max_steps:
        last = t + dt >= t_end
        h = t_end - t if last else dt
        q_new, k7, ev = dp54_step(q, k1, f, h)
        nrhs += 6
        err = dp54_error_norm(q, q_new, ev, rtol, atol)
        if err <= 1.0:
            rho = h211b_ratio(err, err if err_prev is None else err_prev, 1.0 if h_prev is None else h / h_prev)
            q, k1 = q_new, k7
            t = t_end if last else t + h
            accepted.append(h)
            err_prev, h_prev = err, h
            dt = h * step_limiter(rho)
        else:
            rejected += 1
            rho = (CTRL_THETA / err) ** (1.0 / DP54_K) if math.isfinite(err) else 0.0
            dt = h * step_limiter(rho)
    return q, {"accepted": accepted, "rejected": rejected, "rhs": nrhs, "dt_next": dt}


# --------------------------------------------------------------------------------------------
# Budgets and time step
# --------------------------------------------------------------------------------------------

def quadrature_weights(mesh: Mesh) -> torch.Tensor:
    """P J at every node: the tensor-product LGL weights times the Jacobian ([K,N,N,N])."""
    w = mesh.sbp.w
    return w[:, None, None] * w[None, :, None] * w[None, None, :] * mesh.J


def kinetic_energy(q: torch.Tensor, mesh: Mesh) -> torch.Tensor:
    """Integrated kinetic energy sum P J rho|u|^2/2 as a differentiable scalar (Sec. 5.3 diagnostic)."""
    PJ = quadrature_weights(mesh)
    return (PJ * 0.5 * (q[:, 1] ** 2 + q[:, 2] ** 2 + q[:, 3] ** 2) / q[:, 0]).sum()


def budgets(q, dqdt, mesh: Mesh, gas: Gas):
    """(S_total, KE, dS/dt, dKE/dt): P J-weighted sums of S(q), rho|u|^2/2, w.dq/dt and
    dKE/dq.dq/dt with dKE/dq = [-|u|^2/2, u, 0]."""
    q = torch.as_tensor(q, dtype=F64)
    PJ = quadrature_weights(mesh)
    rho, u, _, _ = primitives(q, gas)
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    S = float((PJ * entropy_function(q, gas)).sum())
    KE = float((PJ * 0.5 * rho * usq).sum())
    if dqdt is None:
        return S, KE, 0.0, 0.0
    dqdt = torch.as_tensor(dqdt, dtype=F64)
    w = entropy_variables(q, gas)
    dS = float((PJ * (w * dqdt).sum(dim=1)).sum())
    dKE = float((PJ * (-0.5 * usq * dqdt[:, 0] + u[0] * dqdt[:, 1] + u[1] * dqdt[:, 2]
                       + u[2] * dqdt[:, 3])).sum())
    return S, KE, dS, dKE


def cfl_dt(q, mesh: Mesh, gas: Gas, cfl=0.5) -> float:
    """dt = cfl * min(h/((p+1)^2 max(|u|+c)), h^2/((p+1)^4 nu_max)), nu_max = max(4/3, gamma/Pr) mu/rho_min."""
    q = torch.as_tensor(q, dtype=F64)
    rho, u, _, _ = primitives(q, gas)
    speed = float((torch.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2) + sound_speed(q, gas)).max())
    N = mesh.sbp.N
    dt = mesh.h_min / (N * N * speed)
    if gas.mu > 0.0:
        nu = max(4.0 / 3.0, gas.gamma / gas.Pr) * gas.mu / float(rho.min())
        dt = min(dt, mesh.h_min ** 2 / (N ** 4 * nu))
    return cfl * dt
