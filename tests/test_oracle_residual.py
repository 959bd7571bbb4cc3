"""Pins of the oracle's semi-discrete residual (eq. discEL, eq. MacroForm, eq. NSL) by properties the
paper fixes: linear split form, conservation, entropy conservation/stability, freestream
preservation, the viscous entropy identity, mu-linearity and design-order convergence."""
import math

import numpy as np
import pytest
import sympy as sp
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

TWO_PI = 2 * math.pi


def _setup(p, k, warp=0.0, seed=0, lo=-math.pi, hi=math.pi):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [lo] * 3, [hi] * 3, warp=warp, seed=seed)
    return O.make_mesh(p, x, k, k, k), x


def _linear_flux(a):
    def flux(qa, qb, n, gas):
        an = a[0] * n[0] + a[1] * n[1] + a[2] * n[2]
        return an.unsqueeze(1) * 0.5 * (qa + qb)
    return flux


@pytest.mark.parametrize("warp", [0.0, 0.1])
def test_linear_flux_reduces_to_split_form(warp):
    """With the central flux a.n (u_i+u_j)/2 the Hadamard volume term equals the matrix split form
    -(1/2) sum_lm a_m (D_l A_lm + A_lm D_l) u of eq. convectionsplitdisctele (GCL metrics)."""
    mesh, _ = _setup(3, 2, warp, seed=5)
    a = [0.7, -0.4, 0.25]
    g = torch.Generator().manual_seed(0)
    u = torch.randn(mesh.J.shape[0], 5, 4, 4, 4, generator=g, dtype=torch.float64)
    vol = O.volume_term(u, mesh.Ja, mesh.sbp, None, _linear_flux(a))
    ref = torch.zeros_like(u)
    for l in range(3):
        A = sum(a[m] * mesh.Ja[:, l, m] for m in range(3)).unsqueeze(1)
        ref = ref - 0.5 * (O.dxi(A * u, l, mesh.sbp.D) + A * O.dxi(u, l, mesh.sbp.D))
    assert (vol - ref).abs().max() < 1e-12 * ref.abs().max()


@pytest.mark.parametrize("warp,mu", [(0.0, 0.0), (0.1, 1.0 / 1600), (0.1, 0.05)])
def test_conservation(warp, mu):
    """sum_kappa 1^T P J dq/dt = 0 for every variable on a periodic mesh (telescoping SATs)."""
    mesh, x = _setup(3, 3, warp, seed=1)
    gas = O.Gas.from_mach(0.1, 1.0 / mu if mu > 0 else 0.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=2, rel=1e-2))
    r = O.rhs(q, mesh, gas)
    PJ = O.quadrature_weights(mesh)
    for v in range(5):
        tot = float((PJ * r[:, v]).sum())
        scale = float((PJ * r[:, v].abs()).sum())
        assert abs(tot) < 1e-12 * scale


@pytest.mark.parametrize("warp", [0.0, 0.1])
def test_entropy_conservation_inviscid_ec(warp):
    """Inviscid, no interface dissipation, periodic: sum P J w.dq/dt = 0 to round-off."""
    mesh, x = _setup(3, 3, warp, seed=2)
    gas = O.Gas.from_mach(0.1, 0.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=3, rel=1e-2))
    r = O.rhs(q, mesh, gas, dissipation=False)
    PJ = O.quadrature_weights(mesh)
    prod = PJ * (O.entropy_variables(q, gas) * r).sum(dim=1)
    assert abs(float(prod.sum())) < 1e-13 * float(prod.abs().sum())


def test_entropy_stable_with_dissipation():
    """With the interface dissipation on, the inviscid entropy production is strictly negative."""
    mesh, x = _setup(3, 3, 0.1, seed=2)
    gas = O.Gas.from_mach(0.1, 0.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=3, rel=1e-2))
    _, _, dS, _ = O.budgets(q, O.rhs(q, mesh, gas, dissipation=True), mesh, gas)
    assert dS < 0


def test_freestream_preservation_warped():
    """Uniform flow on the warped mesh: dq/dt = 0 to round-off (discrete GCL + consistent SATs)."""
    mesh, x = _setup(4, 3, 0.1, seed=0)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.freestream(x))
    r = O.rhs(q, mesh, gas)
    flux_scale = (1.0 / (1.4 * 0.01)) / float(mesh.J.min()) * float(mesh.Ja.abs().max())
    assert r.abs().max() < 1e-12 * flux_scale


def test_viscous_entropy_identity():
    """BR1 on a periodic mesh: sum P w.(viscous residual) = -sum P J g^T C g <= 0 exactly, with g the
    lifted physical entropy-variable gradient (C symmetric PSD, eq. Fxment)."""
    mesh, x = _setup(3, 3, 0.1, seed=4)
    gas = O.Gas.from_mach(0.1, 100.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=5, rel=1e-2))
    K = q.shape[0]
    E = torch.arange(K)
    visc = O.viscous_term(q, mesh, gas, E)
    _, g = O.contravariant_viscous_flux(q, mesh, gas, E)
    FV = O.viscous_flux(q, g, gas)
    w = mesh.sbp.w
    P = w[:, None, None] * w[None, :, None] * w[None, None, :]
    lhs = float((P * (O.entropy_variables(q, gas) * visc).sum(dim=1)).sum())
    quad = float((P * mesh.J * (g * FV).sum(dim=(1, 2))).sum())
    assert quad > 0
    assert abs(lhs + quad) < 1e-12 * quad


def test_viscous_part_linear_in_mu():
    mesh, x = _setup(2, 2, 0.1, seed=6)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=7, rel=1e-2))
    g0, g1, g2 = (O.Gas.from_mach(0.1, 0.0), O.Gas.from_mach(0.1, 100.0), O.Gas.from_mach(0.1, 50.0))
    r0, r1, r2 = O.rhs(q, mesh, g0), O.rhs(q, mesh, g1), O.rhs(q, mesh, g2)
    d1, d2 = r1 - r0, r2 - r0
    assert (d2 - 2 * d1).abs().max() < 1e-10 * d2.abs().max()


def test_sampled_elements_match_full():
    """Residual restricted to a few elements (closure of neighbours) equals the full residual there."""
    mesh, x = _setup(3, 3, 0.1, seed=8)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=9, rel=1e-3))
    full = O.rhs(q, mesh, gas)
    E = torch.tensor([0, 5, 13, 26])
    part = O.rhs(q, mesh, gas, elems=E)
    assert (part - full[E]).abs().max() <= 1e-14 * full.abs().max()


def _rate(errs, ks):
    return [math.log(errs[i] / errs[i + 1]) / math.log(ks[i + 1] / ks[i]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("p", [2, 3])
def test_design_order_density_wave(p):
    """Inviscid exact solution rho = 1 + a sin(x+y+z), constant u, p: dq/dt = -u.grad q exactly.
    The nodal residual error converges at (at least) order p on affine meshes."""
    gas = O.Gas.from_mach(0.1, 0.0)
    ks, errs = [4, 8, 16], []
    u = (1.0, 0.5, 0.25)
    for k in ks:
        mesh, x = _setup(p, k)
        q = torch.tensor(I.density_wave(x, amp=0.1, u=u))
        r = O.rhs(q, mesh, gas)
        ph = x[:, 0] + x[:, 1] + x[:, 2]
        drho = -0.1 * np.cos(ph) * sum(u)
        exact = np.stack([drho, u[0] * drho, u[1] * drho, u[2] * drho,
                          0.5 * sum(c * c for c in u) * drho], axis=1)
        errs.append(float(np.abs(r.numpy() - exact).max()))
    rates = _rate(errs, ks)
    assert min(rates) > p - 0.3, (errs, rates)


@pytest.mark.parametrize("case", ["shear", "heat"])
def test_viscous_converges_to_exact_divergence(case):
    """Shear wave u1 = sin(x2): d(rho u1)/dt = -mu sin x2, d(rho E)/dt = mu cos 2x2.  Temperature wave
    T = 1 + a sin x1 at uniform p: d(rho E)/dt = -a kappa sin x1.  Inviscid parts vanish exactly."""
    p, ks, errs = 3, [4, 8, 16], []
    gas = O.Gas.from_mach(0.1, 10.0)
    for k in ks:
        mesh, x = _setup(p, k)
        if case == "shear":
            q = torch.tensor(I.shear_wave(x))
            ex = np.zeros(q.shape)
            ex[:, 1] = -gas.mu * np.sin(x[:, 1])
            ex[:, 4] = gas.mu * np.cos(2 * x[:, 1])
        else:
            q = torch.tensor(I.temperature_wave(x, amp=0.1))
            ex = np.zeros(q.shape)
            ex[:, 4] = -0.1 * gas.kappa * np.sin(x[:, 0])
        r = O.rhs(q, mesh, gas, dissipation=False).numpy()
        errs.append(float(np.abs(r - ex).max()))
    # BR1 converges pointwise at order p-1 at face nodes (faster inside): check the mean rate
    rate = math.log(errs[0] / errs[-1]) / math.log(ks[-1] / ks[0])
    assert rate > 1.8 and errs[-1] < 1e-2 * np.abs(ex).max(), (errs, rate)


def test_tgv_initial_dissipation_rate():
    """Taylor-Green vortex at t = 0 is divergence free, so dKE/dt = -mu <|omega|^2> = -3 mu/4 per unit
    volume (vorticity of the initial field integrated by hand); the ES-C residual reproduces it."""
    mesh, x = _setup(4, 4)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.taylor_green(x))
    _, _, _, dKE = O.budgets(q, O.rhs(q, mesh, gas), mesh, gas)
    rate = dKE / TWO_PI ** 3
    assert abs(rate - (-0.75 / 1600.0)) < 0.02 * 0.75 / 1600.0, rate


def test_tgv_kinetic_energy_closed_form():
    """KE of the initial Taylor-Green field: int rho|u|^2/2 over the box, integrated symbolically."""
    X, Y, Z = sp.symbols("x y z")
    Ma, g = sp.Rational(1, 10), sp.Rational(7, 5)
    rho = 1 + g * Ma ** 2 / 16 * (sp.cos(2 * X) + sp.cos(2 * Y)) * (sp.cos(2 * Z) + 2)
    usq = (sp.sin(X) * sp.cos(Y) * sp.cos(Z)) ** 2 + (sp.cos(X) * sp.sin(Y) * sp.cos(Z)) ** 2
    exact = float(sp.integrate(rho * usq / 2, (X, -sp.pi, sp.pi), (Y, -sp.pi, sp.pi), (Z, -sp.pi, sp.pi)))
    mesh, x = _setup(5, 4)
    _, KE, _, _ = O.budgets(torch.tensor(I.taylor_green(x)), None, mesh, O.Gas.from_mach(0.1))
    assert abs(KE - exact) < 1e-7 * exact


def test_submesh_residual_matches_full_mesh():
    """The residual on sampled elements computed on their two-ring submesh equals the full-mesh one."""
    mesh, x = _setup(3, 6, 0.1, seed=8)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.perturb(I.taylor_green(x), seed=9, rel=1e-3))
    E = torch.tensor([0, 129])
    sub, E2, rows = O.make_submesh(3, x, mesh.nbr, E)
    assert E2.numel() < 6 ** 3
    r_sub = O.rhs(q[E2], sub, gas, elems=rows)
    r_full = O.rhs(q, mesh, gas, elems=E)
    assert (r_sub - r_full).abs().max() <= 1e-14 * r_full.abs().max()


@pytest.mark.parametrize("p,k,warp", [(2, (3, 4, 2), 0.1), (3, (2, 3, 3), 0.0)])
def test_llf_dissipation_entropy_production_face_identity(p, k, warp):
    """Magnitude of the local Lax-Friedrichs interface dissipation (SAT^(I) reading: lambda/2 (q_own -
    q_nbr) lifted by 1/P_ii, lambda = max over both sides of |u.n_J| + c |n_J|).  Its contribution to
    the entropy budget sum P J w.dq/dt is, after pairing the two sides of every interface,
        dS(LLF) - dS(EC) = - sum_interfaces sum_face_nodes w_a w_b lambda/2 (w_L - w_R).(q_L - q_R),
    with w_a w_b the face quadrature weights.  The right side is computed here from the face states
    alone, with this test's own face indexing and sound speed, so a halved or doubled lambda, a dropped
    |n_J|, a wrong lift weight or a dissipation on the wrong side fails it.  The box is anisotropic and
    scaled so that |n_J| is far from 1."""
    kx, ky, kz = k
    s = O.sbp_operator(p)
    lo, hi = [-0.4, -0.9, -0.3], [0.6, 0.3, 0.5]
    x = I.box_coords(s.xi.numpy(), kx, ky, kz, lo, hi, warp=warp, seed=5)
    mesh = O.make_mesh(p, x, kx, ky, kz)
    gas = O.Gas.from_mach(0.3, 0.0)
    q = torch.tensor(I.perturb(I.density_wave(x, amp=0.2, Ma=0.3), seed=4, rel=2e-2))
    dS_llf = O.budgets(q, O.rhs(q, mesh, gas, dissipation=True), mesh, gas)[2]
    dS_ec = O.budgets(q, O.rhs(q, mesh, gas, dissipation=False), mesh, gas)[2]

    g = gas.gamma
    N = p + 1
    wq = s.w.double()
    W2 = wq[:, None] * wq[None, :]                          # face weights (axis order kept)
    w = O.entropy_variables(q, gas)
    nbr = O.box_neighbours(kx, ky, kz)
    total = 0.0
    for l in range(3):
        ax = 4 - l                                           # array axis of xi_{l+1} in [K, 5, N, N, N]
        qL = q.select(ax, N - 1)                            # +xi_l face of every element
        wL = w.select(ax, N - 1)
        R = nbr[:, 2 * l + 1]                                # its neighbour across that face
        qR = q[R].select(ax, 0)
        wR = w[R].select(ax, 0)
        n = mesh.Ja[:, l].select(ax, N - 1)                  # [K, 3, face nodes] contravariant normal
        nmag = torch.sqrt((n ** 2).sum(dim=1))

        def lam(qq):
            rho = qq[:, 0]
            u = qq[:, 1:4] / rho.unsqueeze(1)
            pr = (g - 1.0) * (qq[:, 4] - 0.5 * rho * (u ** 2).sum(dim=1))
            return (u * n).sum(dim=1).abs() + torch.sqrt(g * pr / rho) * nmag

        lmax = torch.maximum(lam(qL), lam(qR))
        quad = ((wL - wR) * (qL - qR)).sum(dim=1)
        total += float((W2 * 0.5 * lmax * quad).sum())
    assert total > 0.0
    assert dS_llf - dS_ec == pytest.approx(-total, rel=1e-11, abs=0.0)
