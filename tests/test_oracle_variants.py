"""Pins of the oracle's SF-KG and DC variants (the paper's comparison discretisations, Sec. 4):
consistency and symmetry of the Kennedy-Gruber flux, kinetic-energy preservation of the split forms
at uniform pressure (which the DC form does not have), the DC volume term as D applied to nodal
contravariant fluxes (equal to the Hadamard form with the central flux of node-own fluxes, since
the rows of D sum to zero), freestream preservation on a warped mesh and global conservation."""
import math

import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

F64 = torch.float64


def _random_states(n, seed, gas):
    g = torch.Generator().manual_seed(seed)
    rho = 0.5 + torch.rand(n, generator=g, dtype=F64)
    u = torch.randn(3, n, generator=g, dtype=F64)
    p = gas.R * (0.5 + torch.rand(n, generator=g, dtype=F64))
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u ** 2).sum(0)
    return torch.stack([rho, rho * u[0], rho * u[1], rho * u[2], E], dim=1)


def test_kg_flux_consistent_symmetric_and_kinetic_energy_form():
    gas = O.Gas.from_mach(0.3, 0.0)
    qa, qb = _random_states(64, 1, gas), _random_states(64, 2, gas)
    n = [torch.randn(64, dtype=F64, generator=torch.Generator().manual_seed(s)) for s in (3, 4, 5)]
    same = O.kg_flux_n(qa, qa, n, gas)
    ref = O.euler_flux_n(qa, n, gas)
    assert torch.allclose(same, ref, rtol=1e-14, atol=1e-12)
    assert torch.equal(O.kg_flux_n(qa, qb, n, gas), O.kg_flux_n(qb, qa, n, gas))
    # momentum flux = mass flux x mean velocity + mean pressure x n (the kinetic-energy form)
    f = O.kg_flux_n(qa, qb, n, gas)
    _, ua, pa, _ = O.primitives(qa, gas)
    _, ub, pb, _ = O.primitives(qb, gas)
    for m in range(3):
        want = f[:, 0] * 0.5 * (ua[m] + ub[m]) + 0.5 * (pa + pb) * n[m]
        assert torch.allclose(f[:, 1 + m], want, rtol=1e-13, atol=1e-12)


def _mesh(p, k, warp, seed, gas_ma=0.3):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), *k, [-math.pi] * 3, [math.pi] * 3, warp=warp, seed=seed)
    return O.make_mesh(p, x, *k), x


@pytest.mark.parametrize("scheme", ["kg", "esc"])
def test_split_forms_preserve_kinetic_energy_at_uniform_pressure(scheme):
    """Inviscid, no interface dissipation, uniform pressure, random density and velocity: the
    kinetic-energy rate sum P J (dKE/dq).dq/dt vanishes to round-off for the split (two-point) forms
    (Jameson's kinetic-energy-preserving momentum flux), and not for DC."""
    gas = O.Gas.from_mach(0.3, 0.0)
    mesh, x = _mesh(3, (3, 2, 2), 0.1, 4)
    g = torch.Generator().manual_seed(9)
    K, N = mesh.J.shape[0], mesh.sbp.N
    rho = 1.0 + 0.3 * torch.rand(K, N, N, N, generator=g, dtype=F64)
    u = 0.3 * torch.randn(3, K, N, N, N, generator=g, dtype=F64)
    p = gas.R * torch.ones(K, N, N, N, dtype=F64)
    q = torch.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                     p / (gas.gamma - 1.0) + 0.5 * rho * (u ** 2).sum(0)], dim=1)
    r = O.rhs(q, mesh, gas, dissipation=False, scheme=scheme)
    _, KE, _, dKE = O.budgets(q, r, mesh, gas)
    PJ = O.quadrature_weights(mesh)
    ke_terms = 0.5 * (u ** 2).sum(0) * r[:, 0].abs() + (u.abs() * r[:, 1:4].abs().movedim(1, 0)).sum(0)
    scale = float((PJ * ke_terms).sum())
    assert abs(dKE) <= 1e-13 * scale, (dKE, scale)
    rd = O.rhs(q, mesh, gas, dissipation=False, scheme="dc")
    _, _, _, dKE_dc = O.budgets(q, rd, mesh, gas)
    assert abs(dKE_dc) > 1e-6 * scale


def test_dc_volume_is_d_times_nodal_contravariant_flux():
    """-sum_l D_l Ftilde_l equals -2 sum_j D_ij (Ftilde_i + Ftilde_j)/2 along every line (the rows of
    D sum to zero), written here with an explicit einsum over the line index."""
    gas = O.Gas.from_mach(0.3, 0.0)
    mesh, x = _mesh(2, (2, 2, 2), 0.1, 5)
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=2, rel=0.05))
    got = O.dc_volume_term(q, mesh.Ja, mesh.sbp, gas)
    want = torch.zeros_like(q)
    for l in range(3):
        Ft = O.euler_flux_n(q, [mesh.Ja[:, l, m] for m in range(3)], gas)
        a = -1 - l
        Ftt = Ft.movedim(a, -1)
        pair = 0.5 * (Ftt.unsqueeze(-1) + Ftt.unsqueeze(-2))
        want = want + (-2.0 * torch.einsum("ij,...ij->...i", mesh.sbp.D, pair)).movedim(-1, a)
    assert torch.allclose(got, want, rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("scheme", ["kg", "dc"])
def test_variants_freestream_and_conservation(scheme):
    gas = O.Gas.from_mach(0.3, 200.0)
    mesh, x = _mesh(3, (3, 3, 2), 0.1, 6)
    qf = torch.tensor(I.freestream(x, Ma=0.3))
    r = O.rhs(qf, mesh, gas, scheme=scheme)
    assert float(r.abs().max()) < 1e-11 * gas.R
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=3, rel=0.02))
    r = O.rhs(q, mesh, gas, scheme=scheme)
    PJ = O.quadrature_weights(mesh)
    for v in range(5):
        tot = float((PJ * r[:, v]).sum())
        mag = float((PJ * r[:, v].abs()).sum())
        assert abs(tot) <= 1e-12 * mag, (v, tot, mag)
