"""Pins of the oracle's optimized metrics (Sec. 3): analytic surface metrics of the interpolated
mapping on the faces, volume metrics that satisfy the discrete GCL with them and are the nearest
ones to the analytic metrics.  Checked against what the definition fixes without reusing its solve:
the adjugate identity and the affine closed form of the cofactor metrics, the agreement of the
surface metrics seen from the two sides of every face, the orthogonality of the correction to an
independently built family of feasible directions (discrete curls of fields that vanish on the
element boundary), and the consequences for the scheme: uniform flow kept on a warped mesh for every
volume flux and interface option, conservation, zero entropy production of the entropy-conservative
scheme, the truncation order on the manufactured solution, and design-order convergence of both
metric constructions to the metrics of the exact (non-polynomial) warped mapping."""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

F64 = torch.float64


def _warped(p, k, seed=0, warp=0.1, lo=-math.pi, hi=math.pi, bounded=(False, False, False)):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [lo] * 3, [hi] * 3, warp=warp, seed=seed)
    return O.make_mesh(p, x, k, k, k, bounded=bounded, metrics="optimized"), x


def test_cofactor_metrics_are_the_adjugate():
    """sum_m Ja_lm dx_m/dxi_a = J delta_la with J = det(dx/dxi) from the independent determinant."""
    p = 3
    s = O.sbp_operator(p)
    x = torch.tensor(I.box_coords(s.xi.numpy(), 2, 2, 2, [0.0] * 3, [1.0] * 3, warp=0.15, seed=4))
    t = O.cofactor_metrics(x, s.D)
    J, _ = O.metric_terms(x, s.D)
    for l in range(3):
        for a in range(3):
            got = sum(t[:, l, m] * O.dxi(x[:, m], a, s.D) for m in range(3))
            want = J if l == a else torch.zeros_like(J)
            assert (got - want).abs().max() < 1e-13 * J.abs().max(), (l, a)


def test_affine_box_optimized_metrics_closed_form():
    """On a box element of sizes h the analytic metrics already meet the discrete GCL, so the
    optimized volume metrics are Ja_lm = delta_lm h_l' h_l''/4 as well."""
    p = 3
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), 2, 3, 4, [0.0, -1.0, 2.0], [1.0, 2.0, 10.0])
    m = O.make_mesh(p, x, 2, 3, 4, metrics="optimized")
    h = np.array([1.0 / 2, 3.0 / 3, 8.0 / 4])
    for l in range(3):
        for mm in range(3):
            expect = (h.prod() / h[l] / 4) if l == mm else 0.0
            assert (m.Ja[:, l, mm] - expect).abs().max() < 1e-14
            assert (m.Ja_face[:, l, mm] - expect).abs().max() < 1e-14


def test_surface_metrics_agree_across_faces():
    """Row l of the cofactor on a face xi_l = +-1 depends only on the face's nodes: the element and
    its neighbour across that face see the same surface metrics (to round-off, periodic faces too)."""
    m, _ = _warped(3, 3)
    t = m.Ja_face
    scale = float(t.abs().max())
    for l in range(3):
        own = O.face(t[:, l], l, 1)                        # face xi_l = +1 of every element
        nbr = O.face(t[m.nbr[:, 2 * l + 1], l], l, 0)      # face xi_l = -1 of its neighbour
        assert (own - nbr).abs().max() < 1e-14 * scale


def _interior_curl(psi, D):
    """Discrete curl_xi of a field psi [3, N, N, N] (xi3, xi2, xi1 axes)."""
    d = lambda u, l: O.dxi(u.unsqueeze(0), l, D)[0]
    return torch.stack([d(psi[2], 1) - d(psi[1], 2), d(psi[0], 2) - d(psi[2], 0), d(psi[1], 0) - d(psi[0], 1)])


@pytest.mark.parametrize("p", [2, 3, 4])
def test_correction_is_orthogonal_to_feasible_directions(p):
    """A curl of a field vanishing at every boundary node satisfies sum_l Q_l^T delta_l = 0 (the
    derivatives commute and delta_l vanishes on the faces xi_l = +-1), so a + delta is feasible too;
    the Euclidean-nearest a has (a - t) orthogonal to every such delta, and a + delta is farther."""
    m, _ = _warped(p, 2, seed=5)
    s = m.sbp
    N = s.N
    g = torch.Generator().manual_seed(7)
    inner = torch.zeros(N, N, N, dtype=F64)
    inner[1:-1, 1:-1, 1:-1] = 1.0
    Ql, El = O.sbp_3d(s)
    for trial in range(4):
        psi = torch.randn(3, N, N, N, generator=g, dtype=F64) * inner
        delta = _interior_curl(psi, s.D)
        # feasibility of delta, checked on the dense operators
        res = sum(Ql[l].T @ delta[l].reshape(-1) for l in range(3))
        assert float(res.abs().max()) < 1e-12 * float(delta.abs().max())
        for e in range(m.Ja.shape[0]):
            for mm in range(3):
                corr = m.Ja[e, :, mm] - m.Ja_face[e, :, mm]
                dot = float((corr * delta).sum())
                assert abs(dot) < 1e-12 * float(corr.abs().max() * delta.abs().sum())
                d0 = float((corr ** 2).sum())
                d1 = float(((corr + 1e-3 * delta) ** 2).sum())
                assert d1 > d0


@pytest.mark.parametrize("scheme,opts", [("esc", {}), ("esc", {"dissipation": "matrix", "ip_coef": 1.0}),
                                         ("kg", {}), ("dc", {})])
def test_freestream_preserved_on_warped_mesh(scheme, opts):
    """A uniform flow stays a steady state with the optimized metrics; with the volume metrics in the
    interface terms instead of the surface ones (an inconsistent pairing) it does not."""
    gas = O.Gas.from_mach(0.3, 200.0)
    m, x = _warped(3, 3, seed=2)
    qf = torch.tensor(I.freestream(x, Ma=0.3))
    r = O.rhs(qf, m, gas, scheme=scheme, **opts)
    assert float(r.abs().max()) < 1e-11 * gas.R
    wrong = O.Mesh(m.sbp, m.x, m.J, m.Ja, m.nbr, m.h_min, None)
    assert float(O.rhs(qf, wrong, gas, scheme=scheme, **opts).abs().max()) > 1e-4 * gas.R


def test_conservation_and_entropy_conservation():
    """Periodic warped mesh: sum P J dq/dt = 0 per variable (viscous, dissipative scheme), and the
    inviscid scheme without interface dissipation produces no entropy, sum P J w.dq/dt = 0."""
    m, x = _warped(3, 3, seed=1)
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=3, rel=0.05))
    PJ = O.quadrature_weights(m)
    gas = O.Gas.from_mach(0.3, 200.0)
    r = O.rhs(q, m, gas)
    for v in range(5):
        tot = float((PJ * r[:, v]).sum())
        mag = float((PJ * r[:, v].abs()).sum())
        assert abs(tot) <= 1e-12 * mag, (v, tot, mag)
    gas0 = O.Gas.from_mach(0.3, 0.0)
    r0 = O.rhs(q, m, gas0, dissipation=False)
    w = O.entropy_variables(q, gas0)
    prod = float((PJ.unsqueeze(1) * w * r0).sum())
    mag = float((PJ.unsqueeze(1) * (w * r0).abs()).sum())
    assert abs(prod) <= 1e-12 * mag, (prod, mag)
    r1 = O.rhs(q, m, gas0)
    assert float((PJ.unsqueeze(1) * w * r1).sum()) < -1e-6 * mag


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_solution_truncation_order(p):
    """Bounded box with the manufactured solution as Dirichlet data: ||R(q_exact) + S|| falls at rate
    >= p - 0.3 with the optimized metrics on a warped mesh."""
    gas = O.Gas.from_mach(I.MMS_MA, I.MMS_RE)
    prim = lambda a, b, c: I.manufactured_primitives(a, b, c, sin=torch.sin, cos=torch.cos)
    errs = []
    for k in (2, 4, 8):
        m, x = _warped(p, k, seed=3, warp=0.05, lo=0.0, hi=1.0, bounded=(True, True, True))
        q = torch.tensor(I.manufactured(x))
        S = O.manufactured_source(prim, x, gas)
        r = O.rhs(q, m, gas, q_ext=q, source=S)
        PJ = O.quadrature_weights(m).unsqueeze(1)
        errs.append(float(torch.sqrt((PJ * r ** 2).sum() / (PJ * S ** 2).sum())))
    rate = math.log2(errs[1] / errs[2])
    assert rate >= p - 0.3, (errs, rate)


def _exact_metrics(xi, k, lo, hi, warp, seed):
    """Cofactor metrics of the exact warped mapping (not its interpolant) at the LGL nodes, by
    autograd of the mapping xi -> x of each element, written out from the warp formula of the input
    module."""
    N = xi.numel()
    lo_t, hi_t = torch.tensor(lo, dtype=F64), torch.tensor(hi, dtype=F64)
    L = hi_t - lo_t
    h = L / k
    phi = torch.tensor(I.warp_phases(seed), dtype=F64)
    g = torch.meshgrid(xi, xi, xi, indexing="ij")                                    # (xi3, xi2, xi1)
    ref = torch.stack([g[2], g[1], g[0]], dim=0).reshape(3, -1)                      # [3 (xi_a), N^3]
    out = torch.empty(k ** 3, 3, 3, N, N, N, dtype=F64)
    for el in range(k ** 3):
        eidx = torch.tensor([el % k, (el // k) % k, el // (k * k)], dtype=F64)
        r = ref.clone().requires_grad_(True)
        X = lo_t[:, None] + (eidx[:, None] + (r + 1.0) * 0.5) * h[:, None]
        ph = 2.0 * math.pi * (X - lo_t[:, None]) / L[:, None]
        x = torch.stack([X[i] + warp * h[i] * torch.prod(torch.sin(ph + phi[i][:, None]), dim=0) for i in range(3)])
        dx = torch.empty(3, 3, N ** 3, dtype=F64)                                   # dx_m / dxi_a
        for m in range(3):
            dx[m] = torch.autograd.grad(x[m].sum(), r, retain_graph=True)[0]
        for l in range(3):
            a, b = (l + 1) % 3, (l + 2) % 3
            for m in range(3):
                m1, m2 = (m + 1) % 3, (m + 2) % 3
                out[el, l, m] = (dx[m1, a] * dx[m2, b] - dx[m2, a] * dx[m1, b]).reshape(N, N, N)
    return out


@pytest.mark.parametrize("p", [2, 3])
def test_metrics_converge_to_the_exact_mapping_metrics(p):
    """Both metric constructions approximate the metrics of the exact (non-polynomial) warped mapping
    at design order: the max error falls at rate >= p - 0.5 from 4^3 to 8^3 elements, and the
    optimized volume metrics are not farther from them than the curl form by more than a few
    percent (they are the nearest feasible ones to the interpolant's analytic metrics)."""
    s = O.sbp_operator(p)
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    errs = {"curl": [], "optimized": []}
    for k in (4, 8):
        x = I.box_coords(s.xi.numpy(), k, k, k, lo, hi, warp=0.1, seed=0)
        ex = _exact_metrics(s.xi, k, lo, hi, 0.1, 0)
        scale = float(ex.abs().max())
        for met in errs:
            m = O.make_mesh(p, x, k, k, k, metrics=met)
            errs[met].append(float((m.Ja - ex).abs().max()) / scale)
    for met, (e4, e8) in errs.items():
        assert math.log2(e4 / e8) >= p - 0.5, (met, e4, e8)
    assert errs["optimized"][1] <= 1.05 * errs["curl"][1], errs
