"""Pins of the oracle's SBP operator and metric terms against closed forms and definitions.

Sec. 2 Definition 1 (SBP operator), Sec. 3 eqs. GCL / discGCLconvection (metric identities).
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgl_closed_form.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        p, xs, ws = [s.strip() for s in line.split("|")]
        env = {"sqrt": math.sqrt}
        rows.append((int(p), [eval(s, env) for s in xs.split(",")], [eval(s, env) for s in ws.split(",")]))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"p{r[0]}")
def test_lgl_closed_form(row):
    p, xs, ws = row
    x, w = O.lgl_nodes_weights(p)
    assert np.allclose(x.numpy(), xs, atol=1e-15, rtol=0)
    assert np.allclose(w.numpy(), ws, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", range(1, 16))
def test_lgl_against_numpy_legendre(p):
    """Interior nodes are the roots of P_p' (numpy's Legendre class); the weights integrate
    polynomials of degree 2p-1 exactly (Gauss-Lobatto quadrature)."""
    x, w = O.lgl_nodes_weights(p)
    if p > 1:
        roots = np.sort(np.polynomial.legendre.Legendre.basis(p).deriv().roots().real)
        assert np.allclose(x.numpy()[1:-1], roots, atol=1e-13)
    for d in range(2 * p):
        exact = (1 - (-1) ** (d + 1)) / (d + 1)
        assert abs(float((w * x ** d).sum()) - exact) < 1e-13


@pytest.mark.parametrize("p", range(1, 16))
def test_sbp_definition(p):
    """Definition 1: D xi^j = j xi^(j-1) for j <= p, P SPD diagonal, Q + Q^T = E."""
    s = O.sbp_operator(p)
    for j in range(p + 1):
        lhs = s.D @ s.xi ** j
        rhs = j * s.xi ** (j - 1) if j > 0 else torch.zeros_like(s.xi)
        assert (lhs - rhs).abs().max() < 1e-11 * max(1, p * p)
    assert (s.w > 0).all()
    assert (s.Q + s.Q.T - s.E).abs().max() < 1e-13
    S = s.Q - 0.5 * s.E
    assert (S + S.T).abs().max() < 1e-13


def _mesh(p, k, warp, seed=0, lo=-math.pi, hi=math.pi):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [lo] * 3, [hi] * 3, warp=warp, seed=seed)
    return O.make_mesh(p, x, k, k, k), x


def test_affine_metrics_closed_form():
    """Box element of size h: J = h1 h2 h3/8 and Ja_lm = delta_lm h_m' h_m''/4."""
    p = 3
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), 2, 3, 4, [0.0, -1.0, 2.0], [1.0, 2.0, 10.0])
    m = O.make_mesh(p, x, 2, 3, 4)
    h = np.array([1.0 / 2, 3.0 / 3, 8.0 / 4])
    assert torch.allclose(m.J, torch.full_like(m.J, h.prod() / 8), rtol=1e-14, atol=0)
    for l in range(3):
        for mm in range(3):
            expect = (h.prod() / h[l] / 4) if l == mm else 0.0
            # the curl form multiplies coordinates (up to |x| = 10 here) by derivatives: round-off
            # grows with |x|, so the bound is relative to the coordinate magnitude
            assert (m.Ja[:, l, mm] - expect).abs().max() < 1e-14 * 10 * 4


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_discrete_gcl_warped(p):
    """eq. discGCLconvection: sum_l D_l A_lm 1 = 0 on the warped periodic mesh."""
    m, _ = _mesh(p, 3, 0.1, seed=0)
    scale = m.Ja.abs().max()
    for mm in range(3):
        g = sum(O.dxi(m.Ja[:, l, mm], l, m.sbp.D) for l in range(3))
        assert g.abs().max() < 1e-13 * scale * p * p


def test_curl_metrics_exact_for_quadratic_map():
    """For a mapping of degree 2 and p >= 4 every product in the curl form is a polynomial of degree
    <= p, so the curl-form metrics equal the cofactors of dx/dxi: sum_m Ja_lm dx_m/dxi_a = J delta_la."""
    p = 4
    s = O.sbp_operator(p)
    N = p + 1
    t = s.xi
    X3, X2, X1 = torch.meshgrid(t, t, t, indexing="ij")
    x = torch.stack([X1 + 0.1 * X2 * X3 + 0.05 * X1 ** 2,
                     X2 + 0.07 * X1 * X3 - 0.03 * X3 ** 2,
                     X3 + 0.09 * X1 * X2 + 0.02 * X2 ** 2], dim=0)[None]
    J, Ja = O.metric_terms(x, s.D)
    for l in range(3):
        for a in range(3):
            acc = sum(Ja[:, l, mm] * O.dxi(x[:, mm], a, s.D) for mm in range(3))
            expect = J if l == a else torch.zeros_like(J)
            assert (acc - expect).abs().max() < 1e-13
    assert N == 5


def test_metrics_converge_to_analytic_cofactors():
    """Curl-form metrics of a smooth (sinusoidal) map approach the exact cofactor matrix spectrally."""
    errs = []
    for p in (3, 5, 7):
        s = O.sbp_operator(p)
        t = s.xi
        X3, X2, X1 = torch.meshgrid(t, t, t, indexing="ij")
        a = 0.1
        x = torch.stack([X1 + a * torch.sin(X2), X2 + a * torch.sin(X3), X3 + a * torch.sin(X1)])[None]
        _, Ja = O.metric_terms(x, s.D)
        # exact Jacobian F[m][a] = dx_m/dxi_a ; cofactor(F)[a][m] = J dxi_a/dx_m
        c1, c2, c3 = a * torch.cos(X2), a * torch.cos(X3), a * torch.cos(X1)
        F = torch.zeros(3, 3, *X1.shape, dtype=torch.float64)
        F[0, 0], F[0, 1] = 1.0, c1
        F[1, 1], F[1, 2] = 1.0, c2
        F[2, 2], F[2, 0] = 1.0, c3
        cof = torch.zeros_like(F)
        for i in range(3):
            for j in range(3):
                i1, i2, j1, j2 = (i + 1) % 3, (i + 2) % 3, (j + 1) % 3, (j + 2) % 3
                cof[j, i] = F[i1, j1] * F[i2, j2] - F[i1, j2] * F[i2, j1]
        errs.append(float((Ja[0] - cof).abs().max()))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-7


def test_face_metrics_match_across_interfaces():
    """Watertight mapping: the contravariant normal Ja_l at a shared face is the same from both sides
    (to round-off), which the conservation of the interface terms rests on."""
    m, _ = _mesh(4, 3, 0.1, seed=3)
    for l in range(3):
        own = O.face(m.Ja[:, l], l, 1)
        nb = O.face(m.Ja[m.nbr[:, 2 * l + 1], l], l, 0)
        assert (own - nb).abs().max() < 1e-13 * m.Ja.abs().max()


def test_jacobian_positive_and_volume():
    """sum P J = volume of the periodic box, also on the warped mesh (displacement is periodic)."""
    m, _ = _mesh(4, 3, 0.1, seed=0)
    assert (m.J > 0).all()
    vol = float(O.quadrature_weights(m).sum())
    assert abs(vol - (2 * math.pi) ** 3) < 1e-10 * vol
