"""CPU tests of the C ABI library: it loads, exports every declared symbol, and its host-side setup
(LGL operator, curl-form metrics, smallest edge, argument checks) matches the oracle.  No kernel is
launched here."""
import ctypes
import math

import numpy as np
import pytest

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import _native as nat
from paper_1911_10966_gb300 import inputs as I


@pytest.fixture(scope="module")
def L():
    return nat.lib()


def test_exports_every_header_symbol(L):
    names = nat.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("p", list(range(1, 8)) + [11, 15])
def test_operators_match_oracle(L, p):
    N = p + 1
    xi, w = np.zeros(N), np.zeros(N)
    D, S = np.zeros(N * N), np.zeros(N * N)
    nat.check(L.esdc_lgl(p, xi.ctypes.data, w.ctypes.data), "lgl")
    nat.check(L.esdc_operators(p, D.ctypes.data, S.ctypes.data), "ops")
    s = O.sbp_operator(p)
    assert np.abs(xi - s.xi.numpy()).max() < 1e-15
    assert np.abs(w - s.w.numpy()).max() < 1e-15
    D = D.reshape(N, N)
    S = S.reshape(N, N)
    assert np.abs(D - s.D.numpy()).max() < 2e-13 * max(1, p * p)
    assert np.abs(S + S.T).max() == 0.0
    Q = np.diag(w) @ D
    E = np.zeros((N, N))
    E[0, 0], E[-1, -1] = -1, 1
    assert np.abs(S + 0.5 * E - Q).max() < 1e-13


def _setup(p, kx, ky, kz, Re=1600.0):
    return nat.Setup(p, kx, ky, kz, 1.4, 0.72, 0.1, Re, 1, 0)


@pytest.mark.parametrize("p,warp", [(2, 0.0), (3, 0.1), (4, 0.1), (7, 0.1), (15, 0.1)])
def test_host_geometry_matches_oracle(L, p, warp):
    k = (3, 2, 2)
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), *k, [-math.pi] * 3, [math.pi] * 3, warp=warp, seed=0)
    K, N3 = x.shape[0], (p + 1) ** 3
    J, Ja, h = np.zeros((K, N3)), np.zeros((K, 9, N3)), ctypes.c_double()
    st = _setup(p, *k)
    nat.check(L.esdc_host_geometry(ctypes.byref(st), np.ascontiguousarray(x).ctypes.data, J.ctypes.data,
                                   Ja.ctypes.data, ctypes.byref(h)), "geometry")
    m = O.make_mesh(p, x, *k)
    Jo = m.J.numpy().reshape(K, N3)
    Jao = m.Ja.numpy().reshape(K, 9, N3)
    # the curl form applies D twice: round-off grows like p^2 up to p = 7 and like |D|^2 beyond, with
    # |D| = p(p+1)/4 (the two sides' D differ by a few ulps of |D|; both are float64)
    tol = 1e-14 * p * p if p <= 7 else 16 * 2.2e-16 * (p * (p + 1) / 4) ** 2
    assert np.abs(J - Jo).max() < tol * np.abs(Jo).max()
    assert np.abs(Ja - Jao).max() < tol * np.abs(Jao).max()
    assert abs(h.value - m.h_min) < 1e-14 * m.h_min


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7])
def test_host_optimized_metrics_match_oracle(L, p):
    """The library's optimized metrics (Sec. 3; solved by fast diagonalisation of the Gram matrix of
    the GCL constraint) against the oracle's (dense pseudo-inverse), volume and surface metrics."""
    k = (3, 2, 2)
    s = O.sbp_operator(p)
    x = np.ascontiguousarray(I.box_coords(s.xi.numpy(), *k, [-math.pi] * 3, [math.pi] * 3, warp=0.1, seed=0))
    K, N = x.shape[0], p + 1
    N2, N3 = N * N, N ** 3
    st = _setup(p, *k)
    st.metrics = 1
    J, Ja, ns = np.zeros((K, N3)), np.zeros((K, 9, N3)), np.zeros((K, 6, 3, N2))
    nat.check(L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, J.ctypes.data, Ja.ctypes.data, None), "geometry")
    nat.check(L.esdc_host_surface_metrics(ctypes.byref(st), x.ctypes.data, ns.ctypes.data), "surface")
    m = O.make_mesh(p, x, *k, metrics="optimized")
    Jao = m.Ja.numpy().reshape(K, 9, N3)
    nso = np.stack([O.face(m.Ja_face[:, l], l, side).numpy().reshape(K, 3, N2) for l in range(3) for side in (0, 1)],
                   axis=1)
    scale = np.abs(Jao).max()
    assert np.abs(Ja - Jao).max() < 1e-14 * p * p * scale
    assert np.abs(ns - nso).max() < 1e-14 * p * p * scale
    assert np.abs(J - m.J.numpy().reshape(K, N3)).max() < 1e-14 * p * p * np.abs(J).max()
    # the curl-form context reports the face values of its volume metrics as its surface metrics
    st.metrics = 0
    nat.check(L.esdc_host_surface_metrics(ctypes.byref(st), x.ctypes.data, ns.ctypes.data), "surface")
    mc = O.make_mesh(p, x, *k)
    ncurl = np.stack([O.face(mc.Ja[:, l], l, side).numpy().reshape(K, 3, N2) for l in range(3) for side in (0, 1)],
                     axis=1)
    assert np.abs(ns - ncurl).max() < 1e-14 * p * p * scale


def test_argument_errors(L):
    xi = np.zeros(17)
    assert L.esdc_lgl(0, xi.ctypes.data, xi.ctypes.data) == nat.ESDC_ERR_ARG
    assert L.esdc_lgl(16, xi.ctypes.data, xi.ctypes.data) == nat.ESDC_ERR_ARG
    assert L.esdc_lgl(3, None, xi.ctypes.data) == nat.ESDC_ERR_ARG
    x = I.box_coords(O.sbp_operator(2).xi.numpy(), 2, 2, 2, [0] * 3, [1] * 3)
    bad = _setup(2, 2, 2, 2)
    bad.gamma = 1.0
    assert L.esdc_host_geometry(ctypes.byref(bad), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    bad = _setup(2, 0, 2, 2)
    assert L.esdc_host_geometry(ctypes.byref(bad), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    out = ctypes.c_void_p()
    assert L.esdc_create(None, x.ctypes.data, ctypes.byref(out)) == nat.ESDC_ERR_ARG
    assert L.esdc_rhs(None, None, None, None) == nat.ESDC_ERR_ARG
    assert b"null" in L.esdc_last_error()


def test_inverted_mesh_rejected(L):
    """A mesh whose elements are mirrored (J < 0) is refused at setup with ESDC_ERR_MESH."""
    p = 2
    x = I.box_coords(O.sbp_operator(p).xi.numpy(), 2, 2, 2, [0] * 3, [1] * 3)
    x = np.ascontiguousarray(x[..., ::-1])       # reverse xi1 inside every element
    st = _setup(p, 2, 2, 2)
    assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_MESH
    out = ctypes.c_void_p()
    assert L.esdc_create(ctypes.byref(st), x.ctypes.data, ctypes.byref(out)) == nat.ESDC_ERR_MESH
    assert out.value is None


def test_strerror(L):
    for c in (0, -1, -2, -3, -4, -5):
        assert len(L.esdc_strerror(c)) > 0


def test_empty_and_out_of_range_sizes(L):
    """No elements, too many elements and degrees outside 1..7 are refused before any allocation."""
    x = np.zeros((1, 3, 2, 2, 2))
    for kx, ky, kz in ((0, 1, 1), (1, 0, 1), (1, 1, -3), (2 ** 20, 2 ** 10, 1)):
        st = _setup(1, kx, ky, kz)
        assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    for p in (0, 16, -1):
        st = _setup(p, 1, 1, 1)
        assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    for p in (8, 14):      # between the per-element kernels (p <= 7) and the p = 15 passes
        st = _setup(p, 1, 1, 1)
        assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_UNSUPPORTED
    st = _setup(15, 1, 1, 1)
    for field, val in (("precision", nat.PREC_FP32), ("dissipation", 2), ("ip_coef", 1.0), ("bounded", 1),
                       ("metrics", 1)):
        bad = _setup(15, 1, 1, 1)
        setattr(bad, field, val)
        assert L.esdc_host_geometry(ctypes.byref(bad), x.ctypes.data, None, None, None) == nat.ESDC_ERR_UNSUPPORTED
    st = _setup(1, 1, 1, 1)
    st.precision = 2
    assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    st = _setup(1, 1, 1, 1)
    st.metrics = 2
    assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_ARG
    st.metrics = 1
    st.precision = nat.PREC_FP32
    # float32 with the optimized metrics passes the setup checks (the all-zero nodes then fail as a mesh)
    assert L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, None, None, None) == nat.ESDC_ERR_MESH
    assert L.esdc_host_surface_metrics(ctypes.byref(st), x.ctypes.data, None) == nat.ESDC_ERR_ARG


def test_single_element_and_p1_geometry(L):
    """Degenerate but valid: one element periodic onto itself, p = 1 (two nodes per direction)."""
    s = O.sbp_operator(1)
    x = np.ascontiguousarray(I.box_coords(s.xi.numpy(), 1, 1, 1, [0] * 3, [2] * 3))
    J = np.zeros((1, 8))
    st = _setup(1, 1, 1, 1)
    nat.check(L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, J.ctypes.data, None, None), "geometry")
    assert np.allclose(J, 1.0)


@pytest.mark.parametrize("p", [7, 15])
def test_high_degree_operators_within_ulps_of_40_digit_reference(L, p):
    """The library's and the oracle's collocation derivatives, each built in its own way (closed form
    in long double; barycentric weights in float64), are both within a few ulps of |D| of D computed
    in 40-digit arithmetic on the exact LGL nodes: their metric terms differ only by round-off."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    N = p + 1
    xi = np.zeros(N)
    w = np.zeros(N)
    D = np.zeros(N * N)
    nat.check(L.esdc_lgl(p, xi.ctypes.data, w.ctypes.data), "lgl")
    nat.check(L.esdc_operators(p, D.ctypes.data, None), "ops")
    dP = lambda t: mp.diff(lambda u: mp.legendre(p, u), t)
    x = [mp.mpf(-1)] + [mp.findroot(dP, mp.mpf(float(xi[i]))) for i in range(1, p)] + [mp.mpf(1)]
    lam = [mp.mpf(1)] * N
    for j in range(N):
        for k in range(N):
            if k != j:
                lam[j] /= x[j] - x[k]
    ref = np.zeros((N, N))
    for i in range(N):
        acc = mp.mpf(0)
        for j in range(N):
            if i != j:
                v = (lam[j] / lam[i]) / (x[i] - x[j])
                ref[i, j] = float(v)
                acc += v
        ref[i, i] = float(-acc)
    scale = np.abs(ref).max() * 2.2e-16
    assert np.abs(D.reshape(N, N) - ref).max() <= 8 * scale
    assert np.abs(O.sbp_operator(p).D.numpy() - ref).max() <= 8 * scale


@pytest.mark.parametrize("p,k,warp,seed", [(2, (3, 2, 4), 0.0, 0), (3, (2, 3, 2), 0.1, 7), (4, (2, 2, 2), 0.15, 2 ** 63 + 5)])
def test_box_generator_matches_inputs(L, p, k, warp, seed):
    """esdc_host_coordinates (the generator behind node_xyz = NULL) equals the input module's box mesh
    with the same splitmix64 phases; geometry from NULL coordinates equals geometry from those nodes."""
    xi = O.sbp_operator(p).xi.numpy()
    lo, hi = [-1.0, 0.0, 2.0], [1.0, 3.0, 2.5]
    st = _setup(p, *k)
    st.lo[:] = lo
    st.hi[:] = hi
    st.warp_amp = warp
    st.warp_seed = seed
    K, N3 = k[0] * k[1] * k[2], (p + 1) ** 3
    x = np.zeros((K, 3, p + 1, p + 1, p + 1))
    nat.check(L.esdc_host_coordinates(ctypes.byref(st), x.ctypes.data), "coordinates")
    want = I.box_coords(xi, *k, lo, hi, warp=warp, phases=I.splitmix64_phases(seed))
    assert np.abs(x - want).max() <= 4e-16 * np.abs(want).max()
    J1, J2 = np.zeros((K, N3)), np.zeros((K, N3))
    nat.check(L.esdc_host_geometry(ctypes.byref(st), None, J1.ctypes.data, None, None), "geometry")
    nat.check(L.esdc_host_geometry(ctypes.byref(st), x.ctypes.data, J2.ctypes.data, None, None), "geometry")
    assert np.array_equal(J1, J2)
    bad = _setup(p, *k)
    bad.lo[:] = lo
    bad.hi[:] = [1.0, 3.0, 2.0]          # hi == lo in x3
    assert L.esdc_host_coordinates(ctypes.byref(bad), x.ctypes.data) == nat.ESDC_ERR_ARG
    bad.hi[:] = hi
    bad.warp_amp = -0.1
    assert L.esdc_host_geometry(ctypes.byref(bad), None, None, None, None) == nat.ESDC_ERR_ARG


def test_splitmix64_published_values():
    """First outputs of splitmix64 from seed 0 as published with the reference implementation
    (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4), checked through the phase mapping."""
    ph = I.splitmix64_phases(0)
    for z, got in ((0xE220A8397B1DCDAF, ph[0, 0]), (0x6E789E6AA1B965F4, ph[0, 1])):
        assert got == float(z >> 11) * 2.0 ** -53 * (2.0 * math.pi)
