"""Pins of the oracle's influence coefficients.

Each check compares the oracle with something other than itself:
- lag sums of the compact coefficients against textbook closed forms of
  static potentials (the partition of unity and discrete moments of the
  B-spline turn sums over g into static integrals);
- gradients and time derivatives of those sums against finite differences
  of the closed forms;
- the paper's closed forms I_n^d (Appendix B) for the tau-form kernel and
  the identity C^(g) = sum_k w^{k,d} U^(g-k) (Section 2.4);
- brute-force 2-D quadrature on cases where the element lies inside one
  knot interval of the retarded time (smooth integrand);
- the free term (self element: C_W^(g) = N(g)/2), rotation/translation
  invariance, and that no adaptive integral stopped on its panel budget.
"""

import numpy as np
import pytest

from oracle import coeffs as oc
from tests.closed_forms import appb_U, slp_static, solid_angle

TRI = np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.3, 0.9, 0.0])
NG = np.array([0.0, 0.0, 1.0])  # (v1 - v0) x (v2 - v0) direction; the paper's normal is -NG
AREA = 0.45
CDT = 0.2
POINTS = [
    (np.array([0.4, 0.3, 0.25]), False),   # above, foot inside
    (np.array([1.5, -0.7, -0.4]), False),  # below, foot outside
    (np.array([0.2, 1.1, 0.05]), False),   # close to the plane, foot outside
    (np.array([0.43, 0.3, 0.0]), True),    # on the element (self)
]
M = {1: 1.0, 2: 1.5, 3: 2.0}  # (d+1)/2


def _window(x, d):
    rmin, rmax = oc.tri_dist(x, TRI)
    return range(max(1, int(np.floor(rmin / CDT)) + 1), int(np.ceil(rmax / CDT + d + 1)))


def _omega_p(x):
    """Solid angle with the sign of the paper's normal (-NG)."""
    return solid_angle(x, TRI)


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pt", range(len(POINTS)))
def test_lag_sums_match_static_closed_forms(d, pt):
    x, self_ = POINTS[pt]
    gs = list(_window(x, d))
    C = np.array([oc.coef(x, -NG, TRI, g, d, CDT, self_=self_, bm=False) for g in gs])
    slp = slp_static(x, TRI)
    # sum_g N(g - r) = 1  ->  sum_g C_U^(g) = (1/4pi) int dS/r
    assert C[:, 0].sum() == pytest.approx(slp / (4 * np.pi), rel=1e-13, abs=1e-15)
    # sum_g g N(g - r) = r + (d+1)/2
    m1 = (np.array(gs) * C[:, 0]).sum()
    assert m1 == pytest.approx((AREA / CDT + M[d] * slp) / (4 * np.pi), rel=1e-13, abs=1e-15)
    # double layer: solid angle (+1/2 on the element, the free term)
    om = 2 * np.pi if self_ else _omega_p(x)
    assert C[:, 1].sum() == pytest.approx(om / (4 * np.pi), rel=1e-13, abs=1e-15)
    if d >= 2:
        # sum_g g^2 C_W = ((m^2 + v) Omega - z int dS/r) / (4 pi), z along the paper normal
        z = 0.0 if self_ else -(NG @ (x - TRI[:3]))
        m2 = (np.array(gs) ** 2 * C[:, 1]).sum()
        ref = ((M[d] ** 2 + (d + 1) / 12.0) * om - (z / CDT) * (slp / CDT)) / (4 * np.pi)
        assert m2 == pytest.approx(ref, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("pt", [0, 1, 2])
def test_gradient_and_time_derivative_sums(d, pt):
    x, _ = POINTS[pt]
    gs = list(_window(x, d))
    P = np.array([oc.coef_parts(x, TRI, g, d, CDT) for g in gs])
    h = 1e-5
    gslp = np.array([(slp_static(x + h * e, TRI) - slp_static(x - h * e, TRI)) / (2 * h) for e in np.eye(3)])
    gom = np.array([(_omega_p(x + h * e) - _omega_p(x - h * e)) / (2 * h) for e in np.eye(3)])
    # normalised units: grad_hat = c dt grad
    assert np.allclose(P[:, 4:7].sum(0), gslp / (4 * np.pi), rtol=1e-8, atol=1e-10)
    assert np.allclose(P[:, 7:10].sum(0), CDT * gom / (4 * np.pi), rtol=1e-8, atol=1e-10)
    g = np.array(gs, dtype=float)
    slp = slp_static(x, TRI)
    # sum_g g N'(g - r) = -1
    assert (g * P[:, 2]).sum() == pytest.approx(-slp / (4 * np.pi * CDT), rel=1e-12, abs=1e-14)
    assert (g * P[:, 3]).sum() == pytest.approx(-_omega_p(x) / (4 * np.pi), rel=1e-12, abs=1e-14)
    assert P[:, 2].sum() == pytest.approx(0.0, abs=1e-13)


@pytest.mark.parametrize("d", [1, 2])
def test_hypersingular_self_term_sum(d):
    # sum over lags of d/dz Chat_W on the element equals the finite part of
    # d/dz of the solid angle, continuous across the element
    x = np.array([0.43, 0.3, 0.0])
    npap = -NG
    gs = list(_window(x, d))
    s = sum(npap @ oc.coef_parts(x, TRI, g, d, CDT, self_=True)[7:10] for g in gs)
    h = 1e-4
    a = (_omega_p(x + h * npap) - _omega_p(x - h * npap) - 4 * np.pi) / (2 * h)
    assert s == pytest.approx(CDT * a / (4 * np.pi), rel=1e-6)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_free_term(d):
    # N^{0,d} at the integer knots (Cox-de Boor values)
    knots = {1: [1.0], 2: [0.5, 0.5], 3: [1 / 6, 2 / 3, 1 / 6]}[d]
    x = np.array([0.43, 0.3, 0.0])
    for g, nv in enumerate(knots, start=1):
        assert oc.coef(x, -NG, TRI, g, d, CDT, self_=True)[1] == pytest.approx(nv / 2, abs=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tau_form_against_appendix_b(d):
    # x above the element with the element wholly inside the sphere r < c t_g
    x = np.array([0.4, 0.3, 0.25])
    for g in (8, 11):
        ref = appb_U(x, TRI, g, d, CDT)
        assert oc.coef_tau(x, TRI, g, d, CDT)[0] == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_compact_equals_kappa_sum_of_tau_form(d):
    for x, self_ in POINTS:
        for g in _window(x, d):
            c = oc.coef(x, -NG, TRI, g, d, CDT, self_=self_, bm=False)
            tu = sum(oc.w(k, d) * oc.coef_tau(x, TRI, g - k, d, CDT, self_=self_)[0]
                     for k in range(d + 2) if g - k > 0)
            tw = sum(oc.w(k, d) * oc.coef_tau(x, TRI, g - k, d, CDT, self_=self_)[1]
                     for k in range(d + 2) if g - k > 0)
            scale = max(abs(oc.coef_tau(x, TRI, g, d, CDT, self_=self_)).max(), 1e-3)
            assert c[0] == pytest.approx(tu, abs=1e-12 * scale)
            assert c[1] == pytest.approx(tw, abs=1e-12 * scale)


def _gauss_triangle(f, v, n=14, sub=3):
    """Brute-force quadrature of a smooth f over the triangle (tensor
    Gauss-Legendre on the collapsed square of each of 4**sub sub-triangles)."""
    v = np.asarray(v).reshape(3, 3)
    xs, ws = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (xs + 1)
    wu = 0.5 * ws
    tris = [v]
    for _ in range(sub):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]), np.array([ab, bc, ca])]
        tris = nxt
    tot = 0.0
    for a, b, c in tris:
        J = np.linalg.norm(np.cross(b - a, c - a))
        for i in range(n):
            for j in range(n):
                s, t = u[i], u[j] * (1 - u[i])
                y = a + s * (b - a) + t * (c - a)
                tot += wu[i] * wu[j] * (1 - u[i]) * J * f(y)
    return tot


@pytest.mark.parametrize("d", [1, 2])
def test_single_piece_brute_force(d):
    # element inside one knot interval of g - r: smooth integrand
    x = np.array([3.0, 2.5, 1.7])
    v = TRI * 0.05 + np.array([0.1, 0.2, 0.0] * 3)
    cdt = 0.5
    r = np.linalg.norm(v.reshape(3, 3) - x / 1.0, axis=1) / cdt
    g = int(np.floor(r.max())) + 1 + 0  # (g - r) in (0, 1) over the element? choose first piece
    assert np.floor(g - r.max()) == np.floor(g - r.min())
    npap = -NG
    for gg in (g, g + 1):
        P = oc.coef_parts(x, v, gg, d, cdt)

        def fu(y):
            rr = np.linalg.norm(x - y) / cdt
            return oc.N(d, gg - rr) / rr

        def fw(y):
            rr = np.linalg.norm(x - y) / cdt
            zz = (npap @ (x - y)) / cdt
            return zz * (oc.N(d, gg - rr) / rr ** 3 + oc.dN(d, gg - rr) / rr ** 2)

        def fdu(y):
            rr = np.linalg.norm(x - y) / cdt
            return oc.dN(d, gg - rr) / rr

        # dS_hat = dS / cdt^2
        assert P[0] == pytest.approx(_gauss_triangle(fu, v) / cdt ** 2 / (4 * np.pi), rel=1e-12)
        assert P[1] == pytest.approx(_gauss_triangle(fw, v) / cdt ** 2 / (4 * np.pi), rel=1e-12)
        assert P[2] == pytest.approx(_gauss_triangle(fdu, v) / cdt ** 2 / (4 * np.pi), rel=1e-12)


def test_rotation_translation_invariance():
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    t = rng.normal(size=3)
    for x, self_ in POINTS[:3]:
        nx = np.array([0.3, -0.4, 0.866])
        nx /= np.linalg.norm(nx)
        vt = (TRI.reshape(3, 3) @ Q.T + t).reshape(9)
        for g in list(_window(x, 2))[:4]:
            a = oc.coef(x, nx, TRI, g, 2, CDT, self_=self_)
            b = oc.coef(Q @ x + t, Q @ nx, vt, g, 2, CDT, self_=self_)
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_no_budget_stops():
    assert oc.budget_hits() == 0
