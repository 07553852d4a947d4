"""Pins of the oracle's time marching.

- The sphere of radius a with uniform Dirichlet data u = f(t) radiates
  u(r, t) = (a/r) f(t - (r-a)/c), so q = du/dn (n into the sphere) is
  f/a + f'/c on the surface; with uniform Neumann data du/dr = f the surface
  value F solves F' = -c (f + F/a), F(0) = 0.  The discrete solutions on
  icospheres approach these at the discretisation rate (not to rounding).
- The compact form equals the paper's literal tau-form marching (Eq.
  bie_disc3, Eq. tau, Eq. sigma, Eq. linear) up to rounding.
- The plane-wave RHS obeys the Burton-Miller operator identity on a smooth
  field.
"""

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import coeffs as oc
from oracle import mot
from synth import workload


def _values_at_collocation(X, d, nt):
    Nv = [oc.N(d, g) for g in range(d + 2)]
    vals = np.zeros((nt, X.shape[1]))
    for a in range(1, nt):
        for g in range(1, d + 1):
            if 0 <= a - g < X.shape[0]:
                vals[a] += Nv[g] * X[a - g]
    return vals


def _sphere_error(name):
    w = workload(name)
    u, q = mot.march(w)
    X = q if w.bc == "dirichlet" else u
    vals = _values_at_collocation(X, w.d, w.nt)
    ts = np.arange(w.nt) * w.dt
    f = mot.gauss(ts, w.sigma, 4 * w.sigma)
    if w.bc == "dirichlet":
        ref = f + mot.dgauss(ts, w.sigma, 4 * w.sigma)  # a = c = 1
    else:
        sol = solve_ivp(lambda t, F: -(mot.gauss(t, w.sigma, 4 * w.sigma) + F), (0, ts[-1]), [0.0],
                        t_eval=ts, rtol=1e-12, atol=1e-14)
        ref = sol.y[0]
    ref = np.repeat(ref[:, None], w.ns, axis=1)
    return np.linalg.norm(vals[1:] - ref[1:]) / np.linalg.norm(ref[1:])


@pytest.mark.parametrize("name,bound", [
    ("sphere320_obie_d1_dirichlet_uniform", 0.06),
    ("sphere320_obie_d1_neumann_uniform", 0.02),
    ("sphere320_bmbie_d2_neumann_uniform", 0.20),
    ("sphere320_bmbie_d1_dirichlet_uniform", 0.25),
])
def test_sphere_closed_form(name, bound):
    assert _sphere_error(name) < bound


def test_sphere_refinement_reduces_error():
    # coarse (80) vs 320 elements, BMBIE d=1 Dirichlet: error must drop
    e80 = _sphere_error("sphere80_bmbie_d1_dirichlet_uniform")
    e320 = _sphere_error("sphere320_bmbie_d1_dirichlet_uniform")
    assert e320 < 0.7 * e80


def test_sphere_refinement_bmbie_d2_neumann():
    """The benchmark's formulation (Burton-Miller, d = 2, Neumann) against the
    closed-form sphere on 80 -> 320 -> 1280 elements (c dt = half the mean
    edge): the error must fall at the discretisation rate, by more than 2x
    per refinement (measured 0.476 -> 0.174 -> 0.051).  A wrong sign or
    factor in the hypersingular or the time-derivative part of the
    Burton-Miller kernels leaves an error that does not shrink."""
    e = [_sphere_error("sphere%d_bmbie_d2_neumann_uniform" % ns) for ns in (80, 320, 1280)]
    assert e[1] < 0.45 * e[0] and e[2] < 0.45 * e[1], e
    assert e[2] < 0.07, e


@pytest.mark.parametrize("name", ["sphere80_obie_d1_dirichlet_uniform", "sphere80_obie_d2_neumann_uniform"])
def test_compact_equals_tau_form(name):
    w = workload(name, nt=24)
    u1, q1 = mot.march(w)
    u2, q2 = mot.march_tau(w)
    for a, b in ((u1, u2), (q1, q2)):
        assert np.linalg.norm(a - b) <= 1e-12 * max(np.linalg.norm(b), 1e-300)


def test_bm_incident_operator():
    # (d/dn - c^-1 d/dt) of the plane pulse by finite differences
    w = workload("ellipsoid80_bmbie_d2_hard_plane_s7")
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    a = 40
    e = mot.incident_rhs(w, xc, n, a)
    h = 1e-5
    t = a * w.dt

    def uin(x, t):
        return mot.gauss(t - (x @ w.direction) / w.c, w.sigma, w.t0)

    fd = (uin(xc + h * n, t) - uin(xc - h * n, t)) / (2 * h) - (uin(xc, t + h) - uin(xc, t - h)) / (2 * h) / w.c
    assert np.allclose(e, fd, atol=1e-8)


def test_raised_cosine_pulse():
    """The pulse of Section 5.1.1: zero outside 0 <= c t - x_1 <= Lambda,
    peak 1 at the middle, area Lambda / (2c) in time, C^1 at both ends, and
    the Burton-Miller right-hand side (d/dn - c^-1 d/dt) u_in by finite
    differences on the paper-shaped sphere."""
    L, c = 0.5, 1.0
    t = np.linspace(-1.0, 2.0, 300001)
    f = mot.raised_cosine(t, L, c, 0.0)
    assert np.all(f[(t < 0) | (t > L / c)] == 0.0)
    assert abs(mot.raised_cosine(np.array([L / (2 * c)]), L, c, 0.0)[0] - 1.0) < 1e-15
    assert abs(np.trapezoid(f, t) - L / (2 * c)) < 1e-9
    h = 1e-7
    for edge in (0.0, L / c):
        assert abs(mot.draised_cosine(np.array([edge]), L, c, 0.0)[0]) < 1e-12
        fd = (mot.raised_cosine(np.array([edge + h]), L, c, 0.0) - mot.raised_cosine(np.array([edge - h]), L, c, 0.0)) / (2 * h)
        assert abs(fd[0]) < 1e-5
    w = workload("paper_sphere80_bmbie_d2_hard")
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    for a in (1, 2, 3):
        e = mot.incident_rhs(w, xc, n, a)
        tt = a * w.dt

        def uin(x, t):
            return mot.raised_cosine(t - (x @ w.direction) / w.c, w.sigma, w.c, w.t0)

        hh = 1e-6
        fd = (uin(xc + hh * n, tt) - uin(xc - hh * n, tt)) / (2 * hh) - (uin(xc, tt + hh) - uin(xc, tt - hh)) / (2 * hh) / w.c
        # atol: central differences across the support's ends, where the
        # pulse's second derivative jumps (O(h f''))
        assert np.allclose(e, fd, atol=1e-4)
        assert np.abs(e).max() > 0.1
