"""Pins of the oracle's field off the boundary (oracle/field.py): the
representation formula applied to the oracle's own marched solution
approaches the closed-form exterior field of a sphere of radius a = 1
(c = 1) under refinement (80 -> 320 elements):

- uniform Dirichlet data u = f(t): u(r, t) = (a/r) f(t - (r - a)/c);
- uniform Neumann data du/dr = f: u(r, t) = (a/r) F(t - (r - a)/c) with F'
  = -c (f + F/a), F(0) = 0 (the surface value).

The opposite overall sign of the formula gives an error near 2, so the
sign convention is pinned too."""

import numpy as np
from scipy.integrate import solve_ivp

from oracle import field, mot
from synth import workload

PTS = np.array([[1.5, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, -3.0]])


def _err(name):
    w = workload(name, nt=64)
    u, q = mot.march(w)
    al = list(range(4, 63, 3))
    t = np.array(al) * w.dt
    F = field.field(w, u, q, PTS, al)
    r = np.linalg.norm(PTS, axis=1)
    tr = t[:, None] - (r[None, :] - 1.0)
    if w.bc == "dirichlet":
        ref = (1.0 / r)[None, :] * mot.gauss(tr, w.sigma, 4 * w.sigma)
    else:
        sol = solve_ivp(lambda tt, Fv: -(mot.gauss(tt, w.sigma, 4 * w.sigma) + Fv), (0, t[-1]), [0.0],
                        dense_output=True, rtol=1e-12, atol=1e-14)
        ref = (1.0 / r)[None, :] * np.where(tr > 0, sol.sol(np.maximum(tr, 0).ravel())[0].reshape(tr.shape), 0.0)
    return np.linalg.norm(F - ref) / np.linalg.norm(ref), np.linalg.norm(-F - ref) / np.linalg.norm(ref)


def test_field_of_sphere_dirichlet_converges():
    # measured 0.33 and 0.15 (BMBIE d = 1; OBIE Dirichlet is unstable on the coarse mesh)
    e80, _ = _err("sphere80_bmbie_d1_dirichlet_uniform")
    e320, flip = _err("sphere320_bmbie_d1_dirichlet_uniform")
    assert e320 < 0.2 and e320 < 0.6 * e80, (e80, e320)
    assert flip > 1.5


def test_field_of_sphere_neumann_converges():
    # measured 0.089 and 0.023
    e80, _ = _err("sphere80_obie_d1_neumann_uniform")
    e320, flip = _err("sphere320_obie_d1_neumann_uniform")
    assert e320 < 0.04 and e320 < 0.4 * e80, (e80, e320)
    assert flip > 1.5
