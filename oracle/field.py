"""The field off the boundary (oracle, TEST INFRASTRUCTURE ONLY).

Plain restatement of the representation formula of the exterior problem
(Section 2.1; Eq. bie is its limit on S), discretised like the boundary
equation (Section 2.4, compact form): at a point x of the exterior domain
and step alpha,

    u(x, t_alpha) = u_in(x, t_alpha)
                  + sum_j sum_{g=1}^{alpha} ( C_U^(g)(x, E_j) q_j^{alpha-g}
                                             - C_W^(g)(x, E_j) u_j^{alpha-g} ),

with the same compact coefficients as on the boundary (oracle.coeffs.coef,
x not on S, so no self term) and the B-spline coefficient histories u, q
of the march.  u_in is the plane pulse of the workload (zero for the
"uniform" workloads).  The overall sign is the one that turns the boundary
equation of the library (0 = e + sum (C_U q - C_W u)) into the extinction
of the total field inside V; it is pinned by the closed-form field of a
sphere (tests/test_oracle_field.py).
"""

import numpy as np

from . import coeffs as oc
from . import mot


def incident(w, points, alpha):
    if w.excitation != "plane":
        return np.zeros(len(points))
    t = alpha * w.dt
    k = np.asarray(w.direction, dtype=np.float64)
    xi = t - (np.asarray(points) @ k) / w.c
    if getattr(w, "shape", 0) == 1:
        return mot.raised_cosine(xi, w.sigma, w.c, w.t0)
    return mot.gauss(xi, w.sigma, w.t0)


def field(w, u, q, points, alphas):
    """u(x_p, t_alpha) for every point and step: [len(alphas), len(points)].
    u, q: coefficient histories [>= max(alphas), ns] (row beta)."""
    cdt = w.c * w.dt
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    ns = xc.shape[0]
    points = np.asarray(points, dtype=np.float64)
    amax = max(alphas)
    out = np.zeros((len(alphas), len(points)))
    zero = np.zeros(3)
    for pi, x in enumerate(points):
        # coefficients of every element at every lag up to amax
        CU = np.zeros((amax + 1, ns))
        CW = np.zeros((amax + 1, ns))
        for j in range(ns):
            rmin, rmax = oc.tri_dist(x, v[j])
            g0 = max(1, int(np.floor(rmin / cdt)) + 1)
            g1 = min(amax, int(np.ceil(rmax / cdt + w.d + 1)) - 1)
            for g in range(g0, g1 + 1):
                c = oc.coef(x, zero, v[j], g, w.d, cdt, self_=False, bm=False)
                CU[g, j], CW[g, j] = c[0], c[1]
        for ai, a in enumerate(alphas):
            s = 0.0
            for g in range(1, a + 1):
                s += CU[g] @ q[a - g] - CW[g] @ u[a - g]
            out[ai, pi] = incident(w, x[None, :], a)[0] + s
    return out
