"""Marching-on-in-time with the direct (no FMM) history sum (oracle).

TEST INFRASTRUCTURE ONLY.  Plain numpy restatement of the time marching of
Section 2.4-2.5 in the compact form (the kappa-sum of Eq. discretised_*
folded into the coefficients by the identity below Eq. bie_disc):

    0 = e_i(t_alpha) + sum_j sum_{beta=0}^{alpha-1}
            ( C_U^(alpha-beta)_ij q_j^beta - C_W^(alpha-beta)_ij u_j^beta )

for alpha = 1 .. Nt-1 (OBIE, Eq. bie_disc, total field with the incident
term e = u_in), or the same with the Burton-Miller coefficients Ubar, Wbar
and e = (d/dn_x - c^-1 d/dt) u_in (BMBIE, Eq. bmbie, Eq. U_W_BM).  At each
alpha the unknowns x^{alpha-1} (u_j where phi_j = 1, q_j where phi_j = 0)
solve the zero-lag system of Eq. linear,

    A x^{alpha-1} = b^{alpha-1},  A_ij = C_U^(1)_ij (1 - phi_j) - C_W^(1)_ij phi_j,

with every known term moved to b (the tilde variables of Eq.
sigma_tau_tilde: the unknown components of the current step are zero in
the history sum).  A is factorised once (dense LU) and reused.

Normals and q follow the paper: n points into the scatterer V and q is the
derivative of u along it.
"""

import numpy as np
import scipy.linalg

from . import coeffs as oc


# ----------------------------------------------------------------------
# excitation (Section 5.1.1 shape: plane pulse; Gaussian profile)
# ----------------------------------------------------------------------

def gauss(t, sigma, t0):
    return np.exp(-(((t - t0) / sigma) ** 2))


def dgauss(t, sigma, t0):
    s = (t - t0) / sigma
    return -2.0 * s / sigma * np.exp(-s * s)


def raised_cosine(t, length, c, t0):
    """The pulse of Section 5.1.1 (Eq. uin) as a function of time at a fixed
    point: 0.5 (1 - Cos(2 pi c (t - t0) / length)), where Cos is the cosine on
    [0, 2 pi] and 1 elsewhere."""
    x = 2.0 * np.pi * c * (np.asarray(t, dtype=np.float64) - t0) / length
    return np.where((x >= 0.0) & (x <= 2.0 * np.pi), 0.5 * (1.0 - np.cos(x)), 0.0)


def draised_cosine(t, length, c, t0):
    x = 2.0 * np.pi * c * (np.asarray(t, dtype=np.float64) - t0) / length
    return np.where((x >= 0.0) & (x <= 2.0 * np.pi), 0.5 * np.sin(x) * 2.0 * np.pi * c / length, 0.0)


def incident_rhs(w, xc, n, alpha):
    """e_i(t_alpha): u_in (OBIE) or (d/dn_x - c^-1 d/dt) u_in (BMBIE) at the
    collocation points, for the plane pulse u_in = g(t - t0 - k.x/c), g the
    Gaussian of width sigma (w.shape 0) or the raised cosine of length sigma
    (w.shape 1)."""
    t = alpha * w.dt
    k = np.asarray(w.direction, dtype=np.float64)
    xi = t - (k @ xc.T) / w.c  # argument shifted by t0 inside g
    if getattr(w, "shape", 0) == 1:
        g, dg = raised_cosine(xi, w.sigma, w.c, w.t0), draised_cosine(xi, w.sigma, w.c, w.t0)
    else:
        g, dg = gauss(xi, w.sigma, w.t0), dgauss(xi, w.sigma, w.t0)
    if w.bie == "obie":
        return g
    # d/dn_x g(t - t0 - k.x/c) = -(k.n / c) g';  c^-1 d/dt g = g' / c
    return -(1.0 + n @ k) / w.c * dg


def known_coefficients(w, nt):
    """B-spline coefficients of prescribed uniform data f(t) = g(t; sigma,
    4 sigma) by collocation at t_alpha, alpha = 1..Nt-1:
    sum_{gamma=1}^{d} N(gamma) fbar^{alpha-gamma} = f(t_alpha)."""
    d = w.d
    Nv = [oc.N(d, float(g)) for g in range(d + 2)]
    f = gauss(np.arange(nt) * w.dt, w.sigma, 4.0 * w.sigma)
    fb = np.zeros(nt)
    for a in range(1, nt):
        s = f[a]
        for g in range(2, d + 1):
            if a - g >= 0:
                s -= Nv[g] * fb[a - g]
        fb[a - 1] = s / Nv[1]
    return fb


def coefficient_kinds(w):
    """Kinds of coefficients the run needs."""
    if w.bie == "obie":
        ku, kw = "cu", "cw"
    else:
        ku, kw = "ub", "wb"
    if w.excitation == "plane":
        return (ku,) if w.bc == "dirichlet" else (kw,)
    return (ku, kw)


def march(w, C=None, nt=None):
    """Run the MOT.  ``C``: dict of dense coefficient arrays [gmax+1, ns, ns]
    (computed here if None).  Returns (u, q), each [Nt-1, ns] holding the
    B-spline coefficients beta = 0..Nt-2."""
    nt = w.nt if nt is None else int(nt)
    cdt = w.c * w.dt
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    ns = xc.shape[0]
    if C is None:
        C = oc.dense(w.xyz, w.tri, w.d, cdt, kinds=coefficient_kinds(w))
    ku, kw = ("cu", "cw") if w.bie == "obie" else ("ub", "wb")
    CU = C.get(ku)
    CW = C.get(kw)
    gmax = (CU if CU is not None else CW).shape[0] - 1
    phi = np.ones(ns) if w.bc == "neumann" else np.zeros(ns)

    # known data (B-spline coefficients) per step
    ubar = np.zeros((nt, ns))
    qbar = np.zeros((nt, ns))
    if w.excitation == "uniform":
        fb = known_coefficients(w, nt)
        if w.bc == "dirichlet":
            ubar[:] = fb[:, None]
        else:
            # prescribed du/dr = f on a sphere about the origin: q = du/dn with
            # n = -r_hat
            qbar[:] = -fb[:, None]

    A = np.zeros((ns, ns))
    if CU is not None:
        A += CU[1] * (1.0 - phi)[None, :]
    if CW is not None:
        A -= CW[1] * phi[None, :]
    lu = scipy.linalg.lu_factor(A)

    u = np.zeros((nt, ns))
    q = np.zeros((nt, ns))
    for a in range(1, nt):
        b = np.zeros(ns)
        if w.excitation == "plane":
            b -= incident_rhs(w, xc, n, a)
        # known part of the current step (lag 1)
        u[a - 1] = ubar[a - 1] * (1.0 - phi)
        q[a - 1] = qbar[a - 1] * phi
        gtop = min(a, gmax)
        for g in range(1, gtop + 1):
            if CU is not None:
                b -= CU[g] @ q[a - g]
            if CW is not None:
                b += CW[g] @ u[a - g]
        x = scipy.linalg.lu_solve(lu, b)
        u[a - 1] += phi * x
        q[a - 1] += (1.0 - phi) * x
    return u[: nt - 1], q[: nt - 1]


def march_tau(w, nt=None):
    """OBIE marching written literally in the paper's tau-form (Eq.
    bie_disc3 with Eq. tau / Eq. sigma and the zero-lag system of Eq. linear
    with the tilde variables of Eq. sigma_tau_tilde), beta* = 0, with the
    truncated-power coefficients U^(g), W^(g) of Eqs.
    discretised_single_layer_potential / discretised_double_layer_potential.
    Used to check the compact form ``march`` (equal up to rounding)."""
    assert w.bie == "obie"
    nt = w.nt if nt is None else int(nt)
    d = w.d
    cdt = w.c * w.dt
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    ns = xc.shape[0]
    U = np.zeros((nt + 1, ns, ns))
    W = np.zeros((nt + 1, ns, ns))
    for g in range(1, nt + 1):
        for i in range(ns):
            for j in range(ns):
                U[g, i, j], W[g, i, j] = oc.coef_tau(xc[i], v[j], g, d, cdt, self_=(i == j))
    wk = [oc.w(k, d) for k in range(d + 2)]
    phi = np.ones(ns) if w.bc == "neumann" else np.zeros(ns)
    ubar = np.zeros((nt, ns))
    qbar = np.zeros((nt, ns))
    if w.excitation == "uniform":
        fb = known_coefficients(w, nt)
        if w.bc == "dirichlet":
            ubar[:] = fb[:, None]
        else:
            qbar[:] = -fb[:, None]
    u = np.zeros((nt, ns))
    q = np.zeros((nt, ns))
    A = wk[0] * (W[1] * phi[None, :] - U[1] * (1.0 - phi)[None, :])
    lu = scipy.linalg.lu_factor(A)

    def fold(h, beta):  # sum_{k=0}^{min(d+1, beta)} w^k h^{beta-k}
        return sum(wk[k] * h[beta - k] for k in range(0, min(d + 1, beta) + 1))

    for a in range(1, nt):
        u[a - 1] = ubar[a - 1] * (1.0 - phi)
        q[a - 1] = qbar[a - 1] * phi
        # b = e - sum_{beta=1}^{alpha} (W^(alpha-beta+1) sigma~^{beta-1} - U^(alpha-beta+1) tau~^{beta-1})
        # (the incident term e of the total-field equation 0 = e + sum(U tau - W sigma))
        b = np.zeros(ns)
        if w.excitation == "plane":
            b += incident_rhs(w, xc, n, a)
        for beta in range(1, a + 1):
            sg = fold(u, beta - 1)
            ta = fold(q, beta - 1)
            b -= W[a - beta + 1] @ sg - U[a - beta + 1] @ ta
        x = scipy.linalg.lu_solve(lu, b)
        u[a - 1] += phi * x
        q[a - 1] += (1.0 - phi) * x
    return u[: nt - 1], q[: nt - 1]
