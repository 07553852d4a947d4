"""Plain definitions of the space-time FMM pieces (oracle, TEST
INFRASTRUCTURE ONLY).

The coefficients c_m^p(k) of the O(Nt) M2L recurrence (Formula 1, Eq. cmp)
and n_d, the number of auxiliary local coefficients (Remark aux); the
space-time hierarchy, P2M, the M2L of Eq. m2l_actual (plain, and through
the FFT with equispaced nodes) and L2P.
"""

from math import comb

import numpy as np


def cmp(p, m, k):
    """Eq. (cmp): C(p, m) ((k-1)^{p-m} - 2 k^{p-m} + (k+1)^{p-m}) (-1)^m."""
    e = p - m
    return comb(p, m) * ((k - 1) ** e - 2 * k ** e + (k + 1) ** e) * (-1) ** m


def n_aux(d):
    """Remark aux: n_d = sum_{p=2}^{d} (p - 1)."""
    return sum(p - 1 for p in range(2, d + 1))


# ----------------------------------------------------------------------
# Space-time hierarchy and the interpolated far field (Sections 3-4)
# ----------------------------------------------------------------------
#
# Readings (the paper defers the hierarchy to its earlier study):
# - interpolation: Lagrange polynomials on the p Chebyshev points of the
#   first kind, omega_a = cos((2a+1) pi / (2p)) (any cardinal interpolant
#   fits Formula 1; the paper's cubic Hermite is not used);
# - interpolation boxes of a level-l cell (side s_l = side / 2^l, centre
#   lo + (c + 1/2) s_l): as a source box its cube enlarged by rho = the
#   largest centroid-to-vertex distance of any element, half-width hs_l =
#   s_l/2 + rho, since an element reaches up to rho beyond the cell that
#   holds its centroid; as an observation box the cube itself, half-width
#   ho_l = s_l/2, since the observation points are the centroids;
# - time: a leaf interval holds Lt = floor((s_L - rho) / (c dt)) steps, so
#   that no source of an interval reaches an interaction-list target in the
#   same interval; a level-l interval holds T_l = Lt 2^(L-l) steps.  Source
#   interval J_k covers source indices sigma in [k T, (k+1) T) (time
#   t_sigma), observation interval I_k covers steps alpha in [k T + 1,
#   (k+1) T + 1); J_k has centre (k T + (T-1)/2) dt and half-length
#   T dt / 2, I_k the same shifted by dt;
# - mu: the smallest integer with c (mu T_l + 1) dt > sqrt(3) (3 s_l + hs_l
#   + ho_l) on every level, so that the kernel is an ordinary polynomial of
#   degree d over the node domain of I_{k+mu+1} x J_k (Section 4.2).


def cheb(p):
    return np.cos((2.0 * np.arange(p) + 1.0) * np.pi / (2.0 * p))


def equi(p):
    """p equispaced points on [-1, 1], the ends included (0 for p = 1): the
    nodes of the FFT form of the M2L (Section 4, the estimate after
    Algorithm 1), under which every M2L block is a Toeplitz matrix."""
    return np.linspace(-1.0, 1.0, p) if p > 1 else np.zeros(1)


def lagrange(nodes, xi):
    """Values and derivatives of the Lagrange basis of ``nodes`` at xi."""
    p = len(nodes)
    val = np.ones(p)
    der = np.zeros(p)
    for a in range(p):
        for b in range(p):
            if b == a:
                continue
            f = (xi - nodes[b]) / (nodes[a] - nodes[b])
            der[a] = der[a] * f + val[a] / (nodes[a] - nodes[b])
            val[a] *= f
    return val, der


class Hierarchy:
    """Parameters of the space-time hierarchy of one mesh (see above)."""

    def __init__(self, xyz, tri, L, c, dt, nt, ps, pt, d, mu=0, nodes="cheb"):
        from . import coeffs as oc
        from . import tree as ot
        v, xc, n, _ = oc.geometry(xyz, tri)
        self.v, self.xc, self.n = v, xc, n
        self.L, self.c, self.dt, self.nt, self.ps, self.pt, self.d = L, c, dt, nt, ps, pt, d
        self.T = ot.build(xc, L)
        self.lo, self.side = self.T["lo"], self.T["side"]
        V = v.reshape(-1, 3, 3)
        dv = V - xc[:, None, :]
        self.rho = float(np.sqrt(dv[..., 0] * dv[..., 0] + dv[..., 1] * dv[..., 1] + dv[..., 2] * dv[..., 2]).max())
        cdt = c * dt
        self.s = [self.side / (1 << l) for l in range(L + 1)]
        self.hs = [self.s[l] / 2.0 + self.rho for l in range(L + 1)]
        self.nodes = nodes
        # FFT form: equispaced nodes, and the observation box is the source
        # box, so that node differences depend only on index differences
        self.ho = list(self.hs) if nodes == "equi" else [self.s[l] / 2.0 for l in range(L + 1)]
        self.Lt = int(np.floor((self.s[L] - self.rho) / cdt))
        if self.Lt < 1 or not (2.0 * self.rho < self.s[L]):
            raise ValueError("infeasible hierarchy: leaf cells too small for c dt and the element size")
        self.Tl = [self.Lt * (1 << (L - l)) for l in range(L + 1)]
        m = 0
        for l in range(2, L + 1):
            rmax = np.sqrt(3.0) * (3.0 * self.s[l] + self.hs[l] + self.ho[l])
            m = max(m, int(np.floor((rmax / cdt - 1.0) / self.Tl[l])) + 1)
        self.mu = max(m, mu)
        self.ws, self.wt = (equi(ps), equi(pt)) if nodes == "equi" else (cheb(ps), cheb(pt))
        # cell index of every element at every level
        self.cell = []
        for l in range(L + 1):
            index = {int(k): i for i, k in enumerate(self.T["keys"][l])}
            self.cell.append(np.array([index[int(k) >> (3 * (L - l))] for k in self.T["leafkey"]]))

    def centre(self, l, ci):
        from . import tree as ot
        co = np.array(ot.demorton(int(self.T["keys"][l][ci]), l), dtype=np.float64)
        return self.lo + (co + 0.5) * self.s[l]

    def src_interval(self, l, k):
        T = self.Tl[l]
        return (k * T + (T - 1) / 2.0) * self.dt, T * self.dt / 2.0

    def obs_interval(self, l, k):
        cen, h = self.src_interval(l, k)
        return cen + self.dt, h

    def space_basis(self, l, ci, y, obs=False):
        """ell_b((y - centre)/h) for b = (b1, b2, b3), b1 fastest, and its
        gradient with respect to y ([P_s], [P_s, 3]); h = hs_l on the source
        box, ho_l on the observation box (obs=True)."""
        h = self.ho[l] if obs else self.hs[l]
        xi = (np.asarray(y) - self.centre(l, ci)) / h
        vals, ders = zip(*(lagrange(self.ws, x) for x in xi))
        p = self.ps
        val = np.zeros(p ** 3)
        grad = np.zeros((p ** 3, 3))
        for b3 in range(p):
            for b2 in range(p):
                for b1 in range(p):
                    b = b1 + p * (b2 + p * b3)
                    val[b] = vals[0][b1] * vals[1][b2] * vals[2][b3]
                    grad[b] = [ders[0][b1] * vals[1][b2] * vals[2][b3] / h,
                               vals[0][b1] * ders[1][b2] * vals[2][b3] / h,
                               vals[0][b1] * vals[1][b2] * ders[2][b3] / h]
        return val, grad


def tri_rule(n):
    """Collapsed (Duffy) Gauss-Legendre rule on the reference triangle
    {(s, t): s, t >= 0, s + t <= 1}: exact for polynomials of degree
    2n - 2 in (s, t) (weights sum to 1/2)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for a in range(n):
        for b in range(n):
            s = x[a]
            t = x[b] * (1.0 - s)
            pts.append((s, t))
            wts.append(w[a] * w[b] * (1.0 - s))
    return np.array(pts), np.array(wts)


def _lagrange_many(nodes, xi):
    """Lagrange basis values and derivatives at the points xi [nq] -> [nq, p]
    (the same recurrence as ``lagrange``, over all points at once)."""
    p = len(nodes)
    val = np.ones((len(xi), p))
    der = np.zeros((len(xi), p))
    for a in range(p):
        for b in range(p):
            if b == a:
                continue
            f = (xi - nodes[b]) / (nodes[a] - nodes[b])
            der[:, a] = der[:, a] * f + val[:, a] / (nodes[a] - nodes[b])
            val[:, a] *= f
    return val, der


def p2m_weights(H, l):
    """A^tau_{jb} = int_{E_j} ell_b dS and A^sigma_{jb} = int_{E_j} n_y.grad ell_b dS
    for the level-l source box of each element's cell (moment of Section 3),
    by the collapsed Gauss rule on each triangle (all quadrature points of an
    element at once)."""
    pts, wts = tri_rule(2 * H.ps + 2)
    ns = H.xc.shape[0]
    p = H.ps
    P = p ** 3
    At = np.zeros((ns, P))
    As = np.zeros((ns, P))
    V = H.v.reshape(-1, 3, 3)
    for j in range(ns):
        a, b, c = V[j]
        area2 = np.linalg.norm(np.cross(b - a, c - a))
        Y = a[None, :] + pts[:, :1] * (b - a)[None, :] + pts[:, 1:2] * (c - a)[None, :]  # [nq, 3]
        xi = (Y - H.centre(l, H.cell[l][j])[None, :]) / H.hs[l]
        L = [_lagrange_many(H.ws, xi[:, k]) for k in range(3)]  # per axis ([nq, p], [nq, p])
        # ell_b = ell_{b1}(x) ell_{b2}(y) ell_{b3}(z), b = b1 + p (b2 + p b3)
        v0, v1, v2 = L[0][0], L[1][0], L[2][0]
        d0, d1, d2 = L[0][1], L[1][1], L[2][1]
        val = np.einsum("qi,qj,qk->qkji", v0, v1, v2).reshape(-1, P)
        g0 = np.einsum("qi,qj,qk->qkji", d0, v1, v2).reshape(-1, P) / H.hs[l]
        g1 = np.einsum("qi,qj,qk->qkji", v0, d1, v2).reshape(-1, P) / H.hs[l]
        g2 = np.einsum("qi,qj,qk->qkji", v0, v1, d2).reshape(-1, P) / H.hs[l]
        n = H.n[j]
        At[j] = area2 * (wts @ val)
        As[j] = area2 * (wts @ (g0 * n[0] + g1 * n[1] + g2 * n[2]))
    return At, As


def fold(h, d):
    """tau^sigma = sum_{kappa=0}^{min(d+1, sigma)} w^kappa h^{sigma-kappa} (Eq. tau, Eq. sigma)."""
    from . import coeffs as oc
    out = np.zeros_like(h)
    for s in range(h.shape[0]):
        for k in range(0, min(d + 1, s) + 1):
            out[s] += oc.w(k, d) * h[s - k]
    return out


def moments(H, l, At, As, tau, sig, k):
    """M_{b,n}(S, J_k) for every level-l cell S (P2M of Section 3, taken
    directly from the elements at any level): [ncells, P_s, P_t]."""
    cen, h = H.src_interval(l, k)
    T = H.Tl[l]
    nc = len(H.T["keys"][l])
    M = np.zeros((nc, H.ps ** 3, H.pt))
    pref = 1.0 / (4.0 * np.pi * (H.c * H.dt) ** H.d)
    for sig_i in range(k * T, (k + 1) * T):
        if sig_i >= tau.shape[0]:
            break
        lt, _ = lagrange(H.wt, (sig_i * H.dt - cen) / h)
        src = At * tau[sig_i][:, None] - As * sig[sig_i][:, None]  # [ns, P]
        for j in range(src.shape[0]):
            M[H.cell[l][j]] += pref * np.outer(src[j], lt)
    return M


def kernel(x, y, t, s, c, d):
    """U(x, y, t, s) = (c (t - s) - r)_+^d / r (Eq. U), broadcasting:
    x [A, 3], y [B, 3], t [M], s [N] -> [A, M, B, N]."""
    r = np.linalg.norm(x[:, None, :] - y[None, :, :], axis=2)  # [A, B]
    a = c * (t[:, None] - s[None, :])  # [M, N]
    z = a[None, :, None, :] - r[:, None, :, None]
    return np.where(z > 0, np.maximum(z, 0.0) ** d, 0.0) / r[:, None, :, None]


def node_points(H, l, ci, obs=False):
    p = H.ps
    h = H.ho[l] if obs else H.hs[l]
    cen = H.centre(l, ci)
    pts = np.zeros((p ** 3, 3))
    for b3 in range(p):
        for b2 in range(p):
            for b1 in range(p):
                pts[b1 + p * (b2 + p * b3)] = cen + h * np.array([H.ws[b1], H.ws[b2], H.ws[b3]])
    return pts


def m2l_naive(H, l, Ms, O, k):
    """L(O, I_k) = sum_{k' < k} sum_{S in IL(O)} U(O, S, I_k, J_k') M(S, J_k')
    (Eq. m2l_actual) with U sampled at the interpolation nodes (Eq. Uabmn);
    Ms[k'] are the level-l moments.  Returns [P_s, P_t]."""
    xo = node_points(H, l, O, obs=True)
    ci, hi = H.obs_interval(l, k)
    to = ci + hi * H.wt
    Lloc = np.zeros((H.ps ** 3, H.pt))
    for S in H.T["il"][l][O]:
        ys = node_points(H, l, S)
        for kp in range(k):
            cj, hj = H.src_interval(l, kp)
            ts = cj + hj * H.wt
            U = kernel(xo, ys, to, ts, H.c, H.d)  # [a, m, b, n]
            Lloc += np.einsum("ambn,bn->am", U, Ms[kp][S])
    return Lloc


def _circulant_axis(p, N):
    """Index differences D = a - b (|D| <= p - 1) at their circular positions
    D mod N of an N-point axis (N >= 2p - 1); other positions stay 0."""
    D = np.zeros(N)
    on = np.zeros(N, dtype=bool)
    for t in range(-(p - 1), p):
        D[t % N] = t
        on[t % N] = True
    return D, on


def m2l_fft(H, l, Ms, O, k):
    """The same sum as m2l_naive, each block U(O, S, I_k, J_k') applied by the
    FFT (Section 4, the complexity estimate after Algorithm 1).  With
    equispaced nodes and equal boxes, x_a - y_b = c_O - c_S + h (w_a - w_b)
    and t_m - s_n = c_I - c_J + h_t (w_m - w_n) depend only on a - b and
    m - n, so a block is a four-level Toeplitz matrix.  Embedded in a
    circulant of 2 p_s points per spatial axis and 2 p_t in time, it acts
    as a circular convolution: U M = IFFT(FFT(u) FFT(M padded)) restricted
    to the first p_s^3 x p_t entries.  Returns [P_s, P_t]."""
    if H.nodes != "equi":
        raise ValueError("the FFT form needs equispaced nodes")
    ps, pt = H.ps, H.pt
    Ns, Nt = 2 * ps, 2 * pt
    hsp = H.hs[l] * (2.0 / (ps - 1) if ps > 1 else 0.0)
    Ds, ons = _circulant_axis(ps, Ns)
    Dt, ont = _circulant_axis(pt, Nt)
    ci, hi = H.obs_interval(l, k)
    co = H.centre(l, O)
    Y = np.zeros((Nt, Ns, Ns, Ns), dtype=complex)
    for S in H.T["il"][l][O]:
        dc = co - H.centre(l, S)
        # axes (t, z, y, x): the vector index b1 + p (b2 + p b3) + P3 n
        rx = dc[0] + hsp * Ds[None, None, None, :]
        ry = dc[1] + hsp * Ds[None, None, :, None]
        rz = dc[2] + hsp * Ds[None, :, None, None]
        r = np.sqrt(rx * rx + ry * ry + rz * rz)
        mask = ons[None, None, None, :] & ons[None, None, :, None] & ons[None, :, None, None]
        for kp in range(k):
            cj, hj = H.src_interval(l, kp)
            htp = hj * (2.0 / (pt - 1) if pt > 1 else 0.0)
            tau = (ci - cj) + htp * Dt
            z = H.c * tau[:, None, None, None] - r
            u = np.where((z > 0) & mask & ont[:, None, None, None], np.maximum(z, 0.0) ** H.d, 0.0) / r
            X = np.zeros((Nt, Ns, Ns, Ns))
            X[:pt, :ps, :ps, :ps] = Ms[kp][S].T.reshape(pt, ps, ps, ps)
            Y += np.fft.fftn(u) * np.fft.fftn(X)
    y = np.fft.ifftn(Y).real[:pt, :ps, :ps, :ps]
    return y.reshape(pt, ps ** 3).T.copy()


def l2p(H, l, O, Lloc, i, alpha, bie):
    """Psi(x_i, t_alpha) = sum_{a,m} D_a ell_m(t_alpha) L_{a,m} (Eq. target_m2l);
    BMBIE applies (d/dn_x - c^-1 d/dt) to ell_a ell_m (Section 3)."""
    ci, hi = H.obs_interval(l, (alpha - 1) // H.Tl[l])
    lt, dlt = lagrange(H.wt, (alpha * H.dt - ci) / hi)
    val, grad = H.space_basis(l, O, H.xc[i], obs=True)
    if bie == "obie":
        return float(val @ Lloc @ lt)
    dn = grad @ H.n[i]
    return float(dn @ Lloc @ lt - val @ Lloc @ (dlt / hi) / H.c)


def far_field(H, u, q, alphas, bie, rows=None, m2l=None):
    """The interpolated far field Psi(x_i, t_alpha) of every row for the given
    steps: sum over levels l >= 2 of L2P of the naive M2L of the directly
    computed moments of the interaction-list cells (every past interval).
    u, q: B-spline coefficient histories [>= max(alphas), ns].  m2l: the
    M2L route (m2l_naive, or m2l_fft with equispaced nodes)."""
    m2l = m2l or m2l_naive
    ns = H.xc.shape[0]
    rows = range(ns) if rows is None else rows
    tau = fold(q, H.d)
    sig = fold(u, H.d)
    out = np.zeros((len(alphas), len(rows)))
    for l in range(2, H.L + 1):
        At, As = p2m_weights(H, l)
        kmax = max((a - 1) // H.Tl[l] for a in alphas)
        Ms = [moments(H, l, At, As, tau, sig, k) for k in range(kmax)]
        cache = {}
        for ai, a in enumerate(alphas):
            k = (a - 1) // H.Tl[l]
            for ri, i in enumerate(rows):
                O = H.cell[l][i]
                if (O, k) not in cache:
                    cache[(O, k)] = m2l(H, l, Ms, O, k)
                out[ai, ri] += l2p(H, l, O, cache[(O, k)], i, a, bie)
    return out
