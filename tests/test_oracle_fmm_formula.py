"""Pins of the space-time FMM definitions (oracle side, no GPU).

1. Formula 1 (Eq. m2l_rec, Eq. m2l_expand_rec1, Eq. m2l_expand_rec2, with
   c_m^p(k) of Eq. cmp) reproduces the naive M2L sum of Eq. m2l_actual when
   the kernel is a degree-d polynomial in the interval distance beyond
   mu + 1 intervals (the condition of Section 4.2), for d = 1..4 and random
   moments: the paper's Appendix D argument, checked numerically.
2. The interpolated kernel of one isolated cluster pair converges to the
   exact tau-form coefficient U^(g) as the number of nodes grows.
3. M2M is exact: interpolating a level-l moment through the child nodes
   reproduces the moment computed directly at the parent level.
"""

from math import comb

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import fmm
from synth import workload


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("mu", [2, 8])
def test_formula1_equals_naive_sum(d, mu):
    rng = np.random.default_rng(10 * d + mu)
    K = 40
    T = 0.37
    a = 1.3
    M = rng.standard_normal(K)
    near = rng.standard_normal(mu + 2)  # U(n) for n = 1..mu (index n); U(mu+1) = a^d below
    near[mu + 1] = a ** d

    def U(n):  # kernel between intervals n apart (n >= 1)
        if n <= mu + 1:
            return near[n]
        return sum(comb(d, p) * a ** (d - p) * ((n - mu - 1) * T) ** p for p in range(d + 1))

    # naive: L_k = sum_{l<k} U(k - l) M_l
    naive = np.array([sum(U(k - l) * M[l] for l in range(min(k, K))) for k in range(K + 1)])
    # Algorithm 1
    Lloc = np.zeros(K + mu + 3)
    D = np.zeros(d + 1)
    A = {}
    for p in range(2, d + 1):
        for m in range(p - 1):
            A[(p, m)] = 0.0
    for k in range(K):
        for l in range(1, mu + 2):
            Lloc[k + l] += U(l) * M[k]
        G = [0.0] + [comb(d, p) * a ** (d - p) * M[k] for p in range(1, d + 1)]
        for p in range(1, d + 1):
            D[p] = D[p] + G[p] + sum(fmm.cmp(p, m, k) * A[(p, m)] for m in range(p - 1))
        Lloc[k + mu + 2] = Lloc[k + mu + 1] + sum(D[p] * T ** p for p in range(1, d + 1))
        for p in range(2, d + 1):
            for m in range(p - 1):
                A[(p, m)] += G[p] * k ** m
    for k in range(1, K + 1):
        assert abs(Lloc[k] - naive[k]) <= 1e-9 * (1 + abs(naive[k])), (k, Lloc[k], naive[k])


def test_interpolation_converges_for_an_isolated_pair():
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=40)
    w.d = 1
    cdt = w.c * w.dt
    errs = []
    for p in (2, 4, 6):
        H = fmm.Hierarchy(w.xyz, w.tri, 2, w.c, w.dt, w.nt, p, p, w.d)
        O = 0
        S = H.T["il"][2][O][0]
        i = int(np.nonzero(H.cell[2] == O)[0][0])
        j = int(np.nonzero(H.cell[2] == S)[0][0])
        At, As = fmm.p2m_weights(H, 2)
        xo, ys = fmm.node_points(H, 2, O, obs=True), fmm.node_points(H, 2, S)
        la, _ = H.space_basis(2, O, H.xc[i], obs=True)
        e = emax = 0.0
        for alpha in range(4, 36):
            sg = 1
            kk, kp = (alpha - 1) // H.Tl[2], sg // H.Tl[2]
            if kp >= kk:
                continue
            cj, hj = H.src_interval(2, kp)
            ci, hi = H.obs_interval(2, kk)
            ln, _ = fmm.lagrange(H.wt, (sg * w.dt - cj) / hj)
            lm, _ = fmm.lagrange(H.wt, (alpha * w.dt - ci) / hi)
            Uk = fmm.kernel(xo, ys, ci + hi * H.wt, cj + hj * H.wt, w.c, w.d)
            v = np.einsum("a,m,ambn,b,n->", la, lm, Uk, At[j], ln) / (4 * np.pi * cdt ** w.d)
            exact = oc.coef_tau(H.xc[i], H.v[j], alpha - sg, w.d, cdt)[0]
            e = max(e, abs(v - exact))
            emax = max(emax, abs(exact))
        errs.append(e / emax)
    # measured 0.17, 0.0086, 0.0017 of the largest coefficient at p = 2, 4, 6
    assert errs[2] < errs[1] < errs[0], errs
    assert errs[0] < 0.3 and errs[1] < 0.015 and errs[2] < 0.004, errs


def test_m2m_is_exact():
    w = workload("sphere1280_obie_d1_dirichlet_uniform", nt=20)
    H = fmm.Hierarchy(w.xyz, w.tri, 3, w.c, w.dt, w.nt, 3, 3, w.d)
    rng = np.random.default_rng(4)
    tau = rng.standard_normal((20, w.ns))
    sig = rng.standard_normal((20, w.ns))
    At3, As3 = fmm.p2m_weights(H, 3)
    At2, As2 = fmm.p2m_weights(H, 2)
    Mc = [fmm.moments(H, 3, At3, As3, tau, sig, k) for k in (0, 1)]  # two child intervals
    Mp = fmm.moments(H, 2, At2, As2, tau, sig, 0)
    # interpolate the children's moments onto the parent's nodes
    ps, pt = H.ps, H.pt
    got = np.zeros_like(Mp)
    for c in range(len(H.T["keys"][3])):
        parent = int(np.nonzero(H.T["keys"][2] == (H.T["keys"][3][c] >> 3))[0][0])
        ysc = fmm.node_points(H, 3, c)
        Sv = np.stack([H.space_basis(2, parent, y)[0] for y in ysc])  # [b_child, b_parent]
        for half in (0, 1):
            cj, hj = H.src_interval(3, half)
            cp, hp = H.src_interval(2, 0)
            Tv = np.stack([fmm.lagrange(H.wt, (cj + hj * wn - cp) / hp)[0] for wn in H.wt])  # [n_child, n_parent]
            got[parent] += Sv.T @ Mc[half][c] @ Tv
    assert np.abs(got - Mp).max() <= 1e-12 * np.abs(Mp).max()
