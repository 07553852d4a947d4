"""Pin of the oracle's whole interpolated far field (not only one cluster
pair): on a 320-element ellipsoid (BMBIE d=2, sound-hard, depth 2) it is
compared with the exact far part of the direct history sum, i.e. the
compact coefficients C^(g) of every pair outside the near lists applied to
the same history (Eq. linear), which shares no code with the FMM route
(moments, naive M2L of Eq. m2l_actual, L2P of Eq. target_m2l).  The sign
and normalisation must agree (the error is well below the far field's own
size), the error must fall by at least 2x per added node for p = 2, 3, 4,
and stay below 0.09 of the far field's maximum at p = 4 (measured: 0.64,
0.22 and 0.061 at p = 2, 3, 4).  A mistake of 10-30 % in a box size, a node
map or the time derivative of L2P moves the p = 4 error above that bound."""

import numpy as np

from oracle import coeffs as oc
from oracle import fmm as ofmm
from oracle import mot
from synth import workload


def _exact_far(C, ku, kw, u, q, near, rows, alphas, ns):
    CU, CW = C.get(ku), C.get(kw)
    gmax = (CU if CU is not None else CW).shape[0] - 1
    out = np.zeros((len(alphas), len(rows)))
    for ai, a in enumerate(alphas):
        for ri, i in enumerate(rows):
            far = np.array([j for j in range(ns) if j not in near[i]])
            s = 0.0
            for g in range(1, min(a, gmax) + 1):
                if CU is not None:
                    s += CU[g][i, far] @ q[a - g][far]
                if CW is not None:
                    s -= CW[g][i, far] @ u[a - g][far]
            out[ai, ri] = s
    return out


def test_far_field_approaches_the_exact_far_sum():
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=60)
    C = oc.dense(w.xyz, w.tri, w.d, w.c * w.dt, kinds=mot.coefficient_kinds(w))
    u, q = mot.march(w, C)
    rows = list(range(0, w.ns, 16))
    alphas = [54, 57]
    errs, flips = [], []
    for p in (2, 3, 4):
        H = ofmm.Hierarchy(w.xyz, w.tri, 2, w.c, w.dt, w.nt, p, p, w.d)
        near = [set(int(v) for v in H.T["near"][i]) for i in range(w.ns)]
        exact = _exact_far(C, "ub", "wb", u, q, near, rows, alphas, w.ns)
        got = ofmm.far_field(H, u, q, alphas, w.bie, rows=rows)
        scale = np.abs(exact).max()
        assert scale > 0
        errs.append(np.abs(got - exact).max() / scale)
        flips.append(np.abs(got + exact).max() / scale)
    # a sign or normalisation mistake would put the error near or above 1
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs
    assert errs[2] < 0.09, errs
    assert min(flips) > 1.5, flips
