"""Pins of the oracle's FFT form of the M2L (Section 4, the complexity
estimate after Algorithm 1: the M2L applied by the FFT).

With equispaced nodes and the observation box equal to the source box, node
differences depend only on index differences, so every M2L block is a
four-level Toeplitz matrix and ``oracle.fmm.m2l_fft`` applies it as a
circular convolution by numpy's FFT.
- It must equal the plain sum ``m2l_naive`` of the same hierarchy to
  rounding (the convolution theorem), on random moments, for ps != pt and
  every observation cell with interaction-list cells.
- The far field it yields must approach the exact far part of the direct
  history sum (compact coefficients of every pair outside the near lists,
  which shares no code with the FMM route) as nodes are added: measured
  1.27, 0.40 and 0.10 of the far field's maximum at p = 2, 3, 4 on the
  320-element ellipsoid (Chebyshev nodes: 0.64, 0.22, 0.061), required to
  fall by more than 2x per node and stay below 0.15 at p = 4; a flipped
  sign errs by more than 1.5.
"""

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import fmm as ofmm
from oracle import mot
from synth import workload
from tests.test_oracle_fmm_farfield import _exact_far


def test_equispaced_nodes():
    assert np.allclose(ofmm.equi(4), [-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0])
    assert np.allclose(ofmm.equi(1), [0.0])
    D, on = ofmm._circulant_axis(3, 6)
    assert list(D[on]) == [0, 1, 2, -2, -1] and not on[3]


@pytest.mark.parametrize("ps,pt", [(3, 4), (4, 3), (2, 2)])
def test_fft_m2l_equals_the_plain_sum(ps, pt):
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=60)
    H = ofmm.Hierarchy(w.xyz, w.tri, 2, w.c, w.dt, w.nt, ps, pt, w.d, nodes="equi")
    assert H.ho == H.hs
    nc = len(H.T["keys"][2])
    rng = np.random.default_rng(7)
    Ms = [rng.standard_normal((nc, ps ** 3, pt)) for _ in range(4)]
    checked = 0
    for O in range(nc):
        if len(H.T["il"][2][O]) == 0:
            continue
        a = ofmm.m2l_naive(H, 2, Ms, O, 3)
        b = ofmm.m2l_fft(H, 2, Ms, O, 3)
        assert np.abs(a).max() > 0
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
        checked += 1
        if checked == 3:
            break
    assert checked == 3


def test_fft_m2l_refuses_chebyshev_nodes():
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=20)
    H = ofmm.Hierarchy(w.xyz, w.tri, 2, w.c, w.dt, w.nt, 2, 2, w.d)
    with pytest.raises(ValueError):
        ofmm.m2l_fft(H, 2, [], 0, 1)


def test_fft_far_field_approaches_the_exact_far_sum():
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=60)
    C = oc.dense(w.xyz, w.tri, w.d, w.c * w.dt, kinds=mot.coefficient_kinds(w))
    u, q = mot.march(w, C)
    rows = list(range(0, w.ns, 16))
    alphas = [54, 57]
    errs, flips = [], []
    for p in (2, 3, 4):
        H = ofmm.Hierarchy(w.xyz, w.tri, 2, w.c, w.dt, w.nt, p, p, w.d, nodes="equi")
        near = [set(int(v) for v in H.T["near"][i]) for i in range(w.ns)]
        exact = _exact_far(C, "ub", "wb", u, q, near, rows, alphas, w.ns)
        got = ofmm.far_field(H, u, q, alphas, w.bie, rows=rows, m2l=ofmm.m2l_fft)
        scale = np.abs(exact).max()
        assert scale > 0
        errs.append(np.abs(got - exact).max() / scale)
        flips.append(np.abs(got + exact).max() / scale)
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs
    assert errs[2] < 0.15, errs
    assert min(flips) > 1.5, flips
