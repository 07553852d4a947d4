"""The cancellation study of Section 5.1.3 (the paper's open question
whether the instability for d >= 2 is arithmetic), on the oracle: the
paper's tau-form coefficient sum C^(g) = sum_kappa w^kappa U^(g-kappa)
(Eq. discretised_single_layer_potential, truncated powers that grow like
g^d) against the compact B-spline form, which integrates N^{0,d} directly
and vanishes exactly once the wavefront has passed the element.  For one
element 12 c dt away, error relative to the largest compact coefficient
(measured, FP64 / FP32 kappa-sum of the FP64 U values):

    lag           15       50       100      200
    d=1 FP64   6.6e-15  4.0e-12  5.4e-12  8.2e-11    FP32  1.4e-7 .. 1.8e-5
    d=2 FP64   2.3e-14  2.5e-11  8.8e-10  4.3e-09    FP32  6.2e-7 .. 2.3e-3
    d=3 FP64   8.7e-15  1.6e-09  1.2e-07  1.2e-06    FP32  5.3e-7 .. 2.2e-1

The loss grows like lag^d; the library stores only compact coefficients,
so its marches do not carry it."""

import numpy as np

from oracle import coeffs as oc

V = np.array([0, 0, 0, 1.0, 0, 0, 0, 1.0, 0.0])
X = np.array([0.3, 0.3, 12.0])


def _errors(d, lags):
    w = [oc.w(k, d) for k in range(d + 2)]
    scale = max(abs(oc.coef(X, np.zeros(3), V, g, d, 1.0, bm=False)[0]) for g in range(10, 20))
    e64, e32 = [], []
    for g in lags:
        comp = oc.coef(X, np.zeros(3), V, g, d, 1.0, bm=False)[0]
        U = [oc.coef_tau(X, V, g - k, d, 1.0)[0] for k in range(d + 2)]
        s64 = sum(w[k] * U[k] for k in range(d + 2))
        s32 = np.float32(0)
        for k in range(d + 2):
            s32 = np.float32(s32 + np.float32(w[k]) * np.float32(U[k]))
        e64.append(abs(s64 - comp) / scale)
        e32.append(abs(float(s32) - comp) / scale)
    return e64, e32


def test_tau_form_loses_digits_like_lag_to_the_d():
    lags = (15, 200)
    e1, f1 = _errors(1, lags)
    e3, f3 = _errors(3, lags)
    # near the wavefront both forms agree to rounding
    assert e1[0] < 1e-12 and e3[0] < 1e-12
    # long after it the tau-form sum carries the cancellation of g^d terms
    assert e3[1] > 1e-8 and e3[1] > 100 * e1[1]
    assert f3[1] > 1e-2
    assert e1[1] < 1e-9
