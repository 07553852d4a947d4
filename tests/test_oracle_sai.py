"""Pins of the learned-SAI oracle (oracle/sai.py), independent of its own
per-row formulas:

1. Gradient: every weight block (W1, b1, W2, b2) against central differences
   of the oracle's own loss at random weights.
2. Loss, closed form: with the output layer zero the network's M is the
   first-order Neumann SAI, M = D^-1 - D^-1 R D^-1 on the row patterns (D the
   diagonal of A, R the rest), and the loss equals ||I - M A||_F^2 computed
   as dense matrices.
3. Exactness: for a diagonal A that M is A^-1 and the loss is zero.
"""

import numpy as np

from oracle import sai as osai


def _matrix(ns=14, seed=0, offdiag=True):
    rng = np.random.default_rng(seed)
    A = np.diag(2.0 + rng.random(ns))
    if offdiag:
        for i in range(ns):
            for j in rng.choice(ns, size=3, replace=False):
                if j != i:
                    A[i, j] = 0.2 * rng.standard_normal()
                    A[j, i] = 0.2 * rng.standard_normal()
    xc = rng.standard_normal((ns, 3))
    return A, xc


def _nweights(W, H):
    return H * osai.F * W + H + W * H + W


def test_gradient_matches_central_differences():
    A, xc = _matrix()
    W, H = 8, 6
    rng = np.random.default_rng(1)
    w = 0.3 * rng.standard_normal(_nweights(W, H))
    L0, g = osai.loss_and_grad(w, A, xc, 0.7, W, H)
    assert L0 > 0
    # every block: W1, b1, W2, b2
    blocks = np.cumsum([0, H * osai.F * W, H, W * H, W])
    for b in range(4):
        idx = np.arange(blocks[b], blocks[b + 1])
        for k in idx[:: max(1, len(idx) // 7)]:
            h = 1e-6
            wp, wm = w.copy(), w.copy()
            wp[k] += h
            wm[k] -= h
            fd = (osai.loss_and_grad(wp, A, xc, 0.7, W, H)[0] - osai.loss_and_grad(wm, A, xc, 0.7, W, H)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (b, k, fd, g[k])


def test_zero_output_layer_gives_the_neumann_sai_residual():
    A, xc = _matrix(seed=3)
    ns = A.shape[0]
    W, H = ns, 5  # every off-diagonal entry of a row fits in its slots
    rng = np.random.default_rng(2)
    w = rng.standard_normal(_nweights(W, H))
    W1, b1, W2, b2 = osai.unpack(w, W, H)
    W2[:] = 0.0
    b2[:] = 0.0
    L, _ = osai.loss_and_grad(w, A, xc, 1.0, W, H)
    D = np.diag(np.diag(A))
    R = A - D
    Di = np.linalg.inv(D)
    M = Di - Di @ R @ Di
    ref = np.linalg.norm(np.eye(ns) - M @ A, "fro") ** 2
    assert abs(L - ref) <= 1e-12 * ref


def test_diagonal_matrix_is_inverted_exactly():
    A, xc = _matrix(seed=4, offdiag=False)
    W, H = 4, 3
    w = np.zeros(_nweights(W, H))
    L, g = osai.loss_and_grad(w, A, xc, 1.0, W, H)
    # zero up to the rounding of (1 / a_ii) a_ii
    assert L <= 1e-28
    assert np.abs(g).max() <= 1e-14
