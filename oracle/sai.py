"""Learned sparse approximate inverse of the zero-lag system (oracle, TEST
INFRASTRUCTURE ONLY).

Plain FP64 numpy restatement of the network and the training loss that the
library uses for its zero-lag preconditioner (an addition of the library;
the paper only says the system of Eq. linear is sparse):

- row i's slots: the diagonal, then the off-diagonal entries of A with
  |A_ij| >= 1e-12 |A_ii| by decreasing |A_ij|/|A_ii| quantised to 2^-20
  (ties by column), at most W;
- features per slot: A_ij/A_ii, A_jj/A_ii, A_ji/A_ii, |x_i - x_j|/(c dt), 1
  (zeros past the row's length);
- network: h = relu(W1 f + b1), o = W2 h + b2 + base, M_ij = o_k / A_ii,
  with the analytic part base_0 = 1 (Jacobi) and base_k = -A_ij / A_jj for
  the off-diagonal slots (first Neumann term of A^-1, in units of 1/A_ii);
- loss: sum_i || e_i^T - m_i^T A ||^2, and its gradient.
Weight vector layout: W1 [H, 5W] row-major, b1 [H], W2 [W, H], b2 [W].
"""

import numpy as np


F = 5


def row_slots(A, i, W):
    cols = [int(j) for j in np.nonzero(A[i])[0] if j != i and abs(A[i, j]) >= 1e-12 * abs(A[i, i])]
    # magnitude quantised to 2^-20 of |A_ii| (entries equal up to rounding
    # keep one order), then column
    cols.sort(key=lambda j: (-int(np.floor(abs(A[i, j] * (1.0 / A[i, i])) * 1048576.0)), j))
    return [i] + cols[: W - 1]


def features(A, xc, cdt, i, W):
    cols = row_slots(A, i, W)
    f = np.zeros(F * W)
    for k, j in enumerate(cols):
        f[F * k] = A[i, j] / A[i, i]
        f[F * k + 1] = A[j, j] / A[i, i]
        f[F * k + 2] = A[j, i] / A[i, i]
        f[F * k + 3] = np.linalg.norm(xc[i] - xc[j]) / cdt
        f[F * k + 4] = 1.0
    return cols, f


def unpack(w, W, H):
    Fw = F * W
    o = 0
    W1 = w[o:o + H * Fw].reshape(H, Fw)
    o += H * Fw
    b1 = w[o:o + H]
    o += H
    W2 = w[o:o + W * H].reshape(W, H)
    o += W * H
    b2 = w[o:o + W]
    return W1, b1, W2, b2


def loss_and_grad(w, A, xc, cdt, W, H):
    """Sum over rows of ||e_i^T - m_i^T A||^2 and its gradient (FP64)."""
    W1, b1, W2, b2 = unpack(np.asarray(w, dtype=np.float64), W, H)
    g = np.zeros(len(w))
    gW1, gb1, gW2, gb2 = unpack(g, W, H)
    ns = A.shape[0]
    L = 0.0
    for i in range(ns):
        cols, f = features(A, xc, cdt, i, W)
        z = W1 @ f + b1
        h = np.maximum(z, 0.0)
        base = np.zeros(W)
        for k in range(len(cols)):
            base[k] = 1.0 if k == 0 else -f[F * k] / f[F * k + 1]
        o = W2 @ h + b2 + base
        n = len(cols)
        m = np.zeros(ns)
        for k in range(n):
            m[cols[k]] = o[k] / A[i, i]
        r = m @ A
        r[i] -= 1.0
        L += float(r @ r)
        go = np.zeros(W)
        for k in range(n):
            go[k] = 2.0 * float(r @ A[cols[k]]) / A[i, i]
        gb2 += go
        gW2 += np.outer(go, h)
        gh = (W2.T @ go) * (z > 0)
        gb1 += gh
        gW1 += np.outer(gh, f)
    return L, g
