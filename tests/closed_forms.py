"""Textbook closed forms used to pin the oracle (independent of it).

- ``slp_static``: int_T dS / |x - y| over a flat triangle (the classical
  edge-by-edge formula of the potential of a uniform triangular layer,
  Wilton et al. 1984 / Graglia 1993).
- ``solid_angle``: signed solid angle of a triangle seen from x (Van
  Oosterom & Strackee 1983), positive on the side opposite to
  (v1 - v0) x (v2 - v0).
- ``appb_U``: the paper's closed forms I_n^d, d = 1..3, of Appendix B for the
  tau-form single-layer coefficient U^(g), valid when the element lies inside
  the sphere r < c t_g (no clipping).
"""

import numpy as np


def slp_static(x, v):
    v = np.asarray(v, dtype=float).reshape(3, 3)
    x = np.asarray(x, dtype=float)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    z = n @ (x - v[0])
    rho = x - z * n
    s = 0.0
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        l = (b - a) / np.linalg.norm(b - a)
        m = np.cross(l, n)
        lp, lm, t0 = (b - rho) @ l, (a - rho) @ l, (a - rho) @ m
        R02 = t0 * t0 + z * z
        Rp, Rm = np.sqrt(lp * lp + R02), np.sqrt(lm * lm + R02)
        s += t0 * np.log((Rp + lp) / (Rm + lm))
        s -= abs(z) * (np.arctan(t0 * lp / (R02 + abs(z) * Rp)) - np.arctan(t0 * lm / (R02 + abs(z) * Rm)))
    return s


def solid_angle(x, v):
    v = np.asarray(v, dtype=float).reshape(3, 3)
    R = v - np.asarray(x, dtype=float)
    r = np.linalg.norm(R, axis=1)
    num = R[0] @ np.cross(R[1], R[2])
    den = r[0] * r[1] * r[2] + (R[0] @ R[1]) * r[2] + (R[0] @ R[2]) * r[1] + (R[1] @ R[2]) * r[0]
    return 2.0 * np.arctan2(num, den)


def _In(d, s, x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    R = np.sqrt(y * y + z * z)
    at1 = np.arctan(x / y)
    at2 = np.arctan(x * z / (y * r)) if z != 0 else 0.0
    lg = np.log((x + r) / R)
    if d == 1:
        return x * y / 2 + (s * s + z * z) / 2 * at1 - s * z * at2 - s * y * lg
    if d == 2:
        return (2 * (s ** 3 + 3 * s * z * z) * at1 - 2 * z * (3 * s * s + z * z) * at2
                - x * y * (-6 * s + r) - y * (6 * s * s + y * y + 3 * z * z) * lg) / 6
    if d == 3:
        return (x * y * (18 * s * s + x * x + 3 * y * y + 6 * z * z - 6 * s * r)
                + 3 * (s ** 4 + 6 * s * s * z * z + z ** 4) * at1 - 12 * s * z * (s * s + z * z) * at2
                - 6 * y * s * (2 * s * s + y * y + 3 * z * z) * lg) / 12
    raise ValueError(d)


def appb_U(x, v, g, d, cdt):
    """U^(g) of the truncated-power kernel from the closed forms of
    Appendix B: (4 pi (c dt)^d)^-1 [sum_n I_n^d + I_0^d], summed over the
    three sub-triangles O-V1-V2 with their orientation signs."""
    v = np.asarray(v, dtype=float).reshape(3, 3)
    x = np.asarray(x, dtype=float)
    s = cdt * g
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    z = n @ (x - v[0])
    O = x - z * n
    total = 0.0
    inside = True
    for i in range(3):
        a, b = v[i] - O, v[(i + 1) % 3] - O
        sign = np.sign(np.cross(a, b) @ n)
        if sign < 0:
            inside = False
        e = (b - a) / np.linalg.norm(b - a)
        x1, x2 = a @ e, b @ e
        y = np.linalg.norm(a - x1 * e)
        # the bracket is int_{theta_1}^{theta_2} -(s-r)^{d+1}/(d+1) dtheta with
        # theta = atan(y/x) decreasing in x: its magnitude is the angular
        # integral of (s-r)^{d+1}/(d+1) over the sub-triangle
        J = abs(_In(d, s, x2, y, z) - _In(d, s, x1, y, z))
        phi = abs(np.arctan2(np.linalg.norm(np.cross(a, b)), a @ b))
        total += sign * ((s - abs(z)) ** (d + 1) / (d + 1) * phi - J)
    del inside
    return total / (4 * np.pi * cdt ** d)
