"""Influence coefficients and B-spline basis of the oracle (ctypes binding).

TEST INFRASTRUCTURE ONLY.  The arithmetic lives in ``tdbem_oracle.c``; this
module compiles it with gcc (OpenMP, no FP contraction) into
``oracle/_build/`` on first use and marshals numpy arrays.

Geometry of the collocation scheme (Section 2.3): element E_j is the flat
triangle of three mesh vertices, its collocation point x_j its centroid
(v0 + v1 + v2) / 3, and the paper's normal n_j = -normalise((v1-v0) x
(v2-v0)), i.e. pointing into the scatterer V.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdbem_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libtdbem_oracle.so")
_lib = None


def build(force=False):
    """Compile the oracle's C core (gcc, -O2 -fopenmp -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_w.restype = ctypes.c_double
        L.orc_w.argtypes = [ctypes.c_int, ctypes.c_int]
        for f in (L.orc_N, L.orc_dN, L.orc_G):
            f.restype = ctypes.c_double
            f.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_coef.restype = None
        L.orc_coef.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, dp]
        L.orc_coef_parts.restype = None
        L.orc_coef_parts.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, dp]
        L.orc_coef_tau.restype = None
        L.orc_coef_tau.argtypes = [dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, dp]
        L.orc_tri_dist.restype = None
        L.orc_tri_dist.argtypes = [dp, dp, dp, dp]
        L.orc_dense.restype = ctypes.c_int
        L.orc_dense.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, dp, dp, dp, dp]
        L.orc_rows.restype = None
        L.orc_rows.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_budget_hits.restype = ctypes.c_long
        L.orc_Gc.restype = ctypes.c_double
        L.orc_Gc.argtypes = [ctypes.c_int, ctypes.c_double]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads():
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------
# B-spline temporal basis (Section 2.3)
# ----------------------------------------------------------------------

def w(kappa, d):
    """Eq. (w)."""
    return float(lib().orc_w(int(kappa), int(d)))


def N(d, tau):
    """N^{0,d}(tau) with dt = 1 (Eq. decompose)."""
    return float(lib().orc_N(int(d), float(tau)))


def dN(d, tau):
    return float(lib().orc_dN(int(d), float(tau)))


def G(d, tau):
    return float(lib().orc_G(int(d), float(tau)))


# ----------------------------------------------------------------------
# geometry of the collocation scheme
# ----------------------------------------------------------------------

def geometry(xyz, tri):
    """Triangle vertex coordinates [ns, 9], centroids [ns, 3], the paper's
    normals (into V) [ns, 3] and areas [ns]."""
    v = np.ascontiguousarray(xyz[tri], dtype=np.float64)  # [ns, 3, 3]
    xc = (v[:, 0] + v[:, 1] + v[:, 2]) / 3.0
    ng = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    area = 0.5 * np.linalg.norm(ng, axis=1)
    n = -ng / np.linalg.norm(ng, axis=1, keepdims=True)
    return v.reshape(-1, 9).copy(), np.ascontiguousarray(xc), np.ascontiguousarray(n), area


# ----------------------------------------------------------------------
# coefficients
# ----------------------------------------------------------------------

def coef(x, nx, v, g, d, cdt, self_=False, bm=True):
    """(C_U, C_W, Ubar, Wbar) of collocation point x (normal nx) against the
    triangle v (9 coordinates) at lag g."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nx = np.ascontiguousarray(nx, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(9)
    out = np.zeros(4)
    lib().orc_coef(_p(x), _p(nx), _p(v), float(g), int(d), float(cdt), int(bool(self_)),
                   int(bool(bm)), _p(out))
    return out


def coef_tau(x, v, g, d, cdt, self_=False):
    """Tau-form (U^(g), W^(g)) with the truncated-power kernel."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(9)
    out = np.zeros(2)
    lib().orc_coef_tau(_p(x), _p(v), float(g), int(d), float(cdt), int(bool(self_)), _p(out))
    return out


def tri_dist(x, v):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(9)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_tri_dist(_p(x), _p(v), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def gamma_max(xyz, tri, d, cdt):
    """Largest lag with a non-zero coefficient: max distance / (c dt) + d + 1."""
    span = np.linalg.norm(xyz.max(0) - xyz.min(0))
    return int(np.ceil(span / cdt + d + 1))


def dense(xyz, tri, d, cdt, kinds=("cu", "cw"), gmax=None):
    """All-pairs coefficients as dense arrays [gmax+1, ns, ns] per kind
    (lag 0 is all zero)."""
    v, xc, n, _ = geometry(xyz, tri)
    ns = v.shape[0]
    if gmax is None:
        gmax = gamma_max(xyz, tri, d, cdt)
    out = {k: (np.zeros((gmax + 1, ns, ns)) if k in kinds else None) for k in ("cu", "cw", "ub", "wb")}
    lib().orc_dense(ns, _p(v), _p(xc), _p(n), int(d), float(cdt), int(gmax),
                    _p(out["cu"]), _p(out["cw"]), _p(out["ub"]), _p(out["wb"]))
    return {k: a for k, a in out.items() if a is not None}


def rows(xyz, tri, d, cdt, rows_, kinds=("cu", "cw"), gmax=None):
    """Coefficients of the given rows: arrays [len(rows), gmax+1, ns]."""
    v, xc, n, _ = geometry(xyz, tri)
    ns = v.shape[0]
    if gmax is None:
        gmax = gamma_max(xyz, tri, d, cdt)
    r = np.ascontiguousarray(rows_, dtype=np.int32)
    out = {k: (np.zeros((len(r), gmax + 1, ns)) if k in kinds else None) for k in ("cu", "cw", "ub", "wb")}
    lib().orc_rows(ns, _p(v), _p(xc), _p(n), int(d), float(cdt), int(gmax), len(r),
                   r.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   _p(out["cu"]), _p(out["cw"]), _p(out["ub"]), _p(out["wb"]))
    return {k: a for k, a in out.items() if a is not None}


def coef_parts(x, v, g, d, cdt, self_=False, grad=True):
    """Normalised parts (Chat_U, Chat_W, d/dg Chat_U, d/dg Chat_W,
    grad Chat_U [3], grad Chat_W [3]); lengths in units of c dt."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(9)
    out = np.zeros(10)
    lib().orc_coef_parts(_p(x), _p(v), float(g), int(d), float(cdt), int(bool(self_)),
                         int(bool(grad)), _p(out))
    return out


def budget_hits():
    """Number of adaptive integrals that stopped on the panel budget (must
    stay 0 for results at full accuracy)."""
    return int(lib().orc_budget_hits())


def Gc(d, tau):
    return float(lib().orc_Gc(int(d), float(tau)))
