"""ctypes binding of libtdbem's C ABI (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: the time marching, the coefficients and the solve
all run in the CUDA library.  Status codes other than TDBEM_OK raise
``TdbemError``.  The library must have been built (``build.build()``); if it
is missing, loading fails loudly -- there is no fallback.
"""

import ctypes
import os

import numpy as np

from . import build as _build

TDBEM_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_NOT_CONVERGED", -5: "ERR_DIVERGED",
          -6: "ERR_TIMEOUT", -7: "ERR_INFEASIBLE_HIERARCHY", -8: "ERR_STATE"}


class TdbemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class tdbem_params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int32), ("d", ctypes.c_int32),
                ("bie", ctypes.c_int32), ("algo", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("ps", ctypes.c_int32), ("pt", ctypes.c_int32), ("mu", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("solver_tol", ctypes.c_double), ("solver_maxit", ctypes.c_int32), ("precond", ctypes.c_int32)]


class tdbem_stats(ctypes.Structure):
    _fields_ = [("ms_rhs", ctypes.c_double), ("ms_near", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("launches_rhs", ctypes.c_int64),
                ("launches_near", ctypes.c_int64), ("launches_solve", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_coef", ctypes.c_int64), ("near_bytes_per_step", ctypes.c_int64),
                ("gamma_max", ctypes.c_int32), ("solve_iters", ctypes.c_int32),
                ("solve_contraction", ctypes.c_double), ("ms_prepare", ctypes.c_double),
                ("ms_far", ctypes.c_double), ("launches_far", ctypes.c_int64), ("fmm_lt", ctypes.c_int32),
                ("fmm_mu", ctypes.c_int32), ("ms_m2l", ctypes.c_double), ("launches_m2l", ctypes.c_int64),
                ("m2l_flops", ctypes.c_double), ("m2l_tile_n", ctypes.c_int32 * 11),
                ("ms_gemm", ctypes.c_double), ("launches_gemm", ctypes.c_int64), ("gemm_tc_flops", ctypes.c_double),
                ("m2l_products", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("launches_far_kernels", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["m2l_tile_n"] = list(self.m2l_tile_n)
        return d


_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double
# name -> (restype, argtypes); the declarations of include/tdbem.h
SIGNATURES = {
    "tdbem_create": (ctypes.c_int, [ctypes.POINTER(tdbem_params), _P, ctypes.POINTER(_P)]),
    "tdbem_destroy": (None, [_P]),
    "tdbem_last_error": (ctypes.c_char_p, [_P]),
    "tdbem_set_mesh": (ctypes.c_int, [_P, _P, _I, _P, _I]),
    "tdbem_set_bc": (ctypes.c_int, [_P, _P]),
    "tdbem_set_known": (ctypes.c_int, [_P, _P]),
    "tdbem_set_incident_plane": (ctypes.c_int, [_P, _P, _D, _D, _I]),
    "tdbem_prepare": (ctypes.c_int, [_P]),
    "tdbem_step": (ctypes.c_int, [_P, _I]),
    "tdbem_step_io": (ctypes.c_int, [_P, _I, _P, _P, _I]),
    "tdbem_step_graph": (ctypes.c_int, [_P, _I]),
    "tdbem_checkpoint": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "tdbem_restore": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "tdbem_sai_create": (ctypes.c_int, [_I, _I, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "tdbem_sai_destroy": (None, [_P]),
    "tdbem_sai_last_error": (ctypes.c_char_p, [_P]),
    "tdbem_sai_train": (ctypes.c_int, [_P, ctypes.POINTER(_P), _I, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "tdbem_sai_gradient": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "tdbem_sai_weights": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64), _I]),
    "tdbem_set_precond": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "tdbem_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "tdbem_batch_create_steps": (ctypes.c_int, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(_P)]),
    "tdbem_batch_step": (ctypes.c_int, [_P, _I]),
    "tdbem_batch_sync": (ctypes.c_int, [_P]),
    "tdbem_batch_destroy": (None, [_P]),
    "tdbem_batch_last_error": (ctypes.c_char_p, [_P]),
    "tdbem_steps_done": (ctypes.c_int, [_P, ctypes.POINTER(_I)]),
    "tdbem_get_solution": (ctypes.c_int, [_P, _P, _P, _I, _I, _I]),
    "tdbem_get_rhs": (ctypes.c_int, [_P, _P]),
    "tdbem_get_coefficients": (ctypes.c_int, [_P, _I, _P, _I, _I, _P]),
    "tdbem_get_zero_lag": (ctypes.c_int, [_P, _P]),
    "tdbem_get_far": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "tdbem_get_tree": (ctypes.c_int, [_P, _I, _I, _P, ctypes.POINTER(ctypes.c_int64)]),
    "tdbem_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(tdbem_stats)]),
    "tdbem_reset_stats": (ctypes.c_int, [_P]),
    "tdbem_sync": (ctypes.c_int, [_P]),
    "tdbem_set_overlap": (ctypes.c_int, [_P, _I]),
    "tdbem_zero_lag_solve_static": (ctypes.c_int, [_P, _P, _P, _I]),
    "tdbem_grid_barrier_probe": (ctypes.c_int, [_I, _I, ctypes.POINTER(_I)]),
    "tdbem_eval_field": (ctypes.c_int, [_P, _P, _I, _I, _I, _P]),
    "tdbem_tc_gemm_check": (ctypes.c_int, [_I, _I, _I, _I, _I, _P, _I, _I, _I, _P, _P, _P]),
}

_lib = None


def lib():
    """Load libtdbem.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libtdbem.so is not built (%s); run paper_2111_05205_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _check(ctx, code):
    if code != TDBEM_OK:
        msg = lib().tdbem_last_error(ctx)
        raise TdbemError(code, msg.decode() if msg else "")


def tdbem_create(params, stream=None):
    out = _P()
    code = lib().tdbem_create(ctypes.byref(params), stream, ctypes.byref(out))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_create")
    return out.value


def tdbem_destroy(ctx):
    lib().tdbem_destroy(ctx)


def tdbem_last_error(ctx):
    m = lib().tdbem_last_error(ctx)
    return m.decode() if m else ""


def tdbem_set_mesh(ctx, xyz, tri):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    _check(ctx, lib().tdbem_set_mesh(ctx, _ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0]))


def tdbem_set_bc(ctx, phi):
    phi = np.ascontiguousarray(phi, dtype=np.int8)
    _check(ctx, lib().tdbem_set_bc(ctx, _ptr(phi)))


def tdbem_set_known(ctx, f):
    """f: known samples [(nt-1), ns] at t_1 .. t_{nt-1}, or None."""
    k = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    _check(ctx, lib().tdbem_set_known(ctx, _ptr(k)))


def tdbem_set_incident_plane(ctx, direction, t0, width, shape=0):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    _check(ctx, lib().tdbem_set_incident_plane(ctx, _ptr(d), float(t0), float(width), int(shape)))


def tdbem_prepare(ctx):
    _check(ctx, lib().tdbem_prepare(ctx))


def tdbem_step(ctx, nsteps):
    _check(ctx, lib().tdbem_step(ctx, int(nsteps)))


def tdbem_step_io(ctx, nsteps, exc=None, x_out=None, on_device=False):
    """exc / x_out: numpy arrays (host) or torch CUDA tensors (on_device)."""
    _check(ctx, lib().tdbem_step_io(ctx, int(nsteps), _ptr(exc), _ptr(x_out), int(bool(on_device))))


def tdbem_step_graph(ctx, nsteps):
    _check(ctx, lib().tdbem_step_graph(ctx, int(nsteps)))


def _bcheck(batch, code):
    if code != TDBEM_OK:
        m = lib().tdbem_batch_last_error(batch)
        raise TdbemError(code, m.decode() if m else "")


def tdbem_batch_create(ctxs):
    arr = (_P * len(ctxs))(*ctxs)
    out = _P()
    code = lib().tdbem_batch_create(arr, len(ctxs), ctypes.byref(out))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_batch_create")
    return out.value


def tdbem_batch_create_steps(ctxs, steps_per_launch):
    arr = (_P * len(ctxs))(*ctxs)
    out = _P()
    code = lib().tdbem_batch_create_steps(arr, len(ctxs), int(steps_per_launch), ctypes.byref(out))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_batch_create_steps")
    return out.value


def tdbem_batch_step(batch, nsteps):
    _bcheck(batch, lib().tdbem_batch_step(batch, int(nsteps)))


def tdbem_batch_sync(batch):
    _bcheck(batch, lib().tdbem_batch_sync(batch))


def tdbem_batch_destroy(batch):
    lib().tdbem_batch_destroy(batch)


def tdbem_batch_last_error(batch):
    m = lib().tdbem_batch_last_error(batch)
    return m.decode() if m else ""


def _scheck(sai, code):
    if code != TDBEM_OK:
        m = lib().tdbem_sai_last_error(sai)
        raise TdbemError(code, m.decode() if m else "")


def tdbem_sai_create(width, hidden, seed):
    out = _P()
    code = lib().tdbem_sai_create(int(width), int(hidden), int(seed), ctypes.byref(out))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_sai_create")
    return out.value


def tdbem_sai_destroy(sai):
    lib().tdbem_sai_destroy(sai)


def tdbem_sai_last_error(sai):
    m = lib().tdbem_sai_last_error(sai)
    return m.decode() if m else ""


def tdbem_sai_train(sai, ctxs, epochs, lr):
    arr = (_P * len(ctxs))(*ctxs)
    loss = ctypes.c_float()
    _scheck(sai, lib().tdbem_sai_train(sai, arr, len(ctxs), int(epochs), float(lr), ctypes.byref(loss)))
    return loss.value


def tdbem_sai_weights(sai, values=None):
    """Get (values None) or set the network weights (float32 numpy)."""
    n = ctypes.c_int64()
    _scheck(sai, lib().tdbem_sai_weights(sai, None, ctypes.byref(n), 0))
    if values is None:
        out = np.zeros(n.value, dtype=np.float32)
        _scheck(sai, lib().tdbem_sai_weights(sai, _ptr(out), ctypes.byref(n), 0))
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    assert v.size == n.value
    _scheck(sai, lib().tdbem_sai_weights(sai, _ptr(v), ctypes.byref(n), 1))
    return v


def tdbem_sai_gradient(sai, ctx):
    n = ctypes.c_int64()
    _scheck(sai, lib().tdbem_sai_weights(sai, None, ctypes.byref(n), 0))
    g = np.zeros(n.value, dtype=np.float32)
    loss = ctypes.c_float()
    _scheck(sai, lib().tdbem_sai_gradient(sai, ctx, _ptr(g), ctypes.byref(loss)))
    return g, loss.value


def tdbem_set_precond(ctx, sai):
    use, sw, q = _I(), _I(), _D()
    _check(ctx, lib().tdbem_set_precond(ctx, sai, ctypes.byref(use), ctypes.byref(sw), ctypes.byref(q)))
    return bool(use.value), sw.value, q.value


def tdbem_checkpoint(ctx):
    """The context's state as bytes."""
    n = ctypes.c_size_t()
    _check(ctx, lib().tdbem_checkpoint(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib().tdbem_checkpoint(ctx, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def tdbem_restore(ctx, data):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(ctx, lib().tdbem_restore(ctx, buf, len(data)))


def tdbem_steps_done(ctx):
    v = _I()
    _check(ctx, lib().tdbem_steps_done(ctx, ctypes.byref(v)))
    return v.value


def tdbem_get_solution(ctx, ns, beta0, nbeta):
    u = np.zeros((nbeta, ns))
    q = np.zeros((nbeta, ns))
    _check(ctx, lib().tdbem_get_solution(ctx, _ptr(u), _ptr(q), int(beta0), int(nbeta), 0))
    return u, q


def tdbem_get_rhs(ctx, ns):
    b = np.zeros(ns)
    _check(ctx, lib().tdbem_get_rhs(ctx, _ptr(b)))
    return b


def tdbem_get_coefficients(ctx, kind, rows, gmax, ns):
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((len(rows), gmax + 1, ns))
    _check(ctx, lib().tdbem_get_coefficients(ctx, int(kind), _ptr(rows), len(rows), int(gmax), _ptr(out)))
    return out


def tdbem_get_far(ctx, ns):
    """(far [Lt, ns], first step) of the current leaf interval (FMM)."""
    a0, n = _I(), _I()
    _check(ctx, lib().tdbem_get_far(ctx, None, ctypes.byref(a0), ctypes.byref(n)))
    out = np.zeros((n.value, ns))
    _check(ctx, lib().tdbem_get_far(ctx, _ptr(out), ctypes.byref(a0), ctypes.byref(n)))
    return out, a0.value


def tdbem_get_zero_lag(ctx, ns):
    out = np.zeros((ns, ns))
    _check(ctx, lib().tdbem_get_zero_lag(ctx, _ptr(out)))
    return out


TREE = {"box": (0, np.float64), "perm": (1, np.int32), "keys": (2, np.uint64), "start": (3, np.int32),
        "nbr_off": (4, np.int32), "nbr": (5, np.int32), "il_off": (6, np.int32), "il": (7, np.int32),
        "near_off": (8, np.int64), "near": (9, np.int32)}


def tdbem_get_tree(ctx, what, level=0):
    """One item of the hierarchy as a numpy array (see include/tdbem.h)."""
    code, dt = TREE[what]
    n = ctypes.c_int64()
    _check(ctx, lib().tdbem_get_tree(ctx, code, int(level), None, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=dt)
    if n.value:
        _check(ctx, lib().tdbem_get_tree(ctx, code, int(level), _ptr(out), ctypes.byref(n)))
    return out


def tdbem_get_stats(ctx):
    s = tdbem_stats()
    _check(ctx, lib().tdbem_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def tdbem_reset_stats(ctx):
    _check(ctx, lib().tdbem_reset_stats(ctx))


def tdbem_sync(ctx):
    _check(ctx, lib().tdbem_sync(ctx))


def tdbem_set_overlap(ctx, overlap):
    _check(ctx, lib().tdbem_set_overlap(ctx, int(overlap)))


def tdbem_zero_lag_solve_static(ctx, b, x, on_device=False):
    """Solve A x = b with no device allocation (see include/tdbem.h).
    b, x: numpy arrays (host) or torch CUDA tensors (on_device)."""
    _check(ctx, lib().tdbem_zero_lag_solve_static(ctx, _ptr(b), _ptr(x), int(bool(on_device))))


def tdbem_grid_barrier_probe(nblocks, starve):
    """Run the bounded grid barrier self-check; True if a wait gave up."""
    out = _I()
    code = lib().tdbem_grid_barrier_probe(int(nblocks), int(starve), ctypes.byref(out))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_grid_barrier_probe")
    return bool(out.value)


def tdbem_tc_gemm_check(a, b, prod, fmt=1, bn=128):
    """Run the tensor-core GEMM self-check: a [nta, m, k] and b [ntb, n, k]
    uint16 bit patterns (BF16 if fmt = 1, FP16 if fmt = 0), prod a list of
    (A term, B term); returns c [n, m] float32."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(b, dtype=np.uint16)
    nta, m, k = a.shape
    ntb, n, k2 = b.shape
    assert k == k2
    pr = np.ascontiguousarray([(s << 4) | t for s, t in prod], dtype=np.int32)
    c = np.zeros((n, m), dtype=np.float32)
    code = lib().tdbem_tc_gemm_check(m, n, k, nta, ntb, _ptr(pr), len(pr), int(fmt), int(bn), _ptr(a), _ptr(b),
                                     _ptr(c))
    if code != TDBEM_OK:
        raise TdbemError(code, "tdbem_tc_gemm_check")
    return c


def tdbem_eval_field(ctx, points, a0, na):
    """Field u(x_p, t_a) at off-surface points for steps a0 .. a0+na-1:
    [na, npts] float64."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((int(na), pts.shape[0]))
    _check(ctx, lib().tdbem_eval_field(ctx, _ptr(pts), pts.shape[0], int(a0), int(na), _ptr(out)))
    return out
