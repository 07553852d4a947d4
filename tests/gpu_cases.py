"""Helpers of the GPU parity tests: run a synthetic workload through the
CUDA library (C ABI) and through the oracle, on the same seeded inputs."""

import numpy as np

from synth import workload


def known_samples(w):
    """Known data of a "uniform" workload at t_1..t_{nt-1}: u = f(t)
    (Dirichlet) or q = -f(t) (Neumann, q = du/dn with n = -r_hat), f the
    Gaussian pulse exp(-((t - 4 sigma)/sigma)^2).  These define the input;
    they are not the method's arithmetic."""
    t = np.arange(1, w.nt) * w.dt
    f = np.exp(-(((t - 4 * w.sigma) / w.sigma) ** 2))
    s = f if w.bc == "dirichlet" else -f
    return np.repeat(s[:, None], w.ns, axis=1)


def phi_of(w):
    return np.full(w.ns, 1 if w.bc == "neumann" else 0, dtype=np.int8)


def gpu_solver(w, stream=None, precision=0, depth=0, fmm=None, precond=0):
    from paper_2111_05205_gb300 import Solver
    inc = (w.direction, w.t0, w.sigma, w.shape) if w.excitation == "plane" else None
    known = known_samples(w) if w.excitation == "uniform" else None
    return Solver(w.xyz, w.tri, w.c, w.dt, w.nt, w.d, w.bie, phi=phi_of(w), known=known, incident=inc,
                  stream=stream, precision=precision, depth=depth, fmm=fmm, precond=precond)


def gpu_march(w, precision=0):
    s = gpu_solver(w, precision=precision)
    try:
        s.step()
        u, q = s.solution()
        st = s.stats()
    finally:
        s.close()
    return u, q, st


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(name, nt=None):
    return workload(name, nt=nt)
