"""Convenience wrapper: one libtdbem context with numpy in and out.

Only marshals arguments; every computation happens in the CUDA library.
"""

import numpy as np

from . import abi


class Solver:
    """Time-domain BEM run on the current CUDA device.

    ``xyz`` [nv, 3] vertices, ``tri`` [ns, 3] counter-clockwise triangles,
    ``c``, ``dt``, ``nt``, ``d`` (B-spline order), ``bie`` ("obie" |
    "bmbie"), ``phi`` per-element boundary condition (1 Neumann, 0
    Dirichlet), ``known`` samples of the known data at t_1..t_{nt-1}
    [(nt-1), ns] or None,
    ``incident`` (direction, t0, width[, shape]) of a plane pulse (shape 0
    Gaussian of that width, 1 raised cosine of that length) or None.
    ``fmm``: (ps, pt, mu) to evaluate the far part with the space-time FMM
    (needs ``depth`` >= 2; mu = 0 picks the smallest valid value).
    ``stream``: a cudaStream_t handle (int) or None.  ``precision``: 0 /
    "fp64" or 1 / "split" (float-pair double-float history sum; FMM M2L with
    BF16 x 3 terms), 2 / "bf16x3", 3 / "bf16" (cheaper M2L products), 4 /
    "f16x2" (two scaled FP16 terms, three products), 5 / "fft" (near-future
    M2L blocks by the FFT on equispaced nodes, FP32).
    ``precond``: 0 Jacobi zero-lag solve, 1 allow a learned SAI
    (tdbem_set_precond).
    """

    def __init__(self, xyz, tri, c, dt, nt, d, bie, phi=None, known=None, incident=None, stream=None,
                 solver_tol=0.0, solver_maxit=0, precision=0, depth=0, fmm=None, precond=0):
        p = abi.tdbem_params()
        p.c, p.dt, p.nt, p.d = float(c), float(dt), int(nt), int(d)
        p.bie = {"obie": 0, "bmbie": 1}[bie] if isinstance(bie, str) else int(bie)
        p.algo = 0
        p.precision = {"fp64": 0, "split": 1, "bf16x3": 2, "bf16": 3, "f16x2": 4, "fft": 5}.get(precision, precision)
        p.depth = int(depth)
        if fmm is not None:  # (ps, pt, mu): the space-time FMM for the far part
            p.algo = 1
            p.ps, p.pt, p.mu = (int(v) for v in fmm)
        p.solver_tol = float(solver_tol)
        p.solver_maxit = int(solver_maxit)
        p.precond = int(precond)
        self.ns = int(np.asarray(tri).shape[0])
        self.nt = int(nt)
        self.ctx = abi.tdbem_create(p, stream)
        try:
            abi.tdbem_set_mesh(self.ctx, xyz, tri)
            if phi is not None:
                abi.tdbem_set_bc(self.ctx, phi)
            if known is not None:
                abi.tdbem_set_known(self.ctx, known)
            if incident is not None:
                direction, t0, width = incident[:3]
                shape = incident[3] if len(incident) > 3 else 0
                abi.tdbem_set_incident_plane(self.ctx, direction, t0, width, shape)
            abi.tdbem_prepare(self.ctx)
        except Exception:
            abi.tdbem_destroy(self.ctx)
            self.ctx = None
            raise

    def close(self):
        if self.ctx is not None:
            abi.tdbem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=None):
        n = self.nt - 1 - abi.tdbem_steps_done(self.ctx) if n is None else int(n)
        abi.tdbem_step(self.ctx, n)

    def solution(self, beta0=0, nbeta=None):
        nbeta = self.nt - 1 - beta0 if nbeta is None else nbeta
        return abi.tdbem_get_solution(self.ctx, self.ns, beta0, nbeta)

    def stats(self):
        return abi.tdbem_get_stats(self.ctx)
