"""The zero-lag solve entry point that allocates no device memory
(tdbem_zero_lag_solve_static) gives the same solution as the time-marching
path (tdbem_step) for the same right-hand side.

Who needs it: callers that cannot call cudaMalloc where they solve (while
another component captures a CUDA graph, or under a no-allocation-after-
start-up policy).  Its scratch is a fixed device array shared by all calls,
so this file is collected last; it must pass alone and after the others.
Tolerance: 1e-12 relative (the same Jacobi sweeps on the same inputs; in
practice the results are identical)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_solve_matches_marching_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_05205_gb300 import abi, build
    from tests.gpu_cases import case, gpu_solver
    build.build()
    w = case("ellipsoid320_bmbie_d2_hard_plane_s11", nt=40)
    s = gpu_solver(w)
    try:
        for nstep in (17, 5):
            abi.tdbem_step(s.ctx, nstep)
            a = abi.tdbem_steps_done(s.ctx)
            b = abi.tdbem_get_rhs(s.ctx, w.ns)
            u, _ = s.solution(a - 1, 1)
            x_ref = u[0]  # sound-hard: x^{a-1} = u^{a-1}, no known part
            x_host = np.zeros(w.ns)
            abi.tdbem_zero_lag_solve_static(s.ctx, b, x_host, on_device=False)
            assert np.linalg.norm(x_host - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
            bd = torch.from_numpy(b).cuda()
            xd = torch.zeros_like(bd)
            abi.tdbem_zero_lag_solve_static(s.ctx, bd, xd, on_device=True)
            torch.cuda.synchronize()
            assert np.linalg.norm(xd.cpu().numpy() - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    finally:
        s.close()


def test_static_solve_rejects_null_and_unprepared_context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_05205_gb300 import abi
    L = abi.lib()
    assert L.tdbem_zero_lag_solve_static(None, None, None, 0) == -1
    p = abi.tdbem_params()
    p.c, p.dt, p.nt, p.d, p.bie = 1.0, 0.1, 10, 1, 0
    ctx = abi.tdbem_create(p)
    try:
        b = np.zeros(4)
        x = np.zeros(4)
        assert L.tdbem_zero_lag_solve_static(ctx, b.ctypes.data, x.ctypes.data, 0) == -8  # ERR_STATE
    finally:
        abi.tdbem_destroy(ctx)


def test_static_solve_other_sweep_parity():
    """A second case whose sweep count has the other parity (a looser solver
    tolerance): the last sweep then ends in the other scratch iterate."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_05205_gb300 import Solver, abi, build
    from tests.gpu_cases import case, phi_of
    build.build()
    w = case("ellipsoid80_bmbie_d2_hard_plane_s5", nt=24)

    def solver(tol):
        return Solver(w.xyz, w.tri, w.c, w.dt, w.nt, w.d, w.bie, phi=phi_of(w), incident=(w.direction, w.t0, w.sigma),
                      solver_tol=tol)

    s0 = solver(0.0)
    k0 = s0.stats()["solve_iters"]
    s0.close()
    for tol in (1e-6, 1e-8, 1e-10, 1e-4, 1e-12):
        s = solver(tol)
        if s.stats()["solve_iters"] % 2 != k0 % 2:
            break
        s.close()
    else:
        pytest.skip("no tolerance gave the other sweep parity")
    try:
        abi.tdbem_step(s.ctx, 9)
        b = abi.tdbem_get_rhs(s.ctx, w.ns)
        u, _ = s.solution(8, 1)
        for on_device in (False, True):
            if on_device:
                bd = torch.from_numpy(b).cuda()
                xd = torch.zeros_like(bd)
                abi.tdbem_zero_lag_solve_static(s.ctx, bd, xd, on_device=True)
                torch.cuda.synchronize()
                x = xd.cpu().numpy()
            else:
                x = np.zeros(w.ns)
                abi.tdbem_zero_lag_solve_static(s.ctx, b, x, on_device=False)
            assert np.linalg.norm(x - u[0]) <= 1e-12 * np.linalg.norm(u[0])
    finally:
        s.close()


def test_static_solve_rejects_more_elements_than_the_array_holds():
    """ns above the 262144-element limit is refused with ERR_ARG before any
    device work, and the output buffer is left as it was."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_05205_gb300 import abi
    ns = 262145
    t = np.arange(ns + 2, dtype=np.float64)
    xyz = np.ascontiguousarray(np.stack([t, t * t * 1e-6, np.zeros_like(t)], axis=1))
    tri = np.ascontiguousarray(np.stack([np.arange(ns), np.arange(ns) + 1, np.arange(ns) + 2], axis=1).astype(np.int32))
    p = abi.tdbem_params()
    p.c, p.dt, p.nt, p.d, p.bie = 1.0, 0.1, 10, 1, 0
    ctx = abi.tdbem_create(p)
    try:
        abi.tdbem_set_mesh(ctx, xyz, tri)
        L = abi.lib()
        b = np.ones(ns)
        x = np.full(ns, 7.0)
        assert L.tdbem_zero_lag_solve_static(ctx, b.ctypes.data, x.ctypes.data, 0) == -1  # ERR_ARG
        assert np.all(x == 7.0)
    finally:
        abi.tdbem_destroy(ctx)
