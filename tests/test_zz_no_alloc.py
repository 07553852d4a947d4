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
