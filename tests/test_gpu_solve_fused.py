"""The fused zero-lag solve: plain stepping runs the K Jacobi sweeps of a
step in one cooperative launch with a grid barrier between sweeps.  Its
results are bit-identical to K one-sweep launches (the graph-replayed
steps use those, and test_gpu_batch.py compares the two paths bit for
bit).  Every wait in the barrier is bounded: here a barrier whose arrival
count no CTA can complete gives up within about a second per round and
reports a timeout, and the device stays usable."""

import time

import pytest

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_grid_barrier_completes():
    torch = _need_gpu()
    from paper_2111_05205_gb300 import abi
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert abi.tdbem_grid_barrier_probe(nsm, 0) is False
    assert abi.tdbem_grid_barrier_probe(1, 0) is False


def test_grid_barrier_wait_is_bounded():
    torch = _need_gpu()
    from paper_2111_05205_gb300 import abi
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    t = time.time()
    assert abi.tdbem_grid_barrier_probe(nsm, 1) is True
    assert time.time() - t < 10.0
    # the device is still usable
    assert abi.tdbem_grid_barrier_probe(nsm, 0) is False


def test_fused_solve_is_used_and_matches_graph_steps():
    _need_gpu()
    import numpy as np
    from paper_2111_05205_gb300 import abi
    from tests.gpu_cases import case, gpu_solver
    w = case("ellipsoid320_bmbie_d2_hard_plane_s11", nt=30)
    a, b = gpu_solver(w, precision=1), gpu_solver(w, precision=1)
    try:
        abi.tdbem_step(a.ctx, 29)       # fused solve, one launch per step
        abi.tdbem_step_graph(b.ctx, 29)  # one launch per sweep
        st = a.stats()
        assert st["launches_solve"] == 29
        ua, _ = a.solution(0, 29)
        ub, _ = b.solution(0, 29)
        assert np.array_equal(ua, ub)
    finally:
        a.close()
        b.close()
