"""Checkpoint at a step, restore into a fresh context, continue: the result
equals the uninterrupted run bit for bit (deterministic kernels), for the
direct path and the FMM path, including a restore point inside a leaf
interval of the FMM.  Restoring the finished context itself (a rewind) and
marching again gives the same result too."""

import numpy as np
import pytest

from synth import workload
from tests.gpu_cases import gpu_solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,k", [("direct", 13), ("fmm", 17), ("fmm", 18)])
def test_checkpoint_resume_is_exact(kind, k):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_05205_gb300 import abi
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=36)
    kw = dict(depth=2, fmm=(3, 3, 0)) if kind == "fmm" else {}
    a = gpu_solver(w, precision=1, **kw)
    b = gpu_solver(w, precision=1, **kw)
    try:
        abi.tdbem_step(a.ctx, k)
        blob = abi.tdbem_checkpoint(a.ctx)
        abi.tdbem_step(a.ctx, 35 - k)
        abi.tdbem_restore(b.ctx, blob)
        assert abi.tdbem_steps_done(b.ctx) == k
        abi.tdbem_step(b.ctx, 35 - k)
        ua, _ = a.solution()
        ub, _ = b.solution()
        assert np.array_equal(ua, ub)
        # rewind the finished context to the checkpoint and march again
        abi.tdbem_restore(a.ctx, blob)
        assert abi.tdbem_steps_done(a.ctx) == k
        abi.tdbem_step(a.ctx, 35 - k)
        ur, _ = a.solution()
        assert np.array_equal(ur, ua)
        with pytest.raises(abi.TdbemError):
            abi.tdbem_restore(b.ctx, blob[:40])
    finally:
        a.close()
        b.close()
