"""The field off the boundary on the GPU (tdbem_eval_field, the
representation formula of the exterior problem, Section 2.1) against the
oracle's (oracle/field.py) on the same marched solution: 1e-11 relative to
the field's largest value (both sides sum the same compact coefficients,
which agree to ~1e-13; the field is a sum over all elements and lags).
Cases: a sound-soft ellipsoid with the Gaussian plane pulse (BMBIE d = 2,
q history, incident term), the sound-hard sphere of Section 5.1.1 with the
raised-cosine pulse (u history), and a point on S refused."""

import numpy as np
import pytest

from oracle import field
from synth import workload
from tests.gpu_cases import gpu_solver

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,nt", [("ellipsoid80_bmbie_d2_soft_plane_s5", 30), ("paper_sphere80_bmbie_d2_hard", 24)])
def test_field_matches_oracle(name, nt):
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    w = workload(name, nt=nt)
    s = gpu_solver(w)
    try:
        s.step()
        u, q = s.solution()
        c = w.xyz.mean(axis=0)
        R = np.linalg.norm(w.xyz - c, axis=1).max()
        pts = c[None, :] + np.array([[1.6 * R, 0, 0], [0, -2.1 * R, 0.3 * R], [0.2 * R, 0.1 * R, 3.0 * R],
                                     [-1.2 * R, 0.9 * R, -0.4 * R]])
        a0, na = 3, nt - 4
        got = abi.tdbem_eval_field(s.ctx, pts, a0, na)
        ref = field.field(w, u, q, pts, list(range(a0, a0 + na)))
        scale = np.abs(ref).max()
        assert scale > 0
        assert np.abs(got - ref).max() <= 1e-11 * scale, np.abs(got - ref).max() / scale
        with pytest.raises(abi.TdbemError):
            abi.tdbem_eval_field(s.ctx, w.xyz[w.tri[0]].mean(axis=0)[None, :], a0, 1)  # a centroid, on S
        done = abi.tdbem_steps_done(s.ctx)
        assert done == nt - 1
        p3 = np.ascontiguousarray(pts)
        out = np.zeros((5, len(pts)))
        code = abi.lib().tdbem_eval_field(s.ctx, p3.ctypes.data, len(pts), done, 5, out.ctypes.data)
        assert code == -1, (code, done)  # steps beyond the ones taken: ERR_ARG
    finally:
        s.close()
