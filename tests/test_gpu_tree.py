"""The device octree and lists are bit-exact with the oracle's definition
(element order, per-level occupied cell keys and cell starts, neighbour and
interaction lists as CSR over cell indices)."""

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import tree as ot
from synth import workload

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _csr(lists):
    off = np.zeros(len(lists) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(x) for x in lists])
    flat = np.array([v for x in lists for v in x], dtype=np.int32)
    return off, flat


def check_tree(ctx, xc, L):
    from paper_2111_05205_gb300 import abi
    T = ot.build(xc, L)
    box = abi.tdbem_get_tree(ctx, "box")
    assert np.array_equal(box[:3], T["lo"]) and box[3] == T["side"]
    assert np.array_equal(abi.tdbem_get_tree(ctx, "perm"), T["perm"].astype(np.int32))
    for lev in range(L + 1):
        assert np.array_equal(abi.tdbem_get_tree(ctx, "keys", lev), T["keys"][lev].astype(np.uint64))
        assert np.array_equal(abi.tdbem_get_tree(ctx, "start", lev), T["start"][lev].astype(np.int32))
        off, flat = _csr(T["nbr"][lev])
        assert np.array_equal(abi.tdbem_get_tree(ctx, "nbr_off", lev), off)
        assert np.array_equal(abi.tdbem_get_tree(ctx, "nbr", lev), flat)
        if lev >= 2:
            off, flat = _csr(T["il"][lev])
            assert np.array_equal(abi.tdbem_get_tree(ctx, "il_off", lev), off)
            assert np.array_equal(abi.tdbem_get_tree(ctx, "il", lev), flat)
    return T


@pytest.mark.parametrize("name,L", [("ellipsoid320_bmbie_d2_hard_plane_s7", 3),
                                    ("ellipsoid80_bmbie_d2_hard_plane_s5", 2),
                                    ("sphere1280_obie_d1_dirichlet_uniform", 4),
                                    ("sphere5120_bmbie_d1_soft_plane", 4),
                                    ("ellipsoid1280_bmbie_d2_hard_plane_s9", 6)])
def test_tree_bit_exact(name, L):
    _need_gpu()
    from tests.gpu_cases import gpu_solver
    w = workload(name, nt=4)
    w.depth = L
    _, xc, _, _ = oc.geometry(w.xyz, w.tri)
    s = gpu_solver(w, depth=L)
    try:
        T = check_tree(s.ctx, xc, L)
        assert len(T["keys"][L]) > 1
    finally:
        s.close()
