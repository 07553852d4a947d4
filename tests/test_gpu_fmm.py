"""Parity of the CUDA space-time FMM with the oracle's interpolated far field.

The GPU evaluates the far part of the history sum with P2M at the leaf
level, separable M2M, the near-/distant-future M2L with the O(Nt)
recurrence of Formula 1 / Algorithm 1, L2L and L2P (Sections 3-4).  The
oracle (``oracle.fmm.far_field``) takes the plain route: moments computed
directly from the elements at every level, the naive M2L of Eq. m2l_actual
over every past interval with the kernel sampled at the nodes, and L2P.
M2M and L2L are exact for the interpolating polynomials and Formula 1 is
exact in the distant-future regime (mu is chosen for that), so the two
agree to rounding, amplified by the far field's cancellation and the
recurrence's polynomial extrapolation (tolerances per precision: _tol).
Both sides use the GPU's own history as input.  The near lists are
bit-exact.
"""

import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import tree as ot
from synth import workload

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    # name, depth, p, nsteps
    ("ellipsoid320_bmbie_d2_hard_plane_s7", 2, 3, 37),
    ("sphere1280_obie_d1_dirichlet_uniform", 3, 2, 29),
    ("sphere1280_bmbie_d1_dirichlet_uniform", 3, 3, 22),
    # long runs: the distant-future recurrence of Formula 1 is active (the
    # observed interval lies far more than mu+1 intervals after the early
    # source intervals)
    ("ellipsoid320_bmbie_d2_hard_plane_s7", 2, 2, 81),
    ("sphere1280_bmbie_d2_neumann_uniform", 3, 2, 81),
]


def _tol(precision, w, nsteps):
    """Far-field tolerance relative to the far field's largest value.

    The tau-form far field (Eq. target) is a sum whose terms are ~1e4-1e5
    times larger than the result (U grows like g^d while tau is a (d+1)-th
    difference), and the distant-future recurrence of Formula 1 extrapolates
    polynomially, so a product's rounding error grows with the square of the
    number of intervals marched for d = 2 (Eq. m2l_expand_rec1).
      precision 0 (FP64): rounding 1e-16 x 1e5 x (40 intervals)^2 < 1e-9
        (measured <= 2.4e-10);
      precision 1 (BF16 x 3 terms, 6 products, FP32 accumulation and FP32
        products: ~6e-8 per entry): 1e-2 on runs of up to 40 steps, 1e-1 on
        the 81-step d = 2 runs (measured 4.4e-3 and 4.1e-2; the d = 1 cases
        stay below 1e-6);
      precision 2 (BF16x3, ~2^-17) and 3 (BF16, ~2^-9): only the d = 1 cases
        (measured <= 2e-6 and <= 1.3e-3); for d = 2 their far field is off
        by 10 % or more, which the precision table in the design notes
        records;
      precision 4 (two FP16 terms scaled per row / per cell, ~2^-22, three
        products, FP32 accumulation): the bounds of precision 1;
      precision 5 (FFT form, equispaced nodes: FP32 transforms and
        products, ~6e-8 per operation times the log of the grid size): the
        bounds of precision 1 (measured 3.1e-3 on the 37-step d = 2 case,
        6.5e-5 and 1.8e-7 on the 81-step ones, <= 3.5e-7 for d = 1)."""
    if precision == 0:
        return 1e-9
    if precision in (1, 4, 5):
        return 1e-1 if (w.d >= 2 and nsteps > 40) else 1e-2
    return 1e-5 if precision == 2 else 1e-2


@pytest.mark.parametrize("precision", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("name,L,p,nsteps", CASES)
def test_fmm_far_field_matches_oracle(name, L, p, nsteps, precision):
    """precision 0: FP64 M2L; 1-4: M2L on the tcgen05 tensor cores with the
    operators and moments split into BF16 (1-3) or scaled FP16 (4) terms
    (FP64 locals and recurrence state); 5: the near-future blocks by the FFT
    on equispaced nodes, against the oracle's hierarchy with the same nodes
    and boxes.  Tolerances: see _tol."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    from tests.gpu_cases import gpu_solver
    w = workload(name, nt=nsteps + 2)
    if precision in (2, 3) and w.d >= 2:
        pytest.skip("BF16x3 / BF16 M2L far fields are not accurate for d = 2 (see _tol)")
    s = gpu_solver(w, depth=L, fmm=(p, p, 0), precision=precision)
    nodes = "equi" if precision == 5 else "cheb"
    try:
        st = s.stats()
        H = ofmm.Hierarchy(w.xyz, w.tri, L, w.c, w.dt, w.nt, p, p, w.d, nodes=nodes)
        assert (st["fmm_lt"], st["fmm_mu"]) == (H.Lt, H.mu)
        # near lists bit-exact with the oracle's leaf neighbour lists
        off = abi.tdbem_get_tree(s.ctx, "near_off")
        near = abi.tdbem_get_tree(s.ctx, "near")
        for i in range(w.ns):
            assert list(near[off[i]:off[i + 1]]) == [int(v) for v in H.T["near"][i]]
        s.step(nsteps)
        far, a0 = abi.tdbem_get_far(s.ctx, w.ns)
        assert a0 > 1
        u, q = s.solution(0, nsteps)
        rows = list(range(0, w.ns, max(1, w.ns // 12)))
        alphas = [a0 + t for t in range(H.Lt)]
        ref = ofmm.far_field(H, u, q, alphas, w.bie, rows=rows, m2l=ofmm.m2l_fft if precision == 5 else None)
        got = far[:, rows]
        scale = np.abs(ref).max()
        assert scale > 0
        err = np.abs(got - ref).max() / scale
        assert err <= _tol(precision, w, nsteps), (err, precision)
    finally:
        s.close()


def test_fmm_infeasible_hierarchy_is_reported():
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    from tests.gpu_cases import gpu_solver
    w = workload("ellipsoid320_bmbie_d2_hard_plane_s7", nt=10)
    with pytest.raises(abi.TdbemError) as e:
        gpu_solver(w, depth=3, fmm=(3, 3, 0))  # leaf cells smaller than 2 rho
    assert e.value.code == -7


@pytest.mark.parametrize("precision", [0, 1, 4, 5])
@pytest.mark.parametrize("p", [4, 5])
def test_fmm_depth4_far_field_two_intervals(p, precision):
    """Depth 4 (levels 2-4 with interaction pairs, every symmetry class of
    the offsets), ps = pt = 4 and 5, on the seeded 5120-element ellipsoid:
    the far field of rows spread over different leaves, observed in two leaf
    intervals of the march, against the oracle's plain route.  These short
    runs stay in the near-future regime where rounding is not yet amplified,
    so the bounds are tighter than _tol's: FP64 1e-10 (measured <= 1.3e-14),
    the tensor-core forms 1e-4 (measured <= 5.4e-6 for precision 1 and
    <= 2.9e-6 for precision 4), the FFT form's FP32 transforms 1e-3
    (measured <= 4.4e-5 at p = 4 and <= 2.9e-4 at p = 5)."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    from tests.gpu_cases import gpu_solver
    w = workload("ellipsoid5120_bmbie_d2_hard_plane_s3", nt=34)
    L = 4
    tol = 1e-10 if precision == 0 else 1e-3 if precision == 5 else 1e-4
    nodes = "equi" if precision == 5 else "cheb"
    H = ofmm.Hierarchy(w.xyz, w.tri, L, w.c, w.dt, w.nt, p, p, w.d, nodes=nodes)
    s = gpu_solver(w, depth=L, fmm=(p, p, 0), precision=precision)
    try:
        st = s.stats()
        assert (st["fmm_lt"], st["fmm_mu"]) == (H.Lt, H.mu)
        # rows from 12 different leaf cells
        leaf = H.cell[L]
        rows, seen = [], set()
        for i in range(0, w.ns, 37):
            if int(leaf[i]) not in seen:
                seen.add(int(leaf[i]))
                rows.append(i)
            if len(rows) == 12:
                break
        for nsteps in (19, 31):
            s.step(nsteps - abi.tdbem_steps_done(s.ctx))
            far, a0 = abi.tdbem_get_far(s.ctx, w.ns)
            u, q = s.solution(0, nsteps)
            alphas = [a0 + t for t in range(H.Lt)]
            ref = ofmm.far_field(H, u, q, alphas, w.bie, rows=rows, m2l=ofmm.m2l_fft if precision == 5 else None)
            scale = np.abs(ref).max()
            assert scale > 0
            err = np.abs(far[:, rows] - ref).max() / scale
            assert err <= tol, (nsteps, err, precision)
    finally:
        s.close()
