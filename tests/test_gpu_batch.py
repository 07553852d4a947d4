"""Graph-replayed steps and the batched multi-instance driver give results
identical (bit for bit) to plain stepping: the same kernels on the same
data, only launched from a captured CUDA graph, and for the batch from one
graph in which each instance is an independent branch.  Instances differ in
mesh size, B-spline order, BIE, boundary condition, precision, Nt and
algorithm (direct path or space-time FMM)."""

import numpy as np
import pytest

from tests.gpu_cases import case, gpu_solver

pytestmark = pytest.mark.gpu

INSTANCES = [
    ("ellipsoid80_bmbie_d2_hard_plane_s7", 0),
    ("ellipsoid320_bmbie_d2_hard_plane_s11", 1),
    ("sphere320_obie_d1_dirichlet_uniform", 0),
    ("sphere80_bmbie_d1_dirichlet_uniform", 1),
    ("ellipsoid80_bmbie_d1_soft_plane_s5", 1),
    ("sphere80_obie_d2_neumann_uniform", 0),
]


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _unknown(s, w, n):
    u, q = s.solution(0, n)
    return u if w.bc == "neumann" else q


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_steps_equal_plain_steps(precision):
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    w = case("ellipsoid320_bmbie_d2_hard_plane_s11", nt=40)
    a, b = gpu_solver(w, precision=precision), gpu_solver(w, precision=precision)
    try:
        abi.tdbem_step(a.ctx, 39)
        abi.tdbem_step(b.ctx, 3)          # mixed: plain, then graph
        abi.tdbem_step_graph(b.ctx, 30)
        abi.tdbem_step_graph(b.ctx, 6)
        assert abi.tdbem_steps_done(b.ctx) == 39
        assert np.array_equal(_unknown(a, w, 39), _unknown(b, w, 39))
    finally:
        a.close()
        b.close()


def test_batch_equals_each_instance_alone():
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    nsteps = 30
    ws = [case(n, nt=nsteps + 1) for n, _ in INSTANCES]
    ref = []
    for w, (n, prec) in zip(ws, INSTANCES):
        s = gpu_solver(w, precision=prec)
        try:
            abi.tdbem_step(s.ctx, nsteps)
            ref.append(_unknown(s, w, nsteps))
        finally:
            s.close()
    sols = [gpu_solver(w, precision=prec) for w, (n, prec) in zip(ws, INSTANCES)]
    try:
        B = abi.tdbem_batch_create([s.ctx for s in sols])
        try:
            abi.tdbem_batch_step(B, 10)
            abi.tdbem_batch_step(B, nsteps - 10)
            abi.tdbem_batch_sync(B)
            abi.tdbem_batch_step(B, 5)  # every instance at Nt-1: nothing happens
            abi.tdbem_batch_sync(B)
        finally:
            abi.tdbem_batch_destroy(B)
        for s, w, r in zip(sols, ws, ref):
            assert abi.tdbem_steps_done(s.ctx) == nsteps
            assert np.array_equal(_unknown(s, w, nsteps), r)
    finally:
        for s in sols:
            s.close()


def test_batch_rejects_fp64_fmm_and_duplicates():
    """The FP64 FMM form's GEMMs are library calls that cannot read the
    device-side step, so its steps are not graph-replayed."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    w = case("ellipsoid320_bmbie_d2_hard_plane_s7", nt=10)
    f = gpu_solver(w, depth=2, fmm=(2, 2, 0))
    d = gpu_solver(w)
    try:
        with pytest.raises(abi.TdbemError):
            abi.tdbem_batch_create([d.ctx, f.ctx])
        with pytest.raises(abi.TdbemError):
            abi.tdbem_batch_create([d.ctx, d.ctx])
        with pytest.raises(abi.TdbemError):
            abi.tdbem_step_graph(f.ctx, 1)
    finally:
        f.close()
        d.close()


# FMM instances: depth 3 crosses leaf boundaries every Lt steps and level-2
# boundaries every 2 Lt; the 81-step runs reach the distant-future
# recurrence of Formula 1
FMM_CASES = [
    ("sphere1280_bmbie_d2_neumann_uniform", 3, (2, 2, 0), 1, 81),
    ("sphere1280_bmbie_d1_dirichlet_uniform", 3, (3, 3, 0), 2, 40),
    ("ellipsoid320_bmbie_d2_hard_plane_s7", 2, (3, 3, 0), 1, 37),
    # the FFT form of the M2L
    ("sphere1280_bmbie_d2_neumann_uniform", 3, (2, 2, 0), 5, 81),
]


@pytest.mark.parametrize("name,L,fmm,precision,nt", FMM_CASES)
def test_graph_fmm_steps_equal_plain_steps(name, L, fmm, precision, nt):
    """FMM steps replayed from one captured graph (every far-field kernel
    decides on the device whether this step is one of its boundaries) give
    the same history, bit for bit, as plain stepping, including plain steps
    before and after graph steps."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    w = case(name, nt=nt)
    a = gpu_solver(w, precision=precision, depth=L, fmm=fmm)
    b = gpu_solver(w, precision=precision, depth=L, fmm=fmm)
    try:
        n = nt - 1
        abi.tdbem_step(a.ctx, n)
        abi.tdbem_step(b.ctx, 5)           # plain, then graph, then plain
        abi.tdbem_step_graph(b.ctx, n - 12)
        abi.tdbem_step(b.ctx, 4)
        abi.tdbem_step_graph(b.ctx, 3)
        assert abi.tdbem_steps_done(b.ctx) == n
        ua, qa = a.solution(0, n)
        ub, qb = b.solution(0, n)
        assert np.abs(ua).max() + np.abs(qa).max() > 0
        assert np.array_equal(ua, ub) and np.array_equal(qa, qb)
    finally:
        a.close()
        b.close()


def test_batch_with_fmm_instances_of_uneven_nt():
    """FMM and direct instances of different meshes, orders, BIEs,
    precisions and Nt in one batch graph: each history equals the instance
    stepped alone (bit for bit)."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    spec = [("sphere1280_bmbie_d2_neumann_uniform", 1, 3, (2, 2, 0), 81),
            ("ellipsoid80_bmbie_d2_hard_plane_s7", 1, 0, None, 30),
            ("sphere1280_bmbie_d1_dirichlet_uniform", 3, 3, (3, 3, 0), 52),
            ("ellipsoid320_bmbie_d2_hard_plane_s7", 1, 2, (3, 3, 0), 37)]
    ws = [case(n, nt=nt) for n, _, _, _, nt in spec]

    def make(w, prec, L, fmm):
        return gpu_solver(w, precision=prec, depth=L, fmm=fmm) if fmm else gpu_solver(w, precision=prec)

    ref = []
    for w, (n, prec, L, fmm, nt) in zip(ws, spec):
        s = make(w, prec, L, fmm)
        try:
            abi.tdbem_step(s.ctx, nt - 1)
            ref.append(s.solution(0, nt - 1))
        finally:
            s.close()
    sols = [make(w, prec, L, fmm) for w, (n, prec, L, fmm, nt) in zip(ws, spec)]
    try:
        # 8 steps of every instance per graph launch (and single steps for
        # the remainders)
        B = abi.tdbem_batch_create_steps([s.ctx for s in sols], 8)
        try:
            abi.tdbem_batch_step(B, 9)
            abi.tdbem_batch_step(B, 40)
            abi.tdbem_batch_step(B, 100)
            abi.tdbem_batch_sync(B)
        finally:
            abi.tdbem_batch_destroy(B)
        for s, r, (n, prec, L, fmm, nt) in zip(sols, ref, spec):
            assert abi.tdbem_steps_done(s.ctx) == nt - 1
            u, q = s.solution(0, nt - 1)
            assert np.array_equal(u, r[0]) and np.array_equal(q, r[1]), n
    finally:
        for s in sols:
            s.close()


def test_batch_of_uneven_nt():
    """Instances of different Nt in one batch: each stops at its own step
    Nt-1 (its kernels see the device-side step counter past the end and do
    nothing) while the others go on, and every history equals the instance
    stepped alone to its end."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    spec = [("ellipsoid80_bmbie_d2_hard_plane_s7", 0, 12), ("ellipsoid320_obie_d1_hard_plane_s3", 1, 30),
            ("sphere80_bmbie_d1_dirichlet_uniform", 1, 21), ("ellipsoid80_bmbie_d2_hard_plane_s9", 1, 40)]
    ws = [case(n, nt=nt) for n, _, nt in spec]
    ref = []
    for w, (n, prec, nt) in zip(ws, spec):
        s = gpu_solver(w, precision=prec)
        try:
            abi.tdbem_step(s.ctx, nt - 1)
            ref.append(_unknown(s, w, nt - 1))
        finally:
            s.close()
    sols = [gpu_solver(w, precision=prec) for w, (n, prec, nt) in zip(ws, spec)]
    try:
        B = abi.tdbem_batch_create([s.ctx for s in sols])
        try:
            abi.tdbem_batch_step(B, 7)
            abi.tdbem_batch_step(B, 25)  # the first instance stops at 11, the third at 20
            abi.tdbem_batch_step(B, 100)  # the last goes to 39
            abi.tdbem_batch_sync(B)
        finally:
            abi.tdbem_batch_destroy(B)
        for s, w, r, (n, prec, nt) in zip(sols, ws, ref, spec):
            assert abi.tdbem_steps_done(s.ctx) == nt - 1
            assert np.array_equal(_unknown(s, w, nt - 1), r)
    finally:
        for s in sols:
            s.close()


@pytest.mark.parametrize("precision", [4, 5])
def test_overlapped_far_field_equals_sequential(precision):
    """Plain FMM stepping runs the part of each boundary's far-field work
    that only later boundaries need on a second stream, beside the following
    steps; the sequential schedule (tdbem_set_overlap 0) gives the same
    history bit for bit, also when the schedule changes mid-march and across
    checkpoint/restore (scaled FP16 GEMM form and FFT form)."""
    _need_gpu()
    from paper_2111_05205_gb300 import abi
    w = case("sphere1280_bmbie_d2_neumann_uniform", nt=81)
    a = gpu_solver(w, precision=precision, depth=3, fmm=(3, 3, 0))
    b = gpu_solver(w, precision=precision, depth=3, fmm=(3, 3, 0))
    try:
        abi.tdbem_set_overlap(b.ctx, 0)
        abi.tdbem_step(a.ctx, 40)
        blob = abi.tdbem_checkpoint(a.ctx)
        abi.tdbem_step(a.ctx, 40)
        abi.tdbem_step(b.ctx, 25)
        abi.tdbem_set_overlap(b.ctx, 1)
        abi.tdbem_step(b.ctx, 30)
        abi.tdbem_set_overlap(b.ctx, 0)
        abi.tdbem_step(b.ctx, 25)
        ua, qa = a.solution()
        ub, qb = b.solution()
        assert np.abs(ua).max() > 0
        assert np.array_equal(ua, ub) and np.array_equal(qa, qb)
        # rewind the overlapped context and march again
        abi.tdbem_restore(a.ctx, blob)
        abi.tdbem_step(a.ctx, 40)
        assert np.array_equal(a.solution()[0], ua)
        with pytest.raises(abi.TdbemError):
            abi.tdbem_set_overlap(a.ctx, 2)
    finally:
        a.close()
        b.close()
