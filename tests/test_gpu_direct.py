"""Parity of the CUDA direct time-marching path with the FP64 oracle.

Every case runs the same seeded synthetic workload through the C ABI and
through ``oracle.mot`` / ``oracle.coeffs`` and compares element by element.
Tolerances (floating point, FP64 on both sides): influence coefficients
1e-13 relative to the largest coefficient of the kind (both sides integrate
to ~1e-15); the zero-lag matrix likewise; whole solution histories 1e-12
relative L2 for the FP64 path (the error of the zero-lag iteration is
bounded by 1e-16 per step) and 1e-11 for the split-precision history sum
(48-bit float-pair products).  Integer lag windows
bit-exact against the oracle's support bound.
"""

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import mot
from tests.gpu_cases import case, gpu_march, gpu_solver, known_samples, phi_of, rel_l2

pytestmark = pytest.mark.gpu

KIND = {"cu": 0, "cw": 1, "ub": 2, "wb": 3}


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(autouse=True, scope="module")
def _built():
    _need_gpu()
    from paper_2111_05205_gb300 import build
    build.build()


MOT_CASES = [
    "sphere320_obie_d1_dirichlet_uniform",   # 320 elements: 10 row blocks, ragged tail of 0
    "sphere80_obie_d1_neumann_uniform",      # 80: ragged 2.5 blocks
    "sphere80_obie_d2_neumann_uniform",
    "sphere80_bmbie_d2_neumann_uniform",
    "sphere80_bmbie_d1_dirichlet_uniform",
    "sphere80_bmbie_d3_neumann_uniform",
    "ellipsoid80_bmbie_d2_hard_plane_s7",
    "ellipsoid80_bmbie_d1_soft_plane_s5",
    "ellipsoid320_bmbie_d2_hard_plane_s11",
    # the paper's sphere (Section 5.1.1) with its raised-cosine pulse
    "paper_sphere80_bmbie_d2_hard",
    "paper_sphere80_bmbie_d1_soft",
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", MOT_CASES)
def test_direct_march_matches_oracle(name, precision):
    w = case(name, nt=48 if "320" in name else 40)
    u, q, st = gpu_march(w, precision=precision)
    uo, qo = mot.march(w)
    X, Xo = (u, uo) if w.bc == "neumann" else (q, qo)
    assert np.isfinite(X).all()
    # FP64: 1e-12.  Split: each product carries ~2^-46 relative error (48-bit
    # float pairs), 128x the FP64 rounding, so 1e-11 on the same cases (the
    # OBIE ones amplify rounding through the marching).
    tol = 1e-12 if precision == 0 else 1e-11
    assert rel_l2(X, Xo) <= tol, (rel_l2(X, Xo), st)
    # the known component is the collocated input (for d = 3 the collocation
    # recurrence itself grows without bound, amplifying rounding)
    K, Ko = (q, qo) if w.bc == "neumann" else (u, uo)
    assert rel_l2(K, Ko) <= (1e-14 if w.d < 3 else 1e-12) or np.linalg.norm(Ko) == 0


@pytest.mark.parametrize("name,kinds", [
    ("sphere80_obie_d1_dirichlet_uniform", ("cu", "cw")),
    ("sphere80_bmbie_d2_neumann_uniform", ("ub", "wb")),
    ("ellipsoid80_bmbie_d3_neumann_uniform_s3", ("ub", "wb")),
])
def test_coefficients_match_oracle(name, kinds):
    if name.startswith("ellipsoid"):
        w = case("ellipsoid80_bmbie_d2_hard_plane_s3")
        w.d, w.excitation, w.nt = 3, "uniform", 40
    else:
        w = case(name, nt=40)
    cdt = w.c * w.dt
    s = gpu_solver(w)
    try:
        gmax = min(oc.gamma_max(w.xyz, w.tri, w.d, cdt), w.nt - 1)
        dense = oc.dense(w.xyz, w.tri, w.d, cdt, kinds=kinds, gmax=gmax)
        from paper_2111_05205_gb300 import abi
        rows = np.arange(w.ns)
        for k in kinds:
            g = abi.tdbem_get_coefficients(s.ctx, KIND[k], rows, gmax, w.ns)  # [i, g, j]
            o = dense[k].transpose(1, 0, 2)
            scale = np.abs(o).max()
            assert np.abs(g - o).max() <= 1e-13 * scale, (k, np.abs(g - o).max(), scale)
    finally:
        s.close()


def test_zero_lag_matrix_matches_oracle():
    from paper_2111_05205_gb300 import abi
    w = case("ellipsoid80_bmbie_d2_hard_plane_s7", nt=8)
    cdt = w.c * w.dt
    s = gpu_solver(w)
    try:
        A = abi.tdbem_get_zero_lag(s.ctx, w.ns)
        C = oc.dense(w.xyz, w.tri, w.d, cdt, kinds=("wb",), gmax=1)
        Ao = -C["wb"][1]  # sound-hard: phi = 1, A = -Wbar^(1)
        assert np.abs(A - Ao).max() <= 1e-13 * np.abs(Ao).max()
        st = s.stats()
        assert 0 < st["solve_contraction"] < 1
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_deterministic_bitwise(precision):
    w = case("ellipsoid80_bmbie_d2_hard_plane_s7", nt=30)
    u1, _, _ = gpu_march(w, precision)
    u2, _, _ = gpu_march(w, precision)
    assert np.array_equal(u1, u2)


def test_split_coefficients_round_trip():
    """The float-pair store keeps 48 significant bits of every coefficient."""
    from paper_2111_05205_gb300 import abi
    w = case("sphere80_bmbie_d2_neumann_uniform", nt=20)
    s0, s1 = gpu_solver(w, precision=0), gpu_solver(w, precision=1)
    try:
        rows = np.arange(0, w.ns, 7)
        a = abi.tdbem_get_coefficients(s0.ctx, 3, rows, 19, w.ns)
        b = abi.tdbem_get_coefficients(s1.ctx, 3, rows, 19, w.ns)
        assert np.abs(a - b).max() <= 2.0 ** -47 * np.abs(a).max()
    finally:
        s0.close()
        s1.close()


def test_step_io_excitation_and_output():
    """The excitation supplied per step through tdbem_step_io (here the
    oracle's own incident term, an input) gives the oracle's solution, and
    x_out returns the unknown of each step."""
    from paper_2111_05205_gb300 import abi
    w = case("ellipsoid80_bmbie_d2_hard_plane_s7", nt=30)
    v, xc, n, _ = oc.geometry(w.xyz, w.tri)
    exc = np.stack([mot.incident_rhs(w, xc, n, a) for a in range(1, w.nt)])
    w_noinc = case("ellipsoid80_bmbie_d2_hard_plane_s7", nt=30)
    w_noinc.excitation = "none"
    s = gpu_solver(w_noinc)
    try:
        x = np.zeros((w.nt - 1, w.ns))
        half = (w.nt - 1) // 2
        abi.tdbem_step_io(s.ctx, half, np.ascontiguousarray(exc[:half]), x[:half])
        rest = w.nt - 1 - half
        xo_part = np.zeros((rest, w.ns))
        abi.tdbem_step_io(s.ctx, rest, np.ascontiguousarray(exc[half:]), xo_part)
        x[half:] = xo_part
        u, q = s.solution()
    finally:
        s.close()
    uo, _ = mot.march(w)
    assert rel_l2(u, uo) <= 1e-12
    assert np.array_equal(x, u)


def test_single_step_and_single_element_edge_cases():
    # Nt = 2: exactly one step
    w = case("sphere80_obie_d1_dirichlet_uniform", nt=2)
    u, q, _ = gpu_march(w)
    uo, qo = mot.march(w)
    assert q.shape == (1, 80) and rel_l2(q, qo) <= 1e-12
    # a single element: one 32-pair block with 31 empty lanes
    from paper_2111_05205_gb300 import Solver
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    f = np.exp(-((np.arange(1, 12) * 0.2 - 1.0) / 0.4) ** 2)[:, None]
    s = Solver(xyz, tri, 1.0, 0.2, 12, 2, "obie", phi=np.zeros(1, np.int8), known=f)
    try:
        s.step()
        uu, qq = s.solution()
    finally:
        s.close()
    from synth.workloads import Workload
    ww = Workload("one", xyz, tri, 1.0, 0.2, 12, 2, "obie", "dirichlet", "uniform", sigma=0.4)
    # oracle's known data: gauss(t; sigma, 4 sigma) with 4 sigma = 1.6; use the same f
    ww.sigma = 0.4
    uo, qo = _march_with_known(ww, f[:, 0])
    assert rel_l2(qq[:, 0], qo[:, 0]) <= 1e-12


def _march_with_known(w, f):
    """Oracle march with the known samples f(t_a) given explicitly."""
    import types
    orig = mot.known_coefficients

    def kc(w_, nt):
        d = w_.d
        Nv = [oc.N(d, float(g)) for g in range(d + 2)]
        fb = np.zeros(nt)
        for a in range(1, nt):
            s = f[a - 1]
            for g in range(2, d + 1):
                if a - g >= 0:
                    s -= Nv[g] * fb[a - g]
            fb[a - 1] = s / Nv[1]
        return fb
    mot.known_coefficients = kc
    try:
        return mot.march(w)
    finally:
        mot.known_coefficients = orig


def test_errors_are_reported_not_crashes():
    from paper_2111_05205_gb300 import abi
    w = case("sphere80_obie_d1_dirichlet_uniform", nt=5)
    s = gpu_solver(w)
    try:
        s.step()
        with pytest.raises(abi.TdbemError):
            abi.tdbem_step(s.ctx, 1)  # past Nt-1
        with pytest.raises(abi.TdbemError):
            abi.tdbem_get_coefficients(s.ctx, 3, [0], 4, w.ns)  # kind not stored
    finally:
        s.close()
    p = abi.tdbem_params()
    p.c, p.dt, p.nt, p.d, p.bie = 1.0, 0.1, 10, 7, 0
    with pytest.raises(abi.TdbemError):
        abi.tdbem_create(p)
