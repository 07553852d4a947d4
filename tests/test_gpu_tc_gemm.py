"""The split-precision tensor-core GEMM (tcgen05.mma with TMEM accumulators,
operands loaded by TMA) against a float64 numpy product of the same 16-bit
operands: ragged tile edges in both output dimensions, K not a multiple of
the 64-element chunk, 1-3 split terms per operand, BF16 and FP16, and both
tile widths.  The only rounding on the GPU side is the FP32 accumulation."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _to16(x, fmt):
    """Round float64 -> BF16 (fmt 1) or FP16 (fmt 0), returned as bit patterns
    and as the float64 values they represent (test input preparation)."""
    if fmt == 0:
        h = x.astype(np.float16)
        return h.view(np.uint16), h.astype(np.float64)
    f = x.astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)  # round to nearest even
    back = (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return r, back


def _split(x, nterm, fmt):
    bits, vals, rest = [], [], x.copy()
    for _ in range(nterm):
        b, v = _to16(rest, fmt)
        bits.append(b)
        vals.append(v)
        rest = rest - v
    return np.stack(bits), np.stack(vals)


@pytest.mark.parametrize("m,n,k,nta,ntb,prod,fmt,bn", [
    (200, 300, 100, 1, 1, [(0, 0)], 1, 128),
    (128, 128, 64, 2, 2, [(0, 0), (0, 1), (1, 0)], 1, 128),
    (333, 77, 648, 3, 3, [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)], 1, 128),
    (130, 520, 256, 2, 2, [(0, 0), (0, 1), (1, 0)], 1, 256),
    (257, 129, 200, 2, 2, [(0, 0), (0, 1), (1, 0)], 0, 128),
    # more tiles than SMs: each persistent CTA takes several tiles, both
    # TMEM accumulators and the ring's phases wrap across tile boundaries
    (2600, 2700, 192, 2, 2, [(0, 0), (0, 1), (1, 0)], 1, 128),
    (1300, 6000, 100, 1, 1, [(0, 0)], 1, 256),
])
def test_tc_gemm_matches_numpy(m, n, k, nta, ntb, prod, fmt, bn):
    from paper_2111_05205_gb300 import abi, build
    build.build()
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    if fmt == 0:
        A *= 0.25
        B *= 0.25
    ab, av = _split(A, nta, fmt)
    bb, bv = _split(B, ntb, fmt)
    c = abi.tdbem_tc_gemm_check(ab, bb, prod, fmt=fmt, bn=bn)
    ref = sum(bv[t] @ av[s].T for s, t in prod)  # [n, m]
    bound = sum(np.abs(bv[t]) @ np.abs(av[s]).T for s, t in prod)
    err = np.abs(c.astype(np.float64) - ref)
    assert np.all(err <= 2e-6 * bound + 1e-30), float((err / bound).max())


def test_tc_gemm_split_reaches_fp32_accuracy():
    """Three BF16 terms per operand with the six leading products give a
    product of the FP64 operands to about FP32 accuracy, far better than two
    terms with three products (~2^-17).  Positive operands and K = 3, so
    that neither the FP32 accumulation in tensor memory (~2^-24 per add) nor
    averaging over a long K hides the products' own error."""
    from paper_2111_05205_gb300 import abi, build
    build.build()
    rng = np.random.default_rng(5)
    m, n, k = 256, 128, 3
    A = rng.uniform(0.5, 1.0, (m, k))
    B = rng.uniform(0.5, 1.0, (n, k))
    ref = B @ A.T
    ab3, _ = _split(A, 3, 1)
    bb3, _ = _split(B, 3, 1)
    c3 = abi.tdbem_tc_gemm_check(ab3, bb3, [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)])
    ab2, _ = _split(A, 2, 1)
    bb2, _ = _split(B, 2, 1)
    c2 = abi.tdbem_tc_gemm_check(ab2, bb2, [(0, 0), (0, 1), (1, 0)])
    e3 = np.max(np.abs(c3 - ref) / ref)
    e2 = np.max(np.abs(c2 - ref) / ref)
    assert e3 < 1.5e-6, e3
    assert e3 < 0.1 * e2, (e3, e2)
