"""Split-precision tensor-core GEMM (tcgen05: TF32 x3, BF16 x3, BF16 integer slices) against FP64 numpy.

Error model of the head/tail split product (x = hi + lo, hi.hi + hi.lo + lo.hi
accumulated in FP32): per product term about u^2 |a||b| with u the unit
roundoff of the head type (2^-11 TF32, 2^-8 BF16) plus FP32 accumulation,
2^-24 per addition.  The tests bound the error elementwise by a multiple of
(|A| |B|)_ij and in relative Frobenius norm.

The integer-slice form (Ozaki scheme, TN_BF16S4) accumulates exactly; its only
error is the dropped levels of the truncated 8-bit slices: per term
< (S + 1) 2^-8S of 2^(e_i + f_j) <= 4 max|A_i.| max|B_.j|, i.e. for S = 4
|C - AB|_ij < 20 * 2^-32 * K * max|A_i.| * max|B_.j| (the bound tested below).
Truncation biases each term's error toward zero magnitude, but the signs of the
terms vary, so relative to |C| ~ sqrt(K) the Frobenius error on Gaussian
operands is about 2^-32 times the ratio of the row/column scale to a typical
entry (~4 for Gaussian rows): ~1e-9, bounded at 1e-8.  On integer operands that
the slices hold exactly the product must come out exact.
"""
import numpy as np
import pytest

from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (relative Frobenius, elementwise vs |A||B|) per precision
TOL = {L.TN_TF32X3: (2e-6, 2e-5), L.TN_BF16X3: (6e-5, 3e-4), L.TN_BF16S4: (1e-8, 3e-8), L.TN_F64S7: (1e-14, 1e-14)}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _run(prec, ta, tb, m, n, k, alpha=1.0, beta=0.0, inst=0):
    A = random_matrix((k, m) if ta else (m, k), instance=10 + inst)
    Bm = random_matrix((n, k) if tb else (k, n), instance=20 + inst)
    C0 = random_matrix((m, n), instance=30 + inst)
    dA, dB, dC = _dev(A), _dev(Bm), _dev(C0)
    nb = L.tn_gemm_split_workspace_bytes(prec, m, n, k)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    L.tn_gemm_split(prec, ta, tb, m, n, k, alpha, dA, m if ta else k, dB, k if tb else n, beta, dC, n, work)
    opA = A.T if ta else A
    opB = Bm.T if tb else Bm
    ref = alpha * opA @ opB + beta * C0
    scale = abs(alpha) * np.abs(opA) @ np.abs(opB) + abs(beta) * np.abs(C0)
    return dC.cpu().numpy(), ref, scale


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3, L.TN_BF16S4, L.TN_F64S7])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_split_gemm_ragged(prec, ta, tb):
    """Several tiles with ragged edges in m, n and k, all transpose cases, beta != 0."""
    C, ref, scale = _run(prec, ta, tb, 200, 150, 70, alpha=1.5, beta=-0.5)
    fro, elem = TOL[prec]
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < fro
    assert np.max(np.abs(C - ref) / scale) < elem


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3, L.TN_BF16S4, L.TN_F64S7])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 64, 32), (1024, 1024, 1024), (1024, 80, 1024), (80, 1024, 1024)])
def test_split_gemm_shapes(prec, m, n, k):
    """Single element, one exact tile, the enlarged-corner size N = chi D^2 = 1024 and skinny panels."""
    C, ref, scale = _run(prec, 0, 0, m, n, k, inst=1)
    fro, elem = TOL[prec]
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < fro
    assert np.max(np.abs(C - ref) / scale) < elem


def test_split_gemm_workspace_too_small():
    m = n = k = 64
    A = _dev(np.zeros((m, k)))
    work = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.TnError):
        L.tn_gemm_split(L.TN_TF32X3, 0, 0, m, n, k, 1.0, A, k, A, n, 0.0, A, n, work)


def test_split_gemm_repeatable():
    """Two calls on the same inputs give identical bits (fixed reduction order)."""
    C1, _, _ = _run(L.TN_TF32X3, 0, 1, 300, 260, 500, inst=2)
    C2, _, _ = _run(L.TN_TF32X3, 0, 1, 300, 260, 500, inst=2)
    assert np.array_equal(C1, C2)


def _slices_bound(A, Bm, k):
    """20 * 2^-32 * K * max|A_i.| * max|B_.j| (the dropped-slice bound of the integer-slice form)."""
    return 20.0 * 2.0 ** -32 * k * np.outer(np.abs(A).max(axis=1), np.abs(Bm).max(axis=0))


@pytest.mark.parametrize("m,n,k", [(200, 150, 70), (1024, 1024, 1024), (300, 260, 1000)])
def test_integer_slices_within_dropped_slice_bound(m, n, k):
    """Rows and columns of very different scales (the exponents are per row/column)."""
    rng = np.random.default_rng(m + n + k)
    A = random_matrix((m, k), instance=40) * 10.0 ** rng.uniform(-6, 6, (m, 1))
    Bm = random_matrix((k, n), instance=41) * 10.0 ** rng.uniform(-6, 6, (1, n))
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_BF16S4, m, n, k), dtype=torch.uint8, device="cuda")
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    L.tn_gemm_split(L.TN_BF16S4, 0, 0, m, n, k, 1.0, _dev(A), k, _dev(Bm), n, 0.0, dC, n, work)
    err = np.abs(dC.cpu().numpy() - A @ Bm)
    assert np.all(err <= _slices_bound(A, Bm, k) + 1e-15 * np.abs(A) @ np.abs(Bm))


@pytest.mark.parametrize("ta,tb,k", [(0, 0, 1024), (1, 1, 1000), (0, 1, 4096)])
def test_integer_slices_exact_on_integers(ta, tb, k):
    """Integer operands in [-255, 255] are held exactly by the slices, so every slice
    product, every FP32 partial sum (integers below 2^24) and the result are exact:
    the tensor-core accumulation must not round at all."""
    m, n = 256, 192
    rng = np.random.default_rng(k + ta)
    A = rng.integers(-255, 256, (k, m) if ta else (m, k)).astype(np.float64)
    Bm = rng.integers(-255, 256, (n, k) if tb else (k, n)).astype(np.float64)
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_BF16S4, m, n, k), dtype=torch.uint8, device="cuda")
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    L.tn_gemm_split(L.TN_BF16S4, ta, tb, m, n, k, 1.0, _dev(A), m if ta else k, _dev(Bm), k if tb else n, 0.0,
                    dC, n, work)
    opA = A.T if ta else A
    opB = Bm.T if tb else Bm
    assert np.array_equal(dC.cpu().numpy(), opA @ opB)      # integer sums below 2^53: numpy is exact too


def test_integer_slices_zero_rows_and_columns():
    m, n, k = 130, 70, 90
    A = random_matrix((m, k), instance=42)
    Bm = random_matrix((k, n), instance=43)
    A[[0, 5, 129]] = 0.0
    Bm[:, [3, 69]] = 0.0
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_BF16S4, m, n, k), dtype=torch.uint8, device="cuda")
    dC = torch.full((m, n), 7.0, dtype=torch.float64, device="cuda")
    L.tn_gemm_split(L.TN_BF16S4, 0, 0, m, n, k, 2.0, _dev(A), k, _dev(Bm), n, 0.5, dC, n, work)
    ref = 2.0 * A @ Bm + 3.5
    C = dC.cpu().numpy()
    np.testing.assert_array_equal(C[[0, 5, 129]], ref[[0, 5, 129]])
    np.testing.assert_array_equal(C[:, [3, 69]], ref[:, [3, 69]])
    assert np.abs(C - ref).max() < 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("m,n,k", [(1024, 112, 1024), (1024, 1024, 1024), (112, 112, 1024), (300, 70, 200)])
def test_seven_slices_exact_on_wide_integers(m, n, k):
    """Integers up to 2^20 need three 8-bit slices; all products and sums are exact
    integers below 2^53, so the FP64-accurate form must reproduce them bit for bit
    (panels and Gram blocks run with the K split and its partial sums)."""
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.integers(-2 ** 20, 2 ** 20 + 1, (m, k)).astype(np.float64)
    Bm = rng.integers(-2 ** 20, 2 ** 20 + 1, (k, n)).astype(np.float64)
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_F64S7, m, n, k), dtype=torch.uint8, device="cuda")
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    L.tn_gemm_split(L.TN_F64S7, 0, 0, m, n, k, 1.0, _dev(A), k, _dev(Bm), n, 0.0, dC, n, work)
    assert np.array_equal(dC.cpu().numpy(), A @ Bm)


def test_seven_slices_match_fp64_on_graded_rows():
    """Rows and columns spanning 12 orders of magnitude: relative to each entry's own
    scale (|A||B|) the error stays at the FP64 level."""
    m, n, k = 256, 192, 512
    rng = np.random.default_rng(5)
    A = random_matrix((m, k), instance=44) * 10.0 ** rng.uniform(-6, 6, (m, 1))
    Bm = random_matrix((k, n), instance=45) * 10.0 ** rng.uniform(-6, 6, (1, n))
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_F64S7, m, n, k), dtype=torch.uint8, device="cuda")
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    L.tn_gemm_split(L.TN_F64S7, 0, 0, m, n, k, 1.0, _dev(A), k, _dev(Bm), n, 0.0, dC, n, work)
    err = np.abs(dC.cpu().numpy() - A @ Bm)
    assert np.all(err <= 2.0 ** -50 * k * np.outer(np.abs(A).max(axis=1), np.abs(Bm).max(axis=0))
                  + 1e-15 * np.abs(A) @ np.abs(Bm))
