"""Split-precision tensor-core GEMM (tcgen05, TF32 x3 and BF16 x3) against FP64 numpy.

Error model of the split product (x = hi + lo, hi.hi + hi.lo + lo.hi accumulated
in FP32): per product term about u^2 |a||b| with u the unit roundoff of the
head type (2^-11 TF32, 2^-8 BF16) plus FP32 accumulation, 2^-24 per addition.
The tests bound the error elementwise by a multiple of (|A| |B|)_ij and in
relative Frobenius norm.
"""
import numpy as np
import pytest

from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (relative Frobenius, elementwise vs |A||B|) per precision
TOL = {L.TN_TF32X3: (2e-6, 2e-5), L.TN_BF16X3: (6e-5, 3e-4)}


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


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_split_gemm_ragged(prec, ta, tb):
    """Several tiles with ragged edges in m, n and k, all transpose cases, beta != 0."""
    C, ref, scale = _run(prec, ta, tb, 200, 150, 70, alpha=1.5, beta=-0.5)
    fro, elem = TOL[prec]
    assert np.linalg.norm(C - ref) / np.linalg.norm(ref) < fro
    assert np.max(np.abs(C - ref) / scale) < elem


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3])
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
