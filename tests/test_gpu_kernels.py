"""GPU parity of the kernel-level entry points against numpy (FP64)."""
import numpy as np
import pytest

from oracle.ctmrg import sign_fix
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_batched_ragged(ta, tb):
    m, n, k, batch = 70, 45, 133, 3
    A = random_matrix((batch, k, m) if ta else (batch, m, k), instance=1)
    Bm = random_matrix((batch, n, k) if tb else (batch, k, n), instance=2)
    C = random_matrix((batch, m, n), instance=3)
    dA, dB, dC = _dev(A), _dev(Bm), _dev(C)
    L.tn_gemm_f64(ta, tb, m, n, k, 1.5, dA, m if ta else k, A[0].size, dB, k if tb else n, Bm[0].size,
                  -0.5, dC, n, C[0].size, batch)
    torch.cuda.synchronize()
    opA = A.transpose(0, 2, 1) if ta else A
    opB = Bm.transpose(0, 2, 1) if tb else Bm
    ref = 1.5 * opA @ opB - 0.5 * C
    np.testing.assert_allclose(dC.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)


def test_gemm_large_square():
    n = 1024
    A, Bm = random_matrix((n, n), instance=4), random_matrix((n, n), instance=5)
    dC = torch.empty((n, n), dtype=torch.float64, device="cuda")
    L.tn_gemm_f64(0, 0, n, n, n, 1.0, _dev(A), n, 0, _dev(Bm), n, 0, 0.0, dC, n, 0, 1)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dC.cpu().numpy(), A @ Bm, rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("dims,perm", [((3, 4, 5, 6, 2), (4, 0, 3, 1, 2)), ((7, 9), (1, 0)),
                                        ((2, 3, 4, 5, 2, 3, 2, 2), (7, 6, 5, 4, 3, 2, 1, 0))])
def test_permute(dims, perm):
    x = random_matrix(dims, instance=6)
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    L.tn_permute_f64(_dev(x), out, dims, perm)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().reshape([dims[p] for p in perm]), x.transpose(perm))


@pytest.mark.parametrize("m,n", [(8, 8), (33, 20), (64, 64), (112, 112), (2, 1)])
def test_svd_small(m, n):
    batch = 3
    A = random_matrix((batch, m, n), instance=7)
    dU = torch.empty((batch, m, n), dtype=torch.float64, device="cuda")
    dS = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    dV = torch.empty((batch, n, n), dtype=torch.float64, device="cuda")
    L.tn_svd_small(_dev(A), m, n, batch, dU, dS, dV)
    torch.cuda.synchronize()
    U, S, V = dU.cpu().numpy(), dS.cpu().numpy(), dV.cpu().numpy()
    for b in range(batch):
        Ur, Sr, Vtr = np.linalg.svd(A[b], full_matrices=False)
        Ur, Vr = sign_fix(Ur, Vtr.T)
        np.testing.assert_allclose(S[b], Sr, rtol=0, atol=1e-12 * Sr[0])
        np.testing.assert_allclose((U[b] * S[b]) @ V[b].T, A[b], atol=1e-12 * Sr[0])
        np.testing.assert_allclose(U[b], Ur, atol=1e-8)          # random spectra are well separated
        np.testing.assert_allclose(V[b], Vr, atol=1e-8)


@pytest.mark.parametrize("n", [1, 7, 50, 112])
def test_eigh_small(n):
    batch = 2
    X = random_matrix((batch, n, n), instance=8)
    A = X + X.transpose(0, 2, 1)
    dW = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    dV = torch.empty((batch, n, n), dtype=torch.float64, device="cuda")
    L.tn_eigh_small(_dev(A), n, batch, dW, dV)
    torch.cuda.synchronize()
    W, V = dW.cpu().numpy(), dV.cpu().numpy()
    for b in range(batch):
        wr = np.linalg.eigvalsh(A[b])
        scale = np.abs(wr).max()
        np.testing.assert_allclose(W[b], wr, atol=1e-12 * scale)
        np.testing.assert_allclose((V[b] * W[b]) @ V[b].T, A[b], atol=1e-11 * scale)
        np.testing.assert_allclose(V[b].T @ V[b], np.eye(n), atol=1e-12)


@pytest.mark.parametrize("m,k,warm", [(300, 40, False), (1024, 64, False), (1024, 64, True), (96, 20, False)])
def test_truncated_svd(m, k, warm):
    """Top-k triplets of a matrix with a decaying spectrum, against the exact factors."""
    rng = np.random.default_rng(9)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = 10.0 ** (-np.arange(m) / 6.0)
    M = (Q1 * s) @ Q2.T
    ctx = L.Context(4, 64)
    dU = torch.empty((m, k), dtype=torch.float64, device="cuda")
    dS = torch.empty(k, dtype=torch.float64, device="cuda")
    dV = torch.empty((m, k), dtype=torch.float64, device="cuda")
    Ur, Vr = sign_fix(Q1[:, :k], Q2[:, :k])
    w = _dev(Vr + 1e-3 * rng.standard_normal(Vr.shape)) if warm else None
    L.tn_truncated_svd(ctx, _dev(M), m, k, dU, dS, dV, w)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dS.cpu().numpy(), s[:k], rtol=0, atol=1e-13)
    # singular vectors: accurate where s_i is well above the noise floor
    good = s[:k] > 1e-8
    np.testing.assert_allclose(dU.cpu().numpy()[:, good], Ur[:, good], atol=1e-6)
    np.testing.assert_allclose(dV.cpu().numpy()[:, good], Vr[:, good], atol=1e-6)
    ctx.close()
