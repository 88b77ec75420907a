"""The allocation-free truncated SVD (tn_truncated_svd_noalloc) against tn_truncated_svd.

It serves callers that cannot allocate device memory when they need the
projector SVD (memory held by another allocator, no tolerance for the
synchronisation of cudaMalloc, no context workspace): only their buffers go
in, the scratch is a fixed array inside the library.  Two calls in a row, with
different sizes, check that the shared scratch left by a call does not leak
into the next.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _matrix(m, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = 10.0 ** (-np.arange(m) / 6.0)
    return torch.from_numpy((Q1 * s) @ Q2.T).to("cuda")


def _bufs(m, k):
    return (torch.empty((m, k), dtype=torch.float64, device="cuda"),
            torch.empty(k, dtype=torch.float64, device="cuda"),
            torch.empty((m, k), dtype=torch.float64, device="cuda"))


def test_noalloc_matches_context_version_two_calls():
    ctx = L.Context(4, 64)
    for m, k, seed in ((1024, 64, 1), (300, 40, 2), (96, 20, 3)):   # consecutive calls, shrinking sizes
        M = _matrix(m, seed)
        U0, S0, V0 = _bufs(m, k)
        U1, S1, V1 = _bufs(m, k)
        L.tn_truncated_svd(ctx, M, m, k, U0, S0, V0)
        L.tn_truncated_svd_noalloc(M, m, k, U1, S1, V1)
        torch.cuda.synchronize()
        # same tolerance as the truncated-SVD tests: values to 1e-13, vectors where
        # s_i > 1e-8 s_1 (below that FP64 fixes a direction only to ~eps s_1 / s_i,
        # and the two entry points may sum their products in different orders)
        S = S0.cpu().numpy()
        good = S > 1e-8 * S[0]
        np.testing.assert_allclose(S1.cpu().numpy(), S, rtol=0, atol=1e-13)
        np.testing.assert_allclose(U1.cpu().numpy()[:, good], U0.cpu().numpy()[:, good], atol=1e-6)
        np.testing.assert_allclose(V1.cpu().numpy()[:, good], V0.cpu().numpy()[:, good], atol=1e-6)
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    m, k = 4096, 96
    M = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    U, S, V = _bufs(m, k)
    with pytest.raises(L.TnError) as err:
        L.tn_truncated_svd_noalloc(M, m, k, U, S, V)
    assert err.value.status == L.TN_ESCRATCH
