"""The allocation-free truncated SVD (tn_truncated_svd_noalloc) against tn_truncated_svd.

It serves callers that cannot allocate device memory when they need the
projector SVD (memory held by another allocator, no tolerance for the
synchronisation of cudaMalloc, no context workspace): only their buffers go
in, the scratch is a fixed array inside the library.  Calls in a row, with
different sizes, check that the shared scratch left by a call does not leak
into the next; each result is also checked against the known exact factors.
This file is collected last.
"""
import numpy as np
import pytest

from oracle.ctmrg import sign_fix
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _factors(m, seed):
    """M = Q1 diag(s) Q2^T with s_i = 10^(-i/6): the exact factors are known."""
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = 10.0 ** (-np.arange(m) / 6.0)
    return Q1, s, Q2


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _bufs(m, k):
    return (torch.empty((m, k), dtype=torch.float64, device="cuda"),
            torch.empty(k, dtype=torch.float64, device="cuda"),
            torch.empty((m, k), dtype=torch.float64, device="cuda"))


def _check(U, S, V, Q1, s, Q2, k):
    """Against the exact factors, with the tolerance of the truncated-SVD tests: values to
    1e-13, vectors where s_i > 1e-8 s_1 (below that FP64 fixes a direction only to about
    eps s_1 / s_i)."""
    Ur, Vr = sign_fix(Q1[:, :k], Q2[:, :k])
    good = s[:k] > 1e-8
    np.testing.assert_allclose(S.cpu().numpy(), s[:k], rtol=0, atol=1e-13)
    np.testing.assert_allclose(U.cpu().numpy()[:, good], Ur[:, good], atol=1e-6)
    np.testing.assert_allclose(V.cpu().numpy()[:, good], Vr[:, good], atol=1e-6)


def test_noalloc_matches_context_version_two_calls():
    """Consecutive calls with shrinking sizes: each against the context entry point and
    against the exact factors."""
    ctx = L.Context(4, 64)
    for m, k, seed in ((1024, 64, 1), (300, 40, 2), (96, 20, 3)):
        Q1, s, Q2 = _factors(m, seed)
        M = _dev((Q1 * s) @ Q2.T)
        U0, S0, V0 = _bufs(m, k)
        U1, S1, V1 = _bufs(m, k)
        L.tn_truncated_svd(ctx, M, m, k, U0, S0, V0)
        L.tn_truncated_svd_noalloc(M, m, k, U1, S1, V1)
        torch.cuda.synchronize()
        _check(U0, S0, V0, Q1, s, Q2, k)
        _check(U1, S1, V1, Q1, s, Q2, k)
        good = S0.cpu().numpy() > 1e-8 * S0.cpu().numpy()[0]
        np.testing.assert_allclose(S1.cpu().numpy(), S0.cpu().numpy(), rtol=0, atol=1e-13)
        np.testing.assert_allclose(U1.cpu().numpy()[:, good], U0.cpu().numpy()[:, good], atol=1e-6)
        np.testing.assert_allclose(V1.cpu().numpy()[:, good], V0.cpu().numpy()[:, good], atol=1e-6)
    ctx.close()


def test_noalloc_warm_start_on_side_stream():
    """A warm start (the context version's V) copied into the shared scratch, on a
    non-default stream, twice in a row: the same triplets as the context entry point."""
    m, k = 300, 40
    Q1, s, Q2 = _factors(m, 4)
    M = _dev((Q1 * s) @ Q2.T)
    ctx = L.Context(4, 64)
    U0, S0, V0 = _bufs(m, k)
    L.tn_truncated_svd(ctx, M, m, k, U0, S0, V0)
    U0w, S0w, V0w = _bufs(m, k)
    L.tn_truncated_svd(ctx, M, m, k, U0w, S0w, V0w, warm=V0)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for _ in range(2):
        U1, S1, V1 = _bufs(m, k)
        with torch.cuda.stream(side):
            L.tn_truncated_svd_noalloc(M, m, k, U1, S1, V1, warm=V0, stream=side)
        side.synchronize()
        _check(U1, S1, V1, Q1, s, Q2, k)
        good = s[:k] > 1e-8
        np.testing.assert_allclose(S1.cpu().numpy(), S0w.cpu().numpy(), rtol=0, atol=1e-13)
        np.testing.assert_allclose(U1.cpu().numpy()[:, good], U0w.cpu().numpy()[:, good], atol=1e-6)
        np.testing.assert_allclose(V1.cpu().numpy()[:, good], V0w.cpu().numpy()[:, good], atol=1e-6)
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    m, k = 4096, 96
    M = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    U, S, V = _bufs(m, k)
    with pytest.raises(L.TnError) as err:
        L.tn_truncated_svd_noalloc(M, m, k, U, S, V)
    assert err.value.status == L.TN_ESCRATCH
