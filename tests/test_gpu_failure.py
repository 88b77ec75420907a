"""Failure detection without faulting the GPU (host-made failures, bounded device waits).

* A state poisoned on the host (a NaN copied in through tn_set_state) makes every
  step entry point return TN_ENUMERIC; the context stays usable afterwards.
* Recycling instability (Sec. VI.D and Sec. VII warn that long recycling windows can
  go unstable): with a fidelity threshold no window can meet (F <= 1 always), every
  window is judged unstable, redone as plain steps and the window length halved;
  tn_evolve reports TN_EUNSTABLE and the state equals the plain evolution's exactly.
  With the test off, the same run recycles and reports TN_OK.
* The device-side wait limit of the tensor-core kernels: a kernel waits on a barrier
  nothing arrives on, gives up after about a second and the call reports
  TN_ETIMEOUT; a split-precision product right after it is correct.
"""
import numpy as np
import pytest

from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_matrix, random_peps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _ctx(D=2, chi=8, h=3.0, tau=0.01, inst=8):
    ctx = L.Context(D, chi)
    ctx.tn_set_hamiltonian(1.0, h)
    ctx.tn_set_time_step(tau)
    ctx.tn_set_state(random_peps(2, D, instance=inst))
    return ctx


def test_poisoned_state_is_reported():
    ctx = _ctx()
    A = random_peps(2, 2, instance=8)
    A[1][0, 1, 0, 1, 1] = np.nan
    ctx.tn_set_state(A)
    for call in (lambda: ctx.tn_fu_step(1e-8, 50), ctx.tn_su_step, ctx.tn_step_prepare):
        with pytest.raises(L.TnError) as err:
            call()
        assert err.value.status == L.TN_ENUMERIC
    A[1][0, 1, 0, 1, 1] = np.inf
    ctx.tn_set_state(A)
    with pytest.raises(L.TnError) as err:
        ctx.tn_evolve(3, recycle=True, n_re=2, ctm_tol=1e-8, ctm_max=50)
    assert err.value.status == L.TN_ENUMERIC
    # the context stays usable: a finite state steps normally
    ctx.tn_set_state(random_peps(2, 2, instance=8))
    ctx.tn_fu_step(1e-8, 100)
    assert all(np.isfinite(a).all() for a in ctx.tn_get_state())
    ctx.close()


@pytest.mark.parametrize("mode", [True, "threshold"])
def test_unstable_windows_fall_back_to_plain_steps(mode):
    n = 6
    plain = _ctx()
    rp = plain.tn_evolve(n, recycle=False, ctm_tol=1e-10, ctm_max=300)
    ref = plain.tn_get_state()
    plain.close()
    ctx = _ctx()
    rep = ctx.tn_evolve(n, recycle=mode, n_re=4, ctm_tol=1e-10, ctm_max=300, min_fidelity=2.0,
                        recycle_eps=float("inf") if mode == "threshold" else None)
    assert rep["status"] == L.TN_EUNSTABLE
    assert rep["steps"] == n and rep["fallbacks"] >= 1 and rep["final_n_re"] == 1
    assert rep["env_computations"] == rp["env_computations"] == n
    for a, b in zip(ctx.tn_get_state(), ref):
        np.testing.assert_array_equal(a, b)        # the same plain steps, the same arithmetic
    ctx.close()
    ok = _ctx()
    rep = ok.tn_evolve(n, recycle=mode, n_re=3, ctm_tol=1e-10, ctm_max=300, min_fidelity=0.0,
                       recycle_eps=float("inf") if mode == "threshold" else None)
    assert rep["status"] == L.TN_OK and rep["fallbacks"] == 0 and rep["final_n_re"] == 3
    assert rep["env_computations"] == 2 and 0.99 < rep["last_fidelity"] <= 1.0 + 1e-12
    ok.close()


def test_realistic_fidelity_threshold_passes():
    """A threshold below the fidelities the method reaches (F ~ 0.9999 at tau = 0.01) never triggers."""
    ctx = _ctx()
    rep = ctx.tn_evolve(6, recycle=True, n_re=3, ctm_tol=1e-10, ctm_max=300, min_fidelity=0.99)
    assert rep["status"] == L.TN_OK and rep["fallbacks"] == 0 and rep["final_n_re"] == 3
    ctx.close()


def test_bounded_wait_expires_and_context_survives():
    import time
    t0 = time.perf_counter()
    assert L.tn_selftest_wait_timeout() == L.TN_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.5 < dt < 30.0, dt
    m = n = k = 200
    A, Bm = random_matrix((m, k), instance=11), random_matrix((k, n), instance=12)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(Bm).cuda()
    dC = torch.empty((m, n), dtype=torch.float64, device="cuda")
    work = torch.empty(L.tn_gemm_split_workspace_bytes(L.TN_TF32X3, m, n, k), dtype=torch.uint8, device="cuda")
    L.tn_gemm_split(L.TN_TF32X3, 0, 0, m, n, k, 1.0, dA, k, dB, n, 0.0, dC, n, work)
    torch.cuda.synchronize()
    ref = A @ Bm
    assert np.abs(dC.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()
