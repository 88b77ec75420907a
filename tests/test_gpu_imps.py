"""The 1D iMPS scheme on the GPU (Sec. III and V), against the oracle and the exact chain.

The chain is where the method has an exact answer: e(h) of the infinite
transverse-field Ising chain.  The GPU's plain iTEBD and recycling windows
(tn_imps_itebd, tn_imps_recycle) are compared with the oracle's on the same
seeded tensors: gauge-invariant quantities (the fidelity F of the gauge fix,
<ZZ>, <X>, the energy) to 1e-10, and the converged energy with the closed form.
"""
import numpy as np
import pytest

from oracle import imps as OI
from oracle import model as OM
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _random_mps(chi, instance):
    A = random_matrix((2, chi, chi), instance=instance)
    return A / np.abs(A).max()


def _close(g, o, tol):
    assert abs(g["zz"] - o[0]) < tol and abs(g["x"] - o[1]) < tol
    assert abs(g["e"] - o[2]) < tol * abs(o[2])


@pytest.mark.parametrize("h,chi", [(2.0, 6), (0.6, 8)])
def test_plain_itebd_matches_oracle(h, chi):
    A = _random_mps(chi, 5)
    ref = OI.itebd(A, h, 0.05, chi, 6)
    m = L.IMPS(A)
    m.tn_imps_itebd(h, 0.05, 6)
    _close(m.tn_imps_observables(h), OI.observables(ref, h), 1e-10)
    np.testing.assert_allclose(np.abs(m.state()), np.abs(ref), atol=1e-9)


@pytest.mark.parametrize("h,chi,n_re", [(2.0, 6, 1), (2.0, 6, 4), (0.6, 8, 3)])
def test_recycling_window_matches_oracle(h, chi, n_re):
    A = OI.itebd(_random_mps(chi, 6), h, 0.05, chi, 4)
    ref, F_ref = OI.recycle_window(A, h, 0.05, chi, n_re)
    m = L.IMPS(A)
    F = m.tn_imps_recycle(h, 0.05, n_re)
    assert abs(F - F_ref) < 1e-10 and F <= 1.0 + 1e-12
    _close(m.tn_imps_observables(h), OI.observables(ref, h), 1e-10)


def test_recycling_reaches_exact_chain_energy():
    """Recycled windows (N_Re = 4) after a few plain steps reach e(h) of the infinite chain
    (h = 3, chi = 6, as the oracle's own pin), on the GPU alone."""
    h, chi = 3.0, 6
    m = L.IMPS(_random_mps(chi, 8))
    m.tn_imps_itebd(h, 0.05, 30)
    for _ in range(15):
        F = m.tn_imps_recycle(h, 0.01, 4)
        assert 0.99 < F <= 1.0 + 1e-12
    assert abs(m.tn_imps_observables(h)["e"] - OM.exact_energy_1d(h)) < 1e-5


def test_rejects_bad_arguments():
    m = L.IMPS(_random_mps(4, 1))
    with pytest.raises(L.TnError):
        m.tn_imps_itebd(2.0, -0.1, 1)
    assert L.lib().tn_imps_workspace_bytes(17) == 0 and L.lib().tn_imps_workspace_bytes(16) > 0
