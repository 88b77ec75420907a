"""Simple-update step and the field sweep (m_z(h), full vs simple update) against the oracle."""
import numpy as np
import pytest

from oracle import ctmrg as OC
from oracle import recycle as OR
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_peps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CELL = OC.checkerboard()


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def test_su_step_parity():
    """Three simple-update steps (h = 3, tau = 0.01, D = 2): energy and magnetisations to 1e-10."""
    D, chi, h, tau = 2, 8, 3.0, 0.01
    A = random_peps(2, D, instance=9)
    ctx = L.Context(D, chi)
    ctx.tn_set_hamiltonian(1.0, h)
    ctx.tn_set_time_step(tau)
    ctx.tn_set_state(A)
    cfg = OR.Config(h=h, tau=tau, D=D, chi=chi)
    Ao = A
    for _ in range(3):
        ctx.tn_su_step()
        Ao = OR.su_step(Ao, CELL, cfg)
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    ctx.tn_ctmrg(1e-12, 500)
    g = ctx.tn_measure()
    o = OR.energy(Ao, CELL, cfg, tol=1e-12)
    assert abs(g["e_site"] - o["e_site"]) < 1e-10 * abs(o["e_site"])
    for t in range(2):
        assert abs(g["mx"][t] - o["mx"][t]) < 1e-9
        assert abs(abs(g["mz"][t]) - abs(o["mz"][t])) < 1e-9
    ctx.close()


@pytest.mark.parametrize("method", ["fu", "su"])
def test_field_sweep_against_oracle(method):
    """Two fields on either side of the transition, five steps each: e_site and |m_z| per field."""
    from paper_1411_0391_gb300.sweep import field_sweep
    D, chi, tau, steps = 2, 8, 0.01, 5
    hs = [2.5, 3.5]
    res = field_sweep(hs, D, chi, tau, steps, method=method, ctm_tol=1e-10, ctm_max=500, measure_tol=1e-12,
                      measure_max=500, instance=8)
    for r in res:
        cfg = OR.Config(h=r["h"], tau=tau, D=D, chi=chi, ctm_tol=1e-10, ctm_max=500)
        A = random_peps(2, D, instance=8)
        if method == "su":
            for _ in range(steps):
                A = OR.su_step(A, CELL, cfg)
        else:
            A, _, _ = OR.evolve(A, CELL, cfg, steps)
        o = OR.energy(A, CELL, cfg, tol=1e-12)
        assert abs(r["e_site"] - o["e_site"]) < 1e-9 * abs(o["e_site"])
        mz = np.mean([abs(z) for z in o["mz"].values()])
        assert abs(r["mz"] - mz) < 1e-8


def test_field_sweep_replica_slices():
    """rank r of world w takes h[r::w]: the union of the slices is the sweep, in order."""
    from paper_1411_0391_gb300.sweep import field_sweep
    hs = [2.0, 2.5, 3.0]
    parts = [field_sweep(hs, 2, 4, 0.05, 1, method="su", rank=r, world=2, measure_tol=1e-8) for r in range(2)]
    assert [p["h"] for p in parts[0]] == [2.0, 3.0]
    assert [p["h"] for p in parts[1]] == [2.5]
