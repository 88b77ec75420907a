"""FP64 parity of the paper's own scheme, the full update of the one-site iPEPS
(Sec. VI.B) with environment recycling (Sec. VI.C), against the oracle.

The one-site cell has one tensor A and two link types (h, v); its CTMRG runs
one cut per move.  Sec. VI.B averages the pairs of the links r, l (and d, u)
of the plaquette; with the per-link two-site cluster both members of each
pair are the same network in this cell, so the averages equal the one pair
per link type both sides compute.  Compared (as in the two-site parity tests,
tensors through absolute values, which a sign gauge leaves unchanged): the
weights lambda, the bond environments' eigenvalues, the ALS costs, |W|, F,
and the energies after the step and after N_Re = 3 recycled steps (1e-10).
"""
import numpy as np
import pytest

from oracle import ctmrg as OC
from oracle import fullupdate as OF
from oracle import recycle as OR
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_peps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CELL = OC.single_site()
H, TAU, N_RE = 3.04, 0.01, 3


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _abs_close(x, ref, rtol):
    x, ref = np.abs(np.asarray(x)), np.abs(np.asarray(ref))
    err = float(np.abs(x - ref).max() / max(ref.max(), 1e-300))
    assert err < rtol, err


@pytest.mark.parametrize("D,chi,inst", [(2, 8, 4), (3, 12, 3), (3, 12, 5)])
def test_one_site_full_update_and_recycling(D, chi, inst):
    A = random_peps(1, D, instance=inst)
    cfg = OR.Config(h=H, tau=TAU, D=D, chi=chi, ctm_tol=1e-12, ctm_max=300)
    Ak, env, info = OR.recycle_window(A, CELL, cfg, N_RE)
    assert info['ctm_converged']
    At = OF.assemble(info['Theta'], CELL, info['fu'])
    o_t = OR.energy(At, CELL, cfg, tol=1e-12)
    o_k = OR.energy(Ak, CELL, cfg, tol=1e-12)
    k = 2 * D

    ctx = L.Context(D, chi, cell=L.TN_CELL_SINGLE)
    ctx.tn_set_hamiltonian(1.0, H)
    ctx.tn_set_time_step(TAU)
    ctx.tn_set_state(A)
    ctx.tn_step_prepare()
    rep = ctx.tn_ctmrg(1e-12, 300)
    assert rep['converged']
    upd = ctx.tn_step_update()
    for e, link in enumerate(OF.link_list(CELL)):
        np.testing.assert_allclose(ctx.tn_get_tensor(L.TN_T_LAMBDA, e, (D,)), info['lam'][link], rtol=0, atol=1e-10)
        N4 = OF.bond_env(info['state'], CELL, link, info['Theta'], info['pre'])
        Nr = OF.psd_project(N4 / np.einsum('ccee->', N4)).reshape(k * k, k * k)
        Ng = ctx.tn_get_tensor(L.TN_T_BOND_ENV, e, (k, k, k, k)).reshape(k * k, k * k)
        w_ref = np.linalg.eigvalsh(Nr)
        np.testing.assert_allclose(np.linalg.eigvalsh(Ng), w_ref, rtol=0, atol=1e-10 * w_ref[-1])
        assert abs(upd['als_cost'][e] - info['als'][link][1]) < 1e-10
    At_gpu = ctx.tn_get_state()
    F = ctx.tn_recycle(N_RE)
    assert abs(F - info['F']) < 1e-10
    for e, link in enumerate(OF.link_list(CELL)):
        _abs_close(ctx.tn_get_tensor(L.TN_T_GAUGE_W, e, (D, D)), info['W'][link], 1e-8)
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    ctx.tn_ctmrg(1e-12, 500)
    g_k = ctx.tn_measure()
    ctx.close()
    assert abs(g_k['e_site'] - o_k['e_site']) < 1e-10 * abs(o_k['e_site'])
    assert abs(abs(g_k['mz'][0]) - abs(o_k['mz'][0])) < 1e-9

    m = L.Context(D, chi, cell=L.TN_CELL_SINGLE)
    m.tn_set_hamiltonian(1.0, H)
    m.tn_set_state(At_gpu)
    m.tn_build_double_layer()
    m.tn_reset_env()
    m.tn_ctmrg(1e-12, 500)
    g_t = m.tn_measure()
    m.close()
    assert abs(g_t['e_site'] - o_t['e_site']) < 1e-10 * abs(o_t['e_site'])
    assert abs(g_t['mx'][0] - o_t['mx'][0]) < 1e-9
