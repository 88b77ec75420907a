"""FP64 parity of the whole full-update step, one recycling window and the observables
at D = 3 and D = 4 (rows a7-a14), against the oracle on the same seeded inputs.

Shapes: D = 3, chi = 16 and D = 4, chi = 16 (N = chi D^2 = 144 and 256: the
projector SVD runs the subspace iteration, not the small Jacobi), and D = 3,
chi = 32 (N = 288, the plain-vs-recycling workload's shape).  Inputs are seeded
Gaussian tensors (h = 3.04, tau = 0.005); the seeds are ones whose first CTMRG
converges to 1e-12 in the oracle (near the critical field some seeds leave the
truncated CTMRG map oscillating, which no implementation can be compared on).

What is compared, per link type where it applies:
  canonical weights lambda and |A_c| element by element (a11),
  singular values of the pre-truncation P Q and |P|, |Q| (a7),
  corner spectra of the converged environment (a6),
  the normalised PSD bond environment N: eigenvalues and |N| element by element (a8),
  ALS sweeps and final costs, balanced |P|, |Q| (a9),
  the energy, <X>, |<Z>| and <ZZ> of the updated state (a10, a14),
  the fidelity F, |W| element by element and the energy after N_Re = 3
  recycled steps (a12, a13).
The canonical form fixes each bond only up to a sign per index (the sign rule
acts on every SVD the same way, but rounding can decide an exact tie), so
tensors are compared through absolute values, element by element: a sign gauge
leaves |.| unchanged, a wrong leg order or index permutation does not.
Energies are held to 1e-10 relative, the spectra to 1e-9.
"""
import numpy as np
import pytest

from oracle import canonical as OK
from oracle import ctmrg as OC
from oracle import fullupdate as OF
from oracle import recycle as OR
from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_peps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CELL = OC.checkerboard()
H, TAU, N_RE = 3.04, 0.005, 3
CASES = [(3, 16, 12), (4, 16, 12), (3, 32, 13)]
E_REL = 1e-10
SITES = [(0, 0), (1, 0), (0, 1), (1, 1)]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


_CACHE = {}


def oracle_case(D, chi, inst):
    """Everything the oracle computes for one case (cached across the tests of a case)."""
    key = (D, chi, inst)
    if key in _CACHE:
        return _CACHE[key]
    A = random_peps(2, D, instance=inst)
    cfg = OR.Config(h=H, tau=TAU, D=D, chi=chi, ctm_tol=1e-12, ctm_max=300)
    Ak, env, info = OR.recycle_window(A, CELL, cfg, N_RE)
    assert info['ctm_converged']
    At = OF.assemble(info['Theta'], CELL, info['fu'])
    N = {}
    for e in OF.link_list(CELL):
        N4 = OF.bond_env(info['state'], CELL, e, info['Theta'], info['pre'])
        N[e] = OF.psd_project(N4 / np.einsum('ccee->', N4))
    out = dict(A=A, cfg=cfg, info=info, N=N, At=At, Ak=Ak,
               spectra=OC.corner_spectra(info['state']),
               obs_t=OR.energy(At, CELL, cfg, tol=1e-12),
               obs_k=OR.energy(Ak, CELL, cfg, tol=1e-12))
    _CACHE[key] = out
    return out


def gpu_case(D, chi, inst, precision=L.TN_F64):
    A = random_peps(2, D, instance=inst)
    ctx = L.Context(D, chi, precision=precision)
    ctx.tn_set_hamiltonian(1.0, H)
    ctx.tn_set_time_step(TAU)
    ctx.tn_set_state(A)
    prep = ctx.tn_step_prepare()
    ctm = ctx.tn_ctmrg(1e-12, 300)
    k = 2 * D
    g = dict(prep=prep, ctm=ctm, spectra=ctx.tn_corner_spectra())
    g['lam'] = [ctx.tn_get_tensor(L.TN_T_LAMBDA, e, (D,)) for e in range(4)]
    g['Ac'] = [ctx.tn_get_tensor(L.TN_T_CANON, t, (2,) + (D,) * 4) for t in range(2)]
    g['preP'] = [ctx.tn_get_tensor(L.TN_T_PRE_P, e, (k, D)) for e in range(4)]
    g['preQ'] = [ctx.tn_get_tensor(L.TN_T_PRE_Q, e, (D, k)) for e in range(4)]
    g['upd'] = ctx.tn_step_update()
    g['N'] = [ctx.tn_get_tensor(L.TN_T_BOND_ENV, e, (k, k, k, k)) for e in range(4)]
    g['fuP'] = [ctx.tn_get_tensor(L.TN_T_FU_P, e, (k, D)) for e in range(4)]
    g['fuQ'] = [ctx.tn_get_tensor(L.TN_T_FU_Q, e, (D, k)) for e in range(4)]
    At = ctx.tn_get_state()
    g['F'] = ctx.tn_recycle(N_RE)
    g['W'] = [ctx.tn_get_tensor(L.TN_T_GAUGE_W, e, (D, D)) for e in range(4)]
    g['K'] = [ctx.tn_get_tensor(L.TN_T_GATE_K, i, (k, D)) for i in range(8)]
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    g['ctm_k'] = ctx.tn_ctmrg(1e-12, 500)
    g['obs_k'] = ctx.tn_measure()
    ctx.close()
    m = L.Context(D, chi, precision=precision)
    m.tn_set_hamiltonian(1.0, H)
    m.tn_set_state(At)
    m.tn_build_double_layer()
    m.tn_reset_env()
    g['ctm_t'] = m.tn_ctmrg(1e-12, 500)
    g['obs_t'] = m.tn_measure()
    m.close()
    return g


_GCACHE = {}


def both(case):
    if case not in _GCACHE:
        _GCACHE[case] = gpu_case(*case)
    return oracle_case(*case), _GCACHE[case]


def _abs_close(x, ref, rtol):
    x, ref = np.abs(np.asarray(x)), np.abs(np.asarray(ref))
    err = float(np.abs(x - ref).max() / max(ref.max(), 1e-300))
    assert err < rtol, err


@pytest.mark.parametrize("case", CASES)
def test_canonical_form_and_pretruncation(case):
    o, g = both(case)
    D = case[0]
    lam = o['info']['lam']
    for e, link in enumerate(OF.link_list(CELL)):
        np.testing.assert_allclose(g['lam'][e], lam[link], rtol=0, atol=1e-10)
    for t in range(2):
        _abs_close(g['Ac'][t], o['info']['A0'][t], 1e-9)
    for e, link in enumerate(OF.link_list(CELL)):
        Po, Qo = o['info']['pre'][link]
        s_ref = np.linalg.svd(Po @ Qo, compute_uv=False)
        s_gpu = np.linalg.svd(g['preP'][e] @ g['preQ'][e], compute_uv=False)
        np.testing.assert_allclose(s_gpu, s_ref, rtol=0, atol=1e-9 * s_ref[0])
        _abs_close(g['preP'][e], Po, 1e-8)
        _abs_close(g['preQ'][e], Qo, 1e-8)
    assert g['prep']['canon_iters'] > 0 and D in (3, 4)


@pytest.mark.parametrize("case", CASES)
def test_converged_environment_spectra(case):
    o, g = both(case)
    # both converge to delta < 1e-12; the iteration at which the delta first dips below
    # that floor is not a parity quantity (it differs by ~10 between LAPACK builds)
    assert g['ctm']['converged'] and o['info']['ctm_converged'], (g['ctm'], o['info']['ctm_iters'])
    for i, (x, y) in enumerate(SITES):
        for c in range(4):
            np.testing.assert_allclose(g['spectra'][i, c], o['spectra'][(x, y, 'C%d' % (c + 1))], rtol=0, atol=1e-9)


@pytest.mark.parametrize("case", CASES)
def test_bond_environment_and_als(case):
    o, g = both(case)
    D = case[0]
    k = 2 * D
    for e, link in enumerate(OF.link_list(CELL)):
        Nr = o['N'][link]
        Ng = g['N'][e]
        w_ref = np.linalg.eigvalsh(Nr.reshape(k * k, k * k))
        w_gpu = np.linalg.eigvalsh(Ng.reshape(k * k, k * k))
        np.testing.assert_allclose(w_gpu, w_ref, rtol=0, atol=1e-10 * w_ref[-1])
        _abs_close(Ng, Nr, 1e-9)
        it, cost = o['info']['als'][link]
        assert abs(g['upd']['als_iters'][e] - it) <= 1, (g['upd']['als_iters'][e], it)
        assert abs(g['upd']['als_cost'][e] - cost) < 1e-10, (g['upd']['als_cost'][e], cost)
        Pf, Qf = o['info']['fu'][link]
        _abs_close(g['fuP'][e], Pf, 1e-7)
        _abs_close(g['fuQ'][e], Qf, 1e-7)


@pytest.mark.parametrize("case", CASES)
def test_updated_state_observables(case):
    o, g = both(case)
    ot, gt = o['obs_t'], g['obs_t']
    # the oracle's CTMRG stops at delta < 1e-12; the GPU's may stall just above that
    # rounding floor (D = 3, chi = 32), which the energy parity below tolerates
    assert g['ctm_t']['delta'] < 1e-10, g['ctm_t']
    assert abs(gt['e_site'] - ot['e_site']) < E_REL * abs(ot['e_site'])
    assert abs(gt['e_link'] - ot['e_link']) < E_REL * abs(ot['e_link'])
    for t in range(2):
        assert abs(gt['mx'][t] - ot['mx'][t]) < 1e-9
        assert abs(abs(gt['mz'][t]) - abs(ot['mz'][t])) < 1e-9
    for e, link in enumerate(OF.link_list(CELL)):
        assert abs(gt['zz'][e] - ot['zz'][link]) < 1e-9


@pytest.mark.parametrize("case", CASES)
def test_recycling_window(case):
    o, g = both(case)
    info = o['info']
    assert abs(g['F'] - info['F']) < 1e-10
    for e, link in enumerate(OF.link_list(CELL)):
        _abs_close(g['W'][e], info['W'][link], 1e-8)
        Wg = g['W'][e]
        np.testing.assert_allclose(Wg @ Wg.T, np.eye(case[0]), atol=1e-12)
    for t in range(2):
        for leg, name in enumerate('lrdu'):
            _abs_close(g['K'][4 * t + leg], info['K'][(t, name)], 1e-7)
    ok, gk = o['obs_k'], g['obs_k']
    assert g['ctm_k']['delta'] < 1e-10, g['ctm_k']
    assert abs(gk['e_site'] - ok['e_site']) < E_REL * abs(ok['e_site'])
    for t in range(2):
        assert abs(abs(gk['mz'][t]) - abs(ok['mz'][t])) < 1e-9


def test_fp64_accurate_slice_form_matches_oracle():
    """The same step with every contraction (and the projector SVD's products) as
    FP64-accurate 7-slice tensor-core products: the FP64 bars of the oracle parity."""
    case = (4, 16, 12)
    o = oracle_case(*case)
    g = gpu_case(*case, precision=L.TN_F64S7)
    for i, (x, y) in enumerate(SITES):
        for c in range(4):
            np.testing.assert_allclose(g['spectra'][i, c], o['spectra'][(x, y, 'C%d' % (c + 1))], rtol=0, atol=1e-9)
    for e, link in enumerate(OF.link_list(CELL)):
        assert abs(g['upd']['als_cost'][e] - o['info']['als'][link][1]) < 1e-10
    ot, gt = o['obs_t'], g['obs_t']
    assert abs(gt['e_site'] - ot['e_site']) < E_REL * abs(ot['e_site'])
    ok, gk = o['obs_k'], g['obs_k']
    assert abs(gk['e_site'] - ok['e_site']) < E_REL * abs(ok['e_site'])
    assert abs(g['F'] - o['info']['F']) < 1e-10
