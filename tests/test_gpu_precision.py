"""Precision forms: CTMRG contractions on the tensor cores against the FP64 oracle and the FP64 form.

The products of the environment computation run on the tensor cores, the small
factorisations, the full-update solve, gauge fixing and the observables in
FP64.  The bar of the precision form is 1e-6 relative on the energy.

* TN_BF16S4 (exact-accumulation BF16 integer slices, products ~1e-9 relative)
  is the form that meets it everywhere, from the trivial start at D = 4,
  chi = 64 included.
* TN_TF32X3 (products ~1e-7 relative) meets it on the short D = 2 trajectory;
  from a cold start at D = 4, chi = 64 it does not: the loop matrix there has
  s_64 / s_1 ~ 7e-7, so its smallest kept directions sit at the product error
  and S^{-1/2} carries that error into the environment (measured 1.5e-5).  Its
  full-size check is a regression guard at 3e-5, not the bar.
* TN_BF16X3 (products ~4e-6) is held to 1e-4 and its actual error is recorded
  by the bench.
The converged corner spectra move with the product error times the conditioning
of the truncated fixed point (S^{-1/2} of the loop's kept directions):
3.6e-5 (TF32 x3, products ~1e-7) and 2.5e-3 (BF16 x3) measured at D = 2,
chi = 12, an amplification of ~400 on the value at the truncation edge; for
the 4-slice products (~4e-9 on Gaussian operands) that model gives ~1.6e-6 on
that value (1.9e-6 measured on GB300), so the bound is 5e-6.
"""
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
E_TOL = {L.TN_TF32X3: 1e-6, L.TN_BF16X3: 1e-4, L.TN_BF16S4: 1e-6}
# normalised corner spectra converged in the split form (FP64 start, then split products)
SPEC_TOL = {L.TN_TF32X3: 1e-4, L.TN_BF16X3: 5e-3, L.TN_BF16S4: 5e-6}
CTM_TOL = {L.TN_TF32X3: 1e-7, L.TN_BF16X3: 1e-5, L.TN_BF16S4: 1e-11}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3, L.TN_BF16S4])
def test_converged_spectra_precision(prec):
    D, chi = 2, 12
    A = random_peps(2, D, instance=3)
    ctx = L.Context(D, chi, precision=prec)
    ctx.tn_set_state(A)
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    ctx.tn_ctmrg(CTM_TOL[prec], 300)
    sp = ctx.tn_corner_spectra()
    st, it, d, conv = OC.ctmrg(CELL, [OC.double_layer(x) for x in A], chi, 1e-11, 300)
    ref = OC.corner_spectra(st)
    for i, (x, y) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        for c in range(4):
            np.testing.assert_allclose(sp[i, c], ref[(x, y, 'C%d' % (c + 1))], atol=SPEC_TOL[prec])
    ctx.close()


@pytest.mark.parametrize("prec", [L.TN_TF32X3, L.TN_BF16X3, L.TN_BF16S4])
def test_trajectory_energy_precision(prec):
    """Five plain full-update steps (h = 3, tau = 0.01, D = 2, chi = 8): energy vs the FP64 oracle."""
    D, chi, h, tau, inst = 2, 8, 3.0, 0.01, 8
    A = random_peps(2, D, instance=inst)
    ctx = L.Context(D, chi, precision=prec)
    ctx.tn_set_hamiltonian(1.0, h)
    ctx.tn_set_time_step(tau)
    ctx.tn_set_state(A)
    cfg = OR.Config(h=h, tau=tau, D=D, chi=chi, ctm_tol=1e-10, ctm_max=500)
    env, Ao = None, A
    ctm_tol = 1e-10 if prec == L.TN_BF16S4 else 1e-8
    for _ in range(5):
        ctx.tn_fu_step(ctm_tol, 500)
        Ao, env, info = OR.fu_step(Ao, CELL, cfg, env)
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    ctx.tn_ctmrg(1e-12 if prec == L.TN_BF16S4 else 1e-8, 500)
    g = ctx.tn_measure()
    o = OR.energy(Ao, CELL, cfg, tol=1e-12)
    err = abs(g['e_site'] - o['e_site']) / abs(o['e_site'])
    assert err < E_TOL[prec], err
    ctx.close()


def test_full_size_converged_energy_precision_vs_f64():
    """D = 4, chi = 64, h = 3.04: one evolved state (two FP64 full-update steps from a
    seeded tensor), CTMRG from the trivial start converged in TF32 x3 and in FP64."""
    D, chi = 4, 64
    ref = L.Context(D, chi)
    ref.tn_set_hamiltonian(1.0, 3.04)
    ref.tn_set_time_step(0.005)
    ref.tn_set_state(random_peps(2, D, instance=4))
    for _ in range(2):
        ref.tn_fu_step(1e-8, 40)
    A = ref.tn_get_state()
    ref.close()
    e = {}
    for prec, tol in ((L.TN_F64, 1e-9), (L.TN_TF32X3, 1e-7)):
        ctx = L.Context(D, chi, precision=prec)
        ctx.tn_set_hamiltonian(1.0, 3.04)
        ctx.tn_set_state(A)
        ctx.tn_build_double_layer()
        ctx.tn_reset_env()
        ctx.tn_ctmrg(tol, 80)
        e[prec] = ctx.tn_measure()["e_site"]
        ctx.close()
    # TF32 x3 does not meet the 1e-6 bar from this cold start (measured 1.5e-5; see the
    # module docstring): a regression guard, the bar is tested on the integer-slice form below
    assert abs(e[L.TN_TF32X3] - e[L.TN_F64]) < 3e-5 * abs(e[L.TN_F64])


def test_full_size_converged_energy_slices_vs_f64():
    """The exact-accumulation integer-slice form at D = 4, chi = 64 from the trivial start:
    the energy of the FP64 form to 1e-6 relative (the precision form's bar)."""
    D, chi = 4, 64
    ref = L.Context(D, chi)
    ref.tn_set_hamiltonian(1.0, 3.04)
    ref.tn_set_time_step(0.005)
    ref.tn_set_state(random_peps(2, D, instance=4))
    for _ in range(2):
        ref.tn_fu_step(1e-8, 40)
    A = ref.tn_get_state()
    ref.close()
    e = {}
    for prec, tol in ((L.TN_F64, 1e-9), (L.TN_BF16S4, 1e-9)):
        ctx = L.Context(D, chi, precision=prec)
        ctx.tn_set_hamiltonian(1.0, 3.04)
        ctx.tn_set_state(A)
        ctx.tn_build_double_layer()
        ctx.tn_reset_env()
        ctx.tn_ctmrg(tol, 80)
        e[prec] = ctx.tn_measure()["e_site"]
        ctx.close()
    assert abs(e[L.TN_BF16S4] - e[L.TN_F64]) < 1e-6 * abs(e[L.TN_F64]), e
