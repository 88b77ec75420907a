"""End-to-end pins of the 2D imaginary-time evolution with full update and recycling (Sec. VI).

D = 1 restricts the iPEPS to product states; imaginary-time evolution then
converges (error O(tau^2)) to the mean-field optimum E_site = -2 - h^2/8
(h < 4), which fixes the iPEPO, the double layer, the bond environment, the
ALS solve and the assembly together.  At h = 0 the ferromagnetic product state
is an exact fixed point with E_site = -2.
"""
import json
import os

import numpy as np
import pytest

from oracle import ctmrg as C
from oracle import recycle as R
from paper_1411_0391_gb300.inputs import random_peps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("h", [2.0, 3.0])
def test_d1_reaches_mean_field(h):
    cell = C.checkerboard()
    A = random_peps(2, 1, instance=3)
    cfg = R.Config(h=h, tau=0.05, D=1, chi=2)
    A, env, _ = R.evolve(A, cell, cfg, 100)
    cfg.tau = 0.01
    A, env, _ = R.evolve(A, cell, cfg, 200, env=env)
    m = R.energy(A, cell, cfg)
    assert abs(m['e_site'] - (-2.0 - h * h / 8.0)) < 1e-4
    assert abs(np.mean(list(m['mx'].values())) - h / 4.0) < 1e-2     # first order in the state error


def test_d1_recycled_reaches_mean_field():
    h = 2.0
    cell = C.checkerboard()
    A = random_peps(2, 1, instance=4)
    cfg = R.Config(h=h, tau=0.05, D=1, chi=2)
    A, env, _ = R.evolve(A, cell, cfg, 60)
    cfg.tau = 0.01
    A, env, n_env = R.evolve(A, cell, cfg, 200, n_re=5, recycle=True, env=env)
    assert n_env == 40
    m = R.energy(A, cell, cfg)
    assert abs(m['e_site'] - (-2.0 - h * h / 8.0)) < 1e-4


def test_h0_product_state_is_fixed_point():
    cell = C.checkerboard()
    A = np.zeros((2, 2, 2, 2, 2))
    A[0, 0, 0, 0, 0] = 1.0
    A = A + 1e-6 * np.random.default_rng(0).standard_normal(A.shape)
    A = [A, A.copy()]
    cfg = R.Config(h=0.0, tau=0.01, D=2, chi=4)
    env = None
    for _ in range(5):
        A, env, _ = R.fu_step(A, cell, cfg, env)
    m = R.energy(A, cell, cfg)
    assert abs(m['e_site'] + 2.0) < 1e-10


@pytest.mark.slow
def test_large_field_against_exact_diagonalisation():
    """h = 5: D = 2 full update against the 4x4 torus ground state (loose: D = 2 and finite size)."""
    with open(os.path.join(GOLDEN, "ed_4x4.json")) as f:
        e_ed = json.load(f)["tfim_4x4_e_site_h5.0"]
    cell = C.checkerboard()
    A = random_peps(2, 2, instance=5)
    cfg = R.Config(h=5.0, tau=0.02, D=2, chi=12, ctm_max=200)
    A, env, _ = R.evolve(A, cell, cfg, 80)
    m = R.energy(A, cell, cfg)
    assert abs(m['e_site'] - e_ed) < 3e-3
    assert m['e_site'] > e_ed - 1e-4          # a variational state cannot go below the ground state by more than finite-size effects


# --- simple-update step (the comparison method of Sec. VI.D) ---------------------------------

def test_su_d1_reaches_mean_field():
    """At D = 1 the simple update is mean-field imaginary-time evolution: E_site -> -2 - h^2/8,
    with the second-order Trotter error O(tau^2) (the error quarters when tau halves)."""
    h = 2.0
    cell = C.checkerboard()
    A = random_peps(2, 1, instance=6)
    cfg = R.Config(h=h, tau=0.05, D=1, chi=2)
    for _ in range(100):
        A = R.su_step(A, cell, cfg)
    err = {}
    for tau, n in ((0.01, 200), (0.005, 200)):
        cfg.tau = tau
        for _ in range(n):
            A = R.su_step(A, cell, cfg)
        err[tau] = R.energy(A, cell, cfg)['e_site'] - (-2.0 - h * h / 8.0)
    assert 0.0 < err[0.005] < 1e-4
    assert 3.2 < err[0.01] / err[0.005] < 4.8


def test_su_h0_product_state_is_fixed_point():
    cell = C.checkerboard()
    A = np.zeros((2, 2, 2, 2, 2))
    A[0, 0, 0, 0, 0] = 1.0
    A = A + 1e-6 * np.random.default_rng(1).standard_normal(A.shape)
    A = [A, A.copy()]
    cfg = R.Config(h=0.0, tau=0.01, D=2, chi=4)
    for _ in range(5):
        A = R.su_step(A, cell, cfg)
    m = R.energy(A, cell, cfg)
    assert abs(m['e_site'] + 2.0) < 1e-10


def test_su_above_fu_variationally():
    """Both methods give variational states of the same ansatz; on the ordered side
    (h = 2.5, D = 2) the simple update, which ignores the environment, ends higher."""
    h = 2.5
    cell = C.checkerboard()
    A0 = random_peps(2, 2, instance=7)
    cfg = R.Config(h=h, tau=0.05, D=2, chi=8, ctm_max=200)
    Asu = A0
    for _ in range(40):
        Asu = R.su_step(Asu, cell, cfg)
    Afu, env, _ = R.evolve(A0, cell, cfg, 40)
    esu = R.energy(Asu, cell, cfg)['e_site']
    efu = R.energy(Afu, cell, cfg, env=env)['e_site']
    assert efu < esu


# --- recycling with the threshold trigger ------------------------------------------------

def _thr_setup():
    cell = C.checkerboard()
    A = random_peps(2, 2, instance=8)
    cfg = R.Config(h=3.0, tau=0.01, D=2, chi=8, ctm_tol=1e-10, ctm_max=500)
    return cell, A, cfg


def test_threshold_infinite_eps_is_one_fixed_window():
    """eps = inf never ends the window: the same state as one window of N_Re = n steps."""
    cell, A, cfg = _thr_setup()
    n = 4
    At, _, n_env, n_chk = R.evolve_threshold(A, cell, cfg, n, eps=np.inf, check_every=1, max_window=n)
    Aw, _, _ = R.recycle_window(A, cell, cfg, n)
    assert n_env == 1 and n_chk == n - 1
    for x, y in zip(At, Aw):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-12)


def test_threshold_zero_eps_is_the_plain_trajectory():
    """eps = 0 ends every window after one recycled step, which reproduces the plain step up
    to a gauge.  That gauge is not orthogonal, and the chi-truncated CTMRG of the next steps
    is covariant only under orthogonal gauges, so the trajectories agree to the truncation
    level (5e-7 at chi = 8), not to rounding."""
    cell, A, cfg = _thr_setup()
    n = 3
    At, env_t, n_env, n_chk = R.evolve_threshold(A, cell, cfg, n, eps=0.0, check_every=1)
    Ap, env_p, _ = R.evolve(A, cell, cfg, n)
    assert n_env == n and n_chk == n - 1
    et = R.energy(At, cell, cfg, tol=1e-12)['e_site']
    ep = R.energy(Ap, cell, cfg, tol=1e-12)['e_site']
    assert abs(et - ep) < 2e-6 * abs(ep)


def test_threshold_trigger_limits():
    """Every check exceeds a tiny threshold (one environment computation per step); none
    exceeds an infinite one (one for the whole run); the log records each check's change."""
    cell, A, cfg = _thr_setup()
    n = 4
    log = []
    _, _, n_env, n_chk = R.evolve_threshold(A, cell, cfg, n, eps=1e-14, check_every=1, log=log)
    assert n_env == n and n_chk == n - 1
    assert all(d['change'] > 1e-14 for d in log)
    _, _, n_env, n_chk = R.evolve_threshold(A, cell, cfg, n, eps=np.inf, check_every=2, max_window=n)
    assert n_env == 1 and n_chk == 1
