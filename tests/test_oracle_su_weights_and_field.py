"""Pins of the oracle's simple-update weighting (row a7) and of the 2D large-field limit.

* Pre-truncation (Sec. VI.B, last paragraph): the simple update treats the bond
  weights lambda as the whole environment of the external legs.  For every link the
  pair (P, Q) must then give the best rank-D approximation (Eckart-Young) of the
  lambda-weighted two-site bond matrix X Y, built here directly: X = Theta_t with
  sqrt(lambda) on each external leg, reshaped [rest, link]; Y = Theta_t' likewise,
  reshaped [link, rest].  The weights are non-uniform, so a wrong power of lambda,
  a weight on the wrong leg or the wrong (kappa, D) fusion fails.
* Large field: second-order perturbation theory around |->> gives
  E_site = -h - 1/(2h) + O(h^-3) in 2D (each of the two bonds per site flips two
  spins at cost 4h with matrix element 1).  A D = 2 iPEPS holds the first-order
  state exactly, so the full-update evolution must reproduce the 1/(2h) term.
"""
import numpy as np
import pytest

from oracle import ctmrg as C
from oracle import fullupdate as F
from oracle import recycle as R

LEGS = {'l': 1, 'r': 2, 'd': 3, 'u': 4}


def _weight_external(T, weights):
    """Multiply T[s, l, r, d, u] by the given weight vector on each named leg."""
    X = T
    for name, w in weights.items():
        shape = [1] * 5
        shape[LEGS[name]] = len(w)
        X = X * w.reshape(shape)
    return X


@pytest.mark.parametrize("D", [2, 3])
def test_pretruncation_is_eckart_young_of_weighted_bond(D):
    kappa = 2
    cell = C.checkerboard()
    rng = np.random.default_rng(40 + D)
    Theta = [rng.standard_normal((2,) + (kappa * D,) * 4) for _ in range(2)]
    # non-uniform, normalised weights per link type
    lam = {}
    for e in F.link_list(cell):
        w = np.sort(rng.uniform(0.05, 1.0, D))[::-1]
        lam[e] = w / np.linalg.norm(w)
    pre = F.pretruncation(Theta, cell, lam, D)
    for e in F.link_list(cell):
        t, dr = e
        left, up, pos = F.neighbours(cell)
        x, y = pos[t]
        tq = cell.tid(x + 1, y) if dr == 'h' else cell.tid(x, y + 1)
        lp, lq = ('r', 'l') if dr == 'h' else ('d', 'u')
        # external legs of each side and the links they belong to
        wp = {name: np.tile(np.sqrt(lam[link]), kappa)
              for name, (link, _s) in F.leg_links(cell, t).items() if name != lp}
        wq = {name: np.tile(np.sqrt(lam[link]), kappa)
              for name, (link, _s) in F.leg_links(cell, tq).items() if name != lq}
        X = np.moveaxis(_weight_external(Theta[t], wp), LEGS[lp], -1).reshape(-1, kappa * D)
        Y = np.moveaxis(_weight_external(Theta[tq], wq), LEGS[lq], 0).reshape(kappa * D, -1)
        U, s, Vt = np.linalg.svd(X @ Y)
        best = (U[:, :D] * s[:D]) @ Vt[:D]
        P, Q = pre[e]
        got = X @ P @ Q @ Y
        assert np.abs(got - best).max() < 1e-10 * s[0], (e, np.abs(got - best).max() / s[0])
        # and the truncation is not trivial: the discarded weight is real
        assert s[D] > 1e-3 * s[0]


@pytest.mark.slow
def test_large_field_second_order_energy():
    """E_site + h + 1/(2h) is O(h^-3): below h^-3 at h = 8 and 16 (measured -9.5e-4 and
    -1.15e-4, against the second-order term 1/(2h) = 0.0625 and 0.031), shrinking ~8x."""
    cell = C.checkerboard()
    res = {}
    for h in (8.0, 16.0):
        A = [np.ones((2, 2, 2, 2, 2)) * 0.1 + 0.01 * x for x in
             np.random.default_rng(3).standard_normal((2, 2, 2, 2, 2, 2))]
        cfg = R.Config(h=h, tau=0.02, D=2, chi=4, ctm_tol=1e-10, ctm_max=100)
        A, env, _ = R.evolve(A, cell, cfg, 30)
        cfg.tau = 0.005                                # Trotter error O(tau^2) well below h^-3
        A, env, _ = R.evolve(A, cell, cfg, 30, env=env)
        m = R.energy(A, cell, cfg, tol=1e-12)
        res[h] = m['e_site'] + h + 1.0 / (2.0 * h)
    for h, r in res.items():
        assert abs(r) < 1.0 / h ** 3, (h, r)          # the 1/(2h) coefficient is right
    assert abs(res[8.0]) > 4.0 * abs(res[16.0])       # and the remainder falls like h^-3
