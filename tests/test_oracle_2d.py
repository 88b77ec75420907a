"""Pins of the 2D oracle: canonical form (Eqs. 17-20), gauge fixing (Eq. 25), full update (Eqs. var, var1)."""
import numpy as np
import pytest
from scipy.stats import ortho_group

from oracle import canonical as K
from oracle import ctmrg as C
from oracle import fullupdate as F
from oracle import recycle as R
from paper_1411_0391_gb300.inputs import random_peps, random_matrix


def _gauge(A, cell, G):
    """Insert G_e G_e^{-1} on every link (the state is unchanged, Eq. for B in Sec. IV)."""
    out = []
    for t, T in enumerate(A):
        for name, (e, side) in F.leg_links(cell, t).items():
            M = G[e] if side == 'out' else np.linalg.inv(G[e]).T
            T = F.leg_mul(T, F.LEG[name], M)
        out.append(T)
    return out


@pytest.mark.parametrize("cell", [C.checkerboard(), C.single_site()], ids=["2site", "1site"])
def test_canonical_constraints(cell):
    A = random_peps(int(cell.pattern.max()) + 1, 3, instance=1)
    can = K.canonicalize(A, cell, tol=1e-13, max_iter=2000)
    assert can['converged']
    assert K.canonical_residual(can['Gamma'], can['lam'], cell) < 1e-10


def test_canonical_weights_are_gauge_invariant():
    cell = C.checkerboard()
    A = random_peps(2, 3, instance=2)
    G = {e: np.eye(3) + 0.3 * random_matrix((3, 3), instance=10 + i)
         for i, e in enumerate(F.link_list(cell))}
    la = K.canonicalize(A, cell, tol=1e-13, max_iter=2000)['lam']
    lb = K.canonicalize(_gauge(A, cell, G), cell, tol=1e-13, max_iter=2000)['lam']
    for e in la:
        np.testing.assert_allclose(la[e], lb[e], atol=1e-9)


def test_canonical_maps_reproduce_weighted_tensor():
    cell = C.checkerboard()
    A = random_peps(2, 2, instance=3)
    can = K.canonicalize(A, cell, tol=1e-13)
    for t in range(2):
        T = A[t]
        for name in ('l', 'r', 'd', 'u'):
            T = F.leg_mul(T, F.LEG[name], can['maps'][(t, name)])
        np.testing.assert_allclose(T / np.linalg.norm(T), can['A'][t], atol=1e-10)


@pytest.mark.parametrize("cell,amp,signs", [(C.checkerboard(), 0.3, False), (C.single_site(), 0.3, False)],
                         ids=["2site", "1site"])
def test_gauge_fix_recovers_orthogonal_gauge(cell, amp, signs):
    """B = A x W with orthogonal W: the polar iteration of Sec. IV.B reaches F = 1 and B.

    The iteration is local (started from W = I); the gauges here are rotations
    of angle ~amp (the iteration can stall on large rotations or sign flips), the regime of two
    canonical forms of nearby states.
    """
    from scipy.linalg import expm
    n = int(cell.pattern.max()) + 1
    Ac = K.canonicalize(random_peps(n, 3, instance=4), cell, tol=1e-13)['A']
    rng = np.random.default_rng(21)
    W = {}
    for e in F.link_list(cell):
        X = amp * rng.standard_normal((3, 3))
        S = np.diag(rng.choice([-1.0, 1.0], 3)) if signs else np.eye(3)
        W[e] = S @ expm(X - X.T)
    B = K.transform(Ac, cell, W)
    Wf, Fid, it = K.gauge_fix(Ac, B, cell)
    assert abs(Fid - 1.0) < 1e-10
    for x, y in zip(K.transform(Ac, cell, Wf), B):
        np.testing.assert_allclose(x, y, atol=1e-8)


def test_pair_projectors_give_truncated_svd():
    rng = np.random.default_rng(5)
    Rp, Lq = rng.standard_normal((6, 6)), rng.standard_normal((6, 6))
    P, Q, S = F.pair_projectors(Rp, Lq, 3)
    U, s, Vt = np.linalg.svd(Rp @ Lq)
    np.testing.assert_allclose(Rp @ P @ Q @ Lq, (U[:, :3] * s[:3]) @ Vt[:3], atol=1e-10)


def _product_env(kD, seed):
    rng = np.random.default_rng(seed)
    L, Rm = rng.standard_normal((kD, kD)), rng.standard_normal((kD, kD))
    return L, Rm, np.einsum('ac,bd->abcd', L @ L.T, Rm @ Rm.T)


def test_als_product_environment_is_eckart_young():
    """N = E_L (x) E_R gives f(M) = ||L^T (I - M) R||^2, minimised at rank D by the truncated SVD of L^T R."""
    kD, D = 6, 3
    L, Rm, N4 = _product_env(kD, 6)
    rng = np.random.default_rng(7)
    P, Q, it, f = F.als(N4, rng.standard_normal((kD, D)), rng.standard_normal((D, kD)), tol=1e-14, max_iter=500)
    s = np.linalg.svd(L.T @ Rm, compute_uv=False)
    assert abs(f - np.sum(s[D:] ** 2)) < 1e-9 * np.sum(s ** 2)


def test_als_without_truncation_is_exact():
    kD = 4
    _, _, N4 = _product_env(kD, 8)
    rng = np.random.default_rng(9)
    P, Q, it, f = F.als(N4, rng.standard_normal((kD, kD)), rng.standard_normal((kD, kD)), tol=1e-14)
    assert abs(f) < 1e-10 * np.einsum('ccee->', N4)


def test_als_cost_is_monotone():
    kD, D = 6, 2
    rng = np.random.default_rng(11)
    X = rng.standard_normal((kD * kD, 40))
    N4 = (X @ X.T).reshape(kD, kD, kD, kD)
    P, Q = rng.standard_normal((kD, D)), rng.standard_normal((D, kD))
    costs = []
    for _ in range(15):
        P, Q, it, f = F.als(N4, P, Q, tol=0.0, max_iter=1)
        costs.append(f)
    assert all(b <= a + 1e-10 * abs(a) for a, b in zip(costs, costs[1:]))
    assert min(costs) >= -1e-10


def test_recycling_window_nre1_matches_plain_step():
    """N_Re = 1 reproduces the plain full-update step up to a gauge (Sec. VI.C)."""
    cell = C.checkerboard()
    cfg = R.Config(h=3.0, tau=0.01, D=2, chi=8)
    A = random_peps(2, 2, instance=12)
    A, env, _ = R.fu_step(A, cell, cfg)
    plain, _, _ = R.fu_step(A, cell, cfg, env)
    rec, _, info = R.recycle_window(A, cell, cfg, 1, env)
    assert info['F'] <= 1.0 + 1e-12
    # CTMRG truncation is covariant only under orthogonal gauges: compare both
    # states in their canonical gauge, which leaves an orthogonal gauge between them.
    mp = R.energy(K.canonicalize(plain, cell, tol=1e-13)['A'], cell, cfg, tol=1e-12)
    mr = R.energy(K.canonicalize(rec, cell, tol=1e-13)['A'], cell, cfg, tol=1e-12)
    assert abs(mp['e_site'] - mr['e_site']) < 1e-9
    for t in range(2):
        assert abs(mp['mx'][t] - mr['mx'][t]) < 1e-9


def test_bond_env_of_product_state_factorises():
    """Row a8 pinned directly: at D = 1 the state is a product and the chi = 1 CTMRG is
    exact, so the environment of a link is the tensor product of the two sites' Gram
    matrices of their open link legs (all other legs of Theta pre-truncated to D = 1):
    N[a, b, a', b'] = G_p[a, a'] G_q[b, b'] up to the scale of the environment."""
    from oracle import fullupdate as FU
    from oracle import model as MD
    from oracle import canonical as CN
    cell = C.checkerboard()
    A = random_peps(2, 1, instance=2)
    g = MD.ipepo(3.0, 0.05)
    can = CN.canonicalize(A, cell)
    Theta = [MD.apply_pepo(g, a) for a in can['A']]
    pre = FU.pretruncation(Theta, cell, can['lam'], 1)
    a_list = [C.double_layer(x) for x in FU.pretruncated_sites(Theta, cell, pre)]
    st, _, _, conv = C.ctmrg(cell, a_list, 1, 1e-13, 200)
    _, _, pos = FU.neighbours(cell)

    def gram(T, leg):
        Tm = np.moveaxis(T, FU.LEG[leg], -1)
        Tm = Tm.reshape(-1, Tm.shape[-1])
        return Tm.T @ Tm

    for e in FU.link_list(cell):
        t, dr = e
        x, y = pos[t]
        if dr == 'h':
            tq, lp, lq = cell.tid(x + 1, y), 'r', 'l'
        else:
            tq, lp, lq = cell.tid(x, y + 1), 'd', 'u'
        Gp = gram(FU.truncate_legs(Theta[t], cell, t, pre, lp), lp)
        Gq = gram(FU.truncate_legs(Theta[tq], cell, tq, pre, lq), lq)
        N4 = FU.bond_env(st, cell, e, Theta, pre)
        ref = np.einsum('ac,bd->abcd', Gp, Gq)
        N4 = N4 / np.einsum('ccee->', N4)
        ref = ref / np.einsum('ccee->', ref)
        np.testing.assert_allclose(N4, ref, rtol=0, atol=1e-12)
