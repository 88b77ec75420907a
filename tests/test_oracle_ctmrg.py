"""Pins of the CTMRG oracle (Sec. VI.B item 1, Fig. 21a) against the exactly solved classical Ising model.

The CTMRG is generic in the network it contracts (Sec. I notes the same
machinery computes classical partition functions), so Yang's magnetisation and
Onsager's free energy fix the absorption, projector and renormalisation steps,
the rotations between moves, and the unit-cell bookkeeping (via link gauges
that only a correctly indexed cell cancels).
"""
import numpy as np
import pytest

from oracle import classical as K
from oracle import ctmrg as C
from oracle import observables as O


@pytest.mark.parametrize("beta", [0.5, 0.6])
def test_uniform_cell_yang_and_onsager(beta):
    a, a_s = K.ising_tensors(beta)
    st, it, d, conv = C.ctmrg(C.single_site(), [a], 12, tol=1e-9, max_iter=300, boundary=[1.0, 1.0])
    e = st.e(0, 0)
    Z1, Z0, Zh, Zv = C.site_scalars(e, a)
    m = C.site_scalars(e, a_s)[0] / Z1
    assert abs(abs(m) - K.yang_magnetization(beta)) < 1e-8
    assert abs(np.log(Z1 * Z0 / (Zh * Zv)) - K.onsager_free_energy(beta)) < 1e-9


def test_disordered_phase_free_energy():
    beta = 0.3                                   # above T_c: m = 0
    a, a_s = K.ising_tensors(beta)
    st, it, d, conv = C.ctmrg(C.single_site(), [a], 12, tol=1e-10, max_iter=300, boundary=[1.0, 1.0])
    Z1, Z0, Zh, Zv = C.site_scalars(st.e(0, 0), a)
    assert abs(np.log(Z1 * Z0 / (Zh * Zv)) - K.onsager_free_energy(beta)) < 1e-9
    assert abs(C.site_scalars(st.e(0, 0), a_s)[0] / Z1) < 1e-6    # finite-chi breaking by the boundary


def test_checkerboard_with_link_gauges():
    """Four different random gauges on the four link types of the (A, B) cell leave m unchanged."""
    beta = 0.5
    a, a_s = K.ising_tensors(beta)
    rng = np.random.default_rng(3)
    G, H, Kg, L = [np.eye(2) + 0.3 * rng.standard_normal((2, 2)) for _ in range(4)]
    A, B = K.gauge_pair(a, G, H, Kg, L)
    As, Bs = K.gauge_pair(a_s, G, H, Kg, L)
    cell = C.checkerboard()
    st, it, d, conv = C.ctmrg(cell, [A, B], 12, tol=1e-9, max_iter=400, boundary=[1.0, 1.0])
    for (x, y) in cell.sites():
        T, Ts = ((A, As), (B, Bs))[cell.tid(x, y)]
        e = st.e(x, y)
        m = C.site_scalars(e, Ts)[0] / C.site_scalars(e, T)[0]
        assert abs(abs(m) - K.yang_magnetization(beta)) < 1e-8


def test_rotation_is_order_four():
    cell = C.checkerboard()
    rng = np.random.default_rng(0)
    a = [rng.standard_normal((4, 4, 4, 4)) for _ in range(2)]
    env = C.init_env(cell, 3, 4)
    for e in env.values():
        for k in e:
            e[k] = rng.standard_normal(e[k].shape)
    st = C.State(cell, a, env)
    r = st.rotated().rotated().rotated().rotated()
    assert np.array_equal(r.cell.pattern, cell.pattern)
    for k in env:
        for n in env[k]:
            assert r.env[k][n] is env[k][n]
    for x, y in zip(r.a, a):
        assert np.array_equal(x, y)


def test_enlarged_corner_matches_definition():
    """The matrix form of Q_UL equals the contraction C1 T1 T4 a written out (Fig. 21a)."""
    cell = C.checkerboard()
    rng = np.random.default_rng(1)
    chi, D2 = 3, 4
    a = [rng.standard_normal((D2,) * 4) for _ in range(2)]
    env = C.init_env(cell, chi, D2)
    for e in env.values():
        for k in e:
            e[k] = rng.standard_normal(e[k].shape)
    st = C.State(cell, a, env)
    Q = C.enlarged_corners(st, 0, 0)[0]
    e = st.e(0, 0)
    ref = np.zeros((chi, D2, chi, D2))
    for i in range(chi):          # T4.in
        for s in range(D2):       # a.d
            for o in range(chi):  # T1.out
                for r in range(D2):
                    v = 0.0
                    for c_in in range(chi):
                        for c_out in range(chi):
                            for m1 in range(D2):
                                for m4 in range(D2):
                                    v += (e['C1'][c_in, c_out] * e['T1'][c_out, o, m1] *
                                          e['T4'][i, c_in, m4] * a[0][m4, r, s, m1])
                    ref[i, s, o, r] = v
    np.testing.assert_allclose(Q, ref.reshape(chi * D2, chi * D2), rtol=1e-12, atol=1e-12)


def test_product_state_energy_exact():
    """A ferromagnetic product state has E_site = -2 at h = 0 and <X> = 0 (exact at any chi)."""
    A = np.zeros((2, 2, 2, 2, 2))
    A[0, 0, 0, 0, 0] = 1.0
    A[1, 1, 1, 1, 1] = 1e-3          # a second, decoupled sector of tiny weight
    cell = C.checkerboard()
    st, it, d, conv = C.ctmrg(cell, [C.double_layer(A)] * 2, 6, tol=1e-12, max_iter=50)
    m = O.measure(st, cell, [A, A], 0.0)
    assert abs(m['e_site'] + 2.0) < 1e-12
    assert abs(m['mz'][0] - 1.0) < 1e-12
