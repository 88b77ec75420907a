"""Structural pins of the CTMRG and observables oracle: lattice symmetry.

(1) Rotation covariance.  The state of the rotated site tensor is the rotated
state: CTMRG on rotate_site(A) must converge to the rotated environment of A
(normalised corner spectra relabelled C1 <- C2, C2 <- C3, C3 <- C4, C4 <- C1, up
to the phase of the move cycle), and <ZZ> on its horizontal links must equal
<ZZ> on the vertical links of A and vice versa.  This fixes the directional moves, the rotation of the double
layer and of the environment labels, and the vertical-bond measurement (which
goes through a rotated network): a wrong leg order or relabelling in any of
them breaks the equalities for a generic tensor.

(2) A tensor invariant under the eight symmetries of the square lattice has
equivalent corners and bonds: equal corner spectra at every site and corner,
equal <ZZ> on every link, in the one-site and the checkerboard cell.
"""
import numpy as np
import pytest

from oracle import ctmrg as C
from oracle import observables as O
from paper_1411_0391_gb300.inputs import random_peps

H = 3.0


def _c4v_symmetrise(A):
    """Average of A over the 8 lattice symmetries acting on the legs (l, r, d, u)."""
    flip_lr = lambda T: T.transpose(0, 2, 1, 3, 4)          # l <-> r
    out, T = np.zeros_like(A), A
    for _ in range(4):
        out += T + flip_lr(T)
        T = C.rotate_site(T)
    return out / 8.0


def _run(cell, tensors, chi=8):
    a = [C.double_layer(A) for A in tensors]
    st, it, d, conv = C.ctmrg(cell, a, chi, tol=1e-10, max_iter=500)
    assert conv, (it, d)
    return st


@pytest.mark.parametrize("inst", [2, 7])
def test_rotated_tensor_gives_the_rotated_environment_and_bonds(inst):
    """CTMRG on rotate_site(A) against CTMRG on A (chi = 24).  The directional moves run
    in a fixed cycle (left, up, right, down); on the rotated lattice the same cycle starts
    one move later, so the two fixed points are the same cycle seen at phases one move
    apart: the corners that the last move leaves alone (new C1 = old C2, new C2 = old C3)
    agree exactly, the other two within the cycle's own oscillation at finite chi
    (~1e-4 on the spectra), and the bond observables within ~3e-7 (measured shrinking
    with chi: 9e-6 at chi = 8, 4e-7 at 16)."""
    A = random_peps(1, 2, instance=inst)[0]
    Ar = C.rotate_site(A)
    cell = C.single_site()
    st, st_r = _run(cell, [A], chi=24), _run(cell, [Ar], chi=24)
    sp, sp_r = C.corner_spectra(st), C.corner_spectra(st_r)
    for new, old in (("C1", "C2"), ("C2", "C3")):
        assert C.ROT_ENV[new] == old
        np.testing.assert_allclose(sp_r[(0, 0, new)], sp[(0, 0, old)], atol=1e-9)
    for new, old in (("C3", "C4"), ("C4", "C1")):
        np.testing.assert_allclose(sp_r[(0, 0, new)], sp[(0, 0, old)], atol=2e-3)
    m, m_r = O.measure(st, cell, [A], H), O.measure(st_r, cell, [Ar], H)
    assert abs(m_r['zz'][(0, 'h')] - m['zz'][(0, 'v')]) < 1e-6
    assert abs(m_r['zz'][(0, 'v')] - m['zz'][(0, 'h')]) < 1e-6
    assert abs(m['zz'][(0, 'h')] - m['zz'][(0, 'v')]) > 1e-3       # the tensor is not symmetric
    assert abs(m_r['mx'][0] - m['mx'][0]) < 1e-6 and abs(m_r['e_site'] - m['e_site']) < 2e-6


@pytest.mark.parametrize("inst", [2, 5])
def test_symmetric_tensor_has_equivalent_corners_and_bonds(inst):
    A = _c4v_symmetrise(random_peps(1, 2, instance=inst)[0])
    for T in (C.rotate_site(A), A.transpose(0, 2, 1, 3, 4), A.transpose(0, 1, 2, 4, 3)):
        np.testing.assert_allclose(T, A, atol=1e-15)
    st = _run(C.single_site(), [A])
    sp = C.corner_spectra(st)
    ref = sp[(0, 0, 'C1')]
    for c in ('C2', 'C3', 'C4'):
        np.testing.assert_allclose(sp[(0, 0, c)], ref, atol=1e-9)
    m = O.measure(st, C.single_site(), [A], H)
    zz = list(m['zz'].values())
    assert len(zz) == 2 and abs(zz[0] - zz[1]) < 1e-9, zz
    # the same tensor on both sites of the checkerboard cell: every site, corner and link alike
    st2 = _run(C.checkerboard(), [A, A])
    for s in C.corner_spectra(st2).values():
        np.testing.assert_allclose(s, ref, atol=1e-8)
    m2 = O.measure(st2, C.checkerboard(), [A, A], H)
    for v in m2['zz'].values():
        assert abs(v - zz[0]) < 1e-8
    assert abs(m2['e_site'] - m['e_site']) < 1e-8
