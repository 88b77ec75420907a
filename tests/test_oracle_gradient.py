"""Pins of the oracle's energy gradient of the 1-site iPEPS (the reference for a CTMRG adjoint)."""
import numpy as np
import pytest

from oracle import gradient as G
from paper_1411_0391_gb300.inputs import random_peps

H, CHI = 3.04, 8


@pytest.fixture(scope="module")
def case():
    A = random_peps(1, 2, instance=3)[0]
    g, e = G.grad_fd(A, H, CHI)
    return A, g, e


def test_gradient_orthogonal_to_scaling(case):
    """E(cA) = E(A) for every c: d/dc E(cA) = <A, g> = 0."""
    A, g, _ = case
    assert abs(np.vdot(A, g)) < 1e-7 * np.linalg.norm(A) * np.linalg.norm(g)


@pytest.mark.parametrize("legs", [(1, 2), (3, 4)])
def test_gradient_orthogonal_to_orthogonal_gauges(case, legs):
    """An orthogonal gauge on the horizontal (l, r) or vertical (d, u) bonds leaves E
    unchanged: the gradient is orthogonal to every tangent X.A - A.X with X = -X^T."""
    A, g, _ = case
    rng = np.random.default_rng(11)
    for _ in range(3):
        X = rng.standard_normal((2, 2))
        X = X - X.T
        t = G.gauge_tangent(A, X, *legs)
        assert abs(np.vdot(t, g)) < 1e-7 * np.linalg.norm(t) * np.linalg.norm(g)


def test_gradient_is_not_trivial(case):
    """A generic direction changes E at first order, as the gradient predicts (a central
    difference along the direction): the orthogonality pins above are not vacuous."""
    A, g, e = case
    d = random_peps(1, 2, instance=4)[0]
    step = 1e-4
    _, env = G.energy(A, H, CHI)
    ep, _ = G.energy(A + step * d, H, CHI, env=env)
    em, _ = G.energy(A - step * d, H, CHI, env=env)
    assert abs(np.vdot(g, d)) > 1e-3
    assert abs((ep - em) / (2 * step) - np.vdot(g, d)) < 1e-6 * abs(np.vdot(g, d))


def test_ferromagnet_is_stationary_at_h0():
    """At h = 0 the product state |up> is the ground state: the gradient vanishes there."""
    A = np.zeros((2, 2, 2, 2, 2))
    A[0, 0, 0, 0, 0] = 1.0
    g, e = G.grad_fd(A, 0.0, 4)
    assert abs(e + 2.0) < 1e-12
    assert np.linalg.norm(g) < 1e-8


def test_central_difference_error_is_second_order(case):
    A, g, _ = case
    g2, _ = G.grad_fd(A, H, CHI, eps=2e-6)
    assert np.linalg.norm(g2 - g) < 1e-6 * np.linalg.norm(g)
