"""Pins of the model layer of the oracle: Trotter gates, iMPO/iPEPO, 1D closed form (Sec. V.A, VI.A)."""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.linalg import expm

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kron(*ops):
    out = np.ones((1, 1))
    for o in ops:
        out = np.kron(out, o)
    return out


def test_bond_split_reproduces_gate():
    # sum_k w[k,s] w[k,t] = e^{delta z_s z_t}: the symmetric split of g_I = U S V
    for delta in (0.0, 0.01, 0.3):
        w = model.bond_weights(delta)
        z = np.array([1.0, -1.0])
        np.testing.assert_allclose(w.T @ w, np.exp(delta * np.outer(z, z)), rtol=1e-14, atol=1e-15)


def test_field_gate_is_exponential():
    for h, d in ((3.04, 0.005), (1.0, 0.2)):
        np.testing.assert_allclose(model.field_gate(h, d), expm(h * d / 2 * model.X), rtol=1e-14)


def test_ipepo_on_2x2_torus_equals_trotter_product():
    """The iPEPO contracted on a 2x2 torus equals g_F e^{-delta H_I} g_F built with expm (Sec. VI.A)."""
    h, delta = 1.7, 0.13
    g = model.ipepo(h, delta)
    # bonds: 0.r=1.l (a), 1.r=0.l (b), 2.r=3.l (c), 3.r=2.l (e), 0.d=2.u (f), 2.d=0.u (i), 1.d=3.u (j), 3.d=1.u (k)
    U = np.einsum('pPbafi,qQabjk,rRecif,sScekj->pqrsPQRS', g, g, g, g).reshape(16, 16)
    # sites 0..3 in kron order; every pair is joined by two bonds on the 2x2 torus
    Zs = [_kron(*[model.Z if i == k else model.I2 for i in range(4)]) for k in range(4)]
    HI = -2.0 * (Zs[0] @ Zs[1] + Zs[2] @ Zs[3] + Zs[0] @ Zs[2] + Zs[1] @ Zs[3])
    GF = _kron(*[model.field_gate(h, delta)] * 4)
    np.testing.assert_allclose(U, GF @ expm(-delta * HI) @ GF, rtol=1e-12, atol=1e-14)


def test_impo_on_ring_equals_trotter_product():
    """The iMPO of Eq. (iMPO1) on a 4-site ring equals g_F e^{-delta H_I} g_F (Sec. V.A)."""
    h, delta = 0.9, 0.2
    g = model.impo(h, delta)
    U = np.einsum('pPda,qQab,rRbc,sScd->pqrsPQRS', g, g, g, g).reshape(16, 16)
    Zs = [_kron(*[model.Z if i == k else model.I2 for i in range(4)]) for k in range(4)]
    HI = -sum(Zs[i] @ Zs[(i + 1) % 4] for i in range(4))
    GF = _kron(*[model.field_gate(h, delta)] * 4)
    np.testing.assert_allclose(U, GF @ expm(-delta * HI) @ GF, rtol=1e-12, atol=1e-14)


def test_apply_pepo_fusion_order():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((2, 3, 3, 3, 3))
    g = model.ipepo(2.0, 0.1)
    T = model.apply_pepo(g, A)
    assert T.shape == (2, 6, 6, 6, 6)
    # entry (s', (kl, l), ...) with kappa-major fusion
    ref = np.einsum('pq,q->p', g[:, :, 1, 0, 1, 1], A[:, 2, 0, 1, 2])
    np.testing.assert_allclose(T[:, 1 * 3 + 2, 0 * 3 + 0, 1 * 3 + 1, 1 * 3 + 2], ref, rtol=1e-14)


def test_exact_1d_energy_matches_paper():
    """E_exact ~ -1.306856 at h = 1.05 (Sec. V.C, Fig. 19 caption)."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        ref = json.load(f)["ising_1d_exact_energy_h1.05"]["value"]
    assert abs(model.exact_energy_1d(1.05) - ref) < 5e-7


@pytest.mark.parametrize("h", [0.3, 1.05, 2.0, 7.0])
def test_exact_1d_energy_quadrature(h):
    val = quad(lambda k: np.sqrt(1 + h * h - 2 * h * np.cos(k)), 0, np.pi, epsabs=1e-14)[0]
    assert abs(model.exact_energy_1d(h) + val / np.pi) < 1e-10


def test_exact_1d_energy_limits():
    assert abs(model.exact_energy_1d(0.0) + 1.0) < 1e-12          # classical chain, <ZZ> = 1
    h = 40.0                                                        # -h - 1/(4h) + O(h^-3)
    assert abs(model.exact_energy_1d(h) + h + 1 / (4 * h)) < 1 / h ** 3
