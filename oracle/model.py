"""Transverse-field Ising model, Trotter gates, iMPO and iPEPO (oracle).

Sec. V.A (1D): H = -sum Z_i Z_{i+1} - h sum X_i, second-order Trotter
    e^{-H delta} ~ prod g_F  prod g_I  prod g_F,   g_F = e^{-H_F delta/2},
    g_I = e^{-H_I delta}, and the single-site iMPO of Eq. (iMPO1).
Sec. VI.A (2D): the same with horizontal and vertical ZZ terms; all ZZ terms
    commute, so the iPEPO reproduces e^{-delta H_I} exactly.

Reading (the printed factor order of the iPEPO is garbled): each bond gate is
split symmetrically, e^{delta Z(x)Z} = sum_k (sqrt(c_k) O_k) (x) (sqrt(c_k) O_k)
with O_0 = I, c_0 = cosh(delta), O_1 = Z, c_1 = sinh(delta).  This is the SVD
g_I = U S V of the paper with sqrt(S) given to each side, which is a gauge
choice on the kappa = 2 bond.
"""
import numpy as np

X = np.array([[0.0, 1.0], [1.0, 0.0]])
Z = np.array([[1.0, 0.0], [0.0, -1.0]])
I2 = np.eye(2)


def field_gate(h, delta):
    """g_F = exp(+h delta X / 2): the half field step e^{-H_F delta/2}, H_F = -h X."""
    c, s = np.cosh(h * delta / 2.0), np.sinh(h * delta / 2.0)
    return np.array([[c, s], [s, c]])


def bond_weights(delta):
    """w[k, t] = sqrt(c_k) (O_k)_{tt}: one side of the symmetric split of e^{delta ZZ}.

    e^{delta Z Z} = cosh(delta) I(x)I + sinh(delta) Z(x)Z, both operators are
    diagonal in the Z basis, so each side carries the diagonal weights w.
    Requires delta >= 0 (sinh(delta) >= 0 for the square root).
    """
    if delta < 0:
        raise ValueError("delta must be >= 0")
    z = np.diag(Z)
    return np.stack([np.sqrt(np.cosh(delta)) * np.ones(2),
                     np.sqrt(np.sinh(delta)) * z])


def impo(h, delta):
    """Single-site iMPO g[s', s, kl, kr] of Eq. (iMPO1), kappa = 2 (Fig. 15).

    g = g_F (V S U) g_F: the site carries the right half of the bond to its
    left (kl) and the left half of the bond to its right (kr).
    """
    gf = field_gate(h, delta)
    w = bond_weights(delta)
    return np.einsum('at,kt,mt,tb->abkm', gf, w, w, gf)


def ipepo(h, delta):
    """Single-site iPEPO g[s', s, l, r, d, u], kappa = 2 on each virtual leg (Fig. 20).

    g = g_F (bond halves on l, r, d, u) g_F, i.e. the 2D analogue of Eq. (iMPO1).
    Applying it on every site gives prod g_F . prod_bonds e^{delta ZZ} . prod g_F.
    """
    gf = field_gate(h, delta)
    w = bond_weights(delta)
    return np.einsum('at,it,jt,kt,mt,tb->abijkm', gf, w, w, w, w, gf)


def apply_pepo(g, A):
    """Theta = g A with fused bonds (kappa, D) -> kappa*D, kappa-major (Sec. VI.C).

    A[s, l, r, d, u], g[s', s, l, r, d, u]; returns Theta[s', L, R, Dn, U] with
    L = kl * D + l and likewise for the other legs.
    """
    d, D = A.shape[0], A.shape[1]
    k = g.shape[2]
    T = np.einsum('pqabce,qlrdu->palbrcdeu', g, A)
    return T.reshape(d, k * D, k * D, k * D, k * D)


def apply_mpo(g, A):
    """Theta = g A for an iMPS tensor A[s, l, r]; bonds fused kappa-major (Sec. V.B)."""
    d, chi = A.shape[0], A.shape[1]
    k = g.shape[2]
    T = np.einsum('pqab,qlr->palbr', g, A)
    return T.reshape(d, k * chi, k * chi)


def exact_energy_1d(h, n=20001):
    """Ground-state energy per site of the infinite 1D TFIM (closed form).

    e(h) = -(1/pi) int_0^pi sqrt(1 + h^2 - 2 h cos k) dk, evaluated with the
    composite Simpson rule on n points (the integrand is smooth for h != 1).
    Sec. V.C quotes E_exact ~ -1.306856 at h = 1.05.
    """
    k = np.linspace(0.0, np.pi, n)
    f = np.sqrt(1.0 + h * h - 2.0 * h * np.cos(k))
    dx = k[1] - k[0]
    s = f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum()
    return -(s * dx / 3.0) / np.pi
