"""2D classical Ising model as a tensor network (oracle pin for the CTMRG).

The paper notes that the same environment machinery computes classical
partition functions (Sec. I).  Here the network of the square-lattice Ising
model Z = sum exp(beta sum_<ij> s_i s_j) is fed to the CTMRG of ctmrg.py in
place of a double layer, and compared with Onsager's free energy and Yang's
spontaneous magnetisation, which fix every part of the CTMRG (absorption,
projectors, renormalisation, cell indexing).

Bond weight B = [[e^b, e^-b], [e^-b, e^b]] = W W^T with W = V diag(sqrt(2 cosh b),
sqrt(2 sinh b)), V the Hadamard matrix; site tensor
a[l, r, d, u] = sum_s W[s,l] W[s,r] W[s,d] W[s,u]   (and s * ... for <s>).
"""
import numpy as np


def ising_tensors(beta):
    """(a, a_s): the site tensor and the one carrying the spin s, legs (l, r, d, u), dim 2."""
    V = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    W = V * np.sqrt(np.array([2.0 * np.cosh(beta), 2.0 * np.sinh(beta)]))[None, :]
    spin = np.array([1.0, -1.0])
    a = np.einsum('sl,sr,sd,su->lrdu', W, W, W, W)
    a_s = np.einsum('s,sl,sr,sd,su->lrdu', spin, W, W, W, W)
    return a, a_s


def yang_magnetization(beta):
    """Spontaneous magnetisation (1 - sinh(2 beta)^-4)^(1/8) for beta > beta_c, else 0."""
    x = np.sinh(2.0 * beta) ** -4
    return (1.0 - x) ** 0.125 if x < 1.0 else 0.0


def onsager_free_energy(beta, n=400):
    """-beta f = ln 2 + (1/(8 pi^2)) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)] dt1 dt2.

    The periodic integrand is summed on an n x n midpoint grid (spectrally
    accurate away from the critical point).
    """
    t = (np.arange(n) + 0.5) * 2.0 * np.pi / n
    c1, c2 = np.meshgrid(np.cos(t), np.cos(t))
    f = np.log(np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c1 + c2))
    return np.log(2.0) + f.mean() / 2.0


def gauge_pair(a, G, H, K, L):
    """Checkerboard tensors (A, B) from a with the link gauges inserted (the network is unchanged).

    Horizontal A->B carries G G^-1, B->A carries H H^-1, vertical A->B K K^-1,
    B->A L L^-1; a tensor's out leg takes leg . M, its in leg M^-1 . leg.
    """
    inv = np.linalg.inv
    A = np.einsum('lrdu,rR,dD,Ll,Uu->LRDU', a, G, K, inv(H), inv(L))
    B = np.einsum('lrdu,rR,dD,Ll,Uu->LRDU', a, H, L, inv(G), inv(K))
    return A, B
