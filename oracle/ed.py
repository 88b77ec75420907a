"""Exact diagonalisation of the transverse-field Ising model on small periodic lattices (oracle pin).

H = -sum_<ij> Z_i Z_j - h sum_i X_i on an Lx x Ly torus, lowest eigenvalue by
scipy's Lanczos (eigsh) on the 2^(Lx*Ly) dimensional space.  A loose check of
the 2D energies away from the critical field.
"""
import numpy as np
import scipy.sparse.linalg as sla


def tfim_ground_energy(Lx, Ly, h):
    """Ground-state energy per site of the TFIM on an Lx x Ly torus."""
    n = Lx * Ly
    dim = 1 << n
    states = np.arange(dim, dtype=np.int64)
    z = 1 - 2 * ((states[:, None] >> np.arange(n)) & 1)          # z[state, site] = +-1
    diag = np.zeros(dim)
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            for j in (y * Lx + (x + 1) % Lx, ((y + 1) % Ly) * Lx + x):
                diag -= z[:, i] * z[:, j]
    flips = [states ^ (1 << i) for i in range(n)]

    def matvec(v):
        v = v.ravel()
        out = diag * v
        for f in flips:
            out -= h * v[f]
        return out

    op = sla.LinearOperator((dim, dim), matvec=matvec, dtype=np.float64)
    w = sla.eigsh(op, k=1, which='SA', tol=1e-12)[0]
    return float(w[0]) / n
