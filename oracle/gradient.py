"""Energy gradient of the 1-site iPEPS (oracle; test infrastructure only).

The reference a fixed-point adjoint of CTMRG has to reproduce: E(A) is the
energy per site of the translation-invariant iPEPS with the single tensor A
(1-site cell), its environment converged by the CTMRG of ctmrg.py and its
observables those of Sec. VI.D; dE/dA is taken by central finite differences,
each perturbed energy warm-started from the environment of A so that all
evaluations stay on one CTMRG fixed point.  Slow (two converged CTMRGs per
entry of A), plain, and pinned by exact invariances of E (tests):
  * E(cA) = E(A): the gradient is orthogonal to A;
  * an orthogonal gauge on the bonds, A -> A x_l O x_r O (likewise on d/u),
    leaves E unchanged (the truncated CTMRG is covariant under orthogonal
    gauges): the gradient is orthogonal to the tangent X.A - A.X, X = -X^T;
  * the h = 0 ferromagnet is the ground state, so a stationary point;
  * the error of the central difference is O(eps^2).
"""
import numpy as np

from .ctmrg import single_site, double_layer, ctmrg
from .observables import measure


def energy(A, h, chi, tol=1e-12, max_iter=2000, env=None):
    """(E_site, environment) of the 1-site iPEPS A[s, l, r, d, u]."""
    cell = single_site()
    st, it, delta, conv = ctmrg(cell, [double_layer(A)], chi, tol, max_iter, env=env)
    return measure(st, cell, [A], h)['e_site'], st.env


def grad_fd(A, h, chi, eps=1e-6, tol=1e-12):
    """dE/dA by central differences, every evaluation warm-started from A's environment."""
    e0, env = energy(A, h, chi, tol)
    g = np.zeros_like(A)
    for idx in np.ndindex(A.shape):
        Ap = A.copy()
        Ap[idx] += eps
        Am = A.copy()
        Am[idx] -= eps
        ep, _ = energy(Ap, h, chi, tol, env=env)
        em, _ = energy(Am, h, chi, tol, env=env)
        g[idx] = (ep - em) / (2.0 * eps)
    return g, e0


def gauge_tangent(A, X, axis_in, axis_out):
    """First-order change of A under the bond gauge exp(X) on the leg pair (in, out):
    X acting on the incoming leg minus X acting on the outgoing leg."""
    return np.moveaxis(np.tensordot(X, A, axes=([1], [axis_in])), 0, axis_in) \
        - np.moveaxis(np.tensordot(A, X, axes=([axis_out], [0])), -1, axis_out)
