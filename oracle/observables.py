"""Local observables from the CTM environment (oracle), Sec. VI.D.

m_z = <Psi|Z|Psi> / <Psi|Psi> (Eq. for m_z(h)), and the energy of the 2D TFIM
H = -sum ZZ - h sum X from one- and two-site reduced density matrices built
from the environment of Fig. 21.

Readings: the energy per site of a cell with n tensors is
    E_site = -(1/n) sum_{link types} <Z Z> - h (1/n) sum_t <X>_t,
every tensor owning one horizontal and one vertical link; the energy per link
of Sec. VI.D is E_site / 2 (two links per site).  Each tensor id is measured at
its first site in the cell.
"""
import numpy as np

from .model import X, Z
from .ctmrg import rotate_site
from .fullupdate import neighbours, link_list


def _un(T):
    c = T.shape[0]
    D = int(round(np.sqrt(T.shape[2])))
    return T.reshape(c, c, D, D)


def rdm1(e, A):
    """rho[s, s'] of one site from its eight environment tensors (trace not normalised)."""
    return np.einsum('ia,aoUu,ob,bcRr,ce,enDd,nk,kiLl,sLRDU,tlrdu->st',
                     e['C1'], _un(e['T1']), e['C2'], _un(e['T2']), e['C3'], _un(e['T3']),
                     e['C4'], _un(e['T4']), A, A, optimize='greedy')


def rdm2_h(ep, eq, Ap, Aq):
    """rho[s, t, s', t'] of the horizontal pair p -> q (trace not normalised)."""
    EL = np.einsum('ia,aoUu,jiLl,kj,nkDd,sLRDU,plrdu->onRrsp',
                   ep['C1'], _un(ep['T1']), _un(ep['T4']), ep['C4'], _un(ep['T3']), Ap, Ap,
                   optimize='greedy')
    ER = np.einsum('ab,oaUu,bcRr,ce,enDd,sLRDU,plrdu->onLlsp',
                   eq['C2'], _un(eq['T1']), _un(eq['T2']), eq['C3'], _un(eq['T3']), Aq, Aq,
                   optimize='greedy')
    return np.einsum('onABsp,onABtq->stpq', EL, ER)


def expect1(rho, O):
    return float(np.einsum('st,ts->', rho, O) / np.trace(rho))


def expect2(rho, O1, O2):
    r = rho.reshape(4, 4)
    O = np.kron(O1, O2)
    return float(np.trace(r @ O.T) / np.trace(r))


def measure(st, cell, A, h):
    """E_site, E_link, <X>_t, <Z>_t and <ZZ>_e from a converged CTMRG state of the tensors A."""
    _, _, pos = neighbours(cell)
    mx, mz, zz = {}, {}, {}
    for t in range(len(A)):
        x, y = pos[t]
        rho = rdm1(st.e(x, y), A[t])
        mx[t], mz[t] = expect1(rho, X), expect1(rho, Z)
    sr = st.rotated()
    for e in link_list(cell):
        t, dr = e
        x, y = pos[t]
        if dr == 'h':
            tq = cell.tid(x + 1, y)
            rho = rdm2_h(st.e(x, y), st.e(x + 1, y), A[t], A[tq])
        else:
            tq = cell.tid(x, y + 1)
            xr, yr = cell.rotate_pos(x, y)
            rho = rdm2_h(sr.e(xr, yr), sr.e(xr + 1, yr), rotate_site(A[t]), rotate_site(A[tq]))
        zz[e] = expect2(rho, Z, Z)
    n = len(A)
    e_site = -sum(zz.values()) / n - h * sum(mx.values()) / n
    return dict(e_site=e_site, e_link=e_site / 2.0, mx=mx, mz=mz, zz=zz)
