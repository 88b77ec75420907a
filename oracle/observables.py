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
from .fullupdate import neighbours, link_list, half_env_left, half_env_right


def _ein(spec, x, y):
    return np.einsum(spec, x, y, optimize=True)


def rdm1(e, A):
    """rho[s, s'] of one site from its eight environment tensors (trace not normalised).

    Pairwise: top = C1 T1 C2, bottom = C3 T3 C4, then T2, T4, the ket and the bra.
    """
    chi, D = e['C1'].shape[0], A.shape[1]
    top = _ein('ibm,bc->icm', _ein('ia,abm->ibm', e['C1'], e['T1']), e['C2'])
    bot = _ein('dfx,fj->djx', _ein('de,efx->dfx', e['C3'], e['T3']), e['C4'])
    R1 = _ein('icm,cdn->imdn', top, e['T2'])
    R2 = _ein('imdn,djx->imnjx', R1, bot)
    R3 = _ein('imnjx,jil->mnxl', R2, e['T4']).reshape((D,) * 8)     # [(U u), (R r), (D d), (L l)]
    K1 = _ein('UuRrDdLl,sLRDU->urdls', R3, A)
    return _ein('urdls,tlrdu->st', K1, A)


def rdm2_h(ep, eq, Ap, Aq):
    """rho[s, t, s', t'] of the horizontal pair p -> q (trace not normalised)."""
    EL = half_env_left(ep, Ap, open_phys=True)       # [o, n, R, r, s, s']
    ER = half_env_right(eq, Aq, open_phys=True)      # [o, n, L, l, t, t']
    return np.einsum('onABsp,onABtq->stpq', EL, ER, optimize=True)


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
