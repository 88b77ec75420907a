"""Full-update bond truncation (oracle), Sec. VI.B item 2.

After the iPEPO step every bond of Theta = g A has dimension kappa*D.  For each
link a pair (P, Q), P: kappa*D x D on the left/top site, Q: D x kappa*D on the
right/bottom site, is found by minimising the cost of Eq. (var),
    f = || Psi_g - Psi_zeta ||^2,
one variable at a time through the quadratic form of Eq. (var1), P = R^{-1} S.
The environment is the CTM environment of the pre-truncated tensors (Sec. VI.B,
last paragraph: pre-truncation with simple-update projectors reduces the cost
to O(chi^3 D^6)).

Links.  A link type is (t, 'h') or (t, 'v'): the bond leaving tensor t to the
right or downward.  Leg ownership of tensor t:
    r -> (t, 'h') out side      l -> (left(t), 'h') in side
    d -> (t, 'v') out side      u -> (up(t), 'v') in side
An out leg is multiplied by P (Theta[.., a, ..] P[a, i]); an in leg by Q
(Q[i, b] Theta[.., b, ..]).

Readings (the figures that define E1..E6 are missing):
* Pre-truncation (a7): the simple-update truncation of each link with the
  canonical-form weights lambda as the environment of the external legs.  Each
  external leg of Theta (index kappa*D, kappa-major) carries sqrt(lambda[i]) on
  top of the sqrt(lambda) already absorbed in the weighted canonical tensor.
* Bond environment (a8): only the optimised link keeps dimension kappa*D on its
  ket and bra legs; every other leg of the two sites is pre-truncated; the
  physical legs are traced.  The CTM tensors carry an arbitrary overall sign
  and scale, so N is divided by <g|g> = sum N[a,a,b,b]; then it is symmetrised
  and projected on its positive part.
* 1-site cell (Sec. VI.B): the paper optimises one pair for each link r, d, l, u
  of the plaquette and then averages, P_h = (P_r + P_l)/2, Q_h = (Q_r + Q_l)/2
  (likewise v from d and u).  With the per-link two-site cluster above, built
  from the CTM tensors directly, the clusters around r and l are the same
  network in a 1-site cell (every site carries the same tensor and the same
  environment), so the two pairs coincide and each average equals the single
  pair per link type that full_update computes.
* ALS (a9): start from the pre-truncation pair, alternate P and Q solves with an
  eigenvalue pseudo-inverse (relative cutoff ALS_PINV_CUTOFF = 1e-12; the paper
  writes P = R^{-1} S and is silent on the singular case), stop when the link matrix
  M = P Q changes by less than tol * ||M|| (cap max_iter); then balance the pair
  by the SVD of M: P = U sqrt(S), Q = sqrt(S) V^T.  A link whose projected
  environment has no weight (<g|g> = 0)
  keeps its pre-truncation pair.
"""
import numpy as np

from .ctmrg import sign_fix, State, rotate_site

LEG = {'l': 1, 'r': 2, 'd': 3, 'u': 4}
PINV_CUTOFF = 1e-12          # S^{-1/2} of the simple-update pair projectors
ALS_PINV_CUTOFF = 1e-12      # pseudo-inverse of the ALS normal equations (reading above)


def neighbours(cell):
    """Tensor ids to the left and above each tensor id; the cell must determine them uniquely."""
    left, up, pos = {}, {}, {}
    for (x, y) in cell.sites():
        t = cell.tid(x, y)
        pos.setdefault(t, (x, y))
        for dct, val in ((left, cell.tid(x - 1, y)), (up, cell.tid(x, y - 1))):
            if dct.setdefault(t, val) != val:
                raise ValueError("unit cell does not fix the neighbours of each tensor")
    return left, up, pos


def link_list(cell):
    """Link types in a fixed order: (t, 'h') then (t, 'v') for t = 0, 1, ..."""
    n = int(cell.pattern.max()) + 1
    return [(t, 'h') for t in range(n)] + [(t, 'v') for t in range(n)]


def leg_links(cell, t):
    """For tensor t: leg name -> (link, 'out'|'in')."""
    left, up, _ = neighbours(cell)
    return {'r': ((t, 'h'), 'out'), 'l': ((left[t], 'h'), 'in'),
            'd': ((t, 'v'), 'out'), 'u': ((up[t], 'v'), 'in')}


def leg_mul(T, axis, M):
    """T'[.., j, ..] = sum_i T[.., i, ..] M[i, j] on the given axis."""
    return np.moveaxis(np.tensordot(T, M, axes=([axis], [0])), -1, axis)


def psd_sqrt(G):
    """Symmetric positive square root of a symmetric PSD matrix (negative eigenvalues clipped)."""
    w, V = np.linalg.eigh(0.5 * (G + G.T))
    w = np.clip(w, 0.0, None)
    return (V * np.sqrt(w)) @ V.T


def pair_projectors(Rp, Lq, D):
    """Truncate the bond between Rp [reduced, a] and Lq [b, reduced] to dimension D.

    Rp Lq = U S V^T (sign rule), P = Lq V_D S_D^{-1/2}, Q = S_D^{-1/2} U_D^T Rp,
    so that Rp (P Q) Lq = U_D S_D V_D^T.  Returns P, Q, S_D.
    """
    U, S, Vt = np.linalg.svd(Rp @ Lq)
    U, V = sign_fix(U[:, :D], Vt[:D].T)
    S = S[:D]
    inv = np.zeros_like(S)
    if S[0] > 0:
        keep = S >= PINV_CUTOFF * S[0]
        inv[keep] = 1.0 / np.sqrt(S[keep])
    return Lq @ (V * inv), (U * inv).T @ Rp, S


def pretruncation(Theta, cell, lam, D, kappa=2):
    """Simple-update projectors (P, Q) of every link type (row a7).

    For link e = (t -> t'): G_t is the Gram matrix of Theta_t on its link leg
    with sqrt(lambda) on each other leg, G_t' likewise; Rp = sqrt(G_t),
    Lq = sqrt(G_t') and the pair comes from pair_projectors.
    """
    left, up, _ = neighbours(cell)
    out = {}
    for e in link_list(cell):
        t, dr = e
        tq = _next(cell, t, dr)
        lp, lq = ('r', 'l') if dr == 'h' else ('d', 'u')
        Gp = _weighted_gram(Theta[t], cell, t, lp, lam, kappa)
        Gq = _weighted_gram(Theta[tq], cell, tq, lq, lam, kappa)
        P, Q, _ = pair_projectors(psd_sqrt(Gp), psd_sqrt(Gq), D)
        out[e] = (P, Q)
    return out


def _next(cell, t, dr):
    _, _, pos = neighbours(cell)
    x, y = pos[t]
    return cell.tid(x + 1, y) if dr == 'h' else cell.tid(x, y + 1)


def _weighted_gram(T, cell, t, leg, lam, kappa):
    legs = leg_links(cell, t)
    X = T
    for name, (e, _side) in legs.items():
        if name == leg:
            continue
        w = np.tile(np.sqrt(lam[e]), kappa)        # index k*D + i -> sqrt(lambda[i])
        X = X * _axis_vec(w, LEG[name])
    ax = LEG[leg]
    Xm = np.moveaxis(X, ax, -1).reshape(-1, X.shape[ax])
    return Xm.T @ Xm


def _axis_vec(w, axis):
    shape = [1] * 5
    shape[axis] = len(w)
    return w.reshape(shape)


def truncate_legs(T, cell, t, proj, open_leg=None):
    """Apply the link projectors to every leg of Theta_t except open_leg."""
    for name, (e, side) in leg_links(cell, t).items():
        if name == open_leg:
            continue
        P, Q = proj[e]
        T = leg_mul(T, LEG[name], P if side == 'out' else Q.T)
    return T


def _un(T):
    c = T.shape[0]
    D = int(round(np.sqrt(T.shape[2])))
    return T.reshape(c, c, D, D)


def _ein(spec, x, y):
    return np.einsum(spec, x, y, optimize=True)


def half_env_left(e, Tp, bra=None, open_phys=False):
    """E_L[o, n, R, r(, s, s')] of site p: C1 T1 T4 with the ket and bra of Tp, then C4 T3.

    Contracted pairwise (the order keeps every intermediate at chi^2 D^4 size):
    C1 T1 -> T4 -> ket -> bra -> (C4 T3).  Tp's r leg stays open (ket R, bra r);
    with open_phys the physical legs stay open too.
    """
    bra = Tp if bra is None else bra
    chi, D = e['C1'].shape[0], Tp.shape[1]
    X1 = _ein('ia,aom->iom', e['C1'], e['T1'])
    X2 = _ein('iom,jin->omjn', X1, e['T4']).reshape(chi, D, D, chi, D, D)
    X3 = _ein('oUujLl,sLRDU->oujlsRD', X2, Tp)
    if open_phys:
        X4 = _ein('oujlsRD,tlrdu->ojRDrdst', X3, bra)
    else:
        X4 = _ein('oujlsRD,slrdu->ojRDrd', X3, bra)
    LL = _ein('kj,nkm->jnm', e['C4'], e['T3']).reshape(chi, chi, D, D)
    if open_phys:
        return _ein('ojRDrdst,jnDd->onRrst', X4, LL)
    return _ein('ojRDrd,jnDd->onRr', X4, LL)


def half_env_right(e, Tq, bra=None, open_phys=False):
    """E_R[o, n, L, l(, s, s')] of site q: T1 C2 T2 with the ket and bra of Tq, then C3 T3."""
    bra = Tq if bra is None else bra
    chi, D = e['C2'].shape[0], Tq.shape[2]
    Y1 = _ein('oam,ac->ocm', e['T1'], e['C2'])
    Y2 = _ein('ocm,ctn->omtn', Y1, e['T2']).reshape(chi, D, D, chi, D, D)
    Y3 = _ein('oUutRr,sLRDU->outrsLD', Y2, Tq)
    if open_phys:
        Y4 = _ein('outrsLD,plrdu->otLDldsp', Y3, bra)
    else:
        Y4 = _ein('outrsLD,slrdu->otLDld', Y3, bra)
    LR = _ein('te,enm->tnm', e['C3'], e['T3']).reshape(chi, chi, D, D)
    if open_phys:
        return _ein('otLDldsp,tnDd->onLlsp', Y4, LR)
    return _ein('otLDld,tnDd->onLl', Y4, LR)


def bond_env_h(ep, eq, Tp, Tq):
    """N[a, a', b, b'] of the horizontal link p -> q (Fig. 21b; reading of E1..E6).

    ep, eq: environments of p and q; Tp has its r leg open, Tq its l leg open
    (ket a, bra a' for p; ket b, bra b' for q).  E_L collects C1 T1 T4 C4 T3 of
    p with the two layers of Tp, E_R collects C2 T1 T2 C3 T3 of q with Tq;
    T1_p.out joins T1_q.in and T3_q.out joins T3_p.in.
    """
    EL = half_env_left(ep, Tp)
    ER = half_env_right(eq, Tq)
    return np.einsum('onAa,onBb->AaBb', EL, ER, optimize=True)


def bond_env(st, cell, e, Theta, proj):
    """Bond environment of link type e as N4[a, b, a', b'] (ket a, ket b, bra a', bra b')."""
    _, _, pos = neighbours(cell)
    t, dr = e
    x, y = pos[t]
    if dr == 'h':
        tq = cell.tid(x + 1, y)
        Tp = truncate_legs(Theta[t], cell, t, proj, 'r')
        Tq = truncate_legs(Theta[tq], cell, tq, proj, 'l')
        N = bond_env_h(st.e(x, y), st.e(x + 1, y), Tp, Tq)
    else:
        tq = cell.tid(x, y + 1)
        Tp = rotate_site(truncate_legs(Theta[t], cell, t, proj, 'd'))
        Tq = rotate_site(truncate_legs(Theta[tq], cell, tq, proj, 'u'))
        sr = st.rotated()
        xr, yr = cell.rotate_pos(x, y)
        N = bond_env_h(sr.e(xr, yr), sr.e(xr + 1, yr), Tp, Tq)
    return N.transpose(0, 2, 1, 3)


def psd_project(N4):
    """Symmetrise N as a matrix [(a,b),(a',b')] and clip its negative eigenvalues (reading)."""
    n = N4.shape[0] * N4.shape[1]
    Nm = N4.reshape(n, n)
    w, V = np.linalg.eigh(0.5 * (Nm + Nm.T))
    w = np.clip(w, 0.0, None)
    return ((V * w) @ V.T).reshape(N4.shape)


def pinv_solve(R, s, cutoff=None):
    """x = R^+ s for symmetric PSD R via its eigenvalues (relative cutoff ALS_PINV_CUTOFF)."""
    cutoff = ALS_PINV_CUTOFF if cutoff is None else cutoff
    w, V = np.linalg.eigh(0.5 * (R + R.T))
    inv = np.zeros_like(w)
    if w[-1] > 0:
        keep = w >= cutoff * w[-1]
        inv[keep] = 1.0 / w[keep]
    return V @ (inv * (V.T @ s))


def cost(N4, M):
    """f(M) = <g|g> + <M|M> - 2 <g|M> of Eq. (var) for the link matrix M = P Q."""
    n2 = np.einsum('abcc->ab', N4)
    T = np.einsum('ccee->', N4)
    return T - 2.0 * np.sum(M * n2) + np.einsum('ab,cd,abcd->', M, M, N4, optimize='greedy')


def als(N4, P, Q, tol=1e-12, max_iter=50):
    """Alternating least squares of Eq. (var1) for one link (row a9).

    Fix Q:  R_P[(a,i),(a',i')] = sum Q[i,b] Q[i',b'] N4[a,b,a',b'],
            S_P[(a,i)]         = sum Q[i,b] N4[a,b,c,c],   P = R_P^+ S_P.
    Fix P:  R_Q[(i,b),(i',b')] = sum P[a,i] P[a',i'] N4[a,b,a',b'],
            S_Q[(i,b)]         = sum P[a,i] N4[a,b,c,c],   Q = R_Q^+ S_Q.
    Returns P, Q, iterations, final cost.
    """
    kD, D = P.shape
    n2 = np.einsum('abcc->ab', N4)
    M_old = P @ Q
    it = 0
    for it in range(1, max_iter + 1):
        RP = np.einsum('ib,jc,abdc->aidj', Q, Q, N4, optimize='greedy').reshape(kD * D, kD * D)
        SP = np.einsum('ib,ab->ai', Q, n2).reshape(kD * D)
        P = pinv_solve(RP, SP).reshape(kD, D)
        RQ = np.einsum('ai,dj,abdc->ibjc', P, P, N4, optimize='greedy').reshape(D * kD, D * kD)
        SQ = np.einsum('ai,ab->ib', P, n2).reshape(D * kD)
        Q = pinv_solve(RQ, SQ).reshape(D, kD)
        M = P @ Q
        dM = np.linalg.norm(M - M_old)
        M_old = M
        if dM <= tol * np.linalg.norm(M):
            break
    return P, Q, it, cost(N4, P @ Q)


def balance(P, Q):
    """P Q = U S V^T (sign rule) -> P = U sqrt(S), Q = sqrt(S) V^T, rank D."""
    D = P.shape[1]
    U, S, Vt = np.linalg.svd(P @ Q)
    U, V = sign_fix(U[:, :D], Vt[:D].T)
    r = np.sqrt(S[:D])
    return U * r, (V * r).T


def assemble(Theta, cell, fu):
    """A~_t = Theta_t with P on its out legs and Q on its in legs (row a10), max-abs normalised."""
    out = []
    for t, T in enumerate(Theta):
        A = truncate_legs(T, cell, t, fu)
        out.append(A / np.abs(A).max())
    return out


def full_update(Theta, cell, st, pre, als_tol=1e-12, als_max=50):
    """Rows a8-a10 for every link type: bond env, ALS, balance.  Returns (fu, info)."""
    fu, info = {}, {}
    for e in link_list(cell):
        N4 = bond_env(st, cell, e, Theta, pre)
        P0, Q0 = pre[e]
        norm = np.einsum('ccee->', N4)                # <g|g>: fixes the environment's sign and scale
        if not abs(norm) > 0.0:
            fu[e], info[e] = (P0.copy(), Q0.copy()), (0, np.nan)   # empty environment
            continue
        N4 = psd_project(N4 / norm)
        P, Q, it, f = als(N4, P0.copy(), Q0.copy(), als_tol, als_max)
        fu[e] = balance(P, Q)
        info[e] = (it, f)
    return fu, info


def pretruncated_sites(Theta, cell, pre):
    return [truncate_legs(T, cell, t, pre) for t, T in enumerate(Theta)]


def state_for(cell, a_list, env):
    return State(cell, a_list, env)
