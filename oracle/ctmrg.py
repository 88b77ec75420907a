"""Double layer and CTM environment of an iPEPS (oracle).

Sec. VI.B item 1: the network L(a) of double-layer tensors
    a_{(l1 l2),(r1 r2),(d1 d2),(u1 u2)} = sum_s Theta^s_{l1 r1 d1 u1} (Theta^s_{l2 r2 d2 u2})^*
is surrounded by corners C1..C4 and edges T1..T4 computed with the corner
transfer matrix method (Fig. 21a). The paper only cites the CTMRG moves, so
this module follows one reading of them (directional moves with half-system
projectors) and states each choice where it is made.

Conventions (all tensors real, row-major numpy arrays):

* Site tensor A[s, l, r, d, u]; x grows to the right, y grows downward;
  A's r leg joins the l leg of (x+1, y), its d leg joins the u leg of (x, y+1).
* Double layer a[L, R, Dn, U], each leg the fused pair (ket, bra) -> ket*D+bra.
* Unit cell: pattern[y][x] = tensor id, periodic in x and y.
* Environment of site (x, y): corners C1 (top-left), C2 (top-right),
  C3 (bottom-right), C4 (bottom-left) and edges T1 (top), T2 (right),
  T3 (bottom), T4 (left).  Going clockwise round the boundary every tensor has
  an incoming and an outgoing chi leg: C[in, out] and T[in, out, m], m being the
  fused inward leg that joins the double layer.  C1.out = T1.in, T1.out = C2.in,
  C2.out = T2.in, ... , T4.out = C1.in.
* All environment tensors keep the fixed shape (chi, chi) / (chi, chi, D^2);
  unused directions are exact zeros.

Reading of the moves: a CTMRG iteration is a left, up, right and down move; a
move absorbs the columns of the unit cell one after the other (x = 0..Lx-1).
The up/right/down moves are the left move applied to the lattice rotated by 90
degrees counter-clockwise, once, twice and three times.
"""
import numpy as np

SVD_CUTOFF = 1e-12   # projector singular values below SVD_CUTOFF * s_1 are dropped


# ----------------------------------------------------------------------------
# double layer, cells and rotations
# ----------------------------------------------------------------------------

def double_layer(A):
    """a[(l l'),(r r'),(d d'),(u u')] = sum_s A[s,l,r,d,u] A[s,l',r',d',u'] (Sec. VI.B)."""
    D = A.shape[1]
    a = np.einsum('slrdu,smnop->lmrndoup', A, A)
    return a.reshape(D * D, D * D, D * D, D * D)


def rotate_site(A):
    """Counter-clockwise lattice rotation of a site tensor A[s,l,r,d,u].

    The up leg points left afterwards, the down leg right, the left leg down and
    the right leg up: A'[s, l', r', d', u'] = A[s, d', u', r', l'].
    """
    return A.transpose(0, 4, 3, 1, 2)


def rotate_double(a):
    """The same rotation for a double layer a[L, R, Dn, U]: a'[L',R',D',U'] = a[D',U',R',L']."""
    return a.transpose(3, 2, 0, 1)


class Cell:
    """Periodic unit cell: pattern[y][x] holds the tensor id at site (x, y)."""

    def __init__(self, pattern):
        self.pattern = np.array(pattern, dtype=int)
        self.Ly, self.Lx = self.pattern.shape

    def tid(self, x, y):
        return int(self.pattern[y % self.Ly, x % self.Lx])

    def sites(self):
        return [(x, y) for y in range(self.Ly) for x in range(self.Lx)]

    def rotated(self):
        """Cell after a counter-clockwise rotation: site (x, y) moves to (y, -x)."""
        Lx2, Ly2 = self.Ly, self.Lx
        p = np.empty((Ly2, Lx2), dtype=int)
        for y2 in range(Ly2):
            for x2 in range(Lx2):
                p[y2, x2] = self.tid(-y2, x2)
        return Cell(p)

    def rotate_pos(self, x, y):
        return (y % self.Ly, (-x) % self.Lx)


def checkerboard():
    """The 2-site (A, B) checkerboard cell [[A, B], [B, A]]."""
    return Cell([[0, 1], [1, 0]])


def single_site():
    return Cell([[0]])


ROT_ENV = {'C1': 'C2', 'T1': 'T2', 'C2': 'C3', 'T2': 'T3',
           'C3': 'C4', 'T3': 'T4', 'C4': 'C1', 'T4': 'T1'}
"""After a counter-clockwise rotation the new C1 is the old C2, etc."""


class State:
    """CTMRG state: a cell, one double layer per tensor id and the environment."""

    def __init__(self, cell, a_list, env):
        self.cell, self.a, self.env = cell, list(a_list), env

    def a_at(self, x, y):
        return self.a[self.cell.tid(x, y)]

    def e(self, x, y):
        return self.env[(x % self.cell.Lx, y % self.cell.Ly)]

    def rotated(self):
        """The whole network rotated counter-clockwise; the env tensors are only relabelled."""
        cell2 = self.cell.rotated()
        env2 = {}
        for (x, y), e in self.env.items():
            env2[self.cell.rotate_pos(x, y)] = {k: e[v] for k, v in ROT_ENV.items()}
        return State(cell2, [rotate_double(a) for a in self.a], env2)


def init_env(cell, chi, D2, boundary=None):
    """Trivial boundary: bond dimension 1 padded to chi.

    Reading (the paper is silent on the initial environment): C = 1 and
    T[0, 0, m] = delta_{ket, bra}, i.e. the outward ket and bra legs of the
    boundary are joined by the identity.  The bond dimension then grows by D^2
    per absorption until it reaches chi; the zero padding keeps every tensor at
    its final shape.  A network that is not a double layer passes its own
    boundary vector (length D2).
    """
    if boundary is None:
        D = int(round(np.sqrt(D2)))
        delta = np.eye(D).reshape(D2)
    else:
        delta = np.asarray(boundary, dtype=float)
    env = {}
    for (x, y) in cell.sites():
        e = {}
        for c in ('C1', 'C2', 'C3', 'C4'):
            C = np.zeros((chi, chi))
            C[0, 0] = 1.0
            e[c] = C
        for t in ('T1', 'T2', 'T3', 'T4'):
            T = np.zeros((chi, chi, D2))
            T[0, 0, :] = delta
            e[t] = T
        env[(x, y)] = e
    return env


def copy_env(env):
    return {k: {n: t.copy() for n, t in v.items()} for k, v in env.items()}


# ----------------------------------------------------------------------------
# one left move
# ----------------------------------------------------------------------------

def _corner(C, Tb, Ta, a, legs):
    """Enlarged corner (C . Ta) . Tb . a as [(Tb.in, a.row), (Ta.out, a.col)].

    C[in, out]; Tb is the edge before C going clockwise (Tb.out = C.in), Ta the
    edge after it (Ta.in = C.out).  legs = positions in a[L, R, Dn, U] of
    (leg joined to Tb.m, leg joined to Ta.m, open leg next to Tb.in, open leg
    next to Ta.out).
    """
    chi, D2 = C.shape[0], a.shape[0]
    X = (C @ Ta.reshape(chi, chi * D2)).reshape(chi, chi, D2)        # [C.in, Ta.out, Ta.m]
    Y = np.tensordot(Tb, X, axes=([1], [0]))                          # [Tb.in, Tb.m, Ta.out, Ta.m]
    ab = a.transpose(legs).reshape(D2 * D2, D2 * D2)                  # [(Tb-leg, Ta-leg), (row, col)]
    Z = Y.transpose(0, 2, 1, 3).reshape(chi * chi, D2 * D2) @ ab      # [(Tb.in, Ta.out), (row, col)]
    Z = Z.reshape(chi, chi, D2, D2).transpose(0, 2, 1, 3)
    return Z.reshape(chi * D2, chi * D2)


def enlarged_corners(st, x, y):
    """The four enlarged corners around the cut between rows y and y+1, columns x, x+1.

    Each is returned as a (chi*D^2) x (chi*D^2) matrix.  Going clockwise round
    the 2x2 block they chain  Q_UL [b4 -> b1] Q_UR [b1 -> b2] Q_LR [b2 -> b3]
    Q_LL [b3 -> b4], where b4 is the cut to be truncated (between the upper-left
    and lower-left corners) and b2 the cut opposite to it.  Every row/column
    index is the pair (chi leg, double-layer leg), chi-major.
    """
    ul, ur, lr, ll = st.e(x, y), st.e(x + 1, y), st.e(x + 1, y + 1), st.e(x, y + 1)
    # Q_UL[(T4.in, a.d), (T1.out, a.r)] = C1[a,b] T1[b,c,m] T4[d,a,n] a[n,r,s,m]
    Qul = _corner(ul['C1'], ul['T4'], ul['T1'], st.a_at(x, y), (0, 3, 2, 1))
    # Q_UR[(T1.in, a.l), (T2.out, a.d)] = C2[a,b] T1[c,a,m] T2[b,d,n] a[l,n,s,m]
    Qur = _corner(ur['C2'], ur['T1'], ur['T2'], st.a_at(x + 1, y), (3, 1, 0, 2))
    # Q_LR[(T2.in, a.u), (T3.out, a.l)] = C3[a,b] T2[c,a,m] T3[b,d,n] a[l,m,n,u]
    Qlr = _corner(lr['C3'], lr['T2'], lr['T3'], st.a_at(x + 1, y + 1), (1, 2, 3, 0))
    # Q_LL[(T3.in, a.r), (T4.out, a.u)] = C4[a,b] T3[c,a,m] T4[b,d,n] a[n,r,m,u]
    Qll = _corner(ll['C4'], ll['T3'], ll['T4'], st.a_at(x, y + 1), (2, 0, 1, 3))
    return Qul, Qur, Qlr, Qll


def sign_fix(U, V):
    """Sign rule for singular pairs: the entry of largest |.| of each column of U is positive.

    Ties within a relative 1e-10 of the maximum go to the lowest row index.
    U and V columns are flipped together, so U S V^T is unchanged.
    """
    U, V = U.copy(), V.copy()
    for j in range(U.shape[1]):
        col = np.abs(U[:, j])
        m = col.max()
        if m == 0.0:
            continue
        i = int(np.nonzero(col >= m * (1.0 - 1e-10))[0][0])
        if U[i, j] < 0:
            U[:, j] *= -1.0
            V[:, j] *= -1.0
    return U, V


def truncated_svd(M, k):
    """Top-k singular triplets of M by LAPACK SVD, sign rule applied."""
    U, S, Vt = np.linalg.svd(M)
    U, V = sign_fix(U[:, :k], Vt[:k].T)
    return U, S[:k], V


def projectors(Qul, Qur, Qlr, Qll, chi):
    """Projector pair for the cut b4 from the half systems (reading of the cited CTMRG).

    R_u = Q_UL Q_UR [b4 -> b2] and R_d = Q_LR Q_LL [b2 -> b4].  The loop cut at
    b2 is rho = R_d R_u = U S V^T; keeping the top chi triplets,
        P_up = R_d^T U S^{-1/2}   (joins the bottom leg of the upper part),
        P_lo = R_u   V S^{-1/2}   (joins the top leg of the lower part),
    so that R_d (P_lo P_up^T) R_u equals the rank-chi truncation of rho.
    S^{-1/2} is set to 0 for s < SVD_CUTOFF * s_1 (those directions are dropped
    while every tensor keeps its shape).  Returns P_up, P_lo, s (all chi).
    """
    Ru = Qul @ Qur
    Rd = Qlr @ Qll
    rho = Rd @ Ru
    U, S, V = truncated_svd(rho, chi)
    inv = np.zeros_like(S)
    keep = S >= SVD_CUTOFF * S[0] if S[0] > 0 else np.zeros_like(S, dtype=bool)
    inv[keep] = 1.0 / np.sqrt(S[keep])
    P_up = Rd.T @ (U * inv)
    P_lo = Ru @ (V * inv)
    return P_up, P_lo, S


def normalize(T):
    """Divide by the largest |entry| (reading: CTM tensors are normalised by max abs)."""
    m = np.abs(T).max()
    return T / m if m > 0 else T


def column_projectors(st, x, chi):
    """Projector pairs of every cut (y | y+1) of column x (row a4).

    Returns Pu, Pl (dicts y -> array [chi, D^2, chi]) and the spectra s[y].
    """
    Pu, Pl, spectra = {}, {}, {}
    for y in range(st.cell.Ly):
        P_up, P_lo, s = projectors(*enlarged_corners(st, x, y), chi)
        D2 = st.a_at(x, y).shape[0]
        Pu[y] = P_up.reshape(chi, D2, chi)
        Pl[y] = P_lo.reshape(chi, D2, chi)
        spectra[y] = s
    return Pu, Pl, spectra


def renormalize(e, a, pu_above, pl_above, pu, pl):
    """New C1, T4, C4 of the next column from site environment e and double layer a (row a5).

        C1'[a, o]    = P_up(y-1|y)[(i,m),a] C1[i,c] T1[c,o,m]
        T4'[a, b, r] = P_up(y|y+1)[(i,s),a] P_lo(y-1|y)[(j,t),b] T4[i,j,m] a[m,r,s,t]
        C4'[i3, a]   = C4[c,q] T3[i3,c,m] P_lo(y|y+1)[(q,m),a]
    each divided by its largest |entry|.
    """
    chi, D2 = e['C1'].shape[0], a.shape[0]
    CT = (e['C1'] @ e['T1'].reshape(chi, -1)).reshape(chi, chi, D2)          # [i, o, m]
    C1n = pu_above.reshape(chi * D2, chi).T @ CT.transpose(0, 2, 1).reshape(chi * D2, chi)
    Ta = np.tensordot(e['T4'], a, axes=([2], [0]))                            # [i, j, r, s, t]
    Ta = Ta.transpose(0, 3, 1, 4, 2).reshape(chi * D2, chi * D2 * D2)
    Ta = (pu.reshape(chi * D2, chi).T @ Ta).reshape(chi, chi * D2, D2)      # [a, (j,t), r]
    T4n = np.tensordot(Ta, pl_above.reshape(chi * D2, chi), axes=([1], [0])).transpose(0, 2, 1)
    TC = np.tensordot(e['T3'], e['C4'], axes=([1], [0]))                      # [i3, m, q]
    C4n = TC.transpose(0, 2, 1).reshape(chi, chi * D2) @ pl.reshape(chi * D2, chi)
    return normalize(C1n), normalize(T4n), normalize(C4n)


def left_move(st, chi):
    """Absorb every column of the cell into the left environment, x = 0..Lx-1.

    For column x the projectors of all cuts (y | y+1) are computed first, then
    the new C1, T4, C4 of column x+1 (renormalize).  Returns the projector
    spectra.
    """
    cell = st.cell
    spectra = []
    for x in range(cell.Lx):
        Pu, Pl, sp = column_projectors(st, x, chi)
        spectra.extend(sp[y] for y in range(cell.Ly))
        new = {}
        for y in range(cell.Ly):
            ya = (y - 1) % cell.Ly
            new[y] = renormalize(st.e(x, y), st.a_at(x, y), Pu[ya], Pl[ya], Pu[y], Pl[y])
        for y in range(cell.Ly):
            tgt = st.e(x + 1, y)
            tgt['C1'], tgt['T4'], tgt['C4'] = new[y]
    return spectra


def ctm_iteration(st, chi):
    """One CTMRG iteration: left, up, right and down moves (four left moves on rotated lattices)."""
    for _ in range(4):
        left_move(st, chi)
        st = st.rotated()
    return st


# ----------------------------------------------------------------------------
# convergence
# ----------------------------------------------------------------------------

def corner_spectra(st):
    """Normalised corner singular values: s / sum(s) for every site and corner, sorted descending."""
    out = {}
    for (x, y), e in st.env.items():
        for c in ('C1', 'C2', 'C3', 'C4'):
            s = np.linalg.svd(e[c], compute_uv=False)
            tot = s.sum()
            out[(x, y, c)] = s / tot if tot > 0 else s
    return out


def spectrum_delta(s_new, s_old):
    """max over corners of || s_new - s_old ||_2 (reading of the singular-value change)."""
    return max(float(np.linalg.norm(s_new[k] - s_old[k])) for k in s_new)


def site_scalars(e, a):
    """Contractions of one site's environment (any leg dimension).

    Z1 = C1 T1 C2 T2 C3 T3 C4 T4 with a in the middle; Z0 = C1 C2 C3 C4;
    Zh = C1 T1 C2 C3 T3 C4 (T1.m joined to T3.m); Zv = C1 C2 T2 C3 C4 T4.
    For a translation-invariant network Z1 Z0 / (Zh Zv) is the partition
    function per site.
    """
    C1, C2, C3, C4 = e['C1'], e['C2'], e['C3'], e['C4']
    T1, T2, T3, T4 = e['T1'], e['T2'], e['T3'], e['T4']
    top = np.einsum('ia,abm,bc->icm', C1, T1, C2)       # [C1.in, C2.out, T1.m]
    bot = np.einsum('de,efx,fj->djx', C3, T3, C4)       # [C3.in, C4.out, T3.m]
    Z1 = np.einsum('icu,cdr,djx,jil,lrxu->', top, T2, bot, T4, a, optimize='greedy')
    Z0 = np.einsum('ia,ab,bc,ci->', C1, C2, C3, C4)
    Zh = np.einsum('icm,cim->', top, bot)
    Zv = np.einsum('ia,ab,bcm,cd,de,eim->', C1, C2, T2, C3, C4, T4, optimize='greedy')
    return Z1, Z0, Zh, Zv


def ctmrg(cell, a_list, chi, tol=1e-10, max_iter=500, env=None, min_iter=1, boundary=None):
    """Run CTMRG iterations until the corner spectra change by less than tol.

    Returns (state, iterations, last delta, converged).  A warm start passes the
    previous environment in env (it is copied, not modified).
    """
    D2 = a_list[0].shape[0]
    env = init_env(cell, chi, D2, boundary) if env is None else copy_env(env)
    st = State(cell, a_list, env)
    prev = corner_spectra(st)
    delta, it = np.inf, 0
    for it in range(1, max_iter + 1):
        st = ctm_iteration(st, chi)
        cur = corner_spectra(st)
        delta = spectrum_delta(cur, prev)
        prev = cur
        if it >= min_iter and delta < tol:
            return st, it, delta, True
    return st, it, delta, False
