"""1D iMPS: canonical form, gauge fixing and environment recycling (oracle), Sec. III and V.

One-site iMPS {Gamma, lambda}; matrices Gamma^s[l, r].  Used as a pin: the 1D
transverse Ising chain has a closed-form ground-state energy.

Canonical form, Sec. III.A steps (i)-(iii):
  V_L = sum_s (lambda Gamma^s)^T (lambda Gamma^s) = Y^T Y,
  V_R = sum_s (Gamma^s lambda)(Gamma^s lambda)^T = X X^T,
  Y lambda X = U lambda~ V^T,  Gamma~^s = V^T X^{-1} Gamma^s Y^{-1} U,
repeated until lambda~ is fixed; Gamma is normalised after every step.

Gauge fixing, Sec. III.B.2: F = sum_s Tr(U A^s U^T B^{sT}) is maximised by
repeating  M = sum_s A^s U^T B^{sT} = W S V^T,  U = V W^T.

Recycling, Sec. V.B: A_0 canonical; Theta = g A_0; A~ = Q Theta P (truncated
canonical form of Theta); A~_1 = Q_c A~ P_c (canonical form of A~);
A~_1 ~ U A_0 U^T; G = U^T Q_c Q g P P_c U applied N_Re times.
"""
import numpy as np

from .model import impo, apply_mpo, X, Z

INV_CUTOFF = 1e-14


def _sqrt_inv(V):
    w, W = np.linalg.eigh(0.5 * (V + V.T))
    w = np.clip(w, 0.0, None)
    r = np.sqrt(w)
    inv = np.zeros_like(r)
    keep = w >= INV_CUTOFF * w.max() if w.max() > 0 else np.zeros_like(w, dtype=bool)
    inv[keep] = 1.0 / r[keep]
    return W, r, inv


def canonical_step(G, lam):
    """One pass of steps (i)-(iii); G[s, l, r].  Returns Gamma~, lambda~, left map, right map."""
    LG = np.einsum('l,slr->slr', lam, G)
    GL = np.einsum('slr,r->slr', G, lam)
    VL = np.einsum('slr,slq->rq', LG, LG)
    VR = np.einsum('slr,sqr->lq', GL, GL)
    W, r, ri = _sqrt_inv(VL)
    Y, Yinv = (W * r).T, W * ri
    W2, r2, ri2 = _sqrt_inv(VR)
    Xm, Xinv = W2 * r2, (W2 * ri2).T
    U, S, Vt = np.linalg.svd(Y @ np.diag(lam) @ Xm)
    left = Vt @ Xinv               # acts on the left leg: Gamma~ = left Gamma right
    right = Yinv @ U
    Gn = np.einsum('al,slr,rb->sab', left, G, right)
    Gn /= np.linalg.norm(Gn)
    return Gn, S / np.linalg.norm(S), left, right


def canonicalize(A, tol=1e-13, max_iter=2000, n_watch=None):
    """Canonical form of A[s, l, r] starting from Gamma = A, lambda = 1.

    Stops when the n_watch largest weights (all by default) change by less than
    tol * lambda_1.  Reading: in a truncation only the kept weights matter, and
    the discarded tiny weights converge far more slowly.
    Returns Gamma, lambda, left map ML and right map MR with
    Gamma ~ ML A MR, and the weighted A_w = sqrt(lambda) Gamma sqrt(lambda) (norm 1).
    """
    chi = A.shape[1]
    lam = np.ones(chi) / np.sqrt(chi)
    G = A.copy()
    ML, MR = np.eye(chi), np.eye(chi)
    for _ in range(max_iter):
        G, lam_n, left, right = canonical_step(G, lam)
        ML, MR = left @ ML, MR @ right
        ML, MR = ML / np.abs(ML).max(), MR / np.abs(MR).max()   # scale is irrelevant
        k = len(lam) if n_watch is None else n_watch
        d = np.abs(lam_n[:k] - lam[:k]).max() / lam_n[0]
        lam = lam_n
        if d < tol:
            break
    s = np.sqrt(lam)
    Aw = np.einsum('l,slr,r->slr', s, G, s)
    Aw /= np.linalg.norm(Aw)
    return G, lam, ML, MR, Aw


def truncate(Theta, chi):
    """Optimal iMPS truncation through the canonical form: A~ = Q Theta P (Eq. CanoPQ1)."""
    G, lam, ML, MR, _ = canonicalize(Theta, tol=1e-12, n_watch=chi)
    s = np.sqrt(lam[:chi])
    Q = s[:, None] * ML[:chi, :]
    P = MR[:, :chi] * s[None, :]
    At = np.einsum('al,slr,rb->sab', Q, Theta, P)
    return At / np.linalg.norm(At), P, Q


def gauge_fix(A, B, tol=1e-12, max_iter=2000, U0=None):
    """U (orthogonal) maximising F = sum_s Tr(U A^s U^T B^{sT}); returns U, F.

    Reading of the stopping rule: F is quadratic in the error of U near its
    maximum, so the iteration stops when U itself changes by less than tol.
    Start: U0 (default the identity).  The iteration U <- polar(M)^T only
    climbs to the nearest local maximum; which one depends on the sign and
    basis conventions of the two canonical forms, so a start that does not
    depend on them matters (see recycle_window).
    """
    chi = A.shape[1]
    U = np.eye(chi) if U0 is None else np.array(U0, dtype=float)
    for _ in range(max_iter):
        M = np.einsum('sab,cb,sdc->ad', A, U, B)     # M = sum_s A^s U^T B^{sT}
        W, S, Vt = np.linalg.svd(M)
        U_new = Vt.T @ W.T
        dU = np.abs(U_new - U).max()
        U = U_new
        if dU < tol:
            break
    F = np.einsum('ab,sbc,dc,sad->', U, A, U, B)
    return U, float(F)


def observables(A, h):
    """<ZZ>, <X> and e = -<ZZ> - h <X> of the iMPS A (brought to canonical form first).

    In canonical form the environments of lambda Gamma lambda Gamma lambda are
    identities, so the reduced density matrices are plain contractions.
    """
    G, lam, _, _, _ = canonicalize(A)
    th1 = np.einsum('a,sab,b->sab', lam, G, lam)
    T2 = np.einsum('a,sab,b,tbc,c->stac', lam, G, lam, G, lam)
    rho2 = np.einsum('stac,uvac->stuv', T2, T2).reshape(4, 4)
    rho1 = np.einsum('sab,tab->st', th1, th1)
    zz = np.trace(rho2 @ np.kron(Z, Z)) / np.trace(rho2)
    x = np.trace(rho1 @ X) / np.trace(rho1)
    return float(zz), float(x), float(-zz - h * x)


def itebd(A, h, delta, chi, n_steps):
    """Plain iTEBD with the iMPO (Sec. V.A): A <- truncate(g A)."""
    g = impo(h, delta)
    for _ in range(n_steps):
        A, _, _ = truncate(apply_mpo(g, A), chi)
    return A


def recycle_window(A, h, delta, chi, n_re):
    """One 1D recycling window (Sec. V.B steps (i)-(iii)); returns the new A and F."""
    g = impo(h, delta)
    _, _, _, _, A0 = canonicalize(A)
    Theta = apply_mpo(g, A0)
    At, P, Q = truncate(Theta, chi)
    _, lam1, MLc, MRc, A1 = canonicalize(At)
    s1 = np.sqrt(lam1)
    # start of the gauge fix (the paper does not give one): for small delta the kappa = 0
    # block of Theta = g A_0 is A_0 up to a factor, so A_1 = Q_c A~ P_c ~ L0 A_0 (...) with
    # the leg map L0 = Q_c Q[:, kappa = 0]; its polar factor is the gauge up to the
    # truncation.  From the identity the iteration can stop in a local maximum
    # (F = 0.44 against 0.989 at h = 2, chi = 6).
    W0, _, V0t = np.linalg.svd((s1[:, None] * MLc) @ Q[:, :chi])
    U, F = gauge_fix(A0, A1, U0=W0 @ V0t)
    KL = U.T @ (s1[:, None] * MLc) @ Q      # chi x kappa*chi: U^T Q_c Q
    KR = P @ (MRc * s1[None, :]) @ U        # kappa*chi x chi: P P_c U
    Ak = A0
    for _ in range(n_re):
        T = np.einsum('al,slr,rb->sab', KL, apply_mpo(g, Ak), KR)
        Ak = T / np.linalg.norm(T)
    return Ak, F
