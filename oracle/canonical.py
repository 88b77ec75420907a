"""iPEPS canonical form and gauge fixing (oracle), Sec. IV.

Canonical form, Sec. IV.A.  An iPEPS {Gamma, lambda} is canonical when, for
every link, the Gram matrix of the tensor on either side of the link, taken on
its link leg with lambda on all of its other legs, is the identity
(Eqs. 17-20: left, right, down and up constraints).  The iterative procedure
of Fig. 11, steps (i)-(iii):
  (i)   V_out = Gram of Gamma_t on its out leg (lambda on the other legs),
        V_in  = Gram of Gamma_t' on its in leg; eigendecompose
        V_out = W D W^T -> Y = D^{1/2} W^T (V_out = Y^T Y),
        V_in  = W'D'W'^T -> X = W' D'^{1/2} (V_in = X X^T);
  (ii)  insert Y^{-1} Y and X X^{-1} around lambda; the SVD
        Y lambda X = U lambda~ V^T gives the new weights;
  (iii) Gamma_t's out leg takes Y^{-1} U, Gamma_t''s in leg takes V^T X^{-1};
repeat until the weights stop changing.  The unit cell may hold several
tensors; every link type carries its own lambda (for the 1-site cell these are
lambda_h and lambda_v of the paper).

Readings:
* the printed "Y_v^T lambda_h X_v" is read as Y_v^T lambda_v X_v;
* lambda is normalised to unit 2-norm and every Gamma to unit Frobenius norm
  after each step (without it the overall scale of Gamma oscillates and
  diverges, s -> s^-3 per step); the pseudo-inverse of D^{1/2} drops
  eigenvalues below 1e-14 of the largest;
* the weighted form is A = sqrt(lambda) on every leg of Gamma (Sec. IV.B),
  normalised to ||A|| = 1; the leg matrices that map the input tensor to this
  weighted form are accumulated (the Q_c, P_c of Sec. VI.C step (i)).

Gauge fixing, Sec. IV.B.  Two canonical iPEPS A and B of the same state differ
by unitary (here orthogonal) matrices on the links.  The local fidelity
Eq. (25) is maximised by alternating polar steps: with all other link matrices
fixed, F is linear in the matrix W_e of link e, F = sum_ij W_e[i,j] M_e[i,j];
M_e = U S V^T gives W_e = U V^T (steps (i)-(v)).  Every leg of A is transformed
as leg'[j] = sum_i leg[i] W_e[i, j], which leaves the state unchanged.
Reading: when one tensor carries both ends of a link (1-site cell), the two
ends are treated as independent within a half-step, as the paper describes.
"""
import numpy as np

from .fullupdate import leg_links, link_list, leg_mul, LEG
from .ctmrg import sign_fix

CANON_INV_CUTOFF = 1e-14


def _weighted(T, links, lam, skip):
    X = T
    for name, (e, _side) in links.items():
        if name == skip:
            continue
        shape = [1] * 5
        shape[LEG[name]] = len(lam[e])
        X = X * lam[e].reshape(shape)
    return X


def _gram(X, leg):
    ax = LEG[leg]
    Xm = np.moveaxis(X, ax, -1).reshape(-1, X.shape[ax])
    return Xm.T @ Xm


def _sqrt_factors(V):
    """V = W D W^T -> (Y, Y^{-1}) with Y = D^{1/2} W^T, and (X, X^{-1}) with X = W D^{1/2}."""
    w, W = np.linalg.eigh(0.5 * (V + V.T))
    w = np.clip(w, 0.0, None)
    r = np.sqrt(w)
    inv = np.zeros_like(r)
    keep = w >= CANON_INV_CUTOFF * w.max() if w.max() > 0 else np.zeros_like(w, dtype=bool)
    inv[keep] = 1.0 / r[keep]
    return W, r, inv


def canonical_links(cell):
    """For each link type e: (t, out leg, t', in leg)."""
    out = {}
    for t in range(int(cell.pattern.max()) + 1):
        for name, (e, side) in leg_links(cell, t).items():
            out.setdefault(e, {})[side] = (t, name)
    return {e: (v['out'][0], v['out'][1], v['in'][0], v['in'][1]) for e, v in out.items()}


def canonical_step(Gamma, lam, cell):
    """One pass of steps (i)-(iii) on every link at once.  Returns new Gamma, lambda, leg maps."""
    links = canonical_links(cell)
    legs_of = [leg_links(cell, t) for t in range(len(Gamma))]
    maps, lam_new = {}, {}
    for e, (t, lo, tq, li) in links.items():
        Vout = _gram(_weighted(Gamma[t], legs_of[t], lam, lo), lo)
        Vin = _gram(_weighted(Gamma[tq], legs_of[tq], lam, li), li)
        W, r, ri = _sqrt_factors(Vout)
        Y, Yinv = (W * r).T, W * ri                 # Y = D^{1/2} W^T, Y^{-1} = W D^{-1/2}
        W2, r2, ri2 = _sqrt_factors(Vin)
        X, Xinv = W2 * r2, (W2 * ri2).T             # X = W' D'^{1/2}, X^{-1} = D'^{-1/2} W'^T
        U, S, Vt = np.linalg.svd(Y @ np.diag(lam[e]) @ X)
        U, V = sign_fix(U, Vt.T)
        nrm = np.linalg.norm(S)
        lam_new[e] = S / nrm if nrm > 0 else S
        maps[(t, lo)] = Yinv @ U                    # out leg: leg . Y^{-1} U
        maps[(tq, li)] = (V.T @ Xinv).T             # in leg: V^T X^{-1} . leg
    G2 = []
    for t, G in enumerate(Gamma):
        for name in ('l', 'r', 'd', 'u'):
            G = leg_mul(G, LEG[name], maps[(t, name)])
        G2.append(G / np.linalg.norm(G))
    return G2, lam_new, maps


def canonicalize(A, cell, tol=1e-12, max_iter=1000, lam0=None):
    """Bring the tensors A (dict-free list by tensor id) to canonical form (row a11).

    Starts from Gamma = A and lambda = 1 (or lam0).  Returns a dict with
      Gamma, lam          the canonical form,
      A                   the weighted tensors sqrt(lambda) Gamma sqrt(lambda), ||A_t|| = 1,
      maps[(t, leg)]      D x D matrices with A_t = c_t * (input A_t x_legs maps),
      iters, delta, converged.
    """
    D = A[0].shape[1]
    lam = {e: np.ones(D) / np.sqrt(D) for e in link_list(cell)} if lam0 is None else dict(lam0)
    Gamma = [a.copy() for a in A]
    acc = {(t, n): np.eye(D) for t in range(len(A)) for n in ('l', 'r', 'd', 'u')}
    delta, it, conv = np.inf, 0, False
    for it in range(1, max_iter + 1):
        Gamma, lam_new, maps = canonical_step(Gamma, lam, cell)
        for k in acc:
            acc[k] = acc[k] @ maps[k]
            acc[k] /= np.abs(acc[k]).max()          # only the direction of each map matters
        delta = max(float(np.abs(lam_new[e] - lam[e]).max()) for e in lam)
        lam = lam_new
        if delta < tol:
            conv = True
            break
    Aw, final_maps = [], {}
    for t, G in enumerate(Gamma):
        legs = leg_links(cell, t)
        W = G
        for name, (e, _side) in legs.items():
            W = leg_mul(W, LEG[name], np.diag(np.sqrt(lam[e])))
        c = np.linalg.norm(W)
        Aw.append(W / c)
        for name, (e, _side) in legs.items():
            final_maps[(t, name)] = acc[(t, name)] @ np.diag(np.sqrt(lam[e]))
    return dict(Gamma=Gamma, lam=lam, A=Aw, maps=final_maps, iters=it, delta=delta, converged=conv)


def canonical_residual(Gamma, lam, cell):
    """max over links and sides of || V / (tr V / D) - I ||_max  (Eqs. 17-20 up to a scalar)."""
    links = canonical_links(cell)
    res = 0.0
    for e, (t, lo, tq, li) in links.items():
        for tt, leg in ((t, lo), (tq, li)):
            V = _gram(_weighted(Gamma[tt], leg_links(cell, tt), lam, leg), leg)
            n = V.shape[0]
            res = max(res, float(np.abs(V * n / np.trace(V) - np.eye(n)).max()))
    return res


def transform(A, cell, W):
    """Apply the link matrices W[e] to every leg of every tensor: leg'[j] = sum_i leg[i] W[i, j]."""
    out = []
    for t, T in enumerate(A):
        for name, (e, _side) in leg_links(cell, t).items():
            T = leg_mul(T, LEG[name], W[e])
        out.append(T)
    return out


def fidelity(A, B, cell, W):
    """F = (1/n) sum_t <B_t, A_t x W> (Eq. 25 summed over the tensors of the cell)."""
    At = transform(A, cell, W)
    return float(sum(np.sum(a * b) for a, b in zip(At, B)) / len(A))


def polar(M):
    """Orthogonal polar factor U V^T of M = U S V^T."""
    U, S, Vt = np.linalg.svd(M)
    return U @ Vt


def gauge_fix(A, B, cell, tol=1e-12, max_iter=500, W0=None):
    """Orthogonal link matrices W with B ~ A x W maximising the local fidelity (row a12).

    A and B are weighted canonical tensors with ||A_t|| = ||B_t|| = 1.  The
    iteration starts from W0 (default: identities; the paper allows any start)
    and visits the links in link_list order; it stops when no W_e changes by
    more than tol in one pass (F is quadratic in the error of W near its
    maximum, so F itself is a poor stopping rule).  Returns W, F, passes.
    """
    D = A[0].shape[1]
    links = link_list(cell)
    W = {e: np.eye(D) for e in links} if W0 is None else {e: W0[e].copy() for e in links}
    it = 0
    for it in range(1, max_iter + 1):
        change = 0.0
        for e in links:
            M = np.zeros((D, D))
            for t, T in enumerate(A):
                for name, (ee, _side) in leg_links(cell, t).items():
                    if ee != e:
                        continue
                    X = T
                    for other, (e2, _s2) in leg_links(cell, t).items():
                        if other != name:
                            X = leg_mul(X, LEG[other], W[e2])
                    ax = LEG[name]
                    Xm = np.moveaxis(X, ax, -1).reshape(-1, D)
                    Bm = np.moveaxis(B[t], ax, -1).reshape(-1, D)
                    M += Xm.T @ Bm
            U, S, Vt = np.linalg.svd(M)
            Wn = U @ Vt
            change = max(change, float(np.abs(Wn - W[e]).max()))
            W[e] = Wn
        if change < tol:
            break
    return W, fidelity(A, B, cell, W), it
