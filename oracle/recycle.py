"""Imaginary-time evolution with full update and environment recycling (oracle), Sec. VI.B-C.

Simple-update step (su_step, the comparison method of Sec. VI.D): rows a11,
a1, a7 and the pre-truncated sites, without environment.

Plain step (every row a1-a10):
    A_c   = weighted canonical form of A, with weights lambda           (a11)
    Theta = g A_c                                                        (a1)
    pre   = simple-update projectors with the lambda environment         (a7)
    a     = double layers of the pre-truncated tensors                   (a2)
    env   = CTMRG of a, warm-started from the previous environment       (a3-a6)
    fu    = bond environment + ALS + balance on every link               (a8-a9)
    A~    = Theta with the fu pairs on every leg                         (a10)
Reading: the canonical form is taken before every full update so that the
simple-update pre-truncation has its weights; the full update itself does not
depend on the gauge.

Recycled window (Sec. VI.C steps (i)-(iii)):
    A_0 = A_c of the current A; one plain step gives Theta, fu and A~;
    (i)   canonical form of A~: A~_1 = A~ x_legs maps                  (a11)
    (ii)  gauge fix: A~_1 ~ A_0 x W, started from the kappa = 0 block of
          the leg maps (gauge_start)                                   (a12)
    (iii) renormalised gate: per leg K = P_fu maps W^T (out legs) and
          K = Q_fu^T maps W^T (in legs), kappa*D x D;
          A_k = (g A_{k-1}) x_legs K, k = 1..N_Re, each max-abs normalised (a13)
    A_0 <- A_{N_Re}.
Reading of the printed G of Sec. VI.C: the stray "Q_v" between P_hc and P_v is
dropped, G = U_h^+ U_v^+ Q_hc Q_h Q_vc Q_v g P_h P_hc P_v P_vc U_h U_v.
With N_Re = 1 the window reproduces the plain step up to a gauge.
"""
import numpy as np

from .model import ipepo, apply_pepo
from .ctmrg import double_layer, ctmrg, init_env
from .fullupdate import (pretruncation, pretruncated_sites, full_update, assemble, bond_env, psd_project, link_list,
                         leg_links, leg_mul, LEG)
from .canonical import canonicalize, gauge_fix, polar
from .observables import measure


class Config:
    def __init__(self, h, tau, D, chi, ctm_tol=1e-10, ctm_max=500, als_tol=1e-12, als_max=50,
                 canon_tol=1e-12, canon_max=1000, gauge_tol=1e-12, gauge_max=500):
        self.h, self.tau, self.D, self.chi = h, tau, D, chi
        self.ctm_tol, self.ctm_max = ctm_tol, ctm_max
        self.als_tol, self.als_max = als_tol, als_max
        self.canon_tol, self.canon_max = canon_tol, canon_max
        self.gauge_tol, self.gauge_max = gauge_tol, gauge_max


def fu_step(A, cell, cfg, env=None, g=None):
    """One plain imaginary-time step.  Returns (A~, env, info) with info holding the pieces."""
    g = ipepo(cfg.h, cfg.tau) if g is None else g
    can = canonicalize(A, cell, cfg.canon_tol, cfg.canon_max)
    Ac = can['A']
    Theta = [apply_pepo(g, a) for a in Ac]
    pre = pretruncation(Theta, cell, can['lam'], cfg.D)
    a_list = [double_layer(x) for x in pretruncated_sites(Theta, cell, pre)]
    st, it, delta, conv = ctmrg(cell, a_list, cfg.chi, cfg.ctm_tol, cfg.ctm_max, env=env)
    fu, als_info = full_update(Theta, cell, st, pre, cfg.als_tol, cfg.als_max)
    At = assemble(Theta, cell, fu)
    info = dict(A0=Ac, lam=can['lam'], Theta=Theta, pre=pre, fu=fu, ctm_iters=it,
                ctm_delta=delta, ctm_converged=conv, als=als_info, state=st)
    return At, st.env, info


def su_step(A, cell, cfg, g=None):
    """One simple-update step: the environment-free method of the comparison in Sec. VI.D.

    Canonical form (weights lambda), Theta = g A_c, and every leg truncated by
    the lambda-weighted simple-update projectors of the pre-truncation (a7);
    the result is max-abs normalised.
    """
    g = ipepo(cfg.h, cfg.tau) if g is None else g
    can = canonicalize(A, cell, cfg.canon_tol, cfg.canon_max)
    Theta = [apply_pepo(g, a) for a in can['A']]
    pre = pretruncation(Theta, cell, can['lam'], cfg.D)
    return [x / np.abs(x).max() for x in pretruncated_sites(Theta, cell, pre)]


def gate_legs(cell, fu, maps, W):
    """Renormalised-gate leg matrices K[(t, leg)] (kappa*D x D), step (iii)."""
    K = {}
    n = len({t for (t, _l) in maps})
    for t in range(n):
        for name, (e, side) in leg_links(cell, t).items():
            P, Q = fu[e]
            base = P if side == 'out' else Q.T
            K[(t, name)] = base @ maps[(t, name)] @ W[e].T
    return K


def recycled_step(A, cell, g, K):
    """A <- (g A) x_legs K, max-abs normalised (row a13)."""
    out = []
    for t, a in enumerate(A):
        T = apply_pepo(g, a)
        for name in ('l', 'r', 'd', 'u'):
            T = leg_mul(T, LEG[name], K[(t, name)])
        out.append(T / np.abs(T).max())
    return out


def gauge_start(cell, fu, maps, D):
    """Starting link matrices of the gauge fix (reading; the paper allows any start).

    For small tau the kappa = 0 block of Theta = g A_0 is A_0 itself up to a
    scalar, so the kappa = 0 rows of the leg maps P Q_c (out leg) and Q^T Q_c
    (in leg) of each link estimate the orthogonal W of A~_1 ~ A_0 x W; W starts
    at the polar factor of their sum.
    """
    W0 = {}
    for t in range(len({tt for (tt, _l) in maps})):
        for name, (e, side) in leg_links(cell, t).items():
            P, Q = fu[e]
            base = P[:D, :] if side == 'out' else Q[:, :D].T
            W0[e] = W0.get(e, 0.0) + base @ maps[(t, name)]
    return {e: polar(M) for e, M in W0.items()}


def recycle_window(A, cell, cfg, n_re, env=None, g=None):
    """One environment computation followed by n_re applications of the renormalised gate."""
    g = ipepo(cfg.h, cfg.tau) if g is None else g
    At, env, info = fu_step(A, cell, cfg, env, g)
    can1 = canonicalize(At, cell, cfg.canon_tol, cfg.canon_max)
    W0 = gauge_start(cell, info['fu'], can1['maps'], cfg.D)
    W, F, git = gauge_fix(info['A0'], can1['A'], cell, cfg.gauge_tol, cfg.gauge_max, W0=W0)
    K = gate_legs(cell, info['fu'], can1['maps'], W)
    Ak = info['A0']
    for _ in range(n_re):
        Ak = recycled_step(Ak, cell, g, K)
    info.update(F=F, gauge_iters=git, K=K, A1=can1['A'], W=W)
    return Ak, env, info


def evolve(A, cell, cfg, n_steps, n_re=1, recycle=False, env=None, log=None):
    """n_steps imaginary-time steps, plain (n_re ignored) or recycled in windows of n_re steps.

    Returns (A, env, number of environment computations).
    """
    done, n_env = 0, 0
    while done < n_steps:
        if recycle:
            k = min(n_re, n_steps - done)
            A, env, info = recycle_window(A, cell, cfg, k, env)
            done += k
        else:
            A, env, info = fu_step(A, cell, cfg, env)
            done += 1
        n_env += 1
        if log is not None:
            log.append(dict(step=done, ctm_iters=info['ctm_iters'], F=info.get('F')))
    return A, env, n_env


def bond_envs(A, cell, cfg, env, g=None, ctm_iters=1):
    """Bond environments of the current state: canonical form, Theta, pre-truncation and
    double layers as in a plain step, ctm_iters warm CTMRG iterations, then every N of
    row a8 normalised by <g|g> and projected on its positive part (as the ALS sees it).

    Returns (N dict by link, env after the iterations).
    """
    g = ipepo(cfg.h, cfg.tau) if g is None else g
    can = canonicalize(A, cell, cfg.canon_tol, cfg.canon_max)
    Theta = [apply_pepo(g, a) for a in can['A']]
    pre = pretruncation(Theta, cell, can['lam'], cfg.D)
    a_list = [double_layer(x) for x in pretruncated_sites(Theta, cell, pre)]
    st, _, _, _ = ctmrg(cell, a_list, cfg.chi, 0.0, ctm_iters, env=env)
    out = {}
    for e in link_list(cell):
        N4 = bond_env(st, cell, e, Theta, pre)
        norm = np.einsum('ccee->', N4)
        out[e] = psd_project(N4 / norm) if abs(norm) > 0.0 else N4
    return out, st.env


def env_change(N_new, N_old):
    """max over links of ||N_new - N_old||_F / ||N_old||_F."""
    return max(np.linalg.norm(N_new[e] - N_old[e]) / np.linalg.norm(N_old[e]) for e in N_old)


def evolve_threshold(A, cell, cfg, n_steps, eps=1e-8, check_every=1, max_window=50, env=None, log=None):
    """Recycling with the threshold trigger (the reading of "recycled until the bond-environment
    change exceeds eps"): a window starts with an environment computation (a plain step, whose
    normalised bond environments N_0 are kept) and continues with recycled steps from A_0 with
    the window's renormalised gate; after every check_every recycled steps one warm CTMRG
    iteration on the current state gives its bond environments N, and the window ends (the
    next step recomputes the environment) once env_change(N, N_0) > eps, or after max_window
    steps.  Returns (A, env, number of environment computations, number of checks).
    """
    g = ipepo(cfg.h, cfg.tau)
    done, n_env, n_chk = 0, 0, 0
    while done < n_steps:
        At, env, info = fu_step(A, cell, cfg, env, g)
        n_env += 1
        N0 = {}
        for e in link_list(cell):                     # the N the ALS of this step used
            N4 = bond_env(info['state'], cell, e, info['Theta'], info['pre'])
            norm = np.einsum('ccee->', N4)
            N0[e] = psd_project(N4 / norm) if abs(norm) > 0.0 else N4
        can1 = canonicalize(At, cell, cfg.canon_tol, cfg.canon_max)
        W0 = gauge_start(cell, info['fu'], can1['maps'], cfg.D)
        W, F, _ = gauge_fix(info['A0'], can1['A'], cell, cfg.gauge_tol, cfg.gauge_max, W0=W0)
        K = gate_legs(cell, info['fu'], can1['maps'], W)
        A = info['A0']
        k = 0
        while done < n_steps and k < max_window:
            A = recycled_step(A, cell, g, K)
            k += 1
            done += 1
            if k % check_every == 0 and done < n_steps:
                N, env = bond_envs(A, cell, cfg, env, g)
                n_chk += 1
                d = env_change(N, N0)
                if log is not None:
                    log.append(dict(step=done, change=d, F=F))
                if d > eps:
                    break
    return A, env, n_env, n_chk


def energy(A, cell, cfg, env=None, tol=1e-10, max_iter=500):
    """CTMRG on the double layers of A, then the observables of Sec. VI.D."""
    a_list = [double_layer(x) for x in A]
    st, it, delta, conv = ctmrg(cell, a_list, cfg.chi, tol, max_iter, env=env)
    m = measure(st, cell, A, cfg.h)
    m.update(ctm_iters=it, ctm_delta=delta, ctm_converged=conv, env=st.env)
    return m

