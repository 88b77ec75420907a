"""Field sweep of the 2D transverse-field Ising model: m_z(h) and E(h) with the
full update (environment-based, optionally recycled) or the simple update.

This is the comparison of Sec. VI.D (magnetisation against the field for the
two methods).  Each field value is an independent evolution from the same
seeded tensors, so a sweep spreads over GPUs as replicas: rank r of `world`
takes the fields h[r::world], with no communication (the caller gathers).
Everything runs through the library's C ABI; this module only orchestrates.
"""
from . import _lib as L
from .inputs import random_peps


def run_field(h, D, chi, tau, steps, method="fu", n_re=1, ctm_tol=1e-8, ctm_max=200, measure_tol=1e-9,
              measure_max=300, precision=L.TN_F64, instance=0, device="cuda:0", state=None, recycle_eps=None,
              check_every=1, warmup_plain=0):
    """Evolve one field value and measure it; returns a dict of observables.

    method: "fu" (full update: plain; recycled in windows of n_re steps when
    n_re > 1; or, with recycle_eps, windows of at most n_re steps ended when the
    bond environment drifts by more than recycle_eps) or "su" (simple update).
    tau, steps: one time step and count, or lists for a schedule of stages
    (e.g. tau = [0.01, 0.001], steps = [1000, 1000]).  The measurement converges
    a fresh CTMRG.  The returned tau and steps are the caller's own values
    (scalars stay scalars).
    """
    taus = list(tau) if isinstance(tau, (list, tuple)) else [tau]
    counts = list(steps) if isinstance(steps, (list, tuple)) else [steps]
    if len(taus) != len(counts):
        raise ValueError("tau and steps stages differ in length")
    ctx = L.Context(D, chi, device=device, precision=precision)
    try:
        ctx.tn_set_hamiltonian(1.0, h)
        ctx.tn_set_state(state if state is not None else random_peps(2, D, instance=instance))
        n_env = 0
        for stage, (tau_s, n_s) in enumerate(zip(taus, counts)):
            ctx.tn_set_time_step(tau_s)
            if method == "su":
                for _ in range(n_s):
                    ctx.tn_su_step()
            elif method == "fu":
                if recycle_eps is not None:
                    mode = "threshold"
                else:
                    mode = n_re > 1
                rep = ctx.tn_evolve(n_s, recycle=mode, n_re=max(n_re, 1), ctm_tol=ctm_tol, ctm_max=ctm_max,
                                    recycle_eps=recycle_eps, check_every=check_every,
                                    warmup_plain=warmup_plain if stage == 0 else 0)
                n_env += rep["env_computations"]
            else:
                raise ValueError("method must be 'fu' or 'su'")
        ctx.tn_build_double_layer()
        ctx.tn_reset_env()
        crep = ctx.tn_ctmrg(measure_tol, measure_max)
        m = ctx.tn_measure()
        return dict(h=h, method=method, D=D, chi=chi, tau=tau, steps=steps, n_re=n_re, e_site=m["e_site"],
                    mx=sum(m["mx"]) / len(m["mx"]), mz=sum(abs(z) for z in m["mz"]) / len(m["mz"]),
                    env_computations=n_env, ctm_converged=crep["converged"], state=ctx.tn_get_state())
    finally:
        ctx.close()


def field_sweep(hs, D, chi, tau, steps, method="fu", rank=0, world=1, **kw):
    """run_field for the fields hs[rank::world] (replicas: one slice per GPU/rank)."""
    return [run_field(h, D, chi, tau, steps, method=method, **kw) for h in list(hs)[rank::world]]
