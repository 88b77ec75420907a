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
              measure_max=300, precision=L.TN_F64, instance=0, device="cuda:0", state=None):
    """Evolve one field value and measure it; returns a dict of observables.

    method: "fu" (full update, recycled in windows of n_re steps when n_re > 1)
    or "su" (simple update).  The measurement converges a fresh CTMRG.
    """
    ctx = L.Context(D, chi, device=device, precision=precision)
    try:
        ctx.tn_set_hamiltonian(1.0, h)
        ctx.tn_set_time_step(tau)
        ctx.tn_set_state(state if state is not None else random_peps(2, D, instance=instance))
        n_env = 0
        if method == "su":
            for _ in range(steps):
                ctx.tn_su_step()
        elif method == "fu":
            rep = ctx.tn_evolve(steps, recycle=n_re > 1, n_re=max(n_re, 1), ctm_tol=ctm_tol, ctm_max=ctm_max)
            n_env = rep["env_computations"]
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
