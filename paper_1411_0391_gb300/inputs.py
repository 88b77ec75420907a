"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only draws the initial iPEPS
tensors of the workloads, A ~ N(0, 1) i.i.d. with leg order (s, l, r, d, u),
divided by max |A|, from numpy's default generator seeded with
SEED_BASE + instance.
"""
import numpy as np

SEED_BASE = 14110391


def random_peps(n_tensors, D, d=2, instance=0, seed=None):
    """n_tensors float64 arrays of shape (d, D, D, D, D), each max-abs normalised."""
    rng = np.random.default_rng(SEED_BASE + instance if seed is None else seed)
    out = []
    for _ in range(n_tensors):
        A = rng.standard_normal((d, D, D, D, D))
        out.append(A / np.abs(A).max())
    return out


def random_matrix(shape, instance=0, seed=None):
    """Gaussian float64 array of the given shape (for kernel-level parity cases)."""
    rng = np.random.default_rng(SEED_BASE + 7919 * (instance + 1) if seed is None else seed)
    return rng.standard_normal(shape)
