"""Shared helpers of the GPU parity tests (imported by test_gpu_*.py)."""
import numpy as np

from oracle import ctmrg as OC

SITE_ORDER = {2: [(0, 0), (1, 0), (0, 1), (1, 1)], 1: [(0, 0)]}
NAMES = ['C1', 'C2', 'C3', 'C4', 'T1', 'T2', 'T3', 'T4']


def env_to_dict(buf, n_tensors, chi, leg):
    """Split the flat environment of tn_get_env into {(x, y): {name: array}}."""
    out, off = {}, 0
    for (x, y) in SITE_ORDER[n_tensors]:
        e = {}
        for k in range(4):
            e[NAMES[k]] = buf[off:off + chi * chi].reshape(chi, chi)
            off += chi * chi
        for k in range(4):
            e[NAMES[4 + k]] = buf[off:off + chi * chi * leg].reshape(chi, chi, leg)
            off += chi * chi * leg
        out[(x, y)] = e
    return out


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def oracle_spectra(st):
    sp = OC.corner_spectra(st)
    return sp
