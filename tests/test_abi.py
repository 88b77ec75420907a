"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/tnite.h.

No compute call is made: these run on a machine without a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_1411_0391_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tnite.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("tn_create", "tn_ctmrg", "tn_evolve", "tn_measure", "tn_recycle", "tn_fu_step"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1411_0391_gb300 import _lib
    assert set(_declared()) == set(_lib.EXPORTED)


def test_workspace_size_is_host_only(libpath):
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    ok = _lib.tn_config(4, 64, _lib.TN_CELL_CHECKERBOARD, _lib.TN_F64)
    bad = _lib.tn_config(4, 0, _lib.TN_CELL_CHECKERBOARD, _lib.TN_F64)
    n = L.tn_workspace_bytes(ctypes.byref(ok))
    assert n > (64 * 16) ** 2 * 8          # at least one N x N matrix
    assert L.tn_workspace_bytes(ctypes.byref(bad)) == 0
    small = _lib.tn_config(2, 8, _lib.TN_CELL_CHECKERBOARD, _lib.TN_F64)
    assert 0 < L.tn_workspace_bytes(ctypes.byref(small)) < n


def test_status_strings(libpath):
    from paper_1411_0391_gb300 import _lib
    assert _lib.lib().tn_strerror(_lib.TN_EINVAL) == b"invalid argument"
    assert _lib.lib().tn_strerror(_lib.TN_ENOCONV).startswith(b"iteration cap")


def test_precision_forms_validated_on_host(libpath):
    """Every precision value of tn_config is accepted by the workspace query; others are not."""
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    for prec in (_lib.TN_F64, _lib.TN_TF32X3, _lib.TN_BF16X3, _lib.TN_BF16S4):
        cfg = _lib.tn_config(2, 8, _lib.TN_CELL_CHECKERBOARD, prec)
        assert L.tn_workspace_bytes(ctypes.byref(cfg)) > 0
    bad = _lib.tn_config(2, 8, _lib.TN_CELL_CHECKERBOARD, 7)
    assert L.tn_workspace_bytes(ctypes.byref(bad)) == 0
    bad = _lib.tn_config(2, 8, _lib.TN_CELL_CHECKERBOARD, -1)
    assert L.tn_workspace_bytes(ctypes.byref(bad)) == 0


def test_split_gemm_workspace_is_the_padded_operands(libpath):
    """Head and tail of each operand, K-major, rows padded to the 128 x 64 tile and K to 128 bytes."""
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    def al(x):
        return (x + 255) // 256 * 256
    m, n, k = 200, 150, 70
    # TF32: 4-byte elements, K padded to 32; BF16: 2-byte elements, K padded to 64
    tf = al(2 * 256 * 96 * 4) + al(2 * 192 * 96 * 4)
    bf = al(2 * 256 * 128 * 2) + al(2 * 192 * 128 * 2)
    assert L.tn_gemm_split_workspace_bytes(_lib.TN_TF32X3, m, n, k) == tf
    assert L.tn_gemm_split_workspace_bytes(_lib.TN_BF16X3, m, n, k) == bf
    assert L.tn_gemm_split_workspace_bytes(_lib.TN_F64, m, n, k) == 0
    assert L.tn_gemm_split_workspace_bytes(_lib.TN_TF32X3, 0, n, k) == 0


def test_argument_checks_before_any_device_call(libpath):
    """Calls that fail validation return TN_EINVAL without touching the GPU."""
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    assert L.tn_set_projector_cutoff(None, 1e-12) == _lib.TN_EINVAL
    assert L.tn_su_step(None, None) == _lib.TN_EINVAL
    assert L.tn_fu_step(None, 1e-8, 10, None) == _lib.TN_EINVAL
    assert L.tn_gemm_split(5, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, 0, None) == _lib.TN_EINVAL
    assert L.tn_gemm_split(_lib.TN_TF32X3, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, 0, None) \
        == _lib.TN_EINVAL
    assert L.tn_truncated_svd_noalloc(None, 8, 4, None, None, None, None, None) == _lib.TN_EINVAL
    h = ctypes.c_void_p()
    bad = _lib.tn_config(9, 8, _lib.TN_CELL_CHECKERBOARD, _lib.TN_F64)       # D out of range
    assert L.tn_create(ctypes.byref(h), ctypes.byref(bad), None, 0, None) == _lib.TN_EINVAL


def test_new_status_strings(libpath):
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    assert b"tensor-core" in L.tn_strerror(_lib.TN_ETIMEOUT)
    assert b"allocation-free" in L.tn_strerror(_lib.TN_ESCRATCH)


def test_evolve_options_validated_on_host(libpath):
    """tn_evolve rejects malformed options before it looks at the context (no device call):
    a NaN fidelity threshold, an unknown mode, a zero window, a NaN trigger."""
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    dummy = ctypes.create_string_buffer(64)        # never dereferenced: validation comes first
    ctx = ctypes.cast(dummy, ctypes.c_void_p)
    rep = _lib.tn_evolve_report()
    nan = float("nan")
    cases = [
        _lib.tn_evolve_opts(_lib.TN_RECYCLE_FIXED, 2, 1e-8, 10, 0.0, 1, 0, 1e-12, 50, nan),
        _lib.tn_evolve_opts(7, 2, 1e-8, 10, 0.0, 1, 0, 1e-12, 50, 0.9),
        _lib.tn_evolve_opts(_lib.TN_RECYCLE_FIXED, 0, 1e-8, 10, 0.0, 1, 0, 1e-12, 50, 0.9),
        _lib.tn_evolve_opts(_lib.TN_RECYCLE_THRESHOLD, 2, 1e-8, 10, nan, 1, 0, 1e-12, 50, 0.9),
        _lib.tn_evolve_opts(_lib.TN_RECYCLE_THRESHOLD, 2, 1e-8, 10, 1e-8, 0, 0, 1e-12, 50, 0.9),
        _lib.tn_evolve_opts(_lib.TN_RECYCLE_FIXED, 2, 1e-8, 10, 0.0, 1, -1, 1e-12, 50, 0.9),
    ]
    for o in cases:
        assert L.tn_evolve(ctx, 4, ctypes.byref(o), ctypes.byref(rep)) == _lib.TN_EINVAL
    assert L.tn_evolve(None, 4, ctypes.byref(cases[1]), ctypes.byref(rep)) == _lib.TN_EINVAL
    assert b"unstable" in L.tn_strerror(_lib.TN_EUNSTABLE)


def test_batch_imps_and_autotune_validated_on_host(libpath):
    """The batched runner, the 1D chain and the autotuner switch check their arguments on the
    host: malformed calls return TN_EINVAL without a device call."""
    from paper_1411_0391_gb300 import _lib
    L = _lib.lib()
    o = _lib.tn_evolve_opts(_lib.TN_RECYCLE_OFF, 1, 1e-8, 10, 0.0, 1, 0, 1e-12, 50, 0.0)
    st = (ctypes.c_int * 2)()
    reps = (_lib.tn_evolve_report * 2)()
    assert L.tn_evolve_batch(None, 2, 1, ctypes.byref(o), 0, st, reps) == _lib.TN_EINVAL
    two_null = (ctypes.c_void_p * 2)(None, None)
    assert L.tn_evolve_batch(two_null, 2, 1, ctypes.byref(o), 0, st, reps) == _lib.TN_EINVAL
    assert L.tn_evolve_batch(two_null, 0, 1, ctypes.byref(o), 0, st, reps) == _lib.TN_EINVAL
    assert L.tn_evolve_batch(two_null, 2, 1, None, 0, st, reps) == _lib.TN_EINVAL
    # 1D chain: bond 2 chi <= 32; workspace sizes are host arithmetic
    assert L.tn_imps_workspace_bytes(0) == 0 and L.tn_imps_workspace_bytes(17) == 0
    assert 0 < L.tn_imps_workspace_bytes(4) < L.tn_imps_workspace_bytes(16)
    F = ctypes.c_double()
    out = (ctypes.c_double * 3)()
    assert L.tn_imps_itebd(None, 4, 2.0, 0.05, 1, None, 0, None) == _lib.TN_EINVAL
    assert L.tn_imps_itebd(None, 4, float("nan"), 0.05, 1, None, 0, None) == _lib.TN_EINVAL
    assert L.tn_imps_recycle(None, 4, 2.0, 0.05, 0, ctypes.byref(F), None, 0, None) == _lib.TN_EINVAL
    assert L.tn_imps_observables(None, 4, 2.0, out, None, 0, None) == _lib.TN_EINVAL
    assert L.tn_imps_observables(None, 4, 2.0, None, None, 0, None) == _lib.TN_EINVAL
    # the tile autotuner switch: on/off, returns the number of shapes tuned so far
    n0 = L.tn_set_autotune(1)
    assert n0 >= 0 and L.tn_set_autotune(0) == n0
