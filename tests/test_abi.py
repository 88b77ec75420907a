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
