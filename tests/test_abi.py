"""The C ABI library loads on a machine without a GPU and exports every entry point that
include/dpr1.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "dpr1.h")).read()
    return sorted(set(re.findall(r"DPR1_API\s+[\w\s\*]+?\b(dpr1_\w+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared()
    for must in ("dpr1_eig", "dpr1_eig_batched", "dpr1_eig_backward", "dpr1_stream_status", "dpr1_eig_noalloc"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1405_7537_gb300 import _build
    try:
        path = _build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    # host-only entry points answer without touching a GPU
    lib.dpr1_workspace_size.argtypes = [ctypes.c_int64]
    lib.dpr1_workspace_size.restype = ctypes.c_size_t
    assert lib.dpr1_workspace_size(1000) > 1000 * 100
    lib.dpr1_status_string.restype = ctypes.c_char_p
    assert lib.dpr1_status_string(0) == b"ok"
    lib.dpr1_eig.restype = ctypes.c_int
    lib.dpr1_eig.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 2 + [ctypes.c_double] + [ctypes.c_void_p] * 2 + \
        [ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_size_t] + [ctypes.c_void_p] * 2
    # argument errors are reported on the host before any launch
    assert lib.dpr1_eig(-1, None, None, 1.0, None, None, 0, None, None, None, None, 0, None, None) == 1
    assert lib.dpr1_eig(4, None, None, -1.0, None, None, 0, None, None, None, None, 0, None, None) == 3
    assert lib.dpr1_eig(0, None, None, 1.0, None, None, 0, None, None, None, None, 0, None, None) == 0
