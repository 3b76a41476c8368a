"""The C-ABI library builds, loads without a GPU, and exports every entry
point that the headers under include/ declare."""
import os
import re

import pytest

import paper_2301_12704_gb300 as A
from paper_2301_12704_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names.update(re.findall(r"\b(aifmm_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_header_symbols():
    _build.build()
    lib = A.lib()
    names = _declared()
    assert "aifmm_build" in names and "aifmm_solve" in names and "aifmm_factor" in names
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_without_gpu_work():
    import ctypes as C
    import numpy as np
    lib = A.lib()
    out = C.c_void_p()
    k = A.Kernel(A.LOG2D, 4, 1.0, 1.0)          # dim 4 is invalid
    pts = np.zeros((4, 4))
    st = lib.aifmm_build(C.c_void_p(pts.ctypes.data), 4, C.byref(k), 1e-8, 8, None, C.byref(out))
    assert st == 1 and out.value is None
    assert b"invalid" in lib.aifmm_last_error(None)
    # null handle calls
    assert lib.aifmm_factor(None) == 1
    assert lib.aifmm_solve(None, None, None, 1, 1) == 1
    assert lib.aifmm_levels(None) == 0
    lib.aifmm_destroy(None)
