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


def test_nugget_and_eta_arguments_checked_before_gpu_work():
    """diag = NaN asks for A_ii = kernel(0) + nugget, which is infinite for
    the log and 1/r kernels; an admissibility parameter eta below sqrt(dim)
    would need a wider near field than the touching boxes: both are refused
    before any device work (so without a GPU)."""
    import ctypes as C
    import numpy as np
    lib = A.lib()
    pts = np.random.default_rng(0).uniform(-1, 1, (64, 2))
    out = C.c_void_p()
    k = A.Kernel(A.LOG2D, 2, float("nan"), 1.0, 0.1)
    st = lib.aifmm_build(C.c_void_p(pts.ctypes.data), 64, C.byref(k), 1e-8, 16, None, C.byref(out))
    assert st == 1 and out.value is None and b"kernel(0)" in lib.aifmm_last_error(None)
    k = A.Kernel(A.LOG2D, 2, 64.0, 1.0, 0.0)
    o = A.Options()
    o.eta = 1.0                                   # below sqrt(2)
    st = lib.aifmm_build(C.c_void_p(pts.ctypes.data), 64, C.byref(k), 1e-8, 16, C.byref(o), C.byref(out))
    assert st == 1 and b"eta" in lib.aifmm_last_error(None)
    k = A.Kernel(A.GAUSS, 2, float("inf"), 0.1, 0.0)
    st = lib.aifmm_build(C.c_void_p(pts.ctypes.data), 64, C.byref(k), 1e-8, 16, None, C.byref(out))
    assert st == 1


def test_set_priority_on_a_null_handle_is_refused():
    """aifmm_set_priority validates its handle before any CUDA call."""
    lib = A.lib()
    assert lib.aifmm_set_priority(None, -5) == 1
