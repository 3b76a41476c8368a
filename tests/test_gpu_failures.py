"""Failure paths through the C ABI, made on the host or by the input, never
by a device fault: an injected allocation failure (AIFMM_FAIL_ALLOC_AT)
returns AIFMM_ERR_OOM, and a numerically singular pivot block returns
AIFMM_ERR_SINGULAR from the pivot-magnitude test of the LU."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12704_gb300 as lib
    return lib


def test_injected_allocation_failure_is_reported(A):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np, workloads as W, paper_2301_12704_gb300 as A\n"
        "w = W.log2d(1024, seed=3, leaf=16, tol=1e-8)\n"
        "pts, b = W.points_and_rhs(w)\n"
        "try:\n"
        "    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)\n"
        "    A.aifmm_factor(h)\n"
        "    print('no error')\n"
        "except A.AifmmError as e:\n"
        "    print('status', e.status, e)\n" % ROOT)
    for k in (2, 9, 25):
        env = dict(os.environ, AIFMM_FAIL_ALLOC_AT=str(k))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        assert "status 2" in r.stdout and "injected" in r.stdout, (k, r.stdout)


def test_singular_pivot_is_a_status(A):
    # Gaussian kernel with a length far beyond the domain: every entry is
    # exactly 1.0 in FP64, so each near-field block K_bb has rank one
    w = W.gauss2d(600, seed=4, leaf=16, tol=1e-8)
    pts, b = W.points_and_rhs(w)
    h = A.aifmm_build(pts, w.kernel, 1.0, w.tol, w.leaf, length=1e9)
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_factor(h)
    assert e.value.status == 3
    assert "singular" in str(e.value)
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_solve(h, b)                    # no factorisation to solve with
    assert e.value.status == 4
    # the library stays usable after the error
    w2 = W.log2d(512, seed=5, leaf=16, tol=1e-8)
    p2, b2 = W.points_and_rhs(w2)
    h2 = A.aifmm_build(p2, w2.kernel, w2.diag, w2.tol, w2.leaf)
    A.aifmm_factor(h2)
    x = A.aifmm_solve(h2, b2)
    assert np.all(np.isfinite(x))
