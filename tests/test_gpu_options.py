"""Kernel and admissibility options of aifmm_build on the GPU.

* diag = NaN with a nugget gives A_ii = kernel(0) + nugget (the Gaussian-
  process form of the batched configuration: exp(0) = 1, nugget 1e-2): the
  same solution, bit for bit, as the diagonal 1.01 given explicitly.
* Any admissibility parameter eta >= sqrt(dim) classifies the boxes of a
  uniform tree as the default does (Sec. 2.2): the same solution, bit for
  bit.
* A handle moved to a high-priority stream after its factorisation
  (aifmm_set_priority, for request loops) solves as before, bit for bit,
  twice in a row."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12704_gb300 as lib
    return lib


def _solve(A, w, pts, b, **kw):
    h = A.aifmm_build(pts, w.kernel, kw.pop("diag", w.diag), w.tol, w.leaf, length=w.length, **kw)
    A.aifmm_factor(h)
    x = A.aifmm_solve(h, b)
    A.aifmm_destroy(h)
    return x


def test_nan_diag_takes_kernel_at_zero_plus_nugget(A):
    w = W.gauss2d(900, seed=14, leaf=16, tol=1e-10)
    assert w.diag == 1.0 + 1e-2
    pts, b = W.points_and_rhs(w)
    x0 = _solve(A, w, pts, b)
    x1 = _solve(A, w, pts, b, diag=float("nan"), nugget=1e-2)
    assert np.array_equal(x0, x1)


def test_eta_at_or_above_sqrt_dim_gives_the_same_lists(A):
    w = W.log2d(1024, seed=11, leaf=16, tol=1e-10)
    pts, b = W.points_and_rhs(w)
    x0 = _solve(A, w, pts, b)
    for eta in (np.sqrt(2.0), 3.0):
        assert np.array_equal(x0, _solve(A, w, pts, b, eta=eta))


def test_solves_after_a_priority_change_are_unchanged(A):
    w = W.log2d(3000, seed=15, leaf=32)
    pts, b = W.points_and_rhs(w, nrhs=2)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    A.aifmm_factor(h)
    x0 = A.aifmm_solve(h, b)
    A.aifmm_set_priority(h, -1000)       # clamped to the device's highest
    x1 = A.aifmm_solve(h, b)
    A.aifmm_set_priority(h, 0)
    x2 = A.aifmm_solve(h, b)
    A.aifmm_destroy(h)
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)
