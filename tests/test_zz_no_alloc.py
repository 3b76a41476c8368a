"""The allocation-free solve.

Callers that cannot allocate device memory after start-up (for instance a
request loop that serves solves against a factorisation made at start-up,
under a fixed memory budget) use aifmm_solve_noalloc.  It must give the same
solution as aifmm_solve.  Every call shares one static device array that
keeps the previous call's contents, so the calls below change the layout of
that array between them (other nrhs, another problem size and depth): a part
that should have been cleared shows up as a wrong solution.  This file is
collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    import torch
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_solve_matches_solve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12704_gb300 as A

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.log2d(4096, seed=0)
    pts, b = W.points_and_rhs(w, nrhs=3)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    A.aifmm_factor(h)
    # a second problem of another size and depth, used between the calls
    w2 = W.log2d(1500, seed=7, leaf=16)
    pts2, b2 = W.points_and_rhs(w2, nrhs=2)
    h2 = A.aifmm_build(pts2, w2.kernel, w2.diag, w2.tol, w2.leaf)
    A.aifmm_factor(h2)
    assert A.aifmm_levels(h2) != A.aifmm_levels(h)

    bd = torch.from_numpy(b.T.copy()).to(dev).t()          # column-major N x 3
    ref3 = A.aifmm_solve(h, bd)
    ref1 = A.aifmm_solve(h, bd[:, :1].t().contiguous().t())
    b2d = torch.from_numpy(b2.T.copy()).to(dev).t()
    ref2 = A.aifmm_solve(h2, b2d)
    for k, hh, rhs, ref in ((3, h, bd, ref3), (1, h, bd[:, :1].t().contiguous().t(), ref1),
                            (2, h2, b2d, ref2), (3, h, bd, ref3), (2, h2, b2d, ref2)):
        x = torch.empty((k, rhs.shape[0]), dtype=torch.float64, device=dev).t()
        x.fill_(np.nan)
        A.aifmm_solve_noalloc(hh, rhs, x)
        rel = _rel(x, ref)
        assert rel <= 1e-12, (k, rel)
    # in place (rhs and x alias)
    y = bd.t().contiguous().t()
    A.aifmm_solve_noalloc(h, y, y)
    assert _rel(y, ref3) <= 1e-12
    # sizes beyond the static array are rejected with a clear error
    big = torch.zeros((4096, w.n), dtype=torch.float64, device=dev).t()
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_solve_noalloc(h, big, big)
    assert e.value.status == 8 and "static scratch" in str(e.value)
    # host buffers are refused (staging them would allocate)
    import ctypes as C
    with pytest.raises(A.AifmmError) as e:
        st = A.lib().aifmm_solve_noalloc(h.raw, C.c_void_p(b.ctypes.data), C.c_void_p(b.ctypes.data), 3, w.n)
        A._check(st, h.raw)
    assert e.value.status == 1
    A.aifmm_destroy(h2)
    A.aifmm_destroy(h)
