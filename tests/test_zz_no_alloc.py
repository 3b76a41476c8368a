"""The allocation-free solve.

Callers that cannot allocate device memory after start-up (for instance a
request loop that serves solves against a factorisation made at start-up,
under a fixed memory budget) use aifmm_solve_noalloc.  It must give the same
solution as aifmm_solve.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other
test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12704_gb300 as A

    w = W.log2d(4096, seed=0)
    pts, b = W.points_and_rhs(w, nrhs=3)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    A.aifmm_factor(h)
    dev = torch.device("cuda", 0)
    bd = torch.from_numpy(b.T.copy()).to(dev).t()          # column-major N x 3
    ref = A.aifmm_solve(h, bd)
    for _ in range(2):                                      # two calls in a row
        x = torch.empty((3, w.n), dtype=torch.float64, device=dev).t()
        x.fill_(np.nan)
        A.aifmm_solve_noalloc(h, bd, x)
        rel = float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref))
        assert rel <= 1e-12, rel
    # in place (rhs and x alias)
    y = bd.clone(memory_format=torch.preserve_format)
    y = y.t().contiguous().t()
    A.aifmm_solve_noalloc(h, y, y)
    assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) <= 1e-12
    # sizes beyond the static array are rejected with a clear error
    big = torch.zeros((4096, w.n), dtype=torch.float64, device=dev).t()
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_solve_noalloc(h, big, big)
    assert e.value.status == 8 and "static scratch" in str(e.value)
    # host buffers are refused (staging them would allocate)
    with pytest.raises(A.AifmmError) as e:
        A.lib()
        import ctypes as C
        st = A.lib().aifmm_solve_noalloc(h.raw, C.c_void_p(b.ctypes.data), C.c_void_p(b.ctypes.data), 3, w.n)
        A._check(st, h.raw)
    assert e.value.status == 1
    A.aifmm_destroy(h)
