"""FP32 factorisation (aifmm_options.precision = 1) as the preconditioner of
FP64 GMRES (Sec. 4: AIFMM used as a preconditioner), through the C ABI,
against the oracle.  The oracle has no FP32 mode: what is pinned is that the
FP32 factorisation solves to about single precision on its own and that
preconditioned GMRES reaches the FP64 oracle's solution of the same H^2
system."""
import numpy as np
import pytest

import workloads as W
from oracle import h2 as OH
from oracle.gmres import gmres as ogmres
from oracle.kernels import Kernel
from oracle.nnca import NNCA
from oracle.tree import Tree

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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _h2_solution(w, pts, b):
    """The oracle's unpreconditioned GMRES solution of the H^2 system."""
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag, w.length)
    nn = NNCA(T, K, w.tol)
    perm = T.perm

    def mv(v):
        y = np.empty_like(v)
        y[perm] = OH.matvec(T, K, nn, v[perm])
        return y

    xo, _, hist = ogmres(mv, b, rtol=1e-13, maxit=600, restart=60)
    return xo, K


CASES = [
    W.log2d(1024, seed=31, leaf=16, tol=1e-10),
    W.invr3d(512, seed=32, leaf=8, tol=1e-8),
]
CASES[0].diag = 100.0


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_fp32_factor_preconditions_fp64_gmres(A, w):
    pts, b = W.points_and_rhs(w)
    b = b[:, 0]
    # FP32 rounding of the fill-ins sits near 1e-7 of their size: compress at
    # 1e-6, the low-accuracy factorisation of a preconditioner
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf, length=w.length, fp32=True, factor_tol=1e-6)
    A.aifmm_factor(h)
    xo, K = _h2_solution(w, pts, b)
    # the FP32 factorisation alone (compressed at 1e-6): far from FP64 accuracy
    x1 = A.aifmm_solve(h, b)[:, 0]
    e1 = _rel(x1, xo)
    assert 1e-12 < e1 <= 1e-3, e1
    # as a preconditioner: FP64 GMRES to rtol 1e-11 in a few steps
    x, it, rr = A.aifmm_gmres(h, b, rtol=1e-11, maxit=60, restart=30, use_precond=True)
    assert rr <= 1e-11
    assert it <= 8, it
    assert _rel(x, xo) <= 1e-9
    # unpreconditioned GMRES needs more steps
    _, it0, _ = A.aifmm_gmres(h, b, rtol=1e-11, maxit=600, restart=30, use_precond=False)
    assert it0 > it


def test_fp32_option_checked(A):
    import ctypes as C
    w = CASES[0]
    pts, _ = W.points_and_rhs(w)
    lib = A.lib()
    k = A.Kernel(w.kernel, 2, float(w.diag), 1.0)
    o = A.Options(0, 0, None, 0, 0, 0.0, 0, 0, 7)          # precision 7: invalid
    out = C.c_void_p()
    p = np.ascontiguousarray(pts)
    st = lib.aifmm_build(C.c_void_p(p.ctypes.data), len(p), C.byref(k), w.tol, w.leaf, C.byref(o), C.byref(out))
    assert st == 1 and out.value is None


@pytest.mark.parametrize("trans_a", [False, True], ids=["AB", "AtB"])
def test_tf32_tile_within_its_rounding(A, trans_a):
    """The TF32 tile (aifmm_options.precision = 2) against the FP64 product:
    each operand rounds to 10 mantissa bits (2^-11 relative), the products
    are exact in FP32 and the FP32 sums add ~K 2^-24, so every entry is
    within 2^-9 |op(A)| |B| of the exact one; ragged sizes over several
    tiles and K chunks."""
    import torch
    g = torch.Generator().manual_seed(5)
    m, n, k = 150, 133, 101
    Aop = torch.randn(m, k, generator=g, dtype=torch.float64)
    Bm = torch.randn(k, n, generator=g, dtype=torch.float64)
    C0 = torch.randn(m, n, generator=g, dtype=torch.float64)
    dev = torch.device("cuda", 0)
    Ad = (Aop.t() if trans_a else Aop).to(dev).t().contiguous().t()   # column-major
    Bd = Bm.to(dev).t().contiguous().t()
    Cd = C0.to(dev).t().contiguous().t()
    A.aifmm_gemm_tf32(Ad, Bd, Cd, alpha=-0.5, trans_a=trans_a)
    exact = C0 - 0.5 * Aop @ Bm
    bound = 2.0 ** -9 * 0.5 * (Aop.abs() @ Bm.abs())
    err = (Cd.cpu() - exact).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    assert float((err / bound).max()) > 1e-3            # the rounding is visible: not an FP64 product


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_tf32_factor_preconditions_fp64_gmres(A, w):
    pts, b = W.points_and_rhs(w)
    b = b[:, 0]
    # TF32 rounding of the products sits near 1e-3 of their size: compress
    # at 1e-3, a coarse factorisation that only preconditions
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf, length=w.length, tf32=True, factor_tol=1e-3)
    A.aifmm_factor(h)
    xo, K = _h2_solution(w, pts, b)
    x1 = A.aifmm_solve(h, b)[:, 0]
    e1 = _rel(x1, xo)
    assert 1e-8 < e1 <= 0.5, e1
    x, it, rr = A.aifmm_gmres(h, b, rtol=1e-11, maxit=100, restart=40, use_precond=True)
    assert rr <= 1e-11
    assert _rel(x, xo) <= 1e-9
    _, it0, _ = A.aifmm_gmres(h, b, rtol=1e-11, maxit=600, restart=40, use_precond=False)
    assert it0 > it, (it0, it)
    A.aifmm_destroy(h)
