"""GPU GMRES (aifmm_gmres, through the C ABI) against the oracle's GMRES on
the same H^2 operator, with and without the AIFMM preconditioner."""
import numpy as np
import pytest

import workloads as W
from oracle import factor as OF
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


def _oracle_ops(w, pts, ftol=None):
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag, w.length)
    nn = NNCA(T, K, w.tol)
    F = OF.factor(T, K, nn, ftol if ftol else w.tol, order="colour")
    perm = T.perm

    def mv(v):
        y = np.empty_like(v)
        y[perm] = OH.matvec(T, K, nn, v[perm])
        return y

    def pc(v):
        x = np.empty_like(v)
        x[perm] = OF.solve(F, v[perm])
        return x

    return K, mv, pc


# a diagonal far below N (condition number about 16) makes unpreconditioned
# GMRES(20) need about 36 steps
W_HARD = W.log2d(1024, seed=21, leaf=16, tol=1e-10)
W_HARD.diag = 100.0


def test_gmres_unpreconditioned_matches_oracle(A):
    w = W_HARD
    pts, b = W.points_and_rhs(w)
    b = b[:, 0]
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    x, it, rr = A.aifmm_gmres(h, b, rtol=1e-10, maxit=300, restart=20, use_precond=False)
    K, mv, pc = _oracle_ops(w, pts)
    xo, ito, hist = ogmres(mv, b, rtol=1e-10, maxit=300, restart=20)
    assert rr <= 1e-10 and hist[-1] <= 1e-10
    assert abs(it - ito) <= 1, (it, ito)
    assert it > 20                               # restarts were exercised
    # the residual the library reports is the H^2 residual of its iterate
    assert abs(_rel(mv(x), b) - rr) <= 1e-12
    assert _rel(x, xo) <= 1e-8
    xd = np.linalg.solve(K.dense(pts), b)
    assert _rel(x, xd) <= 1e-7


@pytest.mark.parametrize("ftol", [None, 1e-4])
def test_gmres_preconditioned_matches_oracle(A, ftol):
    """Preconditioner: the factorisation at tol (one or two steps) or at a
    looser compress threshold (Experiment 5: a low-accuracy AIFMM)."""
    w = W.log2d(1024, seed=22, leaf=16, tol=1e-10)
    w.diag = 100.0
    pts, b = W.points_and_rhs(w)
    b = b[:, 0]
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf, factor_tol=ftol or 0.0)
    A.aifmm_factor(h)
    x, it, rr = A.aifmm_gmres(h, b, rtol=1e-11, maxit=50, restart=30, use_precond=True)
    K, mv, pc = _oracle_ops(w, pts, ftol)
    xo, ito, hist = ogmres(mv, b, rtol=1e-11, maxit=50, restart=30, precond=pc)
    assert rr <= 1e-11
    assert abs(it - ito) <= 1, (it, ito)
    assert it <= (3 if ftol is None else 12)
    assert _rel(x, xo) <= 1e-9
    # unpreconditioned GMRES needs more steps on the same system
    _, it0, _ = A.aifmm_gmres(h, b, rtol=1e-11, maxit=400, restart=30, use_precond=False)
    assert it0 > it


def test_gmres_states_and_limits(A):
    w = W.log2d(512, seed=23, leaf=16, tol=1e-8)
    pts, b = W.points_and_rhs(w)
    b = b[:, 0]
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_gmres(h, b, use_precond=True)          # no factor yet
    assert e.value.status == 4
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_gmres(h, b, restart=0, use_precond=False)
    assert e.value.status == 1
    # too few iterations: NOCONV, and the iterate is still returned
    w2 = W.log2d(512, seed=23, leaf=16, tol=1e-8)
    w2.diag = 5.0
    h2 = A.aifmm_build(pts, w2.kernel, w2.diag, w2.tol, w2.leaf)
    x, it, rr = A.aifmm_gmres(h2, b, rtol=1e-14, maxit=3, restart=2, use_precond=False, raise_noconv=False)
    assert it == 3 and 0 < rr < 1
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_gmres(h2, b, rtol=1e-14, maxit=3, restart=2, use_precond=False)
    assert e.value.status == 5
    # zero right-hand side: zero solution without iterations
    x, it, rr = A.aifmm_gmres(h, np.zeros_like(b), use_precond=False)
    assert it == 0 and not x.any()


def test_gmres_device_buffers(A):
    import torch
    w = W.log2d(512, seed=24, leaf=16, tol=1e-10)
    pts, b = W.points_and_rhs(w)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    A.aifmm_factor(h)
    xh, it_h, rr_h = A.aifmm_gmres(h, b[:, 0], rtol=1e-12, use_precond=True)
    bd = torch.from_numpy(b[:, 0].copy()).cuda()
    xd, it_d, rr_d = A.aifmm_gmres(h, bd, rtol=1e-12, use_precond=True)
    assert xd.is_cuda
    assert it_d == it_h
    assert np.array_equal(xd.cpu().numpy(), xh)
