"""Pins of the oracle's extended system, elimination (Algorithm 2) and solve
(Algorithm 3) against dense linear algebra on small problems."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import factor as F
from oracle import h2
from oracle.extended import BlockSystem, assemble, key_lists, rhs_blocks
from oracle.kernels import Kernel, INVR3D
from oracle.nnca import NNCA
from oracle.tree import Tree


def _problem(n=256, leaf=8, eps=1e-8, seed=7, kind=None, d=2):
    if kind is None:
        w = W.log2d(n, seed=seed, leaf=leaf, tol=eps, nrhs=2)
    else:
        w = W.invr3d(n, seed=seed, leaf=leaf, tol=eps, nrhs=2)
    pts, b = W.points_and_rhs(w)
    T = Tree(pts, leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, eps)
    return T, K, nn, b[T.perm]


def _dense_ext_solve(T, K, nn, bt):
    S = assemble(T, K, nn)
    rk, ck = key_lists(S)
    A = S.dense(rk, ck)
    rhs = rhs_blocks(T, S, bt)
    B = np.vstack([rhs[k] for k in rk])
    X = np.linalg.solve(A, B)
    return X[:T.N], A


def test_extended_system_represents_h2_matrix():
    """Solving A~ x~ = [b;0] densely gives x = H^-1 b, H the NNCA H^2 matrix
    (eq. extendedMatrix encodes eqs. X, Y and the locals equation)."""
    T, K, nn, bt = _problem()
    assert T.L == 3
    x_ext, A = _dense_ext_solve(T, K, nn, bt)
    H = h2.dense(T, K, nn)
    x_h = np.linalg.solve(H, bt)
    assert np.linalg.norm(x_ext - x_h) / np.linalg.norm(x_h) < 1e-12
    # the leading N x N block of A~ is the near field only
    near = np.zeros_like(H)
    for b in range(T.nboxes(T.L)):
        s, e = T.range(T.L, b)
        for q in T.neighbours(T.L, b):
            qs, qe = T.range(T.L, q)
            near[s:e, qs:qe] = K.block(T.points, np.arange(s, e), np.arange(qs, qe))
    assert np.array_equal(A[:T.N, :T.N], near)


def test_elimination_without_compression_is_exact_lu():
    """With compression off every fill-in is kept: Algorithm 2 reduces to an
    exact block LU of A~ and must reproduce the dense solve of A~."""
    T, K, nn, bt = _problem()
    x_ext, _ = _dense_ext_solve(T, K, nn, bt)
    fac = F.factor(T, K, nn, 1e-8, order="paper", compress=False)
    x = F.solve(fac, bt)
    assert np.linalg.norm(x - x_ext) / np.linalg.norm(x_ext) < 1e-12
    assert fac.ncompress == 0


@pytest.mark.parametrize("order", ["paper", "colour"])
def test_tiny_tolerance_reproduces_dense_solution(order):
    """eps_A -> 0: the AIFMM solution tends to A^-1 b (the full-rank invariant)."""
    T, K, nn, bt = _problem(n=1024, leaf=16, eps=1e-15)
    assert T.L == 3
    fac = F.factor(T, K, nn, 1e-15, order=order)
    x = F.solve(fac, bt)
    xd = np.linalg.solve(K.dense(T.points), bt)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
    assert fac.ncompress > 0


def test_error_falls_with_tolerance():
    """E_A decreases as eps_A decreases (Sec. 4.1, inference 2)."""
    errs = []
    for eps in (1e-3, 1e-6, 1e-9, 1e-12):
        T, K, nn, bt = _problem(n=600, leaf=16, eps=eps)
        fac = F.factor(T, K, nn, eps, order="colour")
        x = F.solve(fac, bt[:, :1])
        xd = np.linalg.solve(K.dense(T.points), bt[:, :1])
        errs.append(np.linalg.norm(x - xd) / np.linalg.norm(xd))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-10


def test_error_roughly_flat_in_n():
    """At a fixed eps_A the error against the dense solution stays roughly
    constant as N grows (Sec. 4.1, inference 1), here across a change of
    depth (L = 3 to 4)."""
    eps, errs, depths = 1e-6, [], []
    for n in (512, 1024, 2048):
        w = W.log2d(n, seed=11, leaf=16, tol=eps, nrhs=1)
        pts, b = W.points_and_rhs(w)
        T = Tree(pts, w.leaf)
        K = Kernel(w.kernel, w.diag)
        nn = NNCA(T, K, eps)
        bt = b[T.perm]
        x = F.solve(F.factor(T, K, nn, eps, order="colour"), bt)
        xd = np.linalg.solve(K.dense(T.points), bt)
        errs.append(np.linalg.norm(x - xd) / np.linalg.norm(xd))
        depths.append(T.L)
    assert depths[0] < depths[-1]
    assert max(errs) < 10 * min(errs) and max(errs) < 100 * eps, errs


def test_paper_and_colour_order_agree():
    eps = 1e-10
    T, K, nn, bt = _problem(n=700, leaf=16, eps=eps)
    xp = F.solve(F.factor(T, K, nn, eps, order="paper"), bt)
    xc = F.solve(F.factor(T, K, nn, eps, order="colour"), bt)
    assert np.linalg.norm(xp - xc) / np.linalg.norm(xc) < 10 * eps


def test_pair_grouping_tiny_tolerance_reproduces_dense_solution():
    """Algorithm 2 as printed (pair by pair, each P2P fill-in compressed on
    both of its boxes, Sec. 3.2.1-3.2.3) keeps the eps_A -> 0 invariant."""
    T, K, nn, bt = _problem(n=1024, leaf=16, eps=1e-15)
    fac = F.factor(T, K, nn, 1e-15, order="paper", grouping="pair")
    x = F.solve(fac, bt)
    xd = np.linalg.solve(K.dense(T.points), bt)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
    assert fac.ncompress > 0


def test_pair_and_box_grouping_agree():
    """Reading R2 (one RRQR per box side over all its pending fill-ins)
    against the printed pair-by-pair grouping: both stay within O(eps_A) of
    the uncompressed elimination (an exact sparse LU of the same NNCA system),
    and so of each other.  A_ii = 5 so that the fill-ins are not negligible
    against the diagonal (cond(A) = 2.1e4).  O(eps_A) is taken as 30 eps_A:
    each RRQR leaves a residual of eps_A relative to its augmented matrix
    [U | F] (Sec. 3.2.1), and the errors measured are 11 eps_A (box) and
    3 eps_A (pair); a dropped or mis-signed redirect gives O(1)."""
    eps = 1e-6
    w = W.log2d(1024, seed=7, leaf=16, tol=eps, nrhs=2, diag=5.0)
    pts, b = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, eps)
    bt = b[T.perm]
    xn = F.solve(F.factor(T, K, nn, eps, order="paper", compress=False), bt)
    xb = F.solve(F.factor(T, K, nn, eps, order="paper", grouping="box"), bt)
    xp = F.solve(F.factor(T, K, nn, eps, order="paper", grouping="pair"), bt)
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    assert rel(xb, xn) < 30 * eps and rel(xp, xn) < 30 * eps
    assert rel(xp, xb) < 30 * eps
    assert rel(xb, xn) > 1e-12            # the compression did act


def test_symmetric_and_general_compression_agree():
    """Reading R13 (the GPU's default): for a symmetric kernel with V = U one
    RRQR per box gives both new bases.  Against the general two-sided form
    (two RRQRs whose kept directions differ near the threshold in floating
    point): both within O(eps_A) of the uncompressed elimination (30 eps_A,
    as in the grouping test) and within eps_A of each other, with ranks no
    higher."""
    eps = 1e-6
    w = W.log2d(1024, seed=7, leaf=16, tol=eps, nrhs=2, diag=5.0)
    pts, b = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, eps)
    bt = b[T.perm]
    xn = F.solve(F.factor(T, K, nn, eps, order="paper", compress=False), bt)
    fg = F.factor(T, K, nn, eps, order="paper")
    fs = F.factor(T, K, nn, eps, order="paper", symmetric=True)
    xg, xs = F.solve(fg, bt), F.solve(fs, bt)
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    assert rel(xs, xn) < 30 * eps and rel(xs, xg) < eps
    assert max(fs.ranks.values()) <= max(fg.ranks.values())


def test_multiple_rhs_columns_are_independent():
    T, K, nn, bt = _problem(n=512, leaf=16, eps=1e-10)
    fac = F.factor(T, K, nn, 1e-10, order="colour")
    X = F.solve(fac, bt)
    for k in range(bt.shape[1]):
        np.testing.assert_allclose(F.solve(fac, bt[:, k]), X[:, k], rtol=0, atol=1e-14 * np.abs(X).max())


def test_three_dimensional_small():
    eps = 1e-8
    T, K, nn, bt = _problem(n=512, leaf=8, eps=eps, kind=INVR3D)
    assert T.d == 3 and T.L == 2
    x = F.solve(F.factor(T, K, nn, eps, order="colour"), bt[:, 0])
    xd = np.linalg.solve(K.dense(T.points), bt[:, 0])
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 100 * eps


def test_three_dimensional_three_levels_tiny_tolerance():
    """3D 1/r with three levels (L = 3), so that the octree's non-leaf
    levels and their 27-box stencils are eliminated too: eps_A -> 0 gives
    the dense solution.  (At sizes the oracle affords, 3D leaf boxes hold a
    few points and their bases are full rank: this pins the elimination and
    the level transitions, not the truncation, which the 2D pins cover.)"""
    eps = 1e-15
    w = W.invr3d(600, seed=5, leaf=4, tol=eps, nrhs=1)
    pts, b = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, eps)
    assert T.d == 3 and T.L == 3
    bt = b[T.perm]
    x = F.solve(F.factor(T, K, nn, eps, order="colour"), bt)
    xd = np.linalg.solve(K.dense(T.points), bt)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12


def test_qrcp_forced_columns():
    rng = np.random.default_rng(3)
    U = np.linalg.qr(rng.standard_normal((30, 6)))[0]
    Fm = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 50))   # rank 4
    Q, rd = F.qrcp_forced(np.hstack([U, Fm]), 6)
    assert np.allclose(Q.T @ Q, np.eye(30), atol=1e-14)
    # first columns span U exactly; R_kk of unit orthonormal columns is 1
    assert np.allclose(np.abs(rd[:6]), 1.0, atol=1e-14)
    P = Q[:, :6] @ Q[:, :6].T
    assert np.linalg.norm(P @ U - U) < 1e-13
    tau = 1e-10 * np.linalg.norm(Fm, axis=0).max()
    k = F.rrqr_rank(rd, 6, tau)
    assert k == 10
    # rank is monotone in the threshold
    assert F.rrqr_rank(rd, 6, 1e3 * tau) <= k <= F.rrqr_rank(rd, 6, 0.0)
    # residual of the projected fill-in below threshold
    Qk = Q[:, :k]
    assert np.linalg.norm(Fm - Qk @ (Qk.T @ Fm)) < 1e-12 * np.linalg.norm(Fm)


def test_qrcp_matches_library_qr_without_pivoting():
    """With every column forced the routine is plain Householder QR: compare
    with LAPACK's QR up to column signs."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((12, 7))
    Q, rd = F.qrcp_forced(M, 7)
    Ql, Rl = np.linalg.qr(M)
    s = np.sign(np.sum(Q[:, :7] * Ql, axis=0))
    assert np.allclose(Q[:, :7] * s, Ql, atol=1e-13)
    assert np.allclose(rd, np.abs(np.diag(Rl)), atol=1e-13)


def test_singular_pivot_detected():
    S = BlockSystem()
    S.rsize[("r",)] = 2
    S.csize[("c",)] = 2
    S.set(("r",), ("c",), np.array([[1.0, 2.0], [2.0, 4.0]]))
    with pytest.raises(F.SingularPivot):
        F.eliminate(S, [("r",)], [("c",)], box="t")
