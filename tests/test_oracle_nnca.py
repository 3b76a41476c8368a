"""Pins of the oracle's ACA, NNCA operators and H^2 product (Sec. 2.3)
against exact low-rank matrices and the dense interaction matrix."""
import numpy as np
import pytest

import workloads as W
from oracle import h2
from oracle.kernels import GAUSS, INVR2D, INVR3D, LOG2D, Kernel
from oracle.nnca import NNCA, aca
from oracle.tree import Tree


def _cur_error(M, pr, pc):
    C = M[:, pc]
    R = M[pr, :]
    S = M[np.ix_(pr, pc)]
    approx = C @ np.linalg.solve(S, R)
    return np.linalg.norm(M - approx) / np.linalg.norm(M)


def test_kernel_closed_forms():
    p = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, np.e], [0.0, 2.0]])
    K = Kernel(LOG2D, 7.0)
    A = K.block(p, [0, 1], [0, 1, 2])
    assert A[0, 0] == 7.0 and A[1, 1] == 7.0          # same index: diagonal
    assert A[0, 1] == 0.0 and abs(A[0, 2] - 1.0) < 1e-15
    assert abs(A[1, 2] - 0.5 * np.log(1.0 + np.e ** 2)) < 1e-15
    K = Kernel(INVR2D, 3.0)
    assert K.block(p, [0], [3])[0, 0] == 0.5
    K = Kernel(INVR3D, 3.0)
    q = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 4.0]])
    assert K.block(q, [0], [1])[0, 0] == 0.25
    K = Kernel(GAUSS, 1.01, length=0.5)
    assert abs(K.block(p, [0], [1])[0, 0] - np.exp(-4.0)) < 1e-16
    with pytest.raises(ValueError):
        Kernel(LOG2D, 1.0).block(np.zeros((2, 2)), [0], [1])


def test_aca_exact_rank():
    rng = np.random.default_rng(0)
    for k in (1, 3, 7):
        M = rng.standard_normal((40, k)) @ rng.standard_normal((k, 60))
        pr, pc = aca(lambda i: M[i], lambda j: M[:, j], 40, 60, 1e-12)
        assert len(pr) == k
        assert _cur_error(M, pr, pc) < 1e-12
        assert len(set(pr)) == k and len(set(pc)) == k


def test_aca_full_rank_takes_all_rows():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((25, 40))
    pr, pc = aca(lambda i: M[i], lambda j: M[:, j], 25, 40, 0.0)
    assert sorted(pr) == list(range(25))
    assert _cur_error(M, pr, pc) < 1e-12


def test_aca_first_pivot_is_row_zero_argmax():
    M = np.array([[1.0, -5.0, 2.0], [0.5, 0.1, 0.2], [3.0, 1.0, 9.0]])
    pr, pc = aca(lambda i: M[i], lambda j: M[:, j], 3, 3, 1e-15)
    assert pr[0] == 0 and pc[0] == 1
    # second row: argmax of the residual column among unused rows
    u = M[:, 1]
    i2 = 1 + int(np.argmax(np.abs(u[1:])))
    assert pr[1] == i2


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_aca_smooth_block_error(eps):
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (80, 2))
    Y = rng.uniform(3, 4, (120, 2))
    M = 0.5 * np.log(((X[:, None] - Y[None]) ** 2).sum(-1))
    pr, pc = aca(lambda i: M[i], lambda j: M[:, j], 80, 120, eps)
    assert _cur_error(M, pr, pc) < 30 * eps


def _uchain(T, nn, l, b):
    """Basis of box b at level l evaluated at its points (nested product)."""
    if l == T.L:
        return nn.U[l][b]
    blocks = [_uchain(T, nn, l + 1, c) for c in T.children(b)]
    rows = sum(x.shape[0] for x in blocks)
    cols = sum(x.shape[1] for x in blocks)
    D = np.zeros((rows, cols))
    ro = co = 0
    for x in blocks:
        D[ro:ro + x.shape[0], co:co + x.shape[1]] = x
        ro += x.shape[0]
        co += x.shape[1]
    return D @ nn.U[l][b]


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_nnca_admissible_blocks(eps):
    w = W.log2d(2048, seed=3, leaf=32, tol=eps)
    pts, _ = W.points_and_rhs(w)
    T = Tree(pts, 32)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, eps)
    worst = 0.0
    for l in range(2, T.L + 1):
        for b in range(0, T.nboxes(l), 3):
            Ub = _uchain(T, nn, l, b)
            Ib = np.arange(*T.range(l, b))
            for d in T.interaction_list(l, b)[::4]:
                Ud = _uchain(T, nn, l, d)
                Id = np.arange(*T.range(l, d))
                A = K.block(T.points, Ib, Id)
                approx = Ub @ nn.m2l(l, b, d) @ Ud.T
                worst = max(worst, np.linalg.norm(A - approx) / np.linalg.norm(A))
    assert worst < 100 * eps
    # ranks are nested: a parent's rows are exactly its children's pivots
    for l in range(2, T.L):
        for b in range(T.nboxes(l)):
            want = np.concatenate([nn.piv[l + 1][c] for c in T.children(b)])
            assert np.array_equal(nn.rows[l][b], want)


@pytest.mark.parametrize("kind,d,n,leaf,eps", [(LOG2D, 2, 2048, 32, 1e-8),
                                               (INVR3D, 3, 1024, 16, 1e-6)])
def test_h2_matvec_vs_exact(kind, d, n, leaf, eps):
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1, 1, (n, d))
    T = Tree(pts, leaf)
    K = Kernel(kind, float(n))
    nn = NNCA(T, K, eps)
    x = rng.standard_normal((n, 2))
    y = h2.matvec(T, K, nn, x)
    A = K.dense(T.points)
    exact = A @ x
    # measure the far-field error against the far-field part alone
    Aoff = A - np.diag(np.diag(A))
    err = np.linalg.norm(y - exact) / np.linalg.norm(Aoff @ x)
    assert err < 100 * eps
