"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Integer work (tree order, leaf ranges) must match
exactly; floating-point results within the stated tolerances."""
import numpy as np
import pytest

import workloads as W
from oracle import factor as OF
from oracle import h2 as OH
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


def _oracle(w, pts, order="colour"):
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag, w.length)
    nn = NNCA(T, K, w.tol)
    return T, K, nn


def _to_orig(T, xt):
    x = np.empty_like(xt)
    x[T.perm] = xt
    return x


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    W.log2d(1024, seed=11, leaf=16, tol=1e-10),
    W.log2d(1000, seed=12, leaf=16, tol=1e-8),      # ragged occupancy, L=3
    W.invr2d(1500, seed=13, leaf=24, tol=1e-10),
    W.gauss2d(900, seed=14, leaf=16, tol=1e-10),
    W.invr3d(512, seed=15, leaf=8, tol=1e-8),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_tree_and_nnca_match_oracle(A, w):
    pts, _ = W.points_and_rhs(w)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf, length=w.length)
    T, K, nn = _oracle(w, pts)
    perm, starts = A.aifmm_tree_perm(h)
    assert A.aifmm_levels(h) == T.L
    assert np.array_equal(perm, T.perm)                      # bit-exact
    assert np.array_equal(starts, T.start[T.L])
    same = 0
    total = 0
    for l in range(2, T.L + 1):
        r = A.aifmm_level_ranks(h, l, 0)
        ro = np.array([nn.rank[l][b] for b in range(T.nboxes(l))])
        total += len(ro)
        same += int((r == ro).sum())
    # pivots are floating-point decisions (argmax of residuals); allow a rare
    # near-tie to differ, but the bulk must be identical
    assert same >= 0.97 * total, (same, total)


_ORACLE_X = {}


def _oracle_solution(w, pts, b):
    """Oracle (colour order) and dense solutions of one case, computed once."""
    if w.name not in _ORACLE_X:
        T, K, nn = _oracle(w, pts)
        xo = _to_orig(T, OF.solve(OF.factor(T, K, nn, w.tol, order="colour"), b[T.perm]))
        _ORACLE_X[w.name] = (xo, np.linalg.solve(K.dense(pts), b))
    return _ORACLE_X[w.name]


@pytest.mark.parametrize("symmetric,mode", [(True, "mma"), (False, "mma"), (True, "fma"), (True, "tcgen05")],
                         ids=["sym", "general", "sym-fp64fma", "sym-tcgen05"])
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_factor_solve_matches_oracle(A, w, symmetric, mode):
    """Both elimination modes, and the Schur tiles on the warp MMAs, on
    tcgen05 or on FP64 FMAs, against the oracle's general elimination: they
    differ from it only by rounding and the RRQR cut-off, so the same 10 tol
    bound holds."""
    pts, b = W.points_and_rhs(w, nrhs=2)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf, length=w.length, symmetric=symmetric,
                      fma_gemm=mode == "fma", tcgen05=mode == "tcgen05")
    A.aifmm_factor(h)
    x = A.aifmm_solve(h, b)
    xo, xd = _oracle_solution(w, pts, b)
    assert _rel(x, xo) <= 10 * w.tol
    assert _rel(x, xd) <= 100 * w.tol


def test_h2_matvec_matches_oracle(A):
    w = CASES[0]
    pts, b = W.points_and_rhs(w, nrhs=3)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    y = A.aifmm_matvec(h, b)
    T, K, nn = _oracle(w, pts)
    yo = _to_orig(T, OH.matvec(T, K, nn, b[T.perm]))
    assert _rel(y, yo) < 1e-11
    yd = A.aifmm_direct_matvec(h, b)
    ye = K.dense(pts) @ b
    assert _rel(yd, ye) < 1e-13


def test_small_config_full_size(A):
    """The 4,096-point log-kernel configuration: GPU vs oracle within
    10 tol, and both against the dense LU solution."""
    w = W.SMALL
    pts, b = W.points_and_rhs(w)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    A.aifmm_factor(h)
    x = A.aifmm_solve(h, b)[:, 0]
    T, K, nn = _oracle(w, pts)
    xo = _to_orig(T, OF.solve(OF.factor(T, K, nn, w.tol, order="colour"), b[T.perm, 0]))
    rel = _rel(x, xo)
    assert rel <= 10 * w.tol, rel
    xd = np.linalg.solve(K.dense(pts), b[:, 0])
    assert _rel(x, xd) <= 1e-8


def test_state_and_argument_errors(A):
    w = CASES[0]
    pts, b = W.points_and_rhs(w)
    h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_solve(h, b)
    assert e.value.status == 4
    dup = pts.copy()
    dup[5] = dup[9]
    with pytest.raises(A.AifmmError) as e:
        A.aifmm_build(dup, w.kernel, w.diag, w.tol, w.leaf)
    assert e.value.status == 1
