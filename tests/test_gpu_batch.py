"""Many independent problems of uneven size driven concurrently (one handle
and stream each, paper_2301_12704_gb300.batch): each solution equals the one
computed alone, and matches the oracle on the smallest problem."""
import numpy as np
import pytest

import workloads as W
from oracle import factor as OF
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


def test_concurrent_problems_equal_alone(A):
    from paper_2301_12704_gb300 import batch as B
    probs = W.batched_problems(seed=5, count=6, n_lo=600, n_hi=2500)
    xs, m = B.factor_solve_many(probs, workers=3)
    assert m["problems"] == 6
    for (w, p, b), x in zip(probs, xs):
        h = A.aifmm_build(p, w.kernel, w.diag, w.tol, w.leaf, length=w.length)
        A.aifmm_factor(h)
        xa = A.aifmm_solve(h, b)
        A.aifmm_destroy(h)
        assert np.linalg.norm(x - xa) <= 1e-14 * np.linalg.norm(xa)
    # the smallest against the oracle (10 tol) and the dense solution
    w, p, b = min(probs, key=lambda t: len(t[1]))
    x = xs[[len(t[1]) for t in probs].index(len(p))][:, 0]
    T = Tree(p, w.leaf)
    K = Kernel(w.kernel, w.diag, w.length)
    nn = NNCA(T, K, w.tol)
    xt = OF.solve(OF.factor(T, K, nn, w.tol, order="colour"), b[T.perm, 0])
    xo = np.empty_like(xt)
    xo[T.perm] = xt
    assert np.linalg.norm(x - xo) <= 10 * w.tol * np.linalg.norm(xo)
