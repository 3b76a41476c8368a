"""Parity at the benchmark's size: the 65,536-point 2D log-kernel problem
(uniform in [-1,1]^2, seed 1, A_ii = N, leaf 64, eps_A = 1e-10), built,
factored and solved the way bench.py does it (device buffers, the library on
a torch stream, nrhs = 1 and nrhs = 64).

The oracle cannot factor this size in a test, so the checks are the ones
that hold at any size:
* the tree order and leaf ranges equal the oracle's, bit for bit;
* the NNCA pivot sets of every box at every level equal the oracle's
  (Sec. 2.3), up to explained near-ties (see test_gpu_parity);
* the true residual (A x - b)_i on 256 sampled rows i, each row of A
  evaluated by the oracle's kernel on the CPU, is at most 1e-9 of b on those
  rows, for both right-hand-side counts (the method's error is O(eps_A)
  relative; the solve is a product with an approximate inverse whose error
  the residual bounds from above up to the condition number, about 1 here)."""
import numpy as np
import pytest

import workloads as W
from oracle.kernels import Kernel
from oracle.nnca import NNCA
from oracle.tree import Tree

from test_gpu_parity import _compare_pivots

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


def test_bench_configuration(A):
    import torch
    w = W.BENCH
    pts, b64 = W.points_and_rhs(w, nrhs=64)
    b1 = b64[:, :1].copy(order="F")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    pts_d = torch.from_numpy(pts).to(dev)
    b1_d = torch.from_numpy(np.asfortranarray(b1)).to(dev)
    b64_d = torch.from_numpy(b64.T.copy()).to(dev).t()
    with torch.cuda.stream(stream):
        h = A.aifmm_build(pts_d, w.kernel, w.diag, w.tol, w.leaf, stream=stream.cuda_stream)
        A.aifmm_factor(h)
        x1 = A.aifmm_solve(h, b1_d)
        x64 = A.aifmm_solve(h, b64_d)
    stream.synchronize()
    x1, x64 = x1.cpu().numpy(), x64.cpu().numpy()

    # index work, exactly
    T = Tree(pts, w.leaf)
    perm, starts = A.aifmm_tree_perm(h)
    assert A.aifmm_levels(h) == T.L == 5
    assert np.array_equal(perm, T.perm)
    assert np.array_equal(starts, T.start[T.L])
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, w.tol)
    equal, ties, inherited, _, notes = _compare_pivots(A, h, T, nn)
    total = equal + ties + inherited
    print(f"65,536 points: {equal}/{total} boxes with equal pivots, {ties} near-ties, {inherited} inherited; {notes}")
    assert equal >= 0.9 * total

    # true residual on sampled rows, rows of A from the oracle's kernel
    rng = np.random.default_rng(123)
    rows = np.sort(rng.choice(w.n, 256, replace=False))
    Arows = K.block(pts, rows, np.arange(w.n))
    for x, b, name in ((x1, b1, "nrhs=1"), (x64, b64, "nrhs=64")):
        r = Arows @ x - b[rows]
        rel = float(np.linalg.norm(r) / np.linalg.norm(b[rows]))
        print(f"{name}: sampled-row residual {rel:.3e}")
        assert rel <= 1e-9, (name, rel)
    # every column of the 64-column solve equals the single-column solve's
    # operator applied to that column: column 0 against the nrhs=1 result
    assert float(np.linalg.norm(x64[:, 0] - x1[:, 0]) / np.linalg.norm(x1[:, 0])) <= 1e-12
    A.aifmm_destroy(h)
