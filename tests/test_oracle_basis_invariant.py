"""A box's basis changes only at its own compression (Sec. 3.2: the
compress-and-redirect step of box b rewrites U_b; eliminating another box q
updates blocks in q's coupled rows and columns, which never include the
column z_b).  So the basis a box's compression starts from is the one its
level started with, whichever colour step compresses it: the GPU factors
the Householder QR of every box's basis once per level on this basis.
Checked on the oracle, bit for bit, in colour and in paper order."""
import numpy as np
import pytest

import workloads as W
from oracle import factor as OF
from oracle.kernels import Kernel
from oracle.nnca import NNCA
from oracle.tree import Tree


@pytest.mark.parametrize("order", ["colour", "paper"])
def test_basis_at_compression_is_the_level_start_basis(order):
    w = W.log2d(1024, seed=3, leaf=16, tol=1e-8)
    pts, _ = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    assert T.L >= 3
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, w.tol)
    bases = {}
    fac = OF.factor(T, K, nn, w.tol, order=order, symmetric=True, bases=bases)
    checked = 0
    for (l, b), rec in fac.rrqr.items():
        U0 = bases[(l, b)]
        if rec["r_old"] == 0:
            assert U0 is None or U0.size == 0
            continue
        assert U0 is not None and np.array_equal(rec["U"], U0), (l, b)
        checked += 1
    # compressions happen on every level below the top and most boxes have a basis
    assert checked > 20
    assert len({l for (l, _) in fac.rrqr}) >= 2
