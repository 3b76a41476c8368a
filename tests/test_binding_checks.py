"""The Python binding refuses, before any pointer reaches the library, a
buffer whose row count differs from the problem's N (the library reads N
rows of every vector it is given) and malformed points.  No GPU and no
library load needed: the checks run first."""
import numpy as np
import pytest

import paper_2301_12704_gb300 as A


def _handle(n=10):
    return A.Handle(None, n, 2)


def test_short_or_long_rhs_is_refused():
    h = _handle(10)
    for bad in (np.zeros((9, 1)), np.zeros((11, 2)), np.zeros(9)):
        with pytest.raises(ValueError, match="rows"):
            A.aifmm_solve(h, bad)
        with pytest.raises(ValueError, match="rows"):
            A.aifmm_matvec(h, bad)
        with pytest.raises(ValueError, match="rows"):
            A.aifmm_direct_matvec(h, bad)
    with pytest.raises(ValueError, match="rows"):
        A.aifmm_gmres(h, np.zeros(9))
    with pytest.raises(ValueError, match="rows"):
        A.aifmm_gmres(h, np.zeros((10, 2)))          # two columns flatten to 20 entries


def test_points_must_be_a_matrix():
    with pytest.raises(ValueError, match="N x dim"):
        A.aifmm_build(np.zeros(12), 0, 1.0, 1e-8, 16)
