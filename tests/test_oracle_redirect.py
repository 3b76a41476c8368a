"""Pin of one compress-and-redirect step of the oracle (Sec. 3.2.1-3.2.3,
Algorithm 2) against what it must preserve, for both groupings: all of a
box's fill-ins at once (reading R2) and pair by pair (Algorithm 2 as
printed).

Redirecting a box's pending well-separated fill-ins changes the extended
system's auxiliary unknowns (new bases U~_b, V~_b; the fill-ins moved into
the locals row and the multipole column) but not the operator that the
partially eliminated system applies to the particles still to be eliminated.
That operator is the Schur complement of every other unknown of the current
system, G = A_kk - A_ka A_aa^-1 A_ak, with k the particles x_q and equations
X_q of the uneliminated leaf boxes and a everything else.  So:

* with threshold 0 every direction of [U_b | fill-ins] is kept and the
  redirect is exact: G is unchanged to rounding;
* with threshold eps_A the discarded directions have R_kk <= eps_A times the
  largest column of the augmented matrix [U_b | fill-ins] (the relative
  residual of its RRQR, Sec. 3.2.1), so G changes by O(eps_A |[U | F]|),
  |[U | F]| the Frobenius norm of the bases and fill-ins that were
  compressed.

The diagonal is 20 rather than N so that the fill-ins are not negligible
against the rounding of G (with A_ii = N they are ~1e-12 of |G|).
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import factor as F
from oracle.extended import assemble, colset, rowset
from oracle.kernels import Kernel
from oracle.nnca import NNCA
from oracle.tree import Tree


def _reduced(S, keep_r, keep_c):
    rows = [k for k in S.rows if S.rows[k]]
    cols = [k for k in S.cols if S.cols[k]]
    ar = sorted(k for k in rows if k not in keep_r)
    ac = sorted(k for k in cols if k not in keep_c)
    Aaa = S.dense(ar, ac)
    assert Aaa.shape[0] == Aaa.shape[1]
    return S.dense(keep_r, keep_c) - S.dense(keep_r, ac) @ np.linalg.solve(Aaa, S.dense(ar, keep_c))


def _pending(S, T, l, b):
    rs = [k for k in rowset(T, l, b) if S.rsize.get(k, 0)]
    cs = [k for k in colset(T, l, b) if S.csize.get(k, 0)]
    wcols = sorted({ck for rk in rs for ck in S.rows[rk] if F._is_ws_col(T, l, b, ck)})
    wrows = sorted({rk for ck in cs for rk in S.cols[ck] if F._is_ws_row(T, l, b, rk)})
    return rs, cs, wcols, wrows


@pytest.fixture(scope="module")
def state():
    """Leaf level of a 2,048-point log-kernel problem (32 points per leaf
    box), eliminated in paper order up to the first box after the fourth
    that has pending fill-ins and more points than rank."""
    w = W.log2d(2048, seed=7, leaf=64, tol=1e-8, diag=20.0)
    pts, _ = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    nn = NNCA(T, Kernel(w.kernel, w.diag), w.tol)
    S = assemble(T, Kernel(w.kernel, w.diag), nn)
    L = T.L
    order = list(T.order(L, "paper"))
    done, target = [], None
    for i, b in enumerate(order):
        if i >= 4 and T.count(L, b) > nn.rank[L][b] + 2 and any(_pending(S, T, L, b)[2:]):
            target = b
            break
        F.compress_box(S, T, L, b, w.tol)
        F.eliminate(S, rowset(T, L, b) + [("Y", L, b)], colset(T, L, b) + [("z", L, b)], box=(L, b))
        done.append(b)
    assert target is not None
    live = [b for b in order if b not in done and T.count(L, b)]
    keep_r, keep_c = [("X", b) for b in live], [("x", b) for b in live]
    rs, cs, wcols, wrows = _pending(S, T, L, target)
    nF = float(np.hypot(np.linalg.norm(S.dense(rs, wcols)), np.linalg.norm(S.dense(wrows, cs))))
    zb, Yb = ("z", L, target), ("Y", L, target)
    nU = float(np.hypot(np.linalg.norm(S.dense(rs, [zb])), np.linalg.norm(S.dense([Yb], cs))))
    G0 = _reduced(S, keep_r, keep_c)
    return dict(S=S, T=T, L=L, b=target, m=T.count(L, target), keep=(keep_r, keep_c), G0=G0, nF=nF,
                nA=float(np.hypot(nF, nU)))


def _redirect(st, eps, grouping):
    S1 = copy.deepcopy(st["S"])
    if grouping == "box":
        F.compress_box(S1, st["T"], st["L"], st["b"], eps)
    else:
        F.compress_pairs(S1, st["T"], st["L"], st["b"], eps)
    dG = np.linalg.norm(_reduced(S1, *st["keep"]) - st["G0"])
    return dG, S1.csize[("z", st["L"], st["b"])]


@pytest.mark.parametrize("grouping", ["box", "pair"])
def test_exact_redirect_preserves_the_operator(state, grouping):
    dG, r = _redirect(state, 0.0, grouping)
    assert r <= state["m"]
    # a dropped, mis-signed or transposed redirect of the fill-ins changes G
    # by about |F|; rounding of G leaves ~1e-6 |F| here
    assert dG <= 1e-5 * state["nF"], (dG, state["nF"])


@pytest.mark.parametrize("grouping", ["box", "pair"])
def test_truncated_redirect_changes_the_operator_by_order_eps(state, grouping):
    eps = 1e-4
    d0, r0 = _redirect(state, 0.0, grouping)
    dG, r = _redirect(state, eps, grouping)
    assert r < r0                      # directions were discarded
    assert dG <= 10.0 * eps * state["nA"], (dG, eps * state["nA"])
    assert dG >= 10.0 * d0             # the truncation is visible above rounding
