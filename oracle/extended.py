"""The extended sparse system A~ x~ = b~ as a dictionary of dense blocks.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed (Sec. 3.1):
* Table (Notations3): each box i at levels 2..L has particles x_i, multipoles
  y_i and locals z_i; eq. (particleAtNonLeafLevel): the particles of a
  non-leaf box are its children's multipoles.
* Equations Y_i: y_i = V_i^* x_i, and X_i: b_i = U_i z_i + sum_{j in N(i)}
  K_ij x_j (summary box, eqs. EquationY / EquationX); at a non-leaf level the
  right-hand side b_i is the stack of the children's locals (the equation
  after eq. EqXl2), i.e. the locals equation of each child c,
  z_c = U^dag_c z_{parent} + sum_{j in IL(c)} A_cj y_j (eq. EqXl).
* z^(1) = 0 (after eq. EqXl2) and the Remark of Sec. 3.1: no y, z at levels
  0 and 1, so level-2 boxes have no U^dag / V^dag.

Block keys.  Rows: ('X', b) the leaf equation X_b (one row per point of
leaf b), ('Y', l, b) equation Y_b, ('L', l, b) the locals equation of b.
Columns: ('x', b) the leaf particles, ('y', l, b) multipoles, ('z', l, b)
locals.  For a non-leaf box P at level l the paper's X_P rows are the keys
('L', l+1, c) of its children and its particles x_P are ('y', l+1, c): the
level transition of the paper is implicit in this indexing.

Signs: Y_b is written  V_b^T x_b - y_b = 0  and the locals equation as
-z_b + sum_j A_bj y_j + U^dag_b z_P = 0, so the pivot of box b is
[[K_bb, U_b], [V_b^T, 0]] with -I in (Y_b, y_b) and (L_b, z_b).

Parity: pinned by "eliminating the auxiliaries of the dense A~ reproduces the
dense H^2 matrix" (tests/test_oracle_extended.py).
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np


class BlockSystem:
    """Sparse matrix of dense blocks with row/column incidence sets."""

    def __init__(self):
        self.blk = {}
        self.rows = defaultdict(set)   # row key -> column keys present
        self.cols = defaultdict(set)   # column key -> row keys present
        self.rsize = {}
        self.csize = {}

    def get(self, rk, ck):
        return self.blk.get((rk, ck))

    def set(self, rk, ck, M):
        M = np.asarray(M, dtype=np.float64)
        assert M.shape == (self.rsize[rk], self.csize[ck]), (rk, ck, M.shape)
        self.blk[(rk, ck)] = M
        self.rows[rk].add(ck)
        self.cols[ck].add(rk)

    def add(self, rk, ck, M):
        old = self.blk.get((rk, ck))
        self.set(rk, ck, M if old is None else old + M)

    def pop(self, rk, ck):
        M = self.blk.pop((rk, ck), None)
        if M is not None:
            self.rows[rk].discard(ck)
            self.cols[ck].discard(rk)
        return M

    def dense(self, rkeys, ckeys):
        """Dense sub-matrix over the given key lists (missing blocks = 0)."""
        ro = np.cumsum([0] + [self.rsize[k] for k in rkeys])
        co = np.cumsum([0] + [self.csize[k] for k in ckeys])
        out = np.zeros((ro[-1], co[-1]))
        cidx = {k: n for n, k in enumerate(ckeys)}
        for i, rk in enumerate(rkeys):
            for ck in self.rows.get(rk, ()):
                j = cidx.get(ck)
                if j is not None:
                    out[ro[i]:ro[i + 1], co[j]:co[j + 1]] = self.blk[(rk, ck)]
        return out


def rowset(T, l, b):
    """Row keys of the paper's X_b at level l."""
    if l == T.L:
        return [("X", b)]
    return [("L", l + 1, c) for c in T.children(b)]


def colset(T, l, b):
    """Column keys of the paper's x_b at level l."""
    if l == T.L:
        return [("x", b)]
    return [("y", l + 1, c) for c in T.children(b)]


def assemble(T, K, nn):
    """Build A~ (Sec. 3.1) from the tree, kernel and NNCA operators.
    Returns the BlockSystem; keys of size 0 are omitted."""
    S = BlockSystem()
    L = T.L
    pts = T.points
    for b in range(T.nboxes(L)):
        m = T.count(L, b)
        if m:
            S.rsize[("X", b)] = m
            S.csize[("x", b)] = m
    for l in range(L, 1, -1):
        for b in range(T.nboxes(l)):
            r = nn.rank[l][b]
            if r:
                for k in (("Y", l, b), ("L", l, b)):
                    S.rsize[k] = r
                for k in (("y", l, b), ("z", l, b)):
                    S.csize[k] = r
    # leaf near field K_bq (eq. EquationX) and leaf operators
    for b in range(T.nboxes(L)):
        if not T.count(L, b):
            continue
        Ib = np.arange(*T.range(L, b))
        for q in T.neighbours(L, b):
            if T.count(L, q):
                S.set(("X", b), ("x", q), K.block(pts, Ib, np.arange(*T.range(L, q))))
    for l in range(L, 1, -1):
        for b in range(T.nboxes(l)):
            r = nn.rank[l][b]
            if not r:
                continue
            Ub = nn.U[l][b]
            Vb = nn.V(l, b)
            # z_b column in the X_b rows: U_b (leaf) or U^dag of each child
            off = 0
            for rk in rowset(T, l, b):
                n = S.rsize.get(rk, 0)
                if n:
                    S.set(rk, ("z", l, b), Ub[off:off + n])
                off += n
            off = 0
            for ck in colset(T, l, b):
                n = S.csize.get(ck, 0)
                if n:
                    S.set(("Y", l, b), ck, Vb[off:off + n].T)
                off += n
            S.set(("Y", l, b), ("y", l, b), -np.eye(r))
            S.set(("L", l, b), ("z", l, b), -np.eye(r))
            for d in T.interaction_list(l, b):
                if nn.rank[l][d]:
                    S.set(("L", l, b), ("y", l, d), nn.m2l(l, b, d))
    return S


def rhs_blocks(T, S, bvec):
    """b~ = [b; 0] in block form (eq. extendedMatrix): tree-ordered b."""
    bvec = np.asarray(bvec, dtype=np.float64)
    if bvec.ndim == 1:
        bvec = bvec[:, None]
    out = {}
    for k, n in S.rsize.items():
        out[k] = np.zeros((n, bvec.shape[1]))
    for b in range(T.nboxes(T.L)):
        if T.count(T.L, b):
            s, e = T.range(T.L, b)
            out[("X", b)] = bvec[s:e].copy()
    return out


def key_lists(S):
    """Row and column keys in a fixed order: the unknowns x first (so the
    dense A~ has A's layout in its leading N x N block)."""
    rk = sorted(S.rsize, key=lambda k: (k[0] != "X", k))
    ck = sorted(S.csize, key=lambda k: (k[0] != "x", k))
    return rk, ck
