"""NNCA: nested cross approximation operators (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed (Sec. 2.3):
* eq. (NCA): A_{tX sY} ~ A_{tX s^{X,i}} (A_{t^{X,i} s^{X,i}})^-1
  A_{t^{X,i} s^{Y,o}} (A_{t^{Y,o} s^{Y,o}})^-1 A_{t^{Y,o} sY}, with
  t^{X,i} a subset of t^X and s^{X,i} a subset of the far field F^{X,i}.
* eqs. (Fj)/(Fi): the far-field search space of X is the set of points in
  the boxes of IL(X).
* The operator list after eq. (Fi) and Table 2: leaf L2P
  U_B = A_{tB s^{B,i}} (A_{t^{B,i} s^{B,i}})^-1, L2L
  U^dag_B = A_{t^{B,i} s^{P,i}} (A_{t^{P,i} s^{P,i}})^-1, M2L
  A_BD = A_{t^{B,i} s^{D,o}}, P2M/M2M the V-side counterparts.
* eq. (particleAtNonLeafLevel) and Table (Notations2_2): at a non-leaf box
  the "particles" are the children's multipoles, so the rows searched by the
  parent are the children's incoming row pivots, and U_P stacked over the
  children is [U^dag_c]; this makes the bases nested.

Readings where the paper is silent (it defers the pivot search to its NNCA
reference):
* Pivots are found by adaptive cross approximation with partial pivoting
  (ACA) on A[rows(B), F^{B,i}]: start at row 0; the column pivot is the
  largest residual entry of the current row (lowest index on ties); the next
  row is the largest entry of the residual column among unused rows; stop at
  the first term with |u_k||v_k| <= eps ||S_k||_F (S_k the running
  approximation including that term, its Frobenius norm updated exactly);
  that small term is not kept.  The rank is at most min(rows, cols).
* The kernels in scope are symmetric with sources = targets, so the outgoing
  pivots are the incoming ones with roles swapped: t^{B,o} = s^{B,i},
  s^{B,o} = t^{B,i}.  Then V_B = U_B and A_BD = A_{t^{B,i} t^{D,i}}.

Parity: pinned by (i) the low-rank error of every admissible block against
the dense block, (ii) the H^2 product against the exact product (tests
tests/test_oracle_nnca.py); the exact pivot sequence is "parity unpinned"
against the paper's own code, which is not available.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def aca(evalrow, evalcol, nr: int, nc: int, eps: float, trace: list | None = None):
    """ACA with partial pivoting.  Returns (pivot_rows, pivot_cols).

    ``trace`` (a list, optional) receives one record per step with the
    quantities each decision was taken on: the masked |residual row| from
    which the column pivot was picked and the magnitude of the unreduced row
    (the scale of its rounding), the two sides of the stopping test, and the
    masked |residual column| from which the next row was picked with the
    magnitude of the unreduced column.  Recording changes no arithmetic."""
    us, vs, prow, pcol = [], [], [], []
    if nr == 0 or nc == 0:
        return prow, pcol
    used_r = np.zeros(nr, dtype=bool)
    used_c = np.zeros(nc, dtype=bool)
    frob2 = 0.0
    i = 0
    kmax = min(nr, nc)
    while len(us) < kmax:
        row = np.array(evalrow(i), dtype=np.float64)
        for u, v in zip(us, vs):
            row -= u[i] * v
        used_r[i] = True
        a = np.abs(row)
        a[used_c] = -1.0
        j = int(np.argmax(a))
        if not a[j] > 0.0:
            rest = np.flatnonzero(~used_r)
            if rest.size == 0:
                break
            i = int(rest[0])
            continue
        v = row / row[j]
        u = np.array(evalcol(j), dtype=np.float64)
        rec = None
        if trace is not None:
            rec = {"row": i, "col": j, "row_abs": a.copy(),
                   "row_scale": float(np.abs(np.array(evalrow(i), dtype=np.float64)).max()),
                   "col_scale": float(np.abs(u).max())}
            trace.append(rec)
        for uu, vv in zip(us, vs):
            u -= vv[j] * uu
        cross = 0.0
        for uu, vv in zip(us, vs):
            cross += (uu @ u) * (vv @ v)
        nu, nv = float(np.linalg.norm(u)), float(np.linalg.norm(v))
        frob2 += 2.0 * cross + (nu * nv) ** 2
        if rec is not None:
            rec["stop_lhs"], rec["stop_rhs"] = nu * nv, eps * np.sqrt(max(frob2, 0.0))
        if nu * nv <= eps * np.sqrt(max(frob2, 0.0)):
            if rec is not None:
                rec["stopped"] = True
            break                      # the small term is not kept
        us.append(u)
        vs.append(v)
        prow.append(i)
        pcol.append(j)
        used_c[j] = True
        a = np.abs(u)
        a[used_r] = -1.0
        i = int(np.argmax(a))
        if rec is not None:
            rec["col_abs"] = a.copy()
        if a[i] < 0.0:
            break
    return prow, pcol


class NNCA:
    """Operators of every box at levels 2..L.

    For box b at level l (tree positions are point indices):
      rows[l][b]  -- the row index set of the box: its points (leaf) or the
                     concatenated incoming pivots of its children (Morton
                     order of children), i.e. the box's "particles";
      piv[l][b]   -- t^{b,i}, a subset of rows[l][b];
      far[l][b]   -- s^{b,i};
      U[l][b]     -- A_{rows, s^{b,i}} (A_{t^{b,i} s^{b,i}})^-1, len(rows) x r.
    """

    def __init__(self, tree, kernel, eps: float):
        self.tree, self.kernel, self.eps = tree, kernel, eps
        T = tree
        pts = T.points
        self.rows, self.piv, self.far, self.U, self.rank = {}, {}, {}, {}, {}
        for l in range(T.L, 1, -1):
            self.rows[l], self.piv[l], self.far[l], self.U[l], self.rank[l] = {}, {}, {}, {}, {}
            for b in range(T.nboxes(l)):
                if l == T.L:
                    s, e = T.range(l, b)
                    rows = np.arange(s, e, dtype=np.int64)
                else:
                    parts = [self.piv[l + 1][c] for c in T.children(b)]
                    rows = np.concatenate(parts) if parts else np.zeros(0, np.int64)
                cols = [np.arange(*T.range(l, D), dtype=np.int64)
                        for D in T.interaction_list(l, b)]
                cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
                pr, pc = aca(lambda i: kernel.block(pts, rows[i:i + 1], cols)[0],
                             lambda j: kernel.block(pts, rows, cols[j:j + 1])[:, 0],
                             len(rows), len(cols), eps)
                tpiv = rows[np.array(pr, dtype=np.int64)]
                spiv = cols[np.array(pc, dtype=np.int64)]
                r = len(pr)
                if r > 0:
                    S = kernel.block(pts, tpiv, spiv)
                    C = kernel.block(pts, rows, spiv)
                    U = sla.solve(S.T, C.T).T
                else:
                    U = np.zeros((len(rows), 0))
                self.rows[l][b] = rows
                self.piv[l][b] = tpiv
                self.far[l][b] = spiv
                self.U[l][b] = U
                self.rank[l][b] = r

    def box_sets(self, l, b):
        """(rows, far-field columns) of box b at level l, as tree positions:
        the sets its pivots were searched in."""
        T = self.tree
        cols = [np.arange(*T.range(l, D), dtype=np.int64) for D in T.interaction_list(l, b)]
        cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
        return self.rows[l][b], cols

    def trace_box(self, l, b):
        """Re-run the pivot search of box b at level l and return its trace
        (see ``aca``); the operators are not touched."""
        rows, cols = self.box_sets(l, b)
        pts, kernel = self.tree.points, self.kernel
        tr = []
        aca(lambda i: kernel.block(pts, rows[i:i + 1], cols)[0],
            lambda j: kernel.block(pts, rows, cols[j:j + 1])[:, 0],
            len(rows), len(cols), self.eps, trace=tr)
        return rows, cols, tr

    def V(self, l, b):
        """P2M side; equals U for the symmetric kernels in scope."""
        return self.U[l][b]

    def m2l(self, l, b, d):
        """A_bd = A_{t^{b,i} s^{d,o}} with s^{d,o} = t^{d,i}."""
        return self.kernel.block(self.tree.points, self.piv[l][b], self.piv[l][d])

    def udag(self, l, c):
        """U^dag_c: rows of U_{parent(c)} belonging to child c (level l >= 3)."""
        T = self.tree
        P = T.parent(c)
        off = 0
        for cc in T.children(P):
            if cc == c:
                break
            off += self.rank[l][cc]
        return self.U[l - 1][P][off:off + self.rank[l][c], :]
