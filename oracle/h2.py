"""NNCA H^2 matrix-vector product and its dense form (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed: eqs. (EquationY), (EqXl) and (EquationX) read as a
product (Sec. 3.1), with the operators of Sec. 2.3 (Table 2 and Table
Notations2_2):
  upward   y_b = V_b^* x_b at the leaf, y_P = sum_c V^dag*_c y_c above;
  M2L      z_b = sum_{d in IL(b)} A_bd y_d (+ U^dag_b z_parent, downward);
  leaf     (A x)_b = U_b z_b + sum_{j in N(b)} K_bj x_j.
The paper uses this product inside GMRES (Sec. 4, Experiments 2-4) and
defers its details to the NNCA reference; this is the textbook FMM sweep
over the operators defined there.

Parity: pinned against the exact dense product, error O(eps_A)
(tests/test_oracle_nnca.py); the dense H^2 matrix is pinned against the
dense solve of the extended system (tests/test_oracle_extended.py).
"""
from __future__ import annotations

import numpy as np


def matvec(T, K, nn, x_tree: np.ndarray) -> np.ndarray:
    """y = A_H2 x for x in tree order (N or N x k)."""
    x = np.asarray(x_tree, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    L = T.L
    pts = T.points
    ys = {}
    # upward pass
    for l in range(L, 1, -1):
        for b in range(T.nboxes(l)):
            r = nn.rank[l][b]
            if l == L:
                s, e = T.range(L, b)
                xb = x[s:e]
            else:
                xb = np.vstack([ys[(l + 1, c)] for c in T.children(b)]) if True else None
            ys[(l, b)] = nn.V(l, b).T @ xb if r else np.zeros((0, x.shape[1]))
    # M2L and downward pass
    zs = {}
    for l in range(2, L + 1):
        for b in range(T.nboxes(l)):
            r = nn.rank[l][b]
            z = np.zeros((r, x.shape[1]))
            for d in T.interaction_list(l, b):
                if r and nn.rank[l][d]:
                    z += nn.m2l(l, b, d) @ ys[(l, d)]
            if l > 2 and r:
                P = T.parent(b)
                if nn.rank[l - 1][P]:
                    z += nn.udag(l, b) @ zs[(l - 1, P)]
            zs[(l, b)] = z
    y = np.zeros_like(x)
    for b in range(T.nboxes(L)):
        s, e = T.range(L, b)
        if e == s:
            continue
        if nn.rank[L][b]:
            y[s:e] += nn.U[L][b] @ zs[(L, b)]
        for q in T.neighbours(L, b):
            qs, qe = T.range(L, q)
            if qe > qs:
                y[s:e] += K.block(pts, np.arange(s, e), np.arange(qs, qe)) @ x[qs:qe]
    return y[:, 0] if squeeze else y


def dense(T, K, nn) -> np.ndarray:
    """The H^2 matrix as a dense N x N array (tree order), tiny N only."""
    return matvec(T, K, nn, np.eye(T.N))
