"""AIFMM elimination (Algorithm 2) and back substitution (Algorithm 3), oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
* Sec. 3.2: boxes are eliminated in a fixed order, level L first; eliminating
  box i removes x_i and z_i using equations X_i and Y_i (eqs. EquationX2,
  EquationY); the Schur complement creates the fill-ins of Table (Notations):
  P2P, M2P, P2L, M2L between the neighbours of i.
* Algorithm 2 (Sec. 3.5): a fill-in between well-separated boxes is first
  updated, and compressed and redirected once, just before either of its
  boxes is eliminated; M2L fill-ins between two eliminated boxes are added
  to the existing M2L with no compression.
* Sec. 3.2.1-3.2.3: compression by rank-revealing QR of the augmented
  [U_i | fill-in] (column side) and [V_j | fill-in^*] (row side), threshold
  eps_A; the assignments U_i := U~_i, V_j := V~_j, A_ij := L_i A_ij R_j^* +
  R~_ij^*, the other-M2L updates A_ic := L_i A_ic, A_dj := A_dj R_j^*, the
  M2M update V^dag*_j := V^dag*_j R_j^* and the L2L update U^dag_i := L_i
  U^dag_i.
* Algorithm 3 and the Remark after it (Sec. 3.6): the elimination is
  independent of the right-hand side; the solve replays the right-hand-side
  Schur operations in elimination order, solves for the level-2 multipoles
  directly and back-substitutes in reverse order.

How the oracle realises it.  The extended system is a block dictionary
(``extended``).  Eliminating box b at level l is one step of plain block
Gaussian elimination: pivot rows = X_b-rows + Y_b, pivot columns = x_b-cols
+ z_b; every row holding a block in a pivot column and every column holding a
block in a pivot row is updated by  S[R,C] -= A[R,piv] Piv^-1 A[piv,C]
(LU with partial pivoting of the pivot block).  Fill-ins are simply the
blocks this creates.  Nothing is skipped: the coupled rows and columns are
read from the incidence sets, so with compression switched off the routine
is an exact sparse LU of A~ (pinned against a dense solve of A~).

Readings where the paper is silent or ambiguous:
* R1 order: 'paper' = Morton order within a level; 'colour' = distance-2
  colour classes (Morton order inside a class).  Boxes of one colour have
  disjoint neighbourhoods, so they commute.
* R2 grouping ('box'): just before box b is eliminated, ALL pending
  well-separated fill-ins touching b are compressed at once, one RRQR per
  side: [U_b | row fill-ins of X_b] and [V_b | column fill-ins of x_b]^*.
  A P2P_bq fill-in (q not yet eliminated) is compressed on b's row side now;
  its row space L~_bq lands in the locals row of b as a P2L_bq fill-in that
  is compressed on q's column side just before q is eliminated (and
  symmetrically for P2P_qb).  In exact arithmetic this is the same
  redirection as the paper's two-sided P2P formula, split over the two
  boxes' steps.
  Grouping 'pair' is Algorithm 2 as printed: before box i is eliminated,
  each pending vP2P pair (i, q) has P2P_iq and P2P_qi compressed on both of
  their boxes into the M2Ls A_iq, A_qi (Sec. 3.2.1), and each vP2L pair
  (r, i) has P2L_ri and M2P_ir compressed on i's sides into A_ri, A_ir
  (Secs. 3.2.2, 3.2.3); pairs in ascending partner order, ranks equalised
  (R4) per box after each pair.  Both groupings are pinned against the
  uncompressed elimination and against each other.
* R3 RRQR: Householder QR with column pivoting in which the existing basis
  columns U_b are taken first, in order (so U_b = U~_b L_b holds to rounding,
  as the paper's eq. P2P_2a requires), followed by pivoting on the largest
  residual column norm among the fill-in columns; fill-in directions are kept
  while |R_kk| > eps_A * max_j ||[U_b | F]_:j||: the paper asks for a
  relative residual O(eps_A) of the decomposition of the augmented matrix
  [U_b | F] (Sec. 3.2.1), so the scale is that of the augmented matrix, basis
  columns included.  (Measured against the fill-in columns alone, fill-ins
  that are rounding noise next to the basis -- A_ii = N makes them ~1e-17 of
  it -- were kept to ten digits of their own size: ranks followed the
  rounding.)
* R4 equal ranks: the pivot [[K, U],[V^T, 0]] is square only if U_b and V_b
  have equal column counts; both sides keep r' = max(r'_U, r'_V) columns.
  The smaller side is extended by the other side's extra basis columns,
  orthogonalised against its own (taking its own next QRCP columns instead
  can leave V^T U, hence S, nearly singular).
* R5 singular pivot: LU with partial pivoting; the pivot is singular when some
  |u_kk| <= 1e-14 times the largest entry of column k of the pivot block (a
  column-relative test: the block mixes K, of the size of A, with the
  orthonormal U and V).

Parity: pinned by (i) compression off == dense solve of A~ to 1e-12;
(ii) compression on with eps_A -> 0 == dense solve of A to 1e-12;
(iii) error against the dense solution falls with eps_A; (iv) paper order
and colour order agree to a small multiple of eps_A; (v) both groupings stay
within eps_A of the uncompressed elimination (tests/test_oracle_factor.py);
(vi) one compress-and-redirect step leaves the Schur complement onto the
uneliminated particles unchanged at threshold 0 and changes it by
O(eps_A |F|) at eps_A (tests/test_oracle_redirect.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .extended import BlockSystem, assemble, colset, rhs_blocks, rowset


class SingularPivot(RuntimeError):
    pass


def qrcp_forced(M: np.ndarray, nf: int):
    """Householder QR with column pivoting, first ``nf`` columns unpivoted.

    Returns (Q, rdiag): Q is the m x m orthogonal product of the reflectors
    (M P = Q R) and rdiag[k] = |R_kk| for k < min(m, n)."""
    A = np.array(M, dtype=np.float64, copy=True)
    m, n = A.shape
    Q = np.eye(m)
    rdiag = []
    for k in range(min(m, n)):
        if k >= nf:
            norms = np.linalg.norm(A[k:, k:], axis=0)
            j = k + int(np.argmax(norms))
            if j != k:
                A[:, [k, j]] = A[:, [j, k]]
        x = A[k:, k]
        alpha = float(np.linalg.norm(x))
        rdiag.append(alpha)
        if alpha == 0.0:
            continue
        v = x.copy()
        v[0] += alpha if x[0] >= 0 else -alpha
        v /= np.linalg.norm(v)
        A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        Q[:, k:] -= 2.0 * np.outer(Q[:, k:] @ v, v)
    return Q, rdiag


def _colmax(M: np.ndarray) -> float:
    """Largest column 2-norm of M (0 for no columns)."""
    return float(np.linalg.norm(M, axis=0).max()) if M.shape[1] else 0.0


def rrqr_rank(rdiag, nf: int, tau: float) -> int:
    k = nf
    while k < len(rdiag) and rdiag[k] > tau:
        k += 1
    return k


def _equalise(Q, k, Qother, rn):
    """Reading R4: the first ``rn`` basis columns of one side.  A side whose
    own rank k is below rn is extended by the other side's columns k..rn-1,
    made orthogonal to its own k columns by a Householder QR with every column
    forced (so S = V^T K^-1 U keeps the other side's directions)."""
    if k >= rn:
        return Q[:, :rn]
    Qe, _ = qrcp_forced(np.hstack([Q[:, :k], Qother[:, k:rn]]), rn)
    return Qe[:, :rn]


class Factorization:
    """Result of ``factor``: the elimination steps (for the solve) and stats."""

    def __init__(self, tree, nn, eps, order, compress):
        self.tree, self.nn, self.eps = tree, nn, eps
        self.order, self.compress = order, compress
        self.steps = []
        self.ranks = {}          # (l, b) -> final rank r_b
        self.rrqr = {}           # (l, b) -> RRQR record of the box's compression (grouping 'box')
        self.ncompress = 0


def _is_ws_col(T, l, b, ck):
    if ck[0] == "x":
        return not T.is_neighbour(T.L, b, ck[1])
    if ck[0] == "y":
        lev, q = ck[1], ck[2]
        if lev == l + 1:
            return not T.is_neighbour(l, b, T.parent(q))
        if lev == l:
            return not T.is_neighbour(l, b, q)
    return False


def _is_ws_row(T, l, b, rk):
    if rk[0] == "X":
        return not T.is_neighbour(T.L, b, rk[1])
    if rk[0] == "L":
        lev, q = rk[1], rk[2]
        if lev == l + 1:
            return not T.is_neighbour(l, b, T.parent(q))
        if lev == l:
            return not T.is_neighbour(l, b, q)
    return False


def _ensure_aux(S, l, b):
    for k in (("Y", l, b), ("L", l, b)):
        S.rsize.setdefault(k, 0)
    for k in (("y", l, b), ("z", l, b)):
        S.csize.setdefault(k, 0)


def _resize(S, key, new, is_row):
    sizes = S.rsize if is_row else S.csize
    sizes[key] = new


def compress_box(S: BlockSystem, T, l: int, b: int, eps: float, symmetric: bool = False, log: dict | None = None):
    """Compress and redirect every pending well-separated fill-in of box b
    (reading R2): row side into U_b, column side into V_b.  ``symmetric``
    (reading R13, for A = A^T with V = U): the RRQR of the row side gives
    both new bases, V~_b = U~_b.  ``log`` (optional dict) receives, under
    (l, b), the row side's RRQR record: old rank, |R_kk| sequence, threshold,
    new rank and the basis U_b it started from (recording only)."""
    _ensure_aux(S, l, b)
    Yb, Lb, yb, zb = ("Y", l, b), ("L", l, b), ("y", l, b), ("z", l, b)
    rs = [k for k in rowset(T, l, b) if S.rsize.get(k, 0)]
    cs = [k for k in colset(T, l, b) if S.csize.get(k, 0)]
    m = sum(S.rsize[k] for k in rs)
    if m == 0:
        return 0
    r = S.csize[zb]
    assert S.rsize[Yb] == r
    # ---- gather: U_b, row fill-ins; V_b, column fill-ins
    U = S.dense(rs, [zb]) if r else np.zeros((m, 0))
    wcols = sorted({ck for rk in rs for ck in S.rows[rk] if _is_ws_col(T, l, b, ck)})
    Frow = S.dense(rs, wcols)
    V = S.dense([Yb], cs).T if r else np.zeros((m, 0))
    wrows = sorted({rk for ck in cs for rk in S.cols[ck] if _is_ws_row(T, l, b, rk)})
    Fcol = S.dense(wrows, cs).T
    if not wcols and not wrows:
        # nothing pending; the basis is kept as it is
        return 0
    # ---- RRQR on both sides (R3) and equal ranks (R4)
    QU, dU = qrcp_forced(np.hstack([U, Frow]), r)
    QV, dV = (QU, dU) if symmetric else qrcp_forced(np.hstack([V, Fcol]), r)
    tauU = eps * max(_colmax(U), _colmax(Frow))
    tauV = eps * max(_colmax(V), _colmax(Fcol))
    rU = rrqr_rank(dU, r, tauU)
    rV = rU if symmetric else rrqr_rank(dV, r, tauV)
    rn = max(rU, rV)
    if log is not None:
        log[(l, b)] = {"r_old": r, "rdiag": np.array(dU), "tau": tauU, "rank": rn, "m": m,
                       "ncols": Frow.shape[1], "partners": list(wcols), "U": U.copy()}
    assert rn <= m
    if rn == 0:
        # every fill-in column is exactly zero: drop them
        for ck in wcols:
            for rk in rs:
                S.pop(rk, ck)
        for rk in wrows:
            for ck in cs:
                S.pop(rk, ck)
        return 0
    Ut = _equalise(QU, rU, QV, rn)
    Vt = _equalise(QV, rV, QU, rn)
    Lmat, Lfill = Ut.T @ U, Ut.T @ Frow
    Rmat, Rfill = Vt.T @ V, Vt.T @ Fcol
    # ---- row side: locals row of b is multiplied by L_b; U_b := U~_b
    old_row = {ck: S.pop(Lb, ck) for ck in list(S.rows[Lb])}
    for rk in rs:
        S.pop(rk, zb)
    assert not S.cols[zb], "z_b column holds blocks outside X_b and its locals row"
    _resize(S, Lb, rn, True)
    _resize(S, zb, rn, False)
    for ck, M in old_row.items():
        if ck != zb:
            S.set(Lb, ck, Lmat @ M)
    S.set(Lb, zb, -np.eye(rn))
    off = 0
    for rk in rs:
        n = S.rsize[rk]
        S.set(rk, zb, Ut[off:off + n])
        off += n
    # redirected row fill-ins: M2P_br -> A_br += L~ ; P2P_bq -> P2L_bq := L~
    co = 0
    for ck in wcols:
        n = S.csize[ck]
        for rk in rs:
            S.pop(rk, ck)
        S.add(Lb, ck, Lfill[:, co:co + n])
        co += n
    # ---- column side: multipole column of b times R_b^T; V_b := V~_b
    old_col = {rk: S.pop(rk, yb) for rk in list(S.cols[yb])}
    for ck in cs:
        S.pop(Yb, ck)
    assert not S.rows[Yb], "Y_b row holds blocks outside x_b and y_b"
    _resize(S, yb, rn, False)
    _resize(S, Yb, rn, True)
    for rk, M in old_col.items():
        if rk != Yb:
            S.set(rk, yb, M @ Rmat.T)
    S.set(Yb, yb, -np.eye(rn))
    off = 0
    for ck in cs:
        n = S.csize[ck]
        S.set(Yb, ck, Vt[off:off + n].T)
        off += n
    ro = 0
    for rk in wrows:
        n = S.rsize[rk]
        for ck in cs:
            S.pop(rk, ck)
        S.add(rk, yb, Rfill[:, ro:ro + n].T)
        ro += n
    return rn - r


# ---- the paper's literal grouping: pair by pair (Algorithm 2, vP2P / vP2L) --

def _set_row_basis(S: BlockSystem, T, l: int, b: int, Ut: np.ndarray) -> np.ndarray:
    """U_b := Ut, whose orthonormal columns span the old U_b, so that
    U_b = Ut L_b with L_b = Ut^T U_b.  The locals row of b is multiplied by
    L_b: its M2Ls A_bc (the "other M2L" update of Sec. 3.2.1), its L2L
    U^dag_b (the L2L update) and any fill-in it holds.  Returns L_b."""
    _ensure_aux(S, l, b)
    Lb, zb = ("L", l, b), ("z", l, b)
    rs = [k for k in rowset(T, l, b) if S.rsize.get(k, 0)]
    m = sum(S.rsize[k] for k in rs)
    U = S.dense(rs, [zb]) if S.csize[zb] else np.zeros((m, 0))
    Lm = Ut.T @ U
    rn = Ut.shape[1]
    old_row = {ck: S.pop(Lb, ck) for ck in list(S.rows[Lb])}
    for rk in rs:
        S.pop(rk, zb)
    assert not S.cols[zb], "z_b column holds blocks outside X_b and its locals row"
    _resize(S, Lb, rn, True)
    _resize(S, zb, rn, False)
    for ck, M in old_row.items():
        if ck != zb:
            S.set(Lb, ck, Lm @ M)
    S.set(Lb, zb, -np.eye(rn))
    off = 0
    for rk in rs:
        n = S.rsize[rk]
        S.set(rk, zb, Ut[off:off + n])
        off += n
    return Lm


def _set_col_basis(S: BlockSystem, T, l: int, b: int, Vt: np.ndarray) -> np.ndarray:
    """V_b := Vt (orthonormal, spanning the old V_b: V_b = Vt R_b with
    R_b = Vt^T V_b).  The multipole column of b is multiplied by R_b^T: the
    M2Ls A_db (other M2L update), the parent's M2M V^dag*_b (M2M update) and
    any fill-in it holds.  Returns R_b."""
    _ensure_aux(S, l, b)
    Yb, yb = ("Y", l, b), ("y", l, b)
    cs = [k for k in colset(T, l, b) if S.csize.get(k, 0)]
    m = sum(S.csize[k] for k in cs)
    V = S.dense([Yb], cs).T if S.rsize[Yb] else np.zeros((m, 0))
    Rm = Vt.T @ V
    rn = Vt.shape[1]
    old_col = {rk: S.pop(rk, yb) for rk in list(S.cols[yb])}
    for ck in cs:
        S.pop(Yb, ck)
    assert not S.rows[Yb], "Y_b row holds blocks outside x_b and y_b"
    _resize(S, Yb, rn, True)
    _resize(S, yb, rn, False)
    for rk, M in old_col.items():
        if rk != Yb:
            S.set(rk, yb, M @ Rm.T)
    S.set(Yb, yb, -np.eye(rn))
    off = 0
    for ck in cs:
        n = S.csize[ck]
        S.set(Yb, ck, Vt[off:off + n].T)
        off += n
    return Rm


def _grow(Q0: np.ndarray, F: np.ndarray, eps: float) -> np.ndarray:
    """RRQR of [Q0 | F] with Q0's columns taken first (reading R3): the
    orthonormal basis of Q0 plus the directions of F kept above
    eps * max_j ||[Q0 | F]_:j||."""
    r = Q0.shape[1]
    Q, d = qrcp_forced(np.hstack([Q0, F]), r)
    tau = eps * max(_colmax(Q0), _colmax(F))
    return Q[:, :rrqr_rank(d, r, tau)]


def _row_basis(S, T, l, b):
    rs = [k for k in rowset(T, l, b) if S.rsize.get(k, 0)]
    zb = ("z", l, b)
    m = sum(S.rsize[k] for k in rs)
    return rs, (S.dense(rs, [zb]) if S.csize.get(zb, 0) else np.zeros((m, 0)))


def _col_basis(S, T, l, b):
    cs = [k for k in colset(T, l, b) if S.csize.get(k, 0)]
    Yb = ("Y", l, b)
    m = sum(S.csize[k] for k in cs)
    return cs, (S.dense([Yb], cs).T if S.rsize.get(Yb, 0) else np.zeros((m, 0)))


def compress_p2p(S: BlockSystem, T, l: int, i: int, j: int, eps: float) -> None:
    """Sec. 3.2.1 for the fill-in P2P_ij (x_j -> x_i, both boxes not yet
    eliminated): [U_i | P2P_ij] = U~_i [L_i | L~_ij], [V_j | L~_ij^*] =
    V~_j [R_j | R~_ij]; A_ij := L_i A_ij R_j^* + R~_ij^*, U_i := U~_i,
    V_j := V~_j, with the other M2L, M2M and L2L updates."""
    _ensure_aux(S, l, i)
    _ensure_aux(S, l, j)
    rs, U = _row_basis(S, T, l, i)
    cs, V = _col_basis(S, T, l, j)
    P = S.dense(rs, cs)
    if not rs or not cs or not np.any(P):
        return
    Ut = _grow(U, P, eps)
    Lt = Ut.T @ P
    Vt = _grow(V, Lt.T, eps)
    Rt = Vt.T @ Lt.T
    for rk in rs:
        for ck in cs:
            S.pop(rk, ck)
    _set_row_basis(S, T, l, i, Ut)
    _set_col_basis(S, T, l, j, Vt)
    S.add(("L", l, i), ("y", l, j), Rt.T)


def compress_p2l(S: BlockSystem, T, l: int, r: int, s: int, eps: float) -> None:
    """Sec. 3.2.2 for the fill-in P2L_rs (x_s -> locals of the eliminated
    box r): [V_s | P2L_rs^*] = V~_s [R_s | R~_rs]; A_rs := A_rs R_s^* +
    R~_rs^*, V_s := V~_s, with the other M2L and M2M updates."""
    _ensure_aux(S, l, s)
    cs, V = _col_basis(S, T, l, s)
    Lr = ("L", l, r)
    P = S.dense([Lr], cs) if S.rsize.get(Lr, 0) else np.zeros((0, V.shape[0]))
    if not np.any(P):
        return
    Vt = _grow(V, P.T, eps)
    Rt = Vt.T @ P.T
    for ck in cs:
        S.pop(Lr, ck)
    _set_col_basis(S, T, l, s, Vt)
    S.add(Lr, ("y", l, s), Rt.T)


def compress_m2p(S: BlockSystem, T, l: int, s: int, r: int, eps: float) -> None:
    """Sec. 3.2.3 for the fill-in M2P_sr (multipoles of the eliminated box
    r -> x_s): [U_s | M2P_sr] = U~_s [L_s | L~_sr]; A_sr := L_s A_sr +
    L~_sr, U_s := U~_s, with the other M2L and L2L updates."""
    _ensure_aux(S, l, s)
    rs, U = _row_basis(S, T, l, s)
    yr = ("y", l, r)
    P = S.dense(rs, [yr]) if S.csize.get(yr, 0) else np.zeros((U.shape[0], 0))
    if not np.any(P):
        return
    Ut = _grow(U, P, eps)
    Lt = Ut.T @ P
    for rk in rs:
        S.pop(rk, yr)
    _set_row_basis(S, T, l, s, Ut)
    S.add(("L", l, s), yr, Lt)


def equalise_box(S: BlockSystem, T, l: int, b: int) -> None:
    """Reading R4 after a pair's compression: the side with fewer basis
    columns is extended by the other side's extra columns, orthogonalised
    against its own."""
    _ensure_aux(S, l, b)
    rU, rV = S.csize[("z", l, b)], S.rsize[("Y", l, b)]
    if rU == rV:
        return
    _, U = _row_basis(S, T, l, b)
    _, V = _col_basis(S, T, l, b)
    if rU < rV:
        Q, _ = qrcp_forced(np.hstack([U, V[:, rU:rV]]), rV)
        _set_row_basis(S, T, l, b, Q[:, :rV])
    else:
        Q, _ = qrcp_forced(np.hstack([V, U[:, rV:rU]]), rU)
        _set_col_basis(S, T, l, b, Q[:, :rU])


def _partner(T, l: int, key):
    """The level-l box and the kind ('p2p': not yet eliminated, 'p2l':
    eliminated) behind a well-separated row or column key."""
    if key[0] in ("x", "X"):
        return "p2p", key[1]
    lev, q = key[1], key[2]
    if lev == l + 1:
        return "p2p", T.parent(q)
    return "p2l", q


def compress_pairs(S: BlockSystem, T, l: int, i: int, eps: float) -> int:
    """Algorithm 2 as printed: before box i is eliminated, every pending pair
    holding i is compressed and redirected -- first the vP2P pairs (i, q),
    both P2P_iq and P2P_qi, then the vP2L pairs (r, i), P2L_ri and M2P_ir.
    A pair is pending when its well-separated fill-in blocks exist (set
    semantics, reading R7); pairs are taken in ascending partner order."""
    _ensure_aux(S, l, i)
    rs = [k for k in rowset(T, l, i) if S.rsize.get(k, 0)]
    cs = [k for k in colset(T, l, i) if S.csize.get(k, 0)]
    found = set()
    for rk in rs:
        for ck in S.rows[rk]:
            if _is_ws_col(T, l, i, ck):
                found.add(_partner(T, l, ck))
    for ck in cs:
        for rk in S.cols[ck]:
            if _is_ws_row(T, l, i, rk):
                found.add(_partner(T, l, rk))
    for kind, q in sorted(found, key=lambda t: (t[0] != "p2p", t[1])):
        if kind == "p2p":
            compress_p2p(S, T, l, i, q, eps)
            compress_p2p(S, T, l, q, i, eps)
            equalise_box(S, T, l, q)
        else:
            compress_p2l(S, T, l, q, i, eps)
            compress_m2p(S, T, l, i, q, eps)
        equalise_box(S, T, l, i)
    return len(found)


class Step:
    __slots__ = ("PR", "PC", "lu", "rows", "ARP", "cols", "APC", "box")

    def __init__(self, PR, PC, lu, rows, ARP, cols, APC, box):
        self.PR, self.PC, self.lu = PR, PC, lu
        self.rows, self.ARP, self.cols, self.APC, self.box = rows, ARP, cols, APC, box


def eliminate(S: BlockSystem, PR, PC, box=None) -> Step:
    """One block Gaussian elimination step on pivot rows PR / columns PC."""
    PR = [k for k in PR if S.rsize.get(k, 0)]
    PC = [k for k in PC if S.csize.get(k, 0)]
    nr = sum(S.rsize[k] for k in PR)
    nc = sum(S.csize[k] for k in PC)
    if nr != nc:
        raise RuntimeError(f"non-square pivot {nr}x{nc} at {box}")
    if nr == 0:
        return None
    Piv = S.dense(PR, PC)
    lu = sla.lu_factor(Piv, check_finite=True)
    ud = np.abs(np.diag(lu[0]))
    colmax = np.abs(Piv).max(axis=0)
    if not np.all(ud > 1e-14 * colmax):
        raise SingularPivot(f"singular pivot at {box}")
    setR, setC = set(PR), set(PC)
    rows = sorted({rk for ck in PC for rk in S.cols[ck]} - setR)
    cols = sorted({ck for rk in PR for ck in S.rows[rk]} - setC)
    ARP = S.dense(rows, PC)
    APC = S.dense(PR, cols)
    if rows and cols:
        Z = sla.lu_solve(lu, APC)
        upd = ARP @ Z
        ro = np.cumsum([0] + [S.rsize[k] for k in rows])
        co = np.cumsum([0] + [S.csize[k] for k in cols])
        for i, rk in enumerate(rows):
            for j, ck in enumerate(cols):
                S.add(rk, ck, -upd[ro[i]:ro[i + 1], co[j]:co[j + 1]])
    for rk in PR:
        for ck in list(S.rows[rk]):
            S.pop(rk, ck)
    for ck in PC:
        for rk in list(S.cols[ck]):
            S.pop(rk, ck)
    return Step(PR, PC, lu, rows, ARP, cols, APC, box)


def factor(tree, kernel, nn, eps: float, order: str = "paper", compress: bool = True, grouping: str = "box",
           symmetric: bool = False, bases: dict | None = None):
    """Algorithm 2 on the extended system of (tree, kernel, nn).

    order    -- 'paper' or 'colour' (reading R1)
    compress -- False keeps every fill-in as a block (exact sparse LU of A~)
    grouping -- 'box': all of a box's pending fill-ins in one RRQR per side
                (reading R2, the GPU's form); 'pair': pair by pair, each
                P2P fill-in compressed on both of its boxes (Algorithm 2 as
                printed, Sec. 3.2.1-3.2.3)
    symmetric -- per-box grouping with one RRQR per box for both bases
                (reading R13; the kernel must be symmetric)
    bases    -- optional dict, filled with every box's basis U_b (its X_b x
                z_b block) as its level starts, keyed (l, b); None where the
                box has no basis yet (recording only)
    """
    T = tree
    S = assemble(T, kernel, nn)
    F = Factorization(T, nn, eps, order, compress)
    F.sizes_r, F.sizes_c = S.rsize, S.csize
    for l in range(T.L, 1, -1):
        if bases is not None:
            for b in T.order(l, order):
                zb = ("z", l, b)
                rs = [k for k in rowset(T, l, b) if S.rsize.get(k, 0)]
                bases[(l, b)] = S.dense(rs, [zb]) if S.csize.get(zb, 0) and rs else None
        for b in T.order(l, order):
            if compress and grouping == "pair":
                F.ncompress += compress_pairs(S, T, l, b, eps)
            elif compress:
                if compress_box(S, T, l, b, eps, symmetric=symmetric, log=F.rrqr):
                    F.ncompress += 1
            PR = rowset(T, l, b) + [("Y", l, b)]
            PC = colset(T, l, b) + [("z", l, b)]
            st = eliminate(S, PR, PC, box=(l, b))
            if st is not None:
                F.steps.append(st)
            F.ranks[(l, b)] = S.csize.get(("z", l, b), 0)
    # top: the level-2 locals equations in the level-2 multipoles, solved for
    # directly (Algorithm 3)
    PR = sorted(k for k in S.rows if S.rows[k] and k[0] == "L")
    PC = sorted(k for k in S.cols if S.cols[k] and k[0] == "y")
    leftover = [k for k in S.rows if S.rows[k] and k not in PR]
    assert not leftover, leftover
    st = eliminate(S, PR, PC, box=("top",))
    if st is not None:
        F.steps.append(st)
    F.S = S
    return F


def solve(F: Factorization, b_tree: np.ndarray) -> np.ndarray:
    """Forward sweep (right-hand-side Schur operations), top solve and back
    substitution (Algorithm 3).  ``b_tree`` is in tree order; returns x in
    tree order with the same number of columns."""
    T, S = F.tree, F.S
    b2 = np.asarray(b_tree, dtype=np.float64)
    squeeze = b2.ndim == 1
    if squeeze:
        b2 = b2[:, None]
    nrhs = b2.shape[1]
    rhs = rhs_blocks(T, S, b2)

    def get(key):
        v = rhs.get(key)
        if v is None:
            v = np.zeros((S.rsize.get(key, 0), nrhs))
            rhs[key] = v
        return v

    saved = []
    touched = set()
    for st in F.steps:
        if st.box is not None and len(st.box) == 2:
            # self-check: the locals row of a box receives its row transform
            # (compression) before any right-hand-side update reaches it
            assert ("L",) + tuple(st.box) not in touched, st.box
        touched.update(st.rows)
        rP = np.vstack([get(k) for k in st.PR])
        saved.append(rP)
        if st.rows:
            w = sla.lu_solve(st.lu, rP)
            upd = st.ARP @ w
            o = 0
            for rk in st.rows:
                n = S.rsize[rk]
                rhs[rk] = get(rk) - upd[o:o + n]
                o += n
    sol = {}
    for st, rP in zip(reversed(F.steps), reversed(saved)):
        if st.cols:
            xc = np.vstack([sol[ck] for ck in st.cols])
            rP = rP - st.APC @ xc
        v = sla.lu_solve(st.lu, rP)
        o = 0
        for ck in st.PC:
            n = S.csize[ck]
            sol[ck] = v[o:o + n]
            o += n
    x = np.zeros((T.N, nrhs))
    for b in range(T.nboxes(T.L)):
        if T.count(T.L, b):
            s, e = T.range(T.L, b)
            x[s:e] = sol[("x", b)]
    return x[:, 0] if squeeze else x
