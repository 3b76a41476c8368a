"""Uniform 2^d tree, neighbours, interaction lists and colours (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
* Sec. 2.1: the domain Omega is the smallest hypercube holding every point;
  level 0 is Omega and each box at level l splits into 2^d children.
* The depth L (Sec. 2.1 and Algorithm 2).  The paper states L through the
  leaf occupancy (strictly below n_max in Algorithm 2, at most n_max in
  Sec. 2.1).  Reading used here: the average-occupancy rule
  L = max(2, smallest l with (2^d)^l * n_max >= N); ``depth_rule='max'``
  gives the literal maximum-occupancy rule.
* Fig. 1: level-1 numbering is Z order with x as the low bit.  Boxes at
  every level are numbered in Morton (Z) order, which is also the order in
  which the paper-order elimination visits them.
* Sec. 2.2, eq. (adm_condn) with eta = sqrt(d): on a uniform tree two boxes of
  one level are admissible exactly when they do not touch (a shared vertex
  counts as touching).  Table (Notations1b): N(i) = the non-admissible boxes
  of the level (i included); IL(i) = children of N(parent(i)) that are not in
  N(i).

Points are mapped to leaf cells with half-open cells, the last cell closed:
c = min(floor(((p - lo) * n) / side), n - 1) with n = 2^L.

Pins (tests/test_oracle_tree.py): brute-force geometric admissibility on the
box geometry, partition of the points, colour classes with disjoint
neighbourhoods.
"""
from __future__ import annotations

import numpy as np


def depth_for(n: int, dim: int, leaf: int, rule: str = "average", cells=None) -> int:
    """Tree depth L (see module header)."""
    if rule == "average":
        L = 2
        while (1 << (dim * L)) * leaf < n:
            L += 1
        return L
    if rule == "max":
        # smallest L >= 2 with every leaf holding fewer than n_max points;
        # ``cells`` is a function L -> occupancy array
        L = 2
        while cells(L).max() >= leaf:
            L += 1
        return L
    raise ValueError(rule)


def morton(coords: np.ndarray, bits: int) -> np.ndarray:
    """Interleave integer cell coordinates (.., d) into Morton keys; x is the
    lowest bit (Fig. 1, level 1: 0=(0,0), 1=(1,0), 2=(0,1), 3=(1,1))."""
    coords = np.asarray(coords, dtype=np.int64)
    d = coords.shape[-1]
    key = np.zeros(coords.shape[:-1], dtype=np.int64)
    for b in range(bits):
        for k in range(d):
            key |= ((coords[..., k] >> b) & 1) << (b * d + k)
    return key


def demorton(key: np.ndarray, d: int, bits: int) -> np.ndarray:
    key = np.asarray(key, dtype=np.int64)
    out = np.zeros(key.shape + (d,), dtype=np.int64)
    for b in range(bits):
        for k in range(d):
            out[..., k] |= ((key >> (b * d + k)) & 1) << b
    return out


class Tree:
    """The tree T^L over a point set (sources = targets, Sec. 4)."""

    def __init__(self, points: np.ndarray, leaf: int, depth_rule: str = "average", depth: int | None = None):
        pts = np.asarray(points, dtype=np.float64)
        self.N, self.d = pts.shape
        self.lo = pts.min(axis=0)
        self.side = float((pts.max(axis=0) - self.lo).max())
        if not self.side > 0.0:
            raise ValueError("degenerate point set (zero extent)")

        def cells(L):
            n = 1 << L
            c = np.floor(((pts - self.lo) * n) / self.side).astype(np.int64)
            c = np.minimum(c, n - 1)
            key = morton(c, L)
            return np.bincount(key, minlength=1 << (self.d * L))

        # depth: the rule of Sec. 2.1 (reading R0), or a depth fixed by the
        # caller (to reach pivot blocks of a given size in tests)
        self.L = int(depth) if depth else depth_for(self.N, self.d, leaf, depth_rule, cells)
        L = self.L
        n = 1 << L
        c = np.floor(((pts - self.lo) * n) / self.side).astype(np.int64)
        c = np.minimum(c, n - 1)
        self.leaf_key = morton(c, L)
        # tree order: stable sort by leaf Morton key (ties by original index)
        self.perm = np.argsort(self.leaf_key, kind="stable")
        self.points = pts[self.perm]          # points in tree order
        sorted_keys = self.leaf_key[self.perm]
        # per level: box b covers tree positions [start[l][b], start[l][b+1])
        self.start = {}
        for l in range(L + 1):
            nb = 1 << (self.d * l)
            keys_l = sorted_keys >> (self.d * (L - l))
            self.start[l] = np.searchsorted(keys_l, np.arange(nb + 1))

    # ---- boxes -----------------------------------------------------------
    def nboxes(self, l: int) -> int:
        return 1 << (self.d * l)

    def coords(self, l: int, b: int) -> np.ndarray:
        return demorton(np.int64(b), self.d, l)

    def box(self, l: int, coords) -> int:
        return int(morton(np.asarray(coords, dtype=np.int64), l))

    def range(self, l: int, b: int):
        return int(self.start[l][b]), int(self.start[l][b + 1])

    def count(self, l: int, b: int) -> int:
        s, e = self.range(l, b)
        return e - s

    def parent(self, b: int) -> int:
        return b >> self.d

    def children(self, b: int):
        return [(b << self.d) + k for k in range(1 << self.d)]

    def _in_grid(self, l, c):
        n = 1 << l
        return all(0 <= x < n for x in c)

    # ---- Sec. 2.2 lists -----------------------------------------------------
    def neighbours(self, l: int, b: int):
        """N(b): boxes of level l touching b, b included; Morton order."""
        c = self.coords(l, b)
        out = []
        for off in np.ndindex(*(3,) * self.d):
            q = c + np.array(off) - 1
            if self._in_grid(l, q):
                out.append(self.box(l, q))
        return sorted(out)

    def interaction_list(self, l: int, b: int):
        """IL(b): children of N(parent(b)) not in N(b) (empty for l < 2)."""
        if l < 2:
            return []
        near = set(self.neighbours(l, b))
        out = []
        for P in self.neighbours(l - 1, self.parent(b)):
            for c in self.children(P):
                if c not in near:
                    out.append(c)
        return sorted(out)

    def is_neighbour(self, l: int, a: int, b: int) -> bool:
        return int(np.abs(self.coords(l, a) - self.coords(l, b)).max()) <= 1

    def colour(self, l: int, b: int) -> int:
        """Distance-2 colour: boxes of one colour have disjoint N(.)."""
        c = self.coords(l, b)
        return int(sum(int(c[k] % 3) * 3 ** k for k in range(self.d)))

    def order(self, l: int, mode: str):
        """Elimination order e_1.. e_{2^{dl}} of level l.  'paper': Morton
        order; 'colour': by colour, Morton order within a colour."""
        boxes = list(range(self.nboxes(l)))
        if mode == "paper":
            return boxes
        if mode == "colour":
            return sorted(boxes, key=lambda b: (self.colour(l, b), b))
        raise ValueError(mode)
