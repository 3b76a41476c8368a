"""Pins of the oracle's tree, lists and colours (Sec. 2.1-2.2) against the
geometry itself: brute-force admissibility, point partition, Fig. 1."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.tree import Tree, demorton, depth_for, morton

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_fig1_level1_numbering():
    """Fig. 1 (Sec. 2.1): level-1 boxes 0..3 are BL, BR, TL, TR."""
    rows = [l.split() for l in open(os.path.join(GOLD, "fig1_numbering.txt"))
            if l.strip() and not l.startswith("#")]
    for lev, ix, iy, num in (map(int, r) for r in rows):
        assert morton(np.array([ix, iy]), max(lev, 1)) == num
        if lev:
            assert tuple(demorton(np.int64(num), 2, lev)) == (ix, iy)


@pytest.mark.parametrize("n,d,leaf,L", [(4096, 2, 64, 3), (65536, 2, 64, 5),
                                        (262144, 3, 64, 4), (1000, 2, 64, 2),
                                        (100, 2, 64, 2), (4097, 2, 64, 4)])
def test_depth_average_rule(n, d, leaf, L):
    assert depth_for(n, d, leaf) == L


def test_partition_and_ranges():
    w = W.log2d(3000, seed=5, leaf=16)
    pts, _ = W.points_and_rhs(w)
    T = Tree(pts, 16)
    assert sorted(T.perm.tolist()) == list(range(3000))
    n = 1 << T.L
    for l in range(T.L + 1):
        st = T.start[l]
        assert st[0] == 0 and st[-1] == 3000 and np.all(np.diff(st) >= 0)
        side = T.side / (1 << l)
        for b in range(T.nboxes(l)):
            s, e = T.range(l, b)
            c = T.coords(l, b)
            lo = T.lo + c * side
            P = T.points[s:e]
            # every point of box b lies in its closed cell
            assert np.all(P >= lo - 1e-12) and np.all(P <= lo + side + 1e-12)
            # children partition the parent
            if l < T.L:
                ch = T.children(b)
                assert T.range(l + 1, ch[0])[0] == s and T.range(l + 1, ch[-1])[1] == e
    # stable within a leaf: original indices increase
    for b in range(T.nboxes(T.L)):
        s, e = T.range(T.L, b)
        assert np.all(np.diff(T.perm[s:e]) > 0)


def _adm_bruteforce(l, a, qs, d):
    """eq. (adm_condn), eta = sqrt(d), on the exact box geometry in units of
    the box side h: diam = sqrt(d) h, dist = Euclidean gap between the cubes.
    Vectorised over the boxes ``qs``."""
    ca = demorton(np.int64(a), d, l)
    cq = demorton(np.asarray(qs, dtype=np.int64), d, l)
    gap = np.maximum(np.abs(cq - ca) - 1, 0)          # per-axis gap in units h
    dist2 = (gap ** 2).sum(axis=-1)
    # max(diam) <= eta * dist  <=>  d <= d * dist^2   (squares, integers)
    return d <= d * dist2


@pytest.mark.parametrize("d,L", [(2, 4), (3, 3)])
def test_lists_match_geometric_admissibility(d, L):
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1, 1, ((1 << (d * L)) * 2, d))
    T = Tree(pts, 2)
    assert T.L == L
    for l in range(2, L + 1):
        nb = T.nboxes(l)
        qs = np.arange(nb)
        sample = range(nb) if nb <= 64 else rng.choice(nb, 48, replace=False)
        for b in sample:
            N = set(T.neighbours(l, b))
            IL = set(T.interaction_list(l, b))
            assert b in N and not (N & IL)
            adm = _adm_bruteforce(l, b, qs, d)
            par_near = ~_adm_bruteforce(l - 1, b >> d, qs >> d, d)
            assert set(qs[~adm].tolist()) == N
            assert set(qs[adm & par_near].tolist()) == IL
            assert len(N) <= 3 ** d and len(IL) <= 6 ** d - 3 ** d and IL


@pytest.mark.parametrize("d,L", [(2, 4), (3, 3)])
def test_colour_classes_have_disjoint_neighbourhoods(d, L):
    rng = np.random.default_rng(2)
    T = Tree(rng.uniform(0, 1, ((1 << (d * L)), d)), 1)
    assert T.L == L
    for l in range(2, L + 1):
        classes = {}
        for b in range(T.nboxes(l)):
            classes.setdefault(T.colour(l, b), []).append(b)
        assert len(classes) == min(3, 1 << l) ** d
        for members in classes.values():
            # pairwise disjoint  <=>  the union is as large as the sum
            nbrs = [T.neighbours(l, a) for a in members]
            assert len(set().union(*nbrs)) == sum(len(x) for x in nbrs)
        order = T.order(l, "colour")
        assert sorted(order) == list(range(T.nboxes(l)))
