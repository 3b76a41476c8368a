"""Seeded synthetic inputs for the AIFMM workloads.

This module is shared by the FP64 oracle and by the CUDA path.  It draws
random numbers and names workloads; it holds none of the method's
arithmetic (no tree, no kernel evaluation, no factorisation).

Recipe (the paper's experiments all use synthetic inputs, Sec. 4): the
points are i.i.d. uniform in a box, drawn with numpy's PCG64
``default_rng(seed)`` as one ``uniform(lo, hi, (N, d))`` call; the
right-hand sides are drawn afterwards from the same generator as
``standard_normal((nrhs, N))`` and transposed, so that column k of an
nrhs-column draw is the k-th block of N normals (the nrhs=1 draw is the
first column of the nrhs=64 draw).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# kernel kinds, in the order of the C-ABI enum
LOG2D, INVR3D, INVR2D, GAUSS = 0, 1, 2, 3
KERNEL_NAMES = {LOG2D: "log2d", INVR3D: "invr3d", INVR2D: "invr2d", GAUSS: "gauss"}


@dataclass
class Workload:
    name: str
    n: int
    dim: int
    lo: float
    hi: float
    seed: int
    kernel: int
    diag: float            # value of A_ii
    leaf: int              # n_max, target points per leaf box
    tol: float             # NNCA / RRQR tolerance eps_A
    nrhs: int = 1
    length: float = 1.0    # Gaussian length scale
    extra: dict = field(default_factory=dict)


def points_and_rhs(w: Workload, nrhs: int | None = None):
    """Return (points (N, d) float64, rhs (N, nrhs) float64) for workload w."""
    k = w.nrhs if nrhs is None else nrhs
    rng = np.random.default_rng(w.seed)
    pts = rng.uniform(w.lo, w.hi, (w.n, w.dim))
    b = rng.standard_normal((k, w.n)).T.copy()
    return np.ascontiguousarray(pts), np.asfortranarray(b)


def log2d(n: int, seed: int, leaf: int = 64, tol: float = 1e-10, nrhs: int = 1,
          diag: float | None = None) -> Workload:
    """2D log kernel A_ij = log|x_i - x_j|, A_ii = N (the diagonal of the
    2D benchmark configurations), points uniform in [-1,1]^2."""
    return Workload(f"log2d_N{n}", n, 2, -1.0, 1.0, seed, LOG2D,
                    float(n) if diag is None else diag, leaf, tol, nrhs)


def invr2d(n: int, seed: int, leaf: int = 64, tol: float = 1e-10, nrhs: int = 1) -> Workload:
    """2D 1/r kernel with A_ii = sqrt(1000 N) (Sec. 4.3, Experiment 3)."""
    return Workload(f"invr2d_N{n}", n, 2, -1.0, 1.0, seed, INVR2D,
                    math.sqrt(1000.0 * n), leaf, tol, nrhs)


def invr3d(n: int, seed: int, leaf: int = 64, tol: float = 1e-6, nrhs: int = 1) -> Workload:
    """3D 1/r kernel with A_ii = N^(2/3), points uniform in [-1,1]^3."""
    return Workload(f"invr3d_N{n}", n, 3, -1.0, 1.0, seed, INVR3D,
                    float(n) ** (2.0 / 3.0), leaf, tol, nrhs)


def gauss2d(n: int, seed: int, leaf: int = 64, tol: float = 1e-10, nrhs: int = 1) -> Workload:
    """GP-style kernel exp(-|x-y|^2/0.1^2) + 1e-2 I on [0,1]^2."""
    return Workload(f"gauss2d_N{n}", n, 2, 0.0, 1.0, seed, GAUSS, 1.0 + 1e-2,
                    leaf, tol, nrhs, length=0.1)


# The named configurations: the small case the oracle finishes in seconds and
# the single-GPU benchmark case (same kernel and dimension, nrhs 1 and 64).
SMALL = log2d(4096, seed=0)
BENCH = log2d(65536, seed=1)
BENCH64 = log2d(65536, seed=1, nrhs=64)


def serving_trace(seed: int = 4, rate: float = 50.0, duration: float = 8.0, frac_factor: float = 0.1,
                  n_lo: int = 4096, n_hi: int = 32768, nrhs_max: int = 32, recent: int = 4,
                  tol: float = 1e-8, leaf: int = 64):
    """A request stream for the serving loop: Poisson arrivals (exponential
    gaps at ``rate`` per second) over ``duration`` seconds; each request is a
    factor request with probability ``frac_factor`` (the first one always
    is), else a solve request.  Factor requests: 2D log kernel with
    A_ii = N, N log-uniform in [n_lo, n_hi], points uniform in [-1,1]^2.
    Solve requests: nrhs uniform in 1..nrhs_max, b ~ N(0,1), against one of
    the ``recent`` most recently requested factorisations, uniformly.
    Returns a list of dicts (kind, t, fid, and points or rhs)."""
    rng = np.random.default_rng(seed)
    out, t, fids, sizes = [], 0.0, [], {}
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if not fids or rng.random() < frac_factor:
            n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
            fid = len(fids)
            fids.append(fid)
            sizes[fid] = n
            out.append({"kind": "factor", "t": t, "fid": fid, "points": rng.uniform(-1.0, 1.0, (n, 2)),
                        "kernel": LOG2D, "diag": float(n), "tol": tol, "leaf": leaf})
        else:
            fid = fids[-1 - int(rng.integers(0, min(recent, len(fids))))]
            k = int(rng.integers(1, nrhs_max + 1))
            out.append({"kind": "solve", "t": t, "fid": fid,
                        "rhs": np.asfortranarray(rng.standard_normal((k, sizes[fid])).T)})
    return out


def batched_problems(seed: int = 3, count: int = 256, n_lo: int = 2048, n_hi: int = 32768, tol: float = 1e-10,
                     leaf: int = 64):
    """Many independent GP-style problems of uneven size: N log-uniform in
    [n_lo, n_hi] (one generator for all, seed ``seed``), points uniform in
    [0,1]^2, A = exp(-|x-y|^2/0.1^2) + 1e-2 I, one right-hand side
    b ~ N(0,1) each.  Returns a list of (Workload, points, rhs)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        w = Workload(f"gauss2d_batch{i}_N{n}", n, 2, 0.0, 1.0, seed, GAUSS, 1.0 + 1e-2, leaf, tol, 1,
                     length=0.1)
        pts = rng.uniform(0.0, 1.0, (n, 2))
        b = np.asfortranarray(rng.standard_normal((n, 1)))
        out.append((w, pts, b))
    return out
