"""Many independent AIFMM problems of uneven size on one GPU.

Each problem is its own handle with its own CUDA stream; a pool of host
threads drives them (the C-ABI calls release the interpreter lock), so the
colour steps of different problems -- small launches that leave most SMs
idle for one problem alone -- run side by side on the device.  The problems
share nothing, so the results are those of solving each alone.
"""
from __future__ import annotations

import concurrent.futures as cf
import time

import numpy as np

from . import aifmm_build, aifmm_destroy, aifmm_factor, aifmm_solve, aifmm_stats


def _one(points, kernel, diag, tol, leaf, length, rhs, fp32, factor_tol):
    t0 = time.perf_counter()
    h = aifmm_build(points, kernel, diag, tol, leaf, length=length, fp32=fp32, factor_tol=factor_tol)
    t1 = time.perf_counter()
    try:
        aifmm_factor(h)
        x = aifmm_solve(h, rhs)
    except Exception as e:         # e.g. a rank above the compiled-in capacity: reported, not fatal
        aifmm_destroy(h)
        return None, t1 - t0, time.perf_counter() - t1, 0.0, 0, repr(e)
    t2 = time.perf_counter()
    st = aifmm_stats(h)
    aifmm_destroy(h)
    return x, t1 - t0, t2 - t1, st["bytes_resident"], st["max_rank_factor"], None


def factor_solve_many(problems, workers: int = 8, fp32: bool = False, factor_tol: float = 0.0):
    """problems: iterable of (Workload, points, rhs) (workloads.batched_problems).
    Returns (solutions in order, None for a problem whose factorisation
    failed, and metrics; points/s counts the solved problems only)."""
    problems = list(problems)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        futs = [ex.submit(_one, p, w.kernel, w.diag, w.tol, w.leaf, w.length, b, fp32, factor_tol)
                for (w, p, b) in problems]
        res = [f.result() for f in futs]
    wall = time.perf_counter() - t0
    ok = [r[5] is None for r in res]
    npts = sum(len(p) for (_, p, _), g in zip(problems, ok) if g)
    return [r[0] for r in res], {
        "problems": len(problems), "failed": len(ok) - sum(ok),
        "errors": sorted({r[5] for r in res if r[5]})[:3], "points": npts, "workers": workers, "wall_s": wall,
        "points_per_s": npts / wall, "sum_build_s": sum(r[1] for r in res),
        "sum_factor_solve_s": sum(r[2] for r in res), "max_gb": max(r[3] for r in res) / 1e9,
        "max_rank": max(r[4] for r in res)}
