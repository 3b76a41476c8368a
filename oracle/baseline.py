"""The oracle timed as the CPU baseline of the benchmark.

TEST AND MEASUREMENT INFRASTRUCTURE ONLY (see ``oracle/__init__``): run by
``bench.py``'s CPU-baseline leg as a child process, so that the number of
BLAS threads is fixed before numpy loads.

    python -m oracle.baseline --n 4096 --seed 0 --order paper

builds the tree and the NNCA operators (Sec. 2, not timed as part of the
metric, like the GPU's aifmm_build), then times Algorithm 2 (``factor``)
and Algorithm 3 (``solve``) on one right-hand side of the 2D log-kernel
workload (uniform in [-1,1]^2, A_ii = N, leaf 64, eps_A = 1e-10), and prints
one JSON line: points/s = N / (T_factor + T_solve), the phase times and the
thread count the environment asked for.  The oracle runs as it stands, in
the order asked for ('paper': Morton order; 'colour': distance-2 colours);
its block operations use numpy/scipy, whose BLAS uses the threads given by
OMP_NUM_THREADS / OPENBLAS_NUM_THREADS."""
from __future__ import annotations

import argparse
import json
import os
import time


def main() -> None:
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--order", default="paper", choices=["paper", "colour"])
    a = p.parse_args()
    import workloads as W
    from oracle import factor as OF
    from oracle.kernels import Kernel
    from oracle.nnca import NNCA
    from oracle.tree import Tree
    w = W.log2d(a.n, seed=a.seed)
    pts, b = W.points_and_rhs(w)
    t0 = time.perf_counter()
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, w.tol)
    t1 = time.perf_counter()
    fac = OF.factor(T, K, nn, w.tol, order=a.order)
    t2 = time.perf_counter()
    OF.solve(fac, b[T.perm, 0])
    t3 = time.perf_counter()
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS") or str(os.cpu_count())
    print(json.dumps({"n": a.n, "seed": a.seed, "order": a.order, "threads": int(threads), "levels": T.L,
                      "s_build": t1 - t0, "s_factor": t2 - t1, "s_solve": t3 - t2,
                      "points_per_s": a.n / (t3 - t1)}), flush=True)


if __name__ == "__main__":
    main()
