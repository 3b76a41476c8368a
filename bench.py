#!/usr/bin/env python
"""AIFMM factor+solve benchmark on GB300.

One step = one pass of the whole hot path on one synthetic problem: tree,
lists, NNCA operators and extended system (aifmm_build), the colour-batched
elimination (aifmm_factor), and two solves (nrhs = 1 and nrhs = 64).  The
headline metric is the 65,536-point 2D log-kernel configuration's
factor+solve throughput, points/s = N / (T_factor + T_solve(nrhs=1)), each
phase timed with CUDA events on the stream the library runs on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank factors and solves an
independent problem (replicas: the method has no exchange step), value is
the sum of points over the max time over ranks, scaling "weak".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve points/s at rel-err<=1e-8 vs FP64 oracle"
UNIT = "points/s"
# Digit-pair BF16 MMAs per FP64 multiply-add of the 7-digit tensor-core tile
# (pairs of digits s + t <= 8 of seven 7-bit digits per operand).
OZ_PAIRS = 39
TRAFFIC_65536 = {"k_schur": 1.157e8, "k_cmp_qrcp": 1.137e7}
# Roofline denominators when MEASURED_PEAKS.json is absent: the profiling
# recipe's fallback (one earlier GB300 measurement).
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks():
    """HBM copy bandwidth and cuBLAS BF16 rates measured on this machine's
    GB300s (MEASURED_PEAKS.json, written by the test driver), else the
    fallback; with the source named."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {k: float(d[k]) for k in FALLBACK_PEAKS}, "of measured (MEASURED_PEAKS.json)"
    except Exception:
        return dict(FALLBACK_PEAKS), "of fallback (profiling recipe)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--batched", type=int, default=32,
                   help="also run this many independent uneven problems (1 and 8 host threads); 0: skip")
    p.add_argument("--mixed3d", type=int, default=0,
                   help="also run the 3D mixed-precision GMRES configuration at this many points")
    return p.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n_sample=16384):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the
    same kernel, tolerance, leaf size and point density, n_sample points, in
    this process (the reference arm's steps)."""
    import numpy as np
    import workloads as W
    from oracle import factor as OF
    from oracle.kernels import Kernel
    from oracle.nnca import NNCA
    from oracle.tree import Tree
    w = W.log2d(n_sample, seed=1)
    pts, b = W.points_and_rhs(w)
    T = Tree(pts, w.leaf)
    K = Kernel(w.kernel, w.diag)
    nn = NNCA(T, K, w.tol)
    t0 = time.perf_counter()
    fac = OF.factor(T, K, nn, w.tol, order="paper")
    OF.solve(fac, b[T.perm, 0])
    dt = time.perf_counter() - t0
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    return {"value": n_sample / dt, "unit": UNIT, "cores": int(threads), "kind": "oracle",
            "sample": f"{n_sample}-point log2d problem (same kernel, tol 1e-10, leaf 64, density); "
                      f"factor+solve {dt:.1f} s, paper order, numpy/scipy BLAS threads"}


def oracle_runs(n=4096, seed=0):
    """The oracle on the small configuration at full size (4,096 points, the
    same kernel, diagonal, tolerance and leaf size as the timed problem), as
    child processes with their BLAS thread counts fixed: one thread in
    paper (Morton) order, and all host cores in colour order.  The oracle's
    boxes run one after another; its block operations use the BLAS threads."""
    ncpu = os.cpu_count() or 1
    out = {}
    for key, threads, order in (("single_thread", 1, "paper"), ("all_cores", ncpu, "colour")):
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[v] = str(threads)
        env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
        r = subprocess.run([sys.executable, "-m", "oracle.baseline", "--n", str(n), "--seed", str(seed),
                            "--order", order], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
        if r.returncode != 0:
            out[key] = {"error": (r.stderr or r.stdout)[-300:]}
            continue
        out[key] = json.loads(r.stdout.strip().splitlines()[-1])
    return out


def cpu_baseline_full(n=4096, seed=0):
    """The GPU arm's cpu_baseline: oracle_runs; the faster of the two runs is
    the value (with small blocks, BLAS threads can cost more than they give)."""
    runs = oracle_runs(n, seed)
    ok = {k: v for k, v in runs.items() if "points_per_s" in v}
    if not ok:
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "error": runs}
    best = max(ok.values(), key=lambda r: r["points_per_s"])
    desc = "; ".join(f"{r['threads']} BLAS thread(s), {r['order']} order: {r['points_per_s']:.1f} points/s "
                     f"(factor {r['s_factor']:.2f} s + solve {r['s_solve']:.3f} s)" for r in ok.values())
    return {"value": best["points_per_s"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
            "sample": f"the {n}-point configuration of the same workload at full size (log2d, uniform "
                      f"[-1,1]^2, seed {seed}, A_ii = N, leaf 64, tol 1e-10), factor+solve; {desc}; the value is "
                      f"the faster run; the 65,536-point problem does not fit the bounded time (the oracle's "
                      f"cost grows faster than N: about 37 s at 16,384 points)",
            "runs": runs}


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    vals = []
    info = None
    for _ in range(args.warmup):                      # untimed, as in the GPU arm
        cpu_baseline(4096)
    for _ in range(max(1, args.steps)):
        info = cpu_baseline(4096)
        vals.append(info["value"])
    v = statistics.mean(vals)
    info["value"] = v
    info["sample"] = "4,096-point log2d problem per step (same kernel, tol, leaf, density); " + info["sample"].split("; ", 1)[1]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * 4096 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "log2d N=65536 (oracle timed on a 4,096-point sample)",
                                        "kernel": "log|x-y|, A_ii=N", "tol": 1e-10, "leaf": 64},
        "cpu_baseline": info, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def serve(A, duration=8.0, rate=25.0, seed=4):
    """The serving loop (paper_2301_12704_gb300.serve): Poisson arrivals of
    factor requests (10%) and solve requests (nrhs 1..32) against resident
    factorisations, continuous batching of the solves, memory admission
    under a 150 GB cap.  Host arrays in and out; latency from arrival to the
    result on the host."""
    import workloads as W
    from paper_2301_12704_gb300 import serve as S
    trace = W.serving_trace(seed=seed, rate=rate, duration=duration)
    reqs = S.requests_from_trace(trace)
    srv = S.Server(cap_bytes=150e9, max_cols=64)
    m = srv.run(reqs, timeout=600)
    srv.close()
    m["workload"] = (f"Poisson {rate:g} req/s for {duration:g} s (seed {seed}): 10% factor requests (2D log kernel, "
                     "A_ii = N, N log-uniform 4,096..32,768, tol 1e-8, leaf 64), 90% solve requests (nrhs 1..32, "
                     "b ~ N(0,1)) against one of the 4 latest factorisations; batches of up to 64 columns; cap 150 GB")
    return m


def gmres_mode(A, w, pts_d, b1_d, stream, ftol=1e-6, rtol=1e-10, fp32=False, tf32=False):
    """AIFMM as a preconditioner (Sec. 4, Experiment 5): a factorisation with
    a looser compress threshold (and, with fp32, FP32 tile products; with
    tf32, TF32 tensor-core products), then FP64 GMRES on the H^2 product."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    kw = dict(stream=stream.cuda_stream, factor_tol=ftol, fp32=fp32, tf32=tf32)
    h = A.aifmm_build(pts_d, w.kernel, w.diag, w.tol, w.leaf, **kw)
    A.aifmm_factor(h)                                   # warm
    A.aifmm_destroy(h)
    h = A.aifmm_build(pts_d, w.kernel, w.diag, w.tol, w.leaf, **kw)
    ev[0].record(stream)
    A.aifmm_factor(h)
    ev[1].record(stream)
    x, it, rr = A.aifmm_gmres(h, b1_d[:, 0], rtol=rtol, maxit=100, restart=30, use_precond=True,
                              raise_noconv=False)
    ev[2].record(stream)
    stream.synchronize()
    st = A.aifmm_stats(h)
    r = A.aifmm_direct_matvec(h, x)[:, 0] - b1_d[:, 0]
    true = float(torch.linalg.norm(r) / torch.linalg.norm(b1_d[:, 0]))
    A.aifmm_destroy(h)
    tf, tg = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    return {"factor_tol": ftol, "products": "tf32" if tf32 else "fp32" if fp32 else "fp64", "rtol": rtol,
            "ms_factor": tf,
            "ms_gmres": tg, "iterations": it,
            "relres_h2": rr, "residual_direct_sum": true, "max_rank": st["max_rank_factor"],
            "points_per_s": w.n / ((tf + tg) / 1e3)}


def mixed3d(A, dev, n=32768, rtol=1e-10):
    """The 3D mixed-precision configuration (1/r, A_ii = N^(2/3), uniform in
    [-1,1]^3, seed 2, leaf 64, tol 1e-6): the factorisation with FP32 tile
    products as the preconditioner of FP64 GMRES on the H^2 product, beside
    the same with FP64 products; points/s = N / (T_factor + T_gmres).  N is
    the largest size whose capacity-padded blocks fit one GB300 (262,144
    points would need several hundred GB)."""
    import numpy as np
    import torch
    import workloads as W
    w = W.invr3d(n, seed=2)
    pts, b = W.points_and_rhs(w)
    pts_d = torch.from_numpy(pts).to(dev)
    b_d = torch.from_numpy(np.asfortranarray(b)).to(dev)[:, 0]
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": f"invr3d N={n}: uniform [-1,1]^3 (seed 2), A_ij=1/|x_i-x_j|, A_ii=N^(2/3), leaf 64, "
                       f"NNCA and compress tol 1e-6, GMRES rtol {rtol:g}"}
    for fp32 in (True, False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            h = A.aifmm_build(pts_d, w.kernel, w.diag, w.tol, w.leaf, stream=stream.cuda_stream, fp32=fp32)
            ev[1].record(stream)
            A.aifmm_factor(h)
            ev[2].record(stream)
            x, it, rr = A.aifmm_gmres(h, b_d, rtol=rtol, maxit=200, restart=40, use_precond=True)
            ev[3].record(stream)
        stream.synchronize()
        st = A.aifmm_stats(h)
        r = A.aifmm_direct_matvec(h, x)[:, 0] - b_d
        true = float(torch.linalg.norm(r) / torch.linalg.norm(b_d))
        A.aifmm_destroy(h)
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
        out["fp32" if fp32 else "fp64"] = {
            "ms_build": t[0], "ms_factor": t[1], "ms_gmres": t[2], "iterations": it, "relres_h2": rr,
            "residual_direct_sum": true, "levels": st["levels"], "max_rank": st["max_rank_factor"],
            "gb_resident": st["bytes_resident"] / 1e9, "points_per_s": n / ((t[1] + t[2]) / 1e3)}
    return out


def batched(A, count=256, workers=(1, 8), tol=1e-6):
    """Many independent GP-style problems of uneven size (Gaussian kernel,
    length 0.1, + 1e-2 I on [0,1]^2, N log-uniform 2,048..32,768, seed 3,
    leaf 64): factor + solve of all of them, with 1 and with several host
    threads driving one handle and stream per problem; points/s = solved
    points / wall time.  tol 1e-6: at 1e-10 the Gaussian's far-field ranks of
    the larger problems exceed the compiled-in rank capacity of 1,023."""
    import workloads as W
    from paper_2301_12704_gb300 import batch as B
    probs = W.batched_problems(seed=3, count=count, tol=tol)
    out = {"workload": f"{count} problems: Gaussian kernel exp(-r^2/0.1^2) + 1e-2 I on [0,1]^2, N log-uniform "
                       f"2,048..32,768 (seed 3), tol {tol:g}, leaf 64, one rhs each; FP64"}
    for k in workers:
        _, m = B.factor_solve_many(probs, workers=k)
        out[f"workers_{k}"] = m
    return out


def max_over_ranks(vals, dev, ws):
    """Element-wise maximum of per-rank timings over the process group
    (every rank gets it); identity on one process."""
    if ws <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(v) for v in vals], device=dev, dtype=torch.float64)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return [float(v) for v in x.tolist()]


def replica_value(ws, n, steps, ms_max):
    """Whole-job points/s of ws replicas, each factoring and solving steps
    problems of n points: all points over the slowest rank's time."""
    return ws * n * steps / (ms_max / 1e3)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    import paper_2301_12704_gb300 as A
    import workloads as W

    w = W.log2d(args.n, seed=1 + rank)      # rank 0: the 65,536-point configuration
    pts, b1 = W.points_and_rhs(w, nrhs=1)
    _, b64 = W.points_and_rhs(w, nrhs=64)
    dev = torch.device("cuda", local)
    pts_d = torch.from_numpy(pts).to(dev)
    b1_d = torch.from_numpy(np.asfortranarray(b1)).to(dev)
    b64_d = torch.from_numpy(b64.T.copy()).to(dev).t()         # column-major N x 64
    stream = torch.cuda.Stream(device=dev)

    def step(profile):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        h = A.aifmm_build(pts_d, w.kernel, w.diag, w.tol, w.leaf, stream=stream.cuda_stream, profile=profile)
        ev[1].record(stream)
        A.aifmm_factor(h)
        ev[2].record(stream)
        x1 = A.aifmm_solve(h, b1_d)
        ev[3].record(stream)
        x64 = A.aifmm_solve(h, b64_d)
        ev[4].record(stream)
        stream.synchronize()
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        return h, x1, x64, t

    for _ in range(args.warmup):
        h, _, _, _ = step(False)
        A.aifmm_destroy(h)
    # accuracy of the timed configuration: true residuals of both solves with
    # the exact direct-sum product (outside the timed region)
    h, x1, x64, _ = step(False)
    r = A.aifmm_direct_matvec(h, x1) - b1_d
    resid = float(torch.linalg.norm(r) / torch.linalg.norm(b1_d))
    r = A.aifmm_direct_matvec(h, x64) - b64_d
    resid64 = float((torch.linalg.norm(r, dim=0) / torch.linalg.norm(b64_d, dim=0)).max())
    stats0 = A.aifmm_stats(h)
    A.aifmm_destroy(h)
    del x1, x64, r
    # roofline peaks: the FP64 / FP32 FMA rates measured on this GPU now, the
    # HBM and BF16 ones from the pool's measurement
    fp64_peak = A.aifmm_fma_rate(False, stream.cuda_stream)
    fp32_peak = A.aifmm_fma_rate(True, stream.cuda_stream)
    peaks, peak_src = measured_peaks()

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    NG = 5
    times, groups_ms, groups_fl, groups_n, launches = [], [0.0] * NG, [0.0] * NG, [0] * NG, 0
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h, _, _, t = step(True)
            s = A.aifmm_stats(h)
            for g in range(NG):
                groups_ms[g] += s["group_ms"][g]
                groups_fl[g] += s["group_flops"][g]
                groups_n[g] += s["group_launches"][g]
            launches += s["kernel_launches"]
            times.append(t)
            A.aifmm_destroy(h)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
    clocks = clk.summary()
    tf = sum(t[1] for t in times)
    ts1 = sum(t[2] for t in times)
    ts64 = sum(t[3] for t in times)
    tstep = sum(sum(t) for t in times)
    fs_ms = tf + ts1
    fs_ms, tstep = max_over_ranks([fs_ms, tstep], dev, ws)
    value = replica_value(ws, args.n, args.steps, fs_ms)

    # rooflines of single kernels, from their CUDA-event times inside the
    # timed steps (profile mode records events around each launch on the
    # library's stream) and their algorithmic work counted from the run's
    # block sizes
    names = ["compress_other", "pivot_lu", "z_solve", "schur", "qrcp"]
    G_SCHUR, G_QRCP = 3, 4
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum,
    # averaged over one factorisation's launches) from one ncu capture of
    # these kernels as they now stand, at the 65,536-point workload (summary
    # under profiles/); unknown (None) for other sizes
    traffic = TRAFFIC_65536 if args.n == 65536 else {}

    def kernel_roof(g):
        ms, fl, nl = groups_ms[g], groups_fl[g], groups_n[g]
        fp64 = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        base = {"launches": nl, "avg_launch_ms": ms / max(1, nl), "share_of_factor": ms / max(1e-9, tf),
                "flops_per_launch": fl / max(1, nl),
                "traffic": traffic.get("k_cmp_qrcp" if g == G_QRCP else "k_schur")}
        if g == G_QRCP:
            base.update({"kernel": "k_cmp_qrcp", "bound": "alu", "achieved": fp64, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": fp64 / fp64_peak if fp64_peak else None,
                         "peak_source": "FP64 FMA rate measured on this GPU by aifmm_fma_rate"})
        else:
            # FP64-precision products issued as BF16 digit-pair MMAs: the
            # tensor pipe's work is OZ_PAIRS MMA flops per FP64 flop
            tc = OZ_PAIRS * fp64
            base.update({"kernel": "k_schur", "bound": "tensor", "achieved": tc, "peak": peaks["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": tc / peaks["bf16_tflops"],
                         "peak_source": "BF16 dense burst " + peak_src,
                         "fp64_equivalent_tflops": fp64,
                         "fp64_equivalent_frac_of_fp64_fma": fp64 / fp64_peak if fp64_peak else None})
        return base

    roofs = {names[g]: kernel_roof(g) for g in (G_QRCP, G_SCHUR) if groups_ms[g] > 0}
    dom = max((G_QRCP, G_SCHUR), key=lambda g: groups_ms[g])
    roof = roofs[names[dom]]
    # the solve with one right-hand side: HBM-bound by its algorithmic bytes
    bsolve = stats0["bytes_solve"]
    gbs = bsolve / (ts1 / args.steps / 1e3) / 1e9 if ts1 > 0 else 0.0
    roofs["solve_nrhs1"] = {"kernel": "solve sweeps (k_fwd_*, k_lus_*, k_bwd_*), nrhs=1", "bound": "hbm",
                            "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": gbs / peaks["hbm_gbs"], "bytes": bsolve, "traffic": None,
                            "peak_source": "HBM copy " + peak_src}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tstep / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"log2d N={args.n}: uniform [-1,1]^2 (seed 1), A_ij=log|x_i-x_j|, A_ii=N, "
                                  "leaf 64, NNCA/RRQR tol 1e-10, nrhs 1 (metric) and 64",
                      "levels": stats0["levels"], "max_rank": stats0["max_rank_factor"],
                      "gb_resident": stats0["bytes_resident"] / 1e9,
                      "l2": "inputs larger than L2 (factor storage >> 129 MB)",
                      "parallelism": "replicas" if ws > 1 else "single GPU",
                      "step": "build + factor + solve(nrhs=1) + solve(nrhs=64)"},
           "ms_build": sum(t[0] for t in times) / args.steps, "ms_factor": tf / args.steps,
           "ms_solve_nrhs1": ts1 / args.steps, "ms_solve_nrhs64": ts64 / args.steps,
           "solves_per_s_nrhs64": 64.0 / (ts64 / args.steps / 1e3),
           "residual_direct_sum": resid, "residual_direct_sum_nrhs64_max": resid64,
           "flops_factor": stats0["flops_factor"],
           "factor_fp64_tflops": stats0["flops_factor"] / (tf / args.steps / 1e3) / 1e12,
           "group_ms_per_factor": {n: groups_ms[i] / args.steps for i, n in enumerate(names)},
           "group_tflops": {n: (groups_fl[i] / (groups_ms[i] / 1e3) / 1e12 if groups_ms[i] > 0 else 0.0)
                            for i, n in enumerate(names)},
           "roofline": roof, "rooflines": roofs,
           "peaks": {"fp64_fma_tflops": fp64_peak, "fp32_fma_tflops": fp32_peak, **peaks,
                     "source": "FMA rates: aifmm_fma_rate on this GPU before the timed steps; HBM, BF16: "
                               + peak_src},
           "bytes_solve": bsolve, "bytes_resident": stats0["bytes_resident"],
           "bytes_resident_over_bytes_solve": stats0["bytes_resident"] / max(1.0, bsolve),
           "gpu_launches": launches, "clocks": clocks, "wall_s_timed": wall}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers (copies inside)
        ee = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = A.aifmm_build(pts, w.kernel, w.diag, w.tol, w.leaf)
            t1 = time.perf_counter()
            A.aifmm_factor(h)
            x = A.aifmm_solve(h, b1)
            t2 = time.perf_counter()
            ee.append((t1 - t0, t2 - t1))
            A.aifmm_destroy(h)
        e_fs = sum(x[1] for x in ee)
        out["e2e"] = {"value": ws * args.n * len(ee) / e_fs, "unit": UNIT,
                      "h2d_bytes_per_step": args.n * 8, "d2h_bytes_per_step": args.n * 8,
                      "note": "wall time of aifmm_factor + aifmm_solve with host rhs in and host x out; "
                              "the host points enter through aifmm_build, which the metric excludes"}
    if not args.no_serve:
        out["serve"] = serve(A)
        out["gmres_mode"] = gmres_mode(A, w, pts_d, b1_d, stream, ftol=1e-4)
        out["gmres_mode_fp32"] = gmres_mode(A, w, pts_d, b1_d, stream, ftol=1e-4, fp32=True)
        out["gmres_mode_tf32"] = gmres_mode(A, w, pts_d, b1_d, stream, ftol=1e-3, tf32=True)
    if args.batched:
        out["batched"] = batched(A, count=args.batched)
    if args.mixed3d:
        out["mixed3d"] = mixed3d(A, dev, n=args.mixed3d)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_full()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
