"""Request loop over resident AIFMM factorisations, with continuous batching.

The paper's factorisation is independent of the right-hand side (Remark
after Algorithm 3): a problem is factored once and then solved for as many
right-hand sides as arrive.  This loop serves two kinds of requests:

* ``factor``: build and factor a new problem (C: aifmm_build, aifmm_factor);
  admitted only while the device bytes it is predicted to hold fit under the
  memory cap next to the resident factorisations; idle factorisations (no
  pending solves) are evicted, oldest first, to make room;
* ``solve``: nrhs right-hand sides against a resident factorisation.

Continuous batching: the solve requests that wait on one factorisation are
concatenated column-wise (up to ``max_cols`` columns) into one multi-RHS
aifmm_solve, and the columns are split back per request.  Factor requests
run on a worker thread, each on its handle's own CUDA stream, so their
kernels overlap on the device with the batched solves issued by the serving
thread on other handles' streams; requests that arrive while others are on
the GPU join the next batch or wait for memory.  Once factored, a handle
moves to a high-priority stream (aifmm_set_priority), so the solve batches
are scheduled ahead of the kernels of factorisations still running.

Memory model: the factorisation's blocks are dense per box and stencil slot,
sized by the level's largest box, so at a fixed depth they grow like
N x (points per leaf box); predicted bytes = 1.25 c_d N occ, occ = N / 2^(dL)
with L from the library's depth rule, c_d learnt per dimension from the
factorisations completed so far (the largest seen; before the first one, a
conservative constant).

Host arrays in, host arrays out: latency is measured from arrival to the
moment the result is on the host.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from . import aifmm_build, aifmm_destroy, aifmm_factor, aifmm_set_priority, aifmm_solve, aifmm_stats

# CUDA stream priority of the solves against finished factorisations (CUDA
# clamps it to the device's highest); factorisations keep the default, the
# lowest, so pending solve kernels are scheduled ahead of theirs
SOLVE_PRIORITY = -1000

# conservative bytes per (point x leaf occupancy) before a factorisation of
# that dimension has been measured
_DEFAULT_BPP = {2: 3.0e4, 3: 1.0e5}


def _occupancy(n: int, d: int, leaf: int) -> float:
    """Average points per leaf box under the depth rule
    L = max(2, min l with 2^(d l) leaf >= N)."""
    L = 2
    while (1 << (d * L)) * leaf < n:
        L += 1
    return n / float(1 << (d * L))


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "factor" or "solve"
    t_arrive: float           # seconds from the start of the run
    # factor: the problem
    fid: int = -1             # factorisation id (factor: the one created; solve: the target)
    points: np.ndarray | None = None
    kernel: int = 0
    diag: float = 0.0
    tol: float = 1e-8
    leaf: int = 64
    length: float = 1.0
    # solve: N x nrhs right-hand sides
    rhs: np.ndarray | None = None
    # results
    x: np.ndarray | None = None
    t_done: float = -1.0
    status: str = "pending"   # pending, done, evicted, error
    batch: int = 0            # columns of the solve batch it ran in


class Server:
    """Serve factor and solve requests; see the module docstring."""

    def __init__(self, cap_bytes: float, max_cols: int = 64):
        self.cap = float(cap_bytes)
        self.max_cols = int(max_cols)
        self.resident: "collections.OrderedDict[int, tuple]" = collections.OrderedDict()  # fid -> (handle, bytes, n)
        self.bpp = dict(_DEFAULT_BPP)
        self.factor_q: "collections.deque[Request]" = collections.deque()
        self.solve_q: "dict[int, collections.deque[Request]]" = collections.defaultdict(collections.deque)
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.in_flight = 0.0          # predicted bytes of the factorisation being built
        self.peak_bytes = 0.0
        self.evictions = 0
        self.t0 = 0.0
        self.stop = False
        self.errors: list = []
        self.measured: set = set()    # dimensions with a measured bytes-per-point
        self.building = -1            # fid being factored by the worker
        self.busy = -1                # fid whose batch the serving thread is solving
        self.worker = threading.Thread(target=self._factor_worker, daemon=True)

    # ---- memory model -----------------------------------------------------
    def predict(self, r: Request) -> float:
        n, d = r.points.shape
        return 1.25 * self.bpp.get(d, _DEFAULT_BPP[3]) * n * _occupancy(n, d, r.leaf)

    def resident_bytes(self) -> float:
        return sum(b for _, b, _ in self.resident.values())

    def _admit(self, r: Request) -> bool:
        """Under the lock: make room for r (evicting idle factorisations,
        oldest first) and reserve its predicted bytes; False if it cannot
        fit now."""
        need = self.predict(r)
        if need > self.cap:
            need = self.cap                       # alone on the device: try anyway
        while self.resident_bytes() + self.in_flight + need > self.cap:
            idle = [f for f in self.resident if not self.solve_q.get(f) and f != self.busy]
            if not idle:
                return False
            f = idle[0]
            h, _, _ = self.resident.pop(f)
            aifmm_destroy(h)
            self.evictions += 1
        self.in_flight += need
        return True

    # ---- requests --------------------------------------------------------
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, r: Request) -> None:
        with self.cv:
            if r.kind == "factor":
                self.factor_q.append(r)
            else:
                self.solve_q[r.fid].append(r)
            self.cv.notify_all()

    def _factor_worker(self) -> None:
        while True:
            with self.cv:
                while not self.stop and not (self.factor_q and self._admit(self.factor_q[0])):
                    self.cv.wait(0.002)
                if self.stop:
                    return
                r = self.factor_q.popleft()
                reserved = min(self.predict(r), self.cap)
                self.building = r.fid
            try:
                h = aifmm_build(r.points, r.kernel, r.diag, r.tol, r.leaf, length=r.length)
                aifmm_factor(h)
                aifmm_set_priority(h, SOLVE_PRIORITY)
                nbytes = float(aifmm_stats(h)["bytes_resident"])
                st = "done"
            except Exception as e:      # reported on the request, the loop goes on
                h, nbytes, st = None, 0.0, "error"
                self.errors.append((r.rid, repr(e)))
            with self.cv:
                self.in_flight -= reserved
                self.building = -1
                if h is not None:
                    n, d = r.points.shape
                    ratio = nbytes / (n * _occupancy(n, d, r.leaf))
                    self.bpp[d] = max(self.bpp[d], ratio) if d in self.measured else ratio
                    self.measured.add(d)
                    self.resident[r.fid] = (h, nbytes, n)
                    self.peak_bytes = max(self.peak_bytes, self.resident_bytes())
                r.status, r.t_done = st, self.now()
                self.cv.notify_all()

    def _next_batch(self):
        """Under the lock: the oldest waiting solve's factorisation and as
        many of its waiting requests as fit in max_cols columns."""
        best, t_best = None, None
        for f, q in self.solve_q.items():
            if q and f in self.resident and (t_best is None or q[0].t_arrive < t_best):
                best, t_best = f, q[0].t_arrive
        if best is None:
            return None, None, []
        q = self.solve_q[best]
        take, cols = [], 0
        while q and (not take or cols + q[0].rhs.shape[1] <= self.max_cols):
            r = q.popleft()
            take.append(r)
            cols += r.rhs.shape[1]
        return best, self.resident[best][0], take

    def _drop_orphans(self) -> None:
        """Under the lock: solves whose factorisation failed or was evicted
        before they could run."""
        live = set(self.resident) | {r.fid for r in self.factor_q} | {self.building}
        for f, q in self.solve_q.items():
            if q and f not in live:
                while q:
                    r = q.popleft()
                    r.status, r.t_done = "evicted", self.now()

    def serve_step(self) -> bool:
        """Run one solve batch if any is ready; True if one ran."""
        with self.cv:
            f, h, take = self._next_batch()
            if take:
                self.busy = f                     # not evicted while it is being solved
        if not take:
            return False
        try:
            B = np.asfortranarray(np.hstack([r.rhs for r in take]))
            X = aifmm_solve(h, B)
        finally:
            with self.cv:
                self.busy = -1
                self.cv.notify_all()
        t = self.now()
        c = 0
        for r in take:
            k = r.rhs.shape[1]
            r.x = np.array(X[:, c:c + k])
            r.status, r.t_done, r.batch = "done", t, B.shape[1]
            c += k
        return True

    def run(self, requests: "list[Request]", timeout: float = 600.0) -> dict:
        """Replay requests at their arrival times (seconds from now) and
        serve them; returns the metrics."""
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        self.t0 = time.perf_counter()
        self.worker.start()
        i = 0
        try:
            while True:
                now = self.now()
                while i < len(reqs) and reqs[i].t_arrive <= now:
                    self.submit(reqs[i])
                    i += 1
                ran = self.serve_step()
                done = all(r.status != "pending" for r in reqs)
                if done and i == len(reqs):
                    break
                if now > timeout:
                    raise TimeoutError("serving run exceeded its time limit")
                if not ran:
                    with self.cv:
                        self._drop_orphans()
                    time.sleep(0.0005)
        finally:
            with self.cv:
                self.stop = True
                self.cv.notify_all()
            self.worker.join()
        return metrics(reqs, self.now(), self)

    def close(self) -> None:
        for h, _, _ in self.resident.values():
            aifmm_destroy(h)
        self.resident.clear()


def metrics(reqs, wall: float, srv: Server) -> dict:
    out = {"wall_s": wall, "requests": len(reqs), "evictions": srv.evictions,
           "peak_resident_gb": srv.peak_bytes / 1e9, "cap_gb": srv.cap / 1e9}
    for kind in ("factor", "solve"):
        rs = [r for r in reqs if r.kind == kind and r.status == "done"]
        lat = np.array([r.t_done - r.t_arrive for r in rs]) * 1e3
        out[kind] = {"done": len(rs), "failed": sum(1 for r in reqs if r.kind == kind and r.status != "done"),
                     "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                     "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None}
    sol = [r for r in reqs if r.kind == "solve" and r.status == "done"]
    cols = sum(r.rhs.shape[1] for r in sol)
    out["solves_per_s"] = cols / wall if wall > 0 else 0.0
    out["requests_per_s"] = sum(1 for r in reqs if r.status == "done") / wall if wall > 0 else 0.0
    out["mean_batch_cols"] = float(np.mean([r.batch for r in sol])) if sol else 0.0
    return out


def requests_from_trace(trace) -> "list[Request]":
    """Requests of a trace made by workloads.serving_trace."""
    out = []
    for i, e in enumerate(trace):
        if e["kind"] == "factor":
            out.append(Request(i, "factor", e["t"], fid=e["fid"], points=e["points"], kernel=e["kernel"],
                               diag=e["diag"], tol=e["tol"], leaf=e["leaf"]))
        else:
            out.append(Request(i, "solve", e["t"], fid=e["fid"], rhs=e["rhs"]))
    return out
