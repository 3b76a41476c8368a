"""The serving loop's scheduling (paper_2301_12704_gb300.serve) on the CPU,
with the C-ABI calls replaced by a dense stand-in: batching splits the
columns back to the right requests, memory admission keeps the resident
bytes under the cap by evicting idle factorisations, and every request is
answered."""
import numpy as np
import pytest

import workloads as W
from paper_2301_12704_gb300 import serve as S


class FakeHandle:
    def __init__(self, pts, diag):
        d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=2)
        np.fill_diagonal(d, 1.0)
        self.A = np.log(d)
        np.fill_diagonal(self.A, diag)
        self.alive = True
        self.n = len(pts)
        self.solves = 0
        self.raised = False


@pytest.fixture
def fake(monkeypatch):
    state = {"destroyed": 0, "live": []}

    def build(points, kernel, diag, tol, leaf, length=1.0):
        h = FakeHandle(np.asarray(points), diag)
        state["live"].append(h)
        return h

    def factor(h):
        assert h.alive

    def solve(h, B):
        assert h.alive, "solve on an evicted factorisation"
        assert h.raised, "solve before the factorisation moved to the solve priority"
        h.solves += 1
        return np.linalg.solve(h.A, B)

    def stats(h):
        return {"bytes_resident": 2000.0 * h.n * S._occupancy(h.n, 2, 64)}   # the library's growth

    def destroy(h):
        assert h.alive
        h.alive = False
        state["destroyed"] += 1

    monkeypatch.setattr(S, "aifmm_build", build)
    monkeypatch.setattr(S, "aifmm_factor", factor)
    monkeypatch.setattr(S, "aifmm_solve", solve)
    monkeypatch.setattr(S, "aifmm_stats", stats)
    monkeypatch.setattr(S, "aifmm_destroy", destroy)

    def set_priority(h, p):
        assert h.alive and p == S.SOLVE_PRIORITY
        h.raised = True
        state["raised"] = state.get("raised", 0) + 1

    monkeypatch.setattr(S, "aifmm_set_priority", set_priority)
    return state


def _trace(**kw):
    args = dict(seed=9, rate=400.0, duration=0.4, frac_factor=0.08, n_lo=60, n_hi=120, nrhs_max=6)
    args.update(kw)
    return W.serving_trace(**args)


def test_batched_solves_are_the_requests_own(fake):
    reqs = S.requests_from_trace(_trace())
    srv = S.Server(cap_bytes=1e12, max_cols=16)
    m = srv.run(reqs, timeout=60)
    srv.close()
    assert m["factor"]["failed"] == 0 and m["solve"]["failed"] == 0
    facs = {r.fid: r for r in reqs if r.kind == "factor"}
    for r in reqs:
        if r.kind != "solve":
            continue
        h = FakeHandle(facs[r.fid].points, facs[r.fid].diag)
        x = np.linalg.solve(h.A, r.rhs)
        assert np.allclose(r.x, x, rtol=1e-12, atol=1e-14)
        assert r.batch >= r.rhs.shape[1] and r.batch <= 16 or r.rhs.shape[1] > 16
    # with 400 requests/s several solves wait on one factorisation: batches form
    assert max(r.batch - r.rhs.shape[1] for r in reqs if r.kind == "solve") > 0
    assert m["mean_batch_cols"] > np.mean([r.rhs.shape[1] for r in reqs if r.kind == "solve"])
    # every factorisation moved to the solve priority once factored
    assert fake["raised"] == len(facs)


def test_admission_evicts_idle_factorisations(fake):
    # solves target only the latest factorisation, so older ones go idle
    reqs = S.requests_from_trace(_trace(recent=1, frac_factor=0.2))
    nf = sum(r.kind == "factor" for r in reqs)
    assert nf >= 4
    cap = 2.2 * 1.25 * 2000.0 * 120 * S._occupancy(120, 2, 64)   # two of the largest, with the margin
    srv = S.Server(cap_bytes=cap, max_cols=16)
    m = srv.run(reqs, timeout=60)
    srv.close()
    assert m["factor"]["failed"] == 0 and m["solve"]["failed"] == 0
    assert srv.peak_bytes <= cap
    assert srv.evictions >= nf // 2            # most factorisations had to make room
    assert fake["destroyed"] == nf              # evicted during the run, the rest at close


def test_solves_on_a_failed_factorisation_are_answered(fake, monkeypatch):
    def bad_factor(h):
        raise RuntimeError("singular")
    monkeypatch.setattr(S, "aifmm_factor", bad_factor)
    reqs = S.requests_from_trace(_trace(duration=0.1))
    srv = S.Server(cap_bytes=1e12)
    m = srv.run(reqs, timeout=30)
    srv.close()
    assert all(r.status == "error" for r in reqs if r.kind == "factor")
    assert all(r.status == "evicted" for r in reqs if r.kind == "solve")
    assert m["solve"]["done"] == 0


@pytest.mark.parametrize("n,d", [(100, 2), (4096, 2), (4097, 2), (65536, 2), (30000, 3), (262144, 3)])
def test_occupancy_follows_the_tree_depth_rule(n, d):
    """The memory model's points per leaf box use the same depth as the
    tree (average-occupancy rule, Sec. 2.1): N / 2^(d L)."""
    import numpy as np
    from oracle.tree import Tree
    pts = np.random.default_rng(n + d).uniform(-1.0, 1.0, (n, d))
    L = Tree(pts, 64).L
    assert S._occupancy(n, d, 64) == pytest.approx(n / float(1 << (d * L)))
