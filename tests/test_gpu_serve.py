"""The serving loop on the GPU (through the C ABI): every solve answered in a
mix of factor and solve requests -- batched with other requests, next to a
factorisation running on another stream -- equals the same solve run alone
on a factorisation of the same problem, within 1e-12."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12704_gb300 as lib
    return lib


def test_each_result_same_alone_and_in_the_mix(A):
    from paper_2301_12704_gb300 import serve as S
    trace = W.serving_trace(seed=41, rate=300.0, duration=0.6, frac_factor=0.06, n_lo=1500, n_hi=5000,
                            nrhs_max=6, recent=2)
    reqs = S.requests_from_trace(trace)
    nf = sum(r.kind == "factor" for r in reqs)
    assert nf >= 2
    srv = S.Server(cap_bytes=100e9, max_cols=32)
    m = srv.run(reqs, timeout=300)
    srv.close()
    assert m["factor"]["failed"] == 0 and m["solve"]["failed"] == 0, srv.errors
    # batches formed
    assert max(r.batch - r.rhs.shape[1] for r in reqs if r.kind == "solve") > 0
    # alone: the same problems factored on their own, each request solved alone
    facs = {r.fid: r for r in reqs if r.kind == "factor"}
    worst = 0.0
    for fid, fr in facs.items():
        h = A.aifmm_build(fr.points, fr.kernel, fr.diag, fr.tol, fr.leaf)
        A.aifmm_factor(h)
        for r in reqs:
            if r.kind == "solve" and r.fid == fid:
                x = A.aifmm_solve(h, r.rhs)
                worst = max(worst, float(np.linalg.norm(r.x - x) / np.linalg.norm(x)))
        A.aifmm_destroy(h)
    assert worst <= 1e-12, worst


def test_admission_under_a_small_cap(A):
    from paper_2301_12704_gb300 import serve as S
    trace = W.serving_trace(seed=42, rate=200.0, duration=0.5, frac_factor=0.15, n_lo=2400, n_hi=2600,
                            nrhs_max=4, recent=1)
    reqs = S.requests_from_trace(trace)
    nf = sum(r.kind == "factor" for r in reqs)
    # measure one factorisation, then allow about two at a time
    fr = next(r for r in reqs if r.kind == "factor")
    h = A.aifmm_build(fr.points, fr.kernel, fr.diag, fr.tol, fr.leaf)
    A.aifmm_factor(h)
    one = A.aifmm_stats(h)["bytes_resident"]
    A.aifmm_destroy(h)
    cap = 2.5 * 1.25 * one * (2600 / len(fr.points)) ** 2
    srv = S.Server(cap_bytes=cap, max_cols=16)
    m = srv.run(reqs, timeout=300)
    srv.close()
    assert m["factor"]["failed"] == 0 and m["solve"]["failed"] == 0
    assert srv.peak_bytes <= cap
    assert srv.evictions >= nf - 3
