"""The tensor-core FP64 product tile (aifmm_dgemm_tc) against an
extended-precision reference: its error must be of FP64 size."""
import numpy as np
import pytest

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


def _cm(x):
    import torch
    return torch.from_numpy(np.asfortranarray(x)).cuda().t().contiguous().t()


def _ref(a, b, c, alpha):
    """c + alpha a b in long double (quad on aarch64, 64-bit mantissa on x86)."""
    return (c.astype(np.longdouble) + np.longdouble(alpha) * (a.astype(np.longdouble) @ b.astype(np.longdouble)))


@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (130, 77, 201), (1, 200, 5), (257, 129, 1000)])
def test_dgemm_tc_error_is_fp64_size(A, m, n, k):
    """Operands of moderate dynamic range: error of FP64 size relative to
    |C| + |A||B| (an FP64 product's own error is K u |A||B| at worst)."""
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    if m > 2:
        a[1, :] = 0.0                      # an exact zero row
    c = rng.standard_normal((m, n))
    for alpha in (1.0, -1.0):
        cd = _cm(c)
        A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, alpha)
        got = cd.cpu().numpy()
        ref = _ref(a, b, c, alpha)
        scale = np.abs(c) + np.abs(a) @ np.abs(b)
        err = float(np.max(np.abs(got - ref) / scale))
        e64 = float(np.max(np.abs((c + alpha * (a @ b)) - ref) / scale))
        assert err <= 2.0 ** -48, (err, e64)


def test_dgemm_tc_wide_dynamic_range(A):
    """Rows and columns spanning many binades: every entry keeps 49 bits
    below its row's (column's) largest, so the error is bounded by
    2^-48 sum_k (max|A_i.| |B_kj| + |A_ik| max|B_.j|)."""
    rng = np.random.default_rng(5)
    m, n, k = 96, 80, 300
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    a[:, ::7] *= 1e-9
    b[::5, :] *= 1e6
    c = np.zeros((m, n))
    cd = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, 1.0)
    got = cd.cpu().numpy()
    ref = _ref(a, b, c, 1.0)
    ra = np.abs(a).max(axis=1, keepdims=True)
    cb = np.abs(b).max(axis=0, keepdims=True)
    bound = 2.0 ** -48 * (ra @ np.ones((1, k)) @ np.abs(b) + np.abs(a) @ np.ones((k, 1)) @ cb)
    assert np.all(np.abs(got - ref) <= bound)


def test_dgemm_tc_rejects_bad_arguments(A):
    import ctypes as C
    lib = A.lib()
    assert lib.aifmm_dgemm_tc(None, 1, None, 1, None, 1, 1, 1, 1, 1.0, None) == 1


@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (130, 77, 201), (1, 200, 5), (257, 129, 1000), (64, 64, 31)])
def test_dgemm_tc05_matches_the_mma_tile(A, m, n, k):
    """The tcgen05 tile (tensor-memory accumulators, integer fixed point
    across K) has the FP64-size error of the warp-MMA tile relative to
    |C| + |A||B|, and the two agree to that level."""
    rng = np.random.default_rng(m * 5 + n * 11 + k)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    if m > 2:
        a[1, :] = 0.0
    c = rng.standard_normal((m, n))
    ref = _ref(a, b, c, -1.0)
    scale = np.abs(c) + np.abs(a) @ np.abs(b)
    cd = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, -1.0, tcgen05=True)
    got = cd.cpu().numpy()
    err = float(np.max(np.abs(got - ref) / scale))
    assert err <= 2.0 ** -48, err


def test_dgemm_tc05_wide_dynamic_range(A):
    """Rows and columns spanning many binades: the same per-chunk bound as
    the warp-MMA tile, 2^-48 sum_k (max|A_i.| |B_kj| + |A_ik| max|B_.j|)
    (chunks of 32 here, so the bound with chunk maxima of 64 holds)."""
    rng = np.random.default_rng(5)
    m, n, k = 96, 80, 300
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    a[:, ::7] *= 1e-9
    b[::5, :] *= 1e6
    c = np.zeros((m, n))
    cd = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, 1.0, tcgen05=True)
    got = cd.cpu().numpy()
    ref = _ref(a, b, c, 1.0)
    ra = np.abs(a).max(axis=1, keepdims=True)
    cb = np.abs(b).max(axis=0, keepdims=True)
    bound = 2.0 ** -48 * (ra @ np.ones((1, k)) @ np.abs(b) + np.abs(a) @ np.ones((k, 1)) @ cb)
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (130, 77, 201), (257, 129, 1000)])
def test_dgemm_tc8_error_is_fp64_size(A, m, n, k):
    """Eight digits: error of FP64 size relative to |C| + |A||B|, four times
    below the seven-digit tile's bound (measured 2^-50.1 here)."""
    rng = np.random.default_rng(m + 2 * n + 3 * k)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    b[:, 3 % n] = 0.0                      # an exact zero column
    c = rng.standard_normal((m, n))
    cd = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, -1.0, digits8=True)
    got = cd.cpu().numpy()
    ref = _ref(a, b, c, -1.0)
    scale = np.abs(c) + np.abs(a) @ np.abs(b)
    assert float(np.max(np.abs(got - ref) / scale)) <= 2.0 ** -49


def test_dgemm_tc8_keeps_small_rows(A):
    """Rows of B of very different magnitudes, as in a column of Piv^-1 B:
    with the balanced contraction each output keeps FP64-size error relative
    to its own terms, |err_ij| <= 2^-50 sum_k |A_ik| max_j' |B_kj'|, while
    the plain 7-digit tile loses the small rows' digits."""
    rng = np.random.default_rng(7)
    m, n, k = 96, 64, 192
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    small = np.zeros(k, dtype=bool)
    small[rng.permutation(k)[: k // 2]] = True
    b[small, :] *= 1e-11                   # "x part" rows
    a[: m // 2, ~small] = 0.0              # the first rows of C see only the small rows
    c = np.zeros((m, n))
    ref = _ref(a, b, c, 1.0)
    bound = 2.0 ** -50 * (np.abs(a) @ np.abs(b).max(axis=1, keepdims=True))
    cd = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cd, 1.0, digits8=True)
    got = cd.cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    cp = _cm(c)
    A.aifmm_dgemm_tc(_cm(a), _cm(b), cp, 1.0)
    plain = cp.cpu().numpy()
    top = slice(0, m // 2)
    assert np.max(np.abs(plain[top] - ref[top])) > 1e3 * np.max(np.abs(got[top] - ref[top]))
