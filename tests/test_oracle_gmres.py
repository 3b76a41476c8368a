"""Pins of the oracle's restarted, right-preconditioned GMRES against facts
that do not depend on its code: Krylov-dimension termination, the
minimal-residual property over an independently built Krylov basis,
monotone residuals and one-step convergence with an exact preconditioner."""
import numpy as np
import pytest

from oracle.gmres import gmres


def _rng(seed):
    return np.random.default_rng(seed)


def test_terminates_in_k_steps_for_k_distinct_eigenvalues():
    # A = Q diag(lambda) Q^T with 3 distinct eigenvalues: the minimal
    # polynomial has degree 3, so the Krylov space stops growing after 3 steps
    rng = _rng(0)
    n = 48
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([1.0, 3.0, 7.5], n // 3)
    A = (Q * lam) @ Q.T
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, rtol=1e-13, maxit=n, restart=n)
    assert it == 3
    assert hist[-1] < 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11 * np.linalg.norm(x))


def _krylov_min(A, b, k, Minv):
    """Brute force: minimise ||b - A x|| over x in M^-1 K_k(A M^-1, b), with the
    basis from a QR of the power sequence (no Arnoldi)."""
    AM = A @ Minv
    K = np.empty((len(b), k))
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = AM @ v
    Qk, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(AM @ Qk, b, rcond=None)[0]
    return Minv @ (Qk @ c)


@pytest.mark.parametrize("precond", [False, True])
def test_minimal_residual_over_krylov_space(precond):
    rng = _rng(1)
    n = 40
    A = np.eye(n) * 4.0 + rng.standard_normal((n, n)) / np.sqrt(n)      # nonsymmetric
    b = rng.standard_normal(n)
    if precond:
        Mm = np.diag(np.diag(A)) + np.triu(A, 1) * 0.5                  # some fixed M
        Minv = np.linalg.inv(Mm)
        pc = lambda v: Minv @ v
    else:
        Minv = np.eye(n)
        pc = None
    for k in range(1, 7):
        x, it, hist = gmres(lambda v: A @ v, b, rtol=1e-300, maxit=k, restart=20, precond=pc)
        assert it == k
        xs = _krylov_min(A, b, k, Minv)
        assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs), k
        # the recorded residual is the true one of the iterate
        assert abs(hist[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-12


def test_residuals_do_not_increase_across_restarts():
    rng = _rng(2)
    n = 120
    A = np.eye(n) * 2.0 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, rtol=1e-10, maxit=400, restart=8)
    h = np.array(hist[:-1])
    assert np.all(np.diff(h) <= 1e-12)
    assert hist[-1] <= 1e-10
    assert it > 8                                  # restarts happened


def test_exact_inverse_preconditioner_converges_in_one_step():
    rng = _rng(3)
    n = 30
    A = np.eye(n) + rng.standard_normal((n, n)) / n
    b = rng.standard_normal(n)
    Ainv = np.linalg.inv(A)
    x, it, hist = gmres(lambda v: A @ v, b, rtol=1e-12, maxit=10, restart=10, precond=lambda v: Ainv @ v)
    assert it == 1
    assert hist[-1] < 1e-12


def test_zero_rhs():
    x, it, hist = gmres(lambda v: 2.0 * v, np.zeros(5), rtol=1e-10, maxit=10, restart=5)
    assert it == 0 and not x.any()
