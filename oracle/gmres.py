"""Restarted GMRES with right preconditioning (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed: Sec. 4 uses GMRES (Saad & Schultz) as the iterative
solver, its matrix-vector product being the NNCA H^2 product (Experiments
2-4), with the relative residual ||A x - b|| / ||b|| <= eps_GMRES as the
stopping rule (notation table of Sec. 4); Experiment 5 uses a low-accuracy
AIFMM factorisation as the preconditioner.

What GMRES computes, by definition: after k steps of cycle c the iterate is
    x = x_c + M^-1 V_k y,   y = argmin_y || beta e_1 - H_k y ||,
where V_k (orthonormal) spans the Krylov space K_k(A M^-1, r_c), r_c = b - A x_c,
beta = ||r_c||, and H_k ((k+1) x k) is the Arnoldi Hessenberg matrix, so x
minimises ||b - A x|| over x_c + M^-1 K_k.  The oracle builds V_k and H_k with
modified Gram-Schmidt Arnoldi and solves the small least-squares problem with
numpy's ``lstsq`` (a library primitive), in the textbook order; after each
cycle it restarts from the explicit residual.  The starting guess is zero.

Parity: pinned in tests/test_oracle_gmres.py against properties that do not
depend on this code -- exact convergence in k steps on a matrix with k
distinct eigenvalues, the minimal-residual property checked against a brute
force least squares over an independently built Krylov basis, monotone
residuals, one-step convergence with the exact inverse as preconditioner.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b: np.ndarray, rtol: float, maxit: int, restart: int, precond=None):
    """Solve A x = b.  ``matvec(v)`` returns A v; ``precond(v)`` returns M^-1 v
    (identity when None).  Returns (x, iterations, relres history) where the
    history holds ||b - A x_k|| / ||b|| of every iterate from the least-squares
    residual, and the final entry is the explicit relative residual."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    Minv = precond if precond is not None else (lambda v: v)
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    r = b.copy()
    while True:
        beta = float(np.linalg.norm(r))
        if beta / bnorm <= rtol or it >= maxit:
            break
        V = np.zeros((n, restart + 1))
        H = np.zeros((restart + 1, restart))
        V[:, 0] = r / beta
        k = 0
        y = np.zeros(0)
        for j in range(restart):
            w = matvec(Minv(V[:, j]))
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            it += 1
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            res = float(np.linalg.norm(e1 - H[:k + 1, :k] @ y))
            hist.append(res / bnorm)
            if H[j + 1, j] == 0.0 or res / bnorm <= rtol or it >= maxit:
                break
            V[:, j + 1] = w / H[j + 1, j]
        x = x + Minv(V[:, :k] @ y)
        r = b - matvec(x)
        if hist and hist[-1] <= rtol and np.linalg.norm(r) / bnorm <= rtol:
            break
    hist.append(float(np.linalg.norm(b - matvec(x)) / bnorm))
    return x, it, hist
