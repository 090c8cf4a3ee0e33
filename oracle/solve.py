"""FP64 linear solvers for the oracle: Jacobi-preconditioned CG and dense Cholesky.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves K d = f (Eq. 8) with a direct sparse solver (Section 3.3);
these are the textbook replacements the CUDA path is checked against:
Jacobi-PCG with the relative true residual ||b - A x||_2 / ||b||_2 as the
stopping rule, and a plain column Cholesky for small dense systems.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    true_relres: float
    history: list


def jacobi_pcg(A, b, tol=1e-10, max_iter=100000, x0=None, max_restarts=10) -> PCGResult:
    """Conjugate gradients preconditioned by M = diag(A)^-1, in FP64.

    Per iteration: q = A p; alpha = (r.z)/(p.q); x += alpha p; r -= alpha q;
    z = M r; beta = (r.z)_new/(r.z)_old; p = z + beta p.  The loop stops when the
    recursively updated residual reaches tol*||b||; the true residual is then
    recomputed and, if it is above tol, the iteration restarts from it (at
    most max_restarts times: below FP64's attainable accuracy, about
    cond(A)*eps, restarts no longer help)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    dinv = 1.0 / A.diagonal()
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return PCGResult(np.zeros(n), 0, 0.0, [])
    it = 0
    hist = []
    restarts = 0
    while True:
        r = b - A @ x
        z = dinv * r
        p = z.copy()
        rz = float(r @ z)
        while it < max_iter:
            rn = float(np.linalg.norm(r)) / bnorm
            hist.append(rn)
            if rn <= tol:
                break
            q = A @ p
            alpha = rz / float(p @ q)
            x += alpha * p
            r -= alpha * q
            z = dinv * r
            rz_new = float(r @ z)
            p = z + (rz_new / rz) * p
            rz = rz_new
            it += 1
        true = float(np.linalg.norm(b - A @ x)) / bnorm
        if true <= tol or it >= max_iter or restarts >= max_restarts:
            return PCGResult(x, it, true, hist)
        restarts += 1


def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^T (column by column, no pivoting).
    Raises ValueError if A is not positive definite."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        d = A[j, j] - L[j, :j] @ L[j, :j]
        if not d > 0.0:
            raise ValueError(f"not positive definite at column {j}")
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve A x = b by forward and back substitution on the Cholesky factor."""
    L = cholesky(A)
    n = L.shape[0]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x
