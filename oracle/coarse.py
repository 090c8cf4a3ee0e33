"""Two-level (Jacobi + Galerkin coarse correction) preconditioner in plain
FP64 numpy (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves with a direct method; the library's PCG may add a coarse
correction to its Jacobi preconditioner.  Definitions followed here:

  * coarse space: one trilinear "hat" function per patch centre and
    displacement component on a regular d0 x d1 x d2 grid of patch centres
    over the mesh's bounding box (centre i at lo + (i + 1/2) ext / d), i.e.
    the interpolation of oracle/mlp.py's prolong; Pi is the n x 3P matrix of
    these functions at the nodes, masked by P (zero on prescribed DOFs);
  * Galerkin coarse matrix A_c = Pi^T A Pi (A the masked system matrix);
  * preconditioner M^-1 = D^-1 + Pi A_c^-1 Pi^T (additive two-level);
  * PCG with M^-1 and the usual Fletcher-Reeves beta.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import mlp


def prolongation(xyz: np.ndarray, dims, free: np.ndarray) -> sp.csr_matrix:
    """Pi (3 n_nodes x 3P): column 3j + c is the trilinear function of
    centre j in component c, evaluated at the nodes (rows 3n + c) through
    mlp.prolong applied to unit coarse vectors, then masked by free."""
    P = int(np.prod(dims))
    _, _, lo, ext = mlp.patch_grid(xyz, dims)
    cols = []
    for j in range(3 * P):
        y = np.zeros(3 * P)
        y[j] = 1.0
        cols.append(sp.csr_matrix(mlp.prolong(y.reshape(P, 3), dims, xyz, lo, ext) * free).T)
    return sp.hstack(cols).tocsr()


def galerkin(A: sp.spmatrix, Pi: sp.spmatrix) -> np.ndarray:
    """Dense A_c = Pi^T A Pi."""
    return np.asarray((Pi.T @ (A @ Pi)).todense())


def apply_two_level(r: np.ndarray, dinv: np.ndarray, Pi: sp.spmatrix, Ac: np.ndarray) -> np.ndarray:
    """z = D^-1 r + Pi A_c^-1 Pi^T r (A_c solved by Cholesky)."""
    return dinv * r + Pi @ sla.cho_solve(sla.cho_factor(Ac), Pi.T @ r)


def two_level_pcg(A, b, dinv, Pi, Ac, tol=1e-8, max_iter=100000):
    """PCG with the additive two-level preconditioner; returns (x, iters)
    at the first recursive residual <= tol ||b||."""
    fac = sla.cho_factor(Ac)
    prec = lambda r: dinv * r + Pi @ sla.cho_solve(fac, Pi.T @ r)
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = float(z @ r)
    bn = np.linalg.norm(b)
    for k in range(max_iter):
        q = A @ p
        a = rz / float(p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            return x, k + 1
        z = prec(r)
        rzn = float(z @ r)
        p = z + (rzn / rz) * p
        rz = rzn
    return x, max_iter
