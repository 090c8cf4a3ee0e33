"""Learned coarse solve inside truncated flexible CG, in plain FP64 numpy
(oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component and solves directly.  This is the
reading the build adopts for a network that maps a pooled residual to a
coarse displacement correction (the coarse space of oracle/coarse.py):

  * pooled residual: r_c = Pi^T r, the restriction of r onto the trilinear
    functions of a grid of patch centres (a weighted pooling over the
    patches around each centre);
  * features: x = r_c / RMS(r_c) (zero when r_c = 0);
  * network: mlp.forward with dims (n_c, hidden, n_c), n_c = 3 x centres:
    n_c -> hidden -> GELU -> hidden -> GELU -> n_c;
  * training target: the Galerkin coarse solution y* = A_c^-1 r_c divided by
    its RMS.  Pi^T (r - A Pi y*) = 0, so Pi y* is the A-orthogonal projection
    of the error A^-1 r onto the coarse space: the pairs (r, y*) are
    residual/error pairs of the coarse problem;
  * correction: z = D^-1 r + alpha Pi y with y the network output and
    alpha = y.r_c / y.A_c y (Pi y.r = y.r_c and Pi y.A Pi y = y.A_c y, so
    alpha is the A-optimal step along Pi y), alpha = 0 when y.A_c y <= 0;
  * solver: flexible CG whose new direction is A-orthogonalised against the
    last m directions (truncated FCG, m = 5 by default), exact line search
    along it.  With a fixed SPD preconditioner this is PCG.
"""
from __future__ import annotations

import math

import numpy as np

from . import mlp

HIDDEN = 128


def dims(n_c: int, hidden: int = HIDDEN):
    """Layer widths of the coarse network: n_c -> hidden -> hidden -> n_c
    (returned as input, hidden and output width)."""
    return (n_c, hidden, n_c)


def n_params(n_c: int, hidden: int = HIDDEN) -> int:
    """Parameter count of the coarse network (oracle/mlp.py layout)."""
    return mlp.n_params(n_c, hidden, n_c)


def features(r: np.ndarray, Pi) -> tuple:
    """(x, r_c, s): the restricted residual r_c = Pi^T r, its RMS s and the
    network input x = r_c / s (zeros when s = 0)."""
    rc = Pi.T @ r
    s = math.sqrt(float(np.mean(rc * rc)))
    return (rc / s if s > 0 else np.zeros_like(rc)), rc, s


def target(rc: np.ndarray, Ac: np.ndarray) -> np.ndarray:
    """A_c^-1 r_c divided by its RMS (the Galerkin coarse solution's
    direction; zeros for r_c = 0)."""
    y = np.linalg.solve(Ac, rc)
    s = math.sqrt(float(np.mean(y * y)))
    return y / s if s > 0 else y


def correction(net, r, Pi, Ac, dinv):
    """z = D^-1 r + alpha Pi y for y = net(x); returns (z, alpha).  `net`
    maps the feature vector x (n_c) to y (n_c)."""
    x, rc, s = features(r, Pi)
    if s == 0:
        return dinv * r, 0.0
    y = np.asarray(net(x), dtype=np.float64)
    yAy = float(y @ (Ac @ y))
    alpha = float(y @ rc) / yAy if yAy > 0 else 0.0
    return dinv * r + alpha * (Pi @ y), alpha


def network(theta, n_c: int, hidden: int = HIDDEN, bf16: bool = False):
    """The MLP as a function x -> y (weights rounded to bfloat16 when bf16,
    biases kept in FP32, as the inference path stores them)."""
    th = np.asarray(theta, dtype=np.float64)
    if bf16:
        W1, b1, W2, b2, W3, b3 = mlp.unpack(th, n_c, hidden, n_c)
        th = mlp.pack([mlp.to_bf16(W1), np.float32(b1), mlp.to_bf16(W2), np.float32(b2), mlp.to_bf16(W3),
                       np.float32(b3)])
    return lambda x: mlp.forward(th, np.asarray(x)[None, :], dims(n_c, hidden))[0][0]


def fcg(A, b, prec, m: int = 5, tol: float = 1e-8, max_iter: int = 100000, x0=None, record=None):
    """Truncated flexible CG.  Per iteration: z = prec(r); the direction
    p = z - sum_j (q_j.z / p_j.q_j) p_j over the last m directions (q_j =
    A p_j); q = A p; step a = p.r / p.q; x += a p; r -= a q.  Stops at the
    first recursive residual <= tol ||b||.  record (a list) receives r before
    each preconditioner application.  Returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bn = float(np.linalg.norm(b))
    P, Q, D = [], [], []
    for k in range(max_iter):
        if record is not None:
            record.append(r.copy())
        z = prec(r)
        p = z.copy()
        for pj, qj, dj in zip(P, Q, D):
            p -= (float(qj @ z) / dj) * pj
        q = A @ p
        d = float(p @ q)
        a = float(p @ r) / d
        x += a * p
        r -= a * q
        P.append(p)
        Q.append(q)
        D.append(d)
        if len(P) > m:
            P.pop(0)
            Q.pop(0)
            D.pop(0)
        if np.linalg.norm(r) <= tol * bn:
            return x, k + 1
    return x, max_iter
