"""Pins of the learned coarse solve (oracle/cnet.py): truncated flexible CG
against textbook PCG, the correction's special cases (a network that returns
the Galerkin coarse solution gives the two-level preconditioner of
oracle/coarse.py; a zero output gives Jacobi; alpha is the A-optimal step),
features and targets by their defining properties, and the generic-size
forward pass by a network with a closed-form output."""
import math

import numpy as np
import scipy.sparse as sp

from inputs.kuhn_beam import cantilever
from oracle import cnet as CN
from oracle import coarse as OC
from oracle import fsfem as F
from oracle import mlp as M
from oracle import solve as OS

PHI1 = 0.8413447460685429   # Phi(1) = GELU(1)


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n)) / math.sqrt(n)
    return B @ B.T + 0.1 * np.eye(n), rng


def test_fcg_with_fixed_preconditioner_is_pcg():
    """With a fixed SPD preconditioner, truncated FCG (any m >= 1) produces
    the PCG iterates: same iteration count and solution to rounding (tol
    1e-12), which is the direct solution."""
    A, rng = _spd(40, 1)
    b = rng.normal(size=40)
    dinv = 1.0 / np.diag(A)
    ref = OS.jacobi_pcg(sp.csr_matrix(A), b, tol=1e-12, max_iter=1000, max_restarts=0)
    for m in (1, 3, 8):
        x, it = CN.fcg(A, b, lambda r: dinv * r, m=m, tol=1e-12)
        assert abs(it - ref.iterations) <= 1, (m, it, ref.iterations)
        assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    x_direct = np.linalg.solve(A, b)
    assert np.linalg.norm(x - x_direct) <= 1e-9 * np.linalg.norm(x_direct)


def test_fcg_directions_are_a_orthogonal_within_the_window():
    """With a preconditioner that changes every iteration (a random positive
    diagonal each call), each direction is A-orthogonal to the m before it,
    and the method still converges."""
    A, rng = _spd(30, 2)
    b = rng.normal(size=30)
    calls = []

    def prec(r):
        d = rng.uniform(0.5, 2.0, size=r.size)
        calls.append(d)
        return d * r
    # recompute the directions the way fcg does, recording them
    m = 4
    x = np.zeros(30)
    r = b.copy()
    P, Q, Dd = [], [], []
    allp = []
    for k in range(25):
        z = prec(r)
        p = z.copy()
        for pj, qj, dj in zip(P, Q, Dd):
            p -= (qj @ z) / dj * pj
        q = A @ p
        allp.append(p)
        d = p @ q
        a = (p @ r) / d
        x += a * p
        r -= a * q
        P.append(p); Q.append(q); Dd.append(d)
        if len(P) > m:
            P.pop(0); Q.pop(0); Dd.pop(0)
    for k in range(1, len(allp)):
        for j in range(max(0, k - m), k):
            c = allp[k] @ (A @ allp[j])
            assert abs(c) <= 1e-10 * math.sqrt((allp[k] @ A @ allp[k]) * (allp[j] @ A @ allp[j])), (k, j)
    xs, it = CN.fcg(A, b, prec, m=m, tol=1e-10, max_iter=2000)
    assert it < 2000 and np.linalg.norm(A @ xs - b) <= 1e-9 * np.linalg.norm(b)


def _beam_system():
    p = cantilever(8, 2, 2, seed=2)
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, free, g = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    A = A.tocsr()
    n = A.shape[0]
    freef = np.ones(n)
    freef[p.dir_dofs] = 0
    Pi = OC.prolongation(m.xyz, (3, 2, 2), freef)
    Ac = OC.galerkin(A, Pi)
    return A, b, freef, Pi, Ac, 1.0 / A.diagonal()


def test_correction_special_cases():
    """A network that returns the Galerkin coarse solution's direction makes
    z the two-level preconditioner D^-1 r + Pi A_c^-1 Pi^T r (alpha rescales
    the unit-RMS direction to the solution itself); a zero output gives
    z = D^-1 r and alpha = 0; alpha is the A-optimal step along c = Pi y,
    c.(r - alpha A c) = 0 with the fine A."""
    A, b, freef, Pi, Ac, dinv = _beam_system()
    rng = np.random.default_rng(3)
    r = rng.normal(size=b.size) * freef
    exact = lambda x: CN.target(x, Ac)     # the direction of A_c^-1 x (scale-free)
    z, alpha = CN.correction(exact, r, Pi, Ac, dinv)
    z2 = OC.apply_two_level(r, dinv, Pi, Ac)
    assert np.linalg.norm(z - z2) <= 1e-10 * np.linalg.norm(z2)
    z0, a0 = CN.correction(lambda x: np.zeros_like(x), r, Pi, Ac, dinv)
    assert a0 == 0.0 and np.array_equal(z0, dinv * r)
    y = rng.normal(size=Ac.shape[0])
    z3, a3 = CN.correction(lambda x: y, r, Pi, Ac, dinv)
    c = Pi @ y
    assert abs(c @ (r - a3 * (A @ c))) <= 1e-10 * abs(c @ r)
    assert np.linalg.norm(z3 - dinv * r - a3 * c) <= 1e-12 * np.linalg.norm(z3)


def test_features_and_target_properties():
    """x is scale-invariant with unit RMS; the target, rescaled, solves the
    coarse system A_c y = r_c."""
    A, b, freef, Pi, Ac, dinv = _beam_system()
    rng = np.random.default_rng(4)
    r = rng.normal(size=b.size) * freef
    x, rc, s = CN.features(r, Pi)
    x2, _, s2 = CN.features(7.5 * r, Pi)
    assert np.allclose(x, x2, rtol=1e-13, atol=0) and abs(s2 / s - 7.5) < 1e-12
    assert abs(math.sqrt(np.mean(x * x)) - 1.0) < 1e-13
    t = CN.target(rc, Ac)
    lam = (rc @ t) / (t @ Ac @ t)             # the scale that makes t a solution
    assert np.linalg.norm(Ac @ (lam * t) - rc) <= 1e-10 * np.linalg.norm(rc)
    assert abs(math.sqrt(np.mean(t * t)) - 1.0) < 1e-13
    xz, rcz, sz = CN.features(np.zeros_like(r), Pi)
    assert sz == 0.0 and not xz.any()


def test_forward_generic_sizes_hand_network():
    """forward() at n_in = n_out = 9, hidden 16 on a network whose output is a
    closed form: y0 = 2 GELU(GELU(1) - GELU(-1)) + 0.25 = 2 Phi(1) + 0.25,
    y8 = -Phi(1) (x0 = 1), and y = (0.25, 0, ..) for x = 0."""
    n, h = 9, 16
    W1 = np.zeros((n, h)); b1 = np.zeros(h); W2 = np.zeros((h, h)); b2 = np.zeros(h)
    W3 = np.zeros((h, n)); b3 = np.zeros(n)
    W1[0, 0] = 1.0; W1[0, 2] = -1.0
    W2[0, 1] = 1.0; W2[2, 1] = -1.0
    W3[1, 0] = 2.0; W3[1, 8] = -1.0; b3[0] = 0.25
    theta = M.pack([W1, b1, W2, b2, W3, b3])
    assert theta.size == CN.n_params(n, h)
    X = np.zeros((2, n)); X[0, 0] = 1.0; X[0, 5] = 3.0
    y, _ = M.forward(theta, X, CN.dims(n, h))
    want = np.zeros((2, n)); want[0, 0] = 2 * PHI1 + 0.25; want[0, 8] = -PHI1; want[1, 0] = 0.25
    assert np.abs(y - want).max() < 1e-14
    f = CN.network(theta, n, h)
    assert np.abs(f(X[0]) - want[0]).max() < 1e-14


def test_gradient_generic_sizes_finite_differences():
    rng = np.random.default_rng(5)
    n, h = 7, 12
    d = CN.dims(n, h)
    theta = rng.normal(size=CN.n_params(n, h)) * 0.3
    X = rng.normal(size=(5, n))
    T = rng.normal(size=(5, n))
    loss, g = M.loss_and_grad(theta, X, T, d)
    eps = 1e-6
    for i in list(rng.choice(theta.size, 40, replace=False)) + [0, theta.size - 1]:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (M.loss_and_grad(tp, X, T, d)[0] - M.loss_and_grad(tm, X, T, d)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_learned_fcg_beats_jacobi_when_the_network_is_exact():
    """On a beam, truncated FCG with the exact coarse direction converges in
    far fewer iterations than Jacobi-PCG (the two-level preconditioner's
    count), so the solver loop and the correction fit together."""
    A, b, freef, Pi, Ac, dinv = _beam_system()
    _, kj = CN.fcg(A, b, lambda r: dinv * r, m=5, tol=1e-8)
    exact = lambda x: CN.target(x, Ac)
    _, kl = CN.fcg(A, b, lambda r: CN.correction(exact, r, Pi, Ac, dinv)[0], m=5, tol=1e-8)
    x2, k2 = OC.two_level_pcg(A, b, dinv, Pi, Ac, tol=1e-8)
    assert kl <= k2 + 2 and kl < 0.6 * kj, (kl, k2, kj)
