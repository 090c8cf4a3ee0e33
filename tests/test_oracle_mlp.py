"""Pins of the learned-correction oracle (oracle/mlp.py): closed forms of
GELU, the gradient against central finite differences, one Adam step in
closed form, pooling and prolongation of constant and linear fields,
feature layout and zero padding, bfloat16 rounding, the forward pass of a
network whose output is a closed form in GELU values, and the correction
z = D^-1 r + alpha c on a hand-worked 3-DOF example and by its
A-orthogonality."""
import math

import numpy as np

from inputs.kuhn_beam import kuhn_beam
from oracle import mlp as M


def test_gelu_closed_forms():
    x = np.array([0.0, 1.0, -1.0, 3.0, -3.0, 0.5])
    g = M.gelu(x)
    assert g[0] == 0.0
    # Phi(1) = 0.8413447460685429 (standard normal CDF)
    assert abs(g[1] - 0.8413447460685429) < 1e-15
    # GELU(x) - GELU(-x) = x (Phi(x) + Phi(-x) = 1)
    assert np.allclose(g[[1, 3]] - g[[2, 4]], [1.0, 3.0], atol=1e-15)
    # derivative against a central difference
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.abs(M.gelu_grad(x) - fd).max() < 1e-9


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(size=M.n_params()) * 0.1
    X = rng.normal(size=(7, M.N_IN))
    T = rng.normal(size=(7, M.N_OUT))
    loss, g = M.loss_and_grad(theta, X, T)
    idx = rng.choice(theta.size, 60, replace=False)
    # make sure every layer is probed
    idx = np.concatenate([idx, [0, M.N_IN * M.N_HID, M.N_IN * M.N_HID + M.N_HID + 5, M.n_params() - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_and_grad(tp, X, T)[0] - M.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # the loss is the mean of squared errors over rows
    y, _ = M.forward(theta, X)
    assert np.isclose(loss, np.sum((y - T) ** 2) / 7, rtol=1e-14)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = M.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), step=1, lr=0.01)
    # after one step m_hat = g and v_hat = g^2, so the update is lr*g/(|g|+eps)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_pool_features_prolong():
    mesh = kuhn_beam(8, 4, 4, (4.0, 1.0, 1.0), 0.1, seed=3)
    dims = (4, 2, 2)
    pid, cent, lo, ext = M.patch_grid(mesh.xyz, dims)
    P = 16
    assert pid.min() == 0 and pid.max() == P - 1
    # pooling a constant field gives the constant
    c = np.tile([1.0, -2.0, 3.0], mesh.n_nodes)
    pooled = M.pool(c, pid, P)
    assert np.allclose(pooled, [1.0, -2.0, 3.0])
    # prolonging constant patch values reproduces them; linear values are
    # reproduced inside the hull of the centres
    assert np.allclose(M.prolong(pooled, dims, mesh.xyz, lo, ext), c)
    lin = 0.3 * cent.reshape(-1, 3)[:, 0:1] - 0.7 * cent.reshape(-1, 3)[:, 1:2] + np.array([[1.0, 2.0, 3.0]])
    out = M.prolong(lin, dims, mesh.xyz, lo, ext).reshape(-1, 3)
    inside = np.all((mesh.xyz >= cent[0, 0, 0]) & (mesh.xyz <= cent[-1, -1, -1]), axis=1)
    want = 0.3 * mesh.xyz[:, 0:1] - 0.7 * mesh.xyz[:, 1:2] + np.array([[1.0, 2.0, 3.0]])
    assert inside.sum() > 10
    assert np.abs(out[inside] - want[inside]).max() < 1e-12
    # features: the centre block (offset 13) is the patch's own pooled value
    # scaled by 1/RMS, corners of the grid see zero padding
    rng = np.random.default_rng(1)
    pr = rng.normal(size=(P, 3))
    X = M.features(pr, dims)
    rms = math.sqrt(np.mean(pr ** 2))
    assert np.allclose(X[:, 39:42], pr / rms)
    assert np.allclose(X[0, 0:3], 0.0)                   # (-1,-1,-1) of patch (0,0,0)
    assert np.allclose(X[0, 81:84], [0.5 / 4, 0.5 / 2, 0.5 / 2])
    g = pr.reshape(dims + (3,))
    assert np.allclose(X[0, 3 * 26:3 * 27], g[1, 1, 1] / rms)  # (+1,+1,+1) neighbour


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.0 + 2 ** -9, 3.14159265, -2.5e-3], dtype=np.float32)
    b = M.to_bf16(x)
    assert b[0] == 1.0
    assert b[1] == 1.0                                        # 1 + 2^-8: a tie, rounds to even
    assert b[2] == 1.0                                        # below half an ulp of bf16
    assert abs(b[3] - 3.140625) < 1e-12
    assert np.all(np.abs(b - x) <= np.abs(x) * 2 ** -8)


# Closed-form values used below (standard normal CDF Phi):
#   GELU(0) = 0, GELU(1) = Phi(1) = 0.8413447460685429,
#   GELU(-1) = -(1 - Phi(1)) = -0.15865525393145707,
#   GELU(2) = 2 Phi(2) = 1.9544997361036416.
PHI1 = 0.8413447460685429
GELU2 = 1.9544997361036416


def _hand_network():
    """A network whose output is a closed form in GELU values.

    Layer 1: hidden 0 = X[0], hidden 2 = -X[0], hidden 3 = bias 2.
    Layer 2 (not symmetric): hidden 1 = h1[0] - h1[2], hidden 4 = h1[3] - GELU(2).
    Layer 3: y0 = 2 h2[1] + 0.25, y1 = 10 h2[4], y2 = -h2[1]."""
    W1 = np.zeros((M.N_IN, M.N_HID))
    b1 = np.zeros(M.N_HID)
    W2 = np.zeros((M.N_HID, M.N_HID))
    b2 = np.zeros(M.N_HID)
    W3 = np.zeros((M.N_HID, M.N_OUT))
    b3 = np.zeros(M.N_OUT)
    W1[0, 0] = 1.0
    W1[0, 2] = -1.0
    b1[3] = 2.0
    W2[0, 1] = 1.0
    W2[2, 1] = -1.0
    W2[3, 4] = 1.0
    b2[4] = -GELU2
    W3[1, 0] = 2.0
    W3[4, 1] = 10.0
    W3[1, 2] = -1.0
    b3[0] = 0.25
    return M.pack([W1, b1, W2, b2, W3, b3])


def test_forward_hand_network():
    """Pins forward() by values worked out by hand from GELU closed forms.

    Row 0 (X[0] = 1): h1 = (GELU(1), 0, GELU(-1), GELU(2), 0, ...),
    a2[1] = GELU(1) - GELU(-1) = 1, so h2[1] = GELU(1) = Phi(1); a2[4] = 0.
    Row 1 (X = 0): only the bias unit is on, a2[1] = 0.
    A transposed W2 routes nothing into hidden 1 (y0 = 0.25 on row 0), a GELU
    on the output layer changes y0 = 2 Phi(1) + 0.25, a bias added after the
    GELU of layer 1 leaves a2[4] = 2 - GELU(2) instead of 0."""
    theta = _hand_network()
    X = np.zeros((2, M.N_IN))
    X[0, 0] = 1.0
    X[0, 50] = 7.0          # an input no weight reads
    y, (X_, a1, h1, a2, h2) = M.forward(theta, X)
    assert abs(h1[0, 0] - PHI1) < 1e-15
    assert abs(h1[0, 2] - (-(1.0 - PHI1))) < 1e-15
    assert abs(h1[0, 3] - GELU2) < 1e-15
    assert abs(a2[0, 1] - 1.0) < 1e-15
    want = np.array([[2.0 * PHI1 + 0.25, 0.0, -PHI1],
                     [0.25, 0.0, 0.0]])
    assert np.abs(y - want).max() < 1e-14, y


def _one_node_problem(free):
    """One node (3 DOFs), one patch: pooling returns r, prolongation returns
    the patch value.  A = [[2,1,0],[1,3,0],[0,0,1]], D^-1 = diag(1/2, 1/3, 1)."""
    A = np.array([[2.0, 1.0, 0.0], [1.0, 3.0, 0.0], [0.0, 0.0, 1.0]])
    xyz = np.array([[0.3, 0.2, 0.1]])
    dims = (1, 1, 1)
    pid, _, lo, ext = M.patch_grid(xyz, dims)
    dinv = np.array([0.5, 1.0 / 3.0, 1.0])
    return A, xyz, dims, pid, lo, ext, np.asarray(free, dtype=np.float64), dinv


def test_correction_hand_example():
    """z = D^-1 r + alpha c on a 3-DOF example worked out by hand.

    The network has zero weights and output bias (1, 2, 0), so c = P (1, 2, 0).
    r = (1, 0, 2): all free -> c.r = 1, A c = (4, 7, 0), c.A c = 18,
    alpha = 1/18, z = (1/2 + 1/18, 2/18, 2).  Second DOF prescribed ->
    c = (1, 0, 0), A c = (2, 1, 0), c.A c = 2, alpha = 1/2, z = (1, 0, 2).
    A sign flip in alpha gives z0 = 1/2 - 1/18 (resp. 0)."""
    theta = np.zeros(M.n_params())
    theta[-3:] = [1.0, 2.0, 0.0]
    r = np.array([1.0, 0.0, 2.0])
    A, xyz, dims, pid, lo, ext, free, dinv = _one_node_problem([1, 1, 1])
    z, alpha = M.correction(theta, r, dims, pid, xyz, lo, ext, free, lambda v: A @ v, dinv)
    assert abs(alpha - 1.0 / 18.0) < 1e-16
    assert np.abs(z - [0.5 + 1.0 / 18.0, 2.0 / 18.0, 2.0]).max() < 1e-15
    A, xyz, dims, pid, lo, ext, free, dinv = _one_node_problem([1, 0, 1])
    z, alpha = M.correction(theta, r, dims, pid, xyz, lo, ext, free, lambda v: A @ v, dinv)
    assert abs(alpha - 0.5) < 1e-16
    assert np.abs(z - [1.0, 0.0, 2.0]).max() < 1e-15


def test_correction_orthogonality_and_zero_network():
    """alpha makes the corrected residual A-orthogonal to c,
    c.(r - alpha A c) = 0, on a beam with a random network; a network that
    outputs zero gives z = D^-1 r and alpha = 0."""
    mesh = kuhn_beam(6, 2, 2, (3.0, 1.0, 1.0), 0.1, seed=2)
    dims = (3, 1, 1)
    pid, _, lo, ext = M.patch_grid(mesh.xyz, dims)
    rng = np.random.default_rng(4)
    n = 3 * mesh.n_nodes
    B = rng.normal(size=(n, n)) / math.sqrt(n)
    A = B @ B.T + np.eye(n)                      # symmetric positive definite
    free = (rng.random(n) > 0.2).astype(np.float64)
    dinv = 1.0 / np.diag(A)
    r = rng.normal(size=n) * free
    theta = rng.normal(size=M.n_params()) * 0.2
    z, alpha = M.correction(theta, r, dims, pid, mesh.xyz, lo, ext, free, lambda v: A @ v, dinv)
    c = (z - dinv * r) / alpha
    assert np.all(c[free == 0] == 0.0)
    assert abs(c @ (r - alpha * (A @ c))) <= 1e-12 * abs(c @ r)
    z0, alpha0 = M.correction(np.zeros(M.n_params()), r, dims, pid, mesh.xyz, lo, ext, free,
                              lambda v: A @ v, dinv)
    assert alpha0 == 0.0
    assert np.array_equal(z0, dinv * r)
