"""Pins of the learned-correction oracle (oracle/mlp.py): closed forms of
GELU, the gradient against central finite differences, one Adam step in
closed form, pooling and prolongation of constant and linear fields,
feature layout and zero padding, bfloat16 rounding."""
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
