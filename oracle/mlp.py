"""Learned coarse correction in plain FP64 numpy (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component; this is the reading the build adopts
for a small network that maps a pooled residual to a coarse displacement
correction used inside flexible PCG:

  * patches: a regular grid of np_x x np_y x np_z boxes over the mesh's
    bounding box; node n belongs to the box holding its coordinates;
  * pooling: the mean residual of each patch (3 components);
  * features of patch p: the pooled residuals of the 3x3x3 block of
    patches centred on p (zero outside the grid; 81 values) divided by the
    root-mean-square of all pooled residual components, followed by the
    patch centre normalised to [0, 1]^3 (3 values): 84 inputs;
  * network: 84 -> 128 -> GELU -> 128 -> GELU -> 3, GELU(x) = x Phi(x)
    with the exact error function;
  * prolongation: trilinear interpolation of the patch outputs between
    patch centres (clamped to the outermost centres), masked by P;
  * correction: z = D^-1 r + alpha c with alpha = c.r / c.A c.

Parameters are one flat vector in the order W1 (84x128, row-major:
input-major), b1 (128), W2 (128x128), b2, W3 (128x3), b3.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 84, 128, 3


def n_params(n_in=N_IN, hid=N_HID, n_out=N_OUT) -> int:
    """Parameter count of the three-layer network: W1, b1, W2, b2, W3, b3."""
    return n_in * hid + hid + hid * hid + hid + hid * n_out + n_out


def unpack(theta, n_in=N_IN, hid=N_HID, n_out=N_OUT):
    """Split the flat parameter vector into (W1, b1, W2, b2, W3, b3), W row-major
    (fan_in x fan_out)."""
    sizes = [(n_in, hid), (hid,), (hid, hid), (hid,), (hid, n_out), (n_out,)]
    out, k = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def pack(parts) -> np.ndarray:
    """Inverse of unpack: the parts concatenated in order, FP64."""
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


# ---- patches, pooling, features, prolongation -------------------------------

def patch_grid(xyz: np.ndarray, dims):
    """Box index of every node and the box centres (np_x, np_y, np_z, 3)."""
    lo = xyz.min(axis=0)
    hi = xyz.max(axis=0)
    ext = np.maximum(hi - lo, 1e-300)
    dims = np.asarray(dims, dtype=np.int64)
    q = np.floor((xyz - lo) / ext * dims).astype(np.int64)
    q = np.clip(q, 0, dims - 1)
    pid = (q[:, 0] * dims[1] + q[:, 1]) * dims[2] + q[:, 2]
    cent = np.stack(np.meshgrid(*[lo[a] + (np.arange(dims[a]) + 0.5) * ext[a] / dims[a] for a in range(3)],
                                indexing="ij"), axis=-1)
    return pid, cent, lo, ext


def pool(v: np.ndarray, pid: np.ndarray, n_patches: int) -> np.ndarray:
    """Mean of the nodal 3-vectors v (n_nodes*3) over each patch (empty -> 0)."""
    v3 = v.reshape(-1, 3)
    s = np.zeros((n_patches, 3))
    cnt = np.zeros(n_patches)
    np.add.at(s, pid, v3)
    np.add.at(cnt, pid, 1.0)
    return s / np.maximum(cnt, 1.0)[:, None]


def features(pooled: np.ndarray, dims) -> np.ndarray:
    """(P, 84) inputs: 3x3x3 neighbourhood of pooled residuals / RMS, then
    the normalised patch centre."""
    dx, dy, dz = dims
    g = pooled.reshape(dx, dy, dz, 3)
    rms = math.sqrt(float(np.mean(pooled ** 2)))
    scale = 1.0 / rms if rms > 0 else 0.0
    pad = np.zeros((dx + 2, dy + 2, dz + 2, 3))
    pad[1:-1, 1:-1, 1:-1] = g * scale
    X = np.zeros((dx, dy, dz, N_IN))
    k = 0
    for a in range(3):
        for b in range(3):
            for c in range(3):
                X[..., 3 * k:3 * k + 3] = pad[a:a + dx, b:b + dy, c:c + dz]
                k += 1
    ii, jj, kk = np.meshgrid(np.arange(dx), np.arange(dy), np.arange(dz), indexing="ij")
    X[..., 81] = (ii + 0.5) / dx
    X[..., 82] = (jj + 0.5) / dy
    X[..., 83] = (kk + 0.5) / dz
    return X.reshape(-1, N_IN)


def prolong(c_patch: np.ndarray, dims, xyz, lo, ext) -> np.ndarray:
    """Trilinear interpolation of patch values (P, 3) at the nodes, with the
    patch centres as interpolation points, clamped to the outermost ones.
    Along an axis with a single patch the value is constant."""
    dims = np.asarray(dims, dtype=np.int64)
    g = c_patch.reshape(dims[0], dims[1], dims[2], 3)
    t = (xyz - lo) / ext * dims - 0.5        # continuous patch-centre coordinate
    t = np.clip(t, 0.0, np.maximum(dims - 1, 0).astype(np.float64))
    i0 = np.clip(np.floor(t).astype(np.int64), 0, np.maximum(dims - 2, 0))
    f = np.where(dims > 1, t - i0, 0.0)
    out = np.zeros((xyz.shape[0], 3))
    for a in (0, 1):
        for b in (0, 1):
            for cc in (0, 1):
                idx = np.minimum(i0 + np.array([a, b, cc]), dims - 1)
                w = ((f[:, 0] if a else 1 - f[:, 0]) * (f[:, 1] if b else 1 - f[:, 1]) *
                     (f[:, 2] if cc else 1 - f[:, 2]))
                out += w[:, None] * g[idx[:, 0], idx[:, 1], idx[:, 2]]
    return out.ravel()


# ---- network ------------------------------------------------------------------

def gelu(x):
    """GELU(x) = x Phi(x), Phi the standard normal CDF (Hendrycks and Gimpel 2016)."""
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d GELU / dx = Phi(x) + x phi(x), phi the standard normal density."""
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    Phi = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    return Phi + x * phi


def forward(theta, X, dims=(N_IN, N_HID, N_OUT)):
    """Network outputs (rows, n_out) and the cached pre-activations; dims =
    (n_in, hidden, n_out), the per-patch network's by default."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, *dims)
    a1 = X @ W1 + b1
    h1 = gelu(a1)
    a2 = h1 @ W2 + b2
    h2 = gelu(a2)
    y = h2 @ W3 + b3
    return y, (X, a1, h1, a2, h2)


def loss_and_grad(theta, X, T, dims=(N_IN, N_HID, N_OUT)):
    """Mean-squared error sum((y - T)^2) / rows and its gradient, by the
    chain rule through the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, *dims)
    y, (X_, a1, h1, a2, h2) = forward(theta, X, dims)
    rows = X.shape[0]
    d = y - T
    loss = float(np.sum(d * d) / rows)
    dy = 2.0 * d / rows
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3.T
    da2 = dh2 * gelu_grad(a2)
    gW2 = h1.T @ da2
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2.T
    da1 = dh1 * gelu_grad(a1)
    gW1 = X_.T @ da1
    gb1 = da1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba): biased moments, bias correction, update.
    Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (round to nearest even), returned as
    float64 for arithmetic."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def correction(theta, r, dims, pid, xyz, lo, ext, free, apply_A, dinv):
    """z = D^-1 r + alpha c, c = P prolong(net(features(pool(r)))),
    alpha = c.r / c.A c (0 when c.A c <= 0)."""
    P = int(np.prod(dims))
    X = features(pool(r, pid, P), dims)
    y, _ = forward(theta, X)
    c = prolong(y, dims, xyz, lo, ext) * free
    Ac = apply_A(c)
    cAc = float(c @ Ac)
    alpha = float(c @ r) / cAc if cAc > 0 else 0.0
    return dinv * r + alpha * c, alpha
