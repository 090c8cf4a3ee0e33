"""Pins of the oracle's NS-FEM-T4 and ES-FEM-T4 stiffnesses (oracle/nsfem.py,
oracle/esfem.py) against what the mathematics fixes: a single tet gives the
textbook FEM-T4 stiffness (every node or edge domain is a part of the tet
with its own gradients), rigid motions lie in the null space, a linear field
is in equilibrium at interior nodes (the patch test), K is symmetric, and
both are softer than FEM-T4 (K_FEM - K positive semi-definite: on each
smoothing domain the mean strain's energy is at most the mean energy, by
convexity)."""
import numpy as np
import pytest

from inputs.kuhn_beam import kuhn_beam
from oracle import fsfem as F
from oracle import esfem as ES
from oracle import nsfem as N

ASSEMBLE = {"ns": N.assemble_ns, "es": ES.assemble_es}


def _rigid(xyz):
    n = xyz.shape[0]
    out = []
    for a in range(3):
        t = np.zeros((n, 3))
        t[:, a] = 1.0
        out.append(t.ravel())
    for w in np.eye(3):
        out.append(np.cross(w[None, :], xyz).ravel())
    return np.stack(out, 1)


@pytest.mark.parametrize("model", ["ns", "es"])
def test_single_tet_is_fem(model):
    xyz = np.array([[0.1, 0.0, 0.2], [1.3, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.2, 1.1]])
    tets = np.array([[0, 1, 2, 3]])
    Kns = ASSEMBLE[model](xyz, tets, 210e9, 0.3).toarray()
    Kfem = F.dense_K_fem(xyz, tets, 210e9, 0.3)
    assert np.abs(Kns - Kfem).max() <= 1e-12 * np.abs(Kfem).max()


@pytest.mark.parametrize("model", ["ns", "es"])
def test_null_space_symmetry_and_patch(model):
    m = kuhn_beam(3, 3, 3, (1.0, 2.0, 1.5), 0.1, seed=11)
    K = ASSEMBLE[model](m.xyz, m.tets, 210e9, 0.3)
    Kd = K.toarray()
    scale = np.abs(Kd).max()
    assert np.abs(Kd - Kd.T).max() <= 1e-12 * scale
    R = _rigid(m.xyz)
    assert np.abs(K @ R).max() <= 1e-10 * scale * np.abs(R).max()
    H = np.random.default_rng(4).standard_normal((3, 3)) * 1e-3
    u = (m.xyz @ H.T).ravel()
    lat = m.lattice()
    interior = np.all((lat > 0) & (lat < np.array([m.nx, m.ny, m.nz])), axis=1)
    f = (K @ u).reshape(-1, 3)
    assert np.abs(f[interior]).max() <= 1e-10 * scale * np.abs(u).max()
    assert np.abs(f[~interior]).max() > 1e-6 * scale * np.abs(u).max()  # boundary tractions remain


@pytest.mark.parametrize("model", ["ns", "es"])
def test_softer_than_fem(model):
    m = kuhn_beam(2, 1, 1, (2.0, 1.0, 1.0), 0.1, seed=5)
    Kns = ASSEMBLE[model](m.xyz, m.tets, 1.0, 0.3).toarray()
    Kfem = F.dense_K_fem(m.xyz, m.tets, 1.0, 0.3)
    ev = np.linalg.eigvalsh(Kfem - Kns)
    assert ev.min() >= -1e-12 * np.abs(Kfem).max()
    assert ev.max() > 1e-6 * np.abs(Kfem).max()  # strictly softer somewhere
