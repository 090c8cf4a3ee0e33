"""Pins of the oracle's strain and stress recovery (oracle/recover.py)
against closed forms and independent constructions:
- a linear displacement field gives the exact strain sym(H) on every face
  and node (the patch property of the smoothed strain), its stress D sym(H),
  and the von Mises stress of that state from its principal stresses;
- a single tet: every face strain equals the tet's FEM strain, formed from
  the Jacobian-route gradients (not the Eq. 7 route the oracle uses);
- von Mises closed forms: uniaxial, pure shear, hydrostatic;
- the vectorised nodal means against a per-node loop on a small mesh.
"""
import numpy as np

from inputs.kuhn_beam import kuhn_beam
from oracle import fsfem as F
from oracle import recover as R


def _voigt_strain(H):
    e = 0.5 * (H + H.T)
    return np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[2, 0], 2 * e[0, 1]])


def _vm_principal(s):
    T = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
    p = np.linalg.eigvalsh(T)
    return np.sqrt(0.5 * ((p[0] - p[1]) ** 2 + (p[1] - p[2]) ** 2 + (p[2] - p[0]) ** 2))


def test_linear_field_exact():
    m = kuhn_beam(3, 3, 3, (1.0, 2.0, 1.5), 0.1, seed=11)
    rng = np.random.default_rng(3)
    H = rng.standard_normal((3, 3)) * 1e-3
    a = rng.standard_normal(3)
    u = (a[None, :] + m.xyz @ H.T).ravel()
    E, nu = 210e9, 0.3
    r = R.recover(m.xyz, m.tets, E, nu, u)
    want = _voigt_strain(H)
    # rounding scale: the strain sums terms b_I u_I of size |u| / h with the
    # translation a included (cell size h ~ 0.5 here)
    tol = 1e-12 * np.abs(u).max()
    assert np.abs(r.face_strain - want).max() <= tol
    assert np.abs(r.node_strain - want).max() <= tol
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    e = 0.5 * (H + H.T)
    S = lam * np.trace(e) * np.eye(3) + 2 * mu * e
    sig = np.array([S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[2, 0], S[0, 1]])
    assert np.abs(r.face_stress - sig).max() <= 3 * (lam + 2 * mu) * tol
    assert np.abs(r.node_stress - sig).max() <= 3 * (lam + 2 * mu) * tol
    assert np.allclose(r.node_vm, _vm_principal(sig), rtol=1e-10)


def test_single_tet_faces_equal_fem_strain():
    xyz = np.array([[0.1, 0.0, 0.2], [1.3, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.2, 1.1]])
    tets = np.array([[0, 1, 2, 3]])
    u = np.random.default_rng(4).standard_normal(12)
    g = F.tet_gradients_jacobian(xyz, tets)[0]          # (4, 3)
    Hu = u.reshape(4, 3).T @ g                            # du_i / dx_j
    want = _voigt_strain(Hu)
    r = R.recover(xyz, tets, 1.0, 0.25, u)
    assert r.face_strain.shape == (4, 6)
    assert np.allclose(r.face_strain, want[None, :], rtol=1e-12, atol=1e-14)
    assert np.allclose(r.node_strain, want[None, :], rtol=1e-12, atol=1e-14)


def test_von_mises_closed_forms():
    assert np.isclose(R.von_mises(np.array([7.0, 0, 0, 0, 0, 0])), 7.0)
    assert np.isclose(R.von_mises(np.array([0, 0, 0, 0, 0, 2.0])), 2.0 * np.sqrt(3.0))
    assert np.isclose(R.von_mises(np.array([0, 0, 0, 1.5, 0, 0])), 1.5 * np.sqrt(3.0))
    assert abs(R.von_mises(np.array([-4.0, -4.0, -4.0, 0, 0, 0]))) < 1e-12
    s = np.random.default_rng(5).standard_normal(6)
    assert np.isclose(R.von_mises(s), _vm_principal(s))


def test_node_means_against_loop():
    m = kuhn_beam(2, 1, 2, (1.0, 1.0, 1.0), 0.1, seed=12)
    faces = F.build_faces(m.tets)
    dom = F.smoothing_domains_eq7(m.xyz, m.tets, faces)
    vals = np.random.default_rng(6).standard_normal((faces.n, 6))
    got = R.node_means(m.n_nodes, faces.tri, dom.Vk, vals)
    for node in range(m.n_nodes):
        sel = np.nonzero((faces.tri == node).any(axis=1))[0]
        want = (dom.Vk[sel, None] * vals[sel]).sum(0) / dom.Vk[sel].sum()
        assert np.allclose(got[node], want, rtol=1e-13, atol=1e-15)
