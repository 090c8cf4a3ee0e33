"""Strain and stress recovery (the paper's post-processing, Sec. 3.4) in
plain FP64 numpy (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions followed here:

  * face strain: the smoothed strain eps_k = Bbar_k u_k of every face, with
    Bbar_k from the smoothing domains of Eq. 7 (fsfem.smoothing_domains_eq7,
    the Gauss-point route of Table 1) and the strain matrix of Eq. 4: Voigt
    order (xx, yy, zz, yz, zx, xy), engineering shear strains;
  * face stress: sigma_k = D eps_k with the isotropic D of fsfem.material_D;
  * nodal values: for every node, the mean of eps_k (sigma_k) over the faces
    whose triangle contains the node, weighted by V_k (the smoothing domains
    whose closure holds the node); the paper does not say how its nodal
    output is averaged, this is the reading used here;
  * von Mises stress: sqrt(((s_xx - s_yy)^2 + (s_yy - s_zz)^2
    + (s_zz - s_xx)^2) / 2 + 3 (t_yz^2 + t_zx^2 + t_xy^2)).

Faces are in the oracle's canonical order (lexicographic node triples).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fsfem as F


@dataclass
class Recovery:
    faces: F.Faces
    Vk: np.ndarray           # (N_f,)
    face_strain: np.ndarray  # (N_f, 6)
    face_stress: np.ndarray  # (N_f, 6)
    node_strain: np.ndarray  # (N_n, 6)
    node_stress: np.ndarray  # (N_n, 6)
    node_vm: np.ndarray      # (N_n,)


def von_mises(s: np.ndarray) -> np.ndarray:
    """von Mises equivalent of Voigt stresses s (..., 6)."""
    s = np.asarray(s, dtype=np.float64)
    a = s[..., 0] - s[..., 1]
    b = s[..., 1] - s[..., 2]
    c = s[..., 2] - s[..., 0]
    return np.sqrt(0.5 * (a * a + b * b + c * c) + 3.0 * (s[..., 3] ** 2 + s[..., 4] ** 2 + s[..., 5] ** 2))


def node_means(n_nodes: int, tri: np.ndarray, Vk: np.ndarray, values: np.ndarray) -> np.ndarray:
    """V_k-weighted mean over the faces whose triangle contains each node of
    per-face values (N_f, m); nodes on no face get 0."""
    acc = np.zeros((n_nodes, values.shape[1]))
    w = np.zeros(n_nodes)
    for j in range(3):
        np.add.at(acc, tri[:, j], Vk[:, None] * values)
        np.add.at(w, tri[:, j], Vk)
    return np.divide(acc, w[:, None], out=np.zeros_like(acc), where=w[:, None] > 0)


def recover(xyz, tets, E: float, nu: float, u: np.ndarray) -> Recovery:
    """Face strains and stresses and their nodal means for the displacement
    field u (3 n_nodes), by the definitions in the module docstring."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    faces = F.build_faces(tets)
    dom = F.smoothing_domains_eq7(xyz, tets, faces)
    eps = F.smoothed_strains(dom, np.asarray(u, dtype=np.float64))
    sig = eps @ F.material_D(E, nu).T
    n = xyz.shape[0]
    ns = node_means(n, faces.tri, dom.Vk, eps)
    nsig = node_means(n, faces.tri, dom.Vk, sig)
    return Recovery(faces, dom.Vk, eps, sig, ns, nsig, von_mises(nsig))
