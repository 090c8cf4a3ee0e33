"""ES-FEM-T4, the edge-based smoothed FEM (the third S-FEM model the paper
lists with FS-FEM and NS-FEM, Sec. 2.1), in plain FP64 numpy / scipy
(oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions followed here (the edge-domain counterpart of Eq. 2-9):

  * smoothing domain of edge k: a sixth of every tet that contains the edge
    (a tet has six edges), V_k = sum_{e ni k} V_e / 6;
  * smoothed gradient of node I over that domain:
    b_{k,I} = sum_{e ni k, I in e} (V_e / 6) grad N_I^e / V_k;
  * K = sum_k V_k Bbar_k^T D Bbar_k (Eq. 4 strain matrices side by side).

Assembled edge by edge from these definitions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fsfem as F


def edges_of(tets) -> dict:
    """(a, b) with a < b -> the tets that contain the edge, ascending."""
    out: dict = {}
    for e, t in enumerate(np.asarray(tets, dtype=np.int64)):
        for i in range(4):
            for j in range(i + 1, 4):
                a, b = sorted((int(t[i]), int(t[j])))
                out.setdefault((a, b), []).append(e)
    return out


def assemble_es(xyz, tets, E: float, nu: float) -> sp.csr_matrix:
    """The unconstrained ES-FEM stiffness (3 n_nodes square, CSR)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    V = F.tet_volumes(xyz, tets)
    G = F.tet_gradients_jacobian(xyz, tets)
    D = F.material_D(E, nu)
    n = xyz.shape[0]
    rows, cols, vals = [], [], []
    for _, around in sorted(edges_of(tets).items()):
        Vk = sum(V[e] / 6.0 for e in around)
        support = sorted({int(v) for e in around for v in tets[e]})
        where = {v: k for k, v in enumerate(support)}
        b = np.zeros((len(support), 3))
        for e in around:
            for a in range(4):
                b[where[int(tets[e, a])]] += (V[e] / 6.0) * G[e, a]
        b /= Vk
        Bm = F.strain_matrix(b).transpose(1, 0, 2).reshape(6, 3 * len(support))
        Kk = Vk * (Bm.T @ D @ Bm)
        dofs = (3 * np.array(support)[:, None] + np.arange(3)[None, :]).ravel()
        rows.append(np.repeat(dofs, dofs.size))
        cols.append(np.tile(dofs, dofs.size))
        vals.append(Kk.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * n, 3 * n))
    return K.tocsr()
