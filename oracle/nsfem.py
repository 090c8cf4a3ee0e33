"""NS-FEM-T4, the node-based smoothed FEM (one of the S-FEM models the paper
lists beside FS-FEM, Sec. 2.1), in plain FP64 numpy / scipy (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions followed here (the node-domain counterpart of Eq. 2-9):

  * smoothing domain of node n: a quarter of every tet that contains it,
    V_n = sum_{e ni n} V_e / 4;
  * smoothed gradient of node I over that domain:
    b_{n,I} = sum_{e ni n, I in e} (V_e / 4) grad N_I^e / V_n, for every node I
    of the tets around n (the support of the domain);
  * K = sum_n V_n Bbar_n^T D Bbar_n, Bbar_n the strain matrices of Eq. 4 of
    the b_{n,I} side by side.

Assembled node by node from these definitions (the GPU applies the same K
through per-tet strains and per-node stresses).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fsfem as F


def assemble_ns(xyz, tets, E: float, nu: float) -> sp.csr_matrix:
    """The unconstrained NS-FEM stiffness (3 n_nodes square, CSR)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    V = F.tet_volumes(xyz, tets)
    G = F.tet_gradients_jacobian(xyz, tets)     # (n_tets, 4, 3)
    D = F.material_D(E, nu)
    n = xyz.shape[0]
    around = [[] for _ in range(n)]
    for e in range(tets.shape[0]):
        for v in tets[e]:
            around[int(v)].append(e)
    rows, cols, vals = [], [], []
    for node in range(n):
        if not around[node]:
            continue
        Vn = sum(V[e] / 4.0 for e in around[node])
        support = sorted({int(v) for e in around[node] for v in tets[e]})
        where = {v: k for k, v in enumerate(support)}
        b = np.zeros((len(support), 3))
        for e in around[node]:
            for a in range(4):
                b[where[int(tets[e, a])]] += (V[e] / 4.0) * G[e, a]
        b /= Vn
        Bm = F.strain_matrix(b).transpose(1, 0, 2).reshape(6, 3 * len(support))
        Kn = Vn * (Bm.T @ D @ Bm)
        dofs = (3 * np.array(support)[:, None] + np.arange(3)[None, :]).ravel()
        rows.append(np.repeat(dofs, dofs.size))
        cols.append(np.tile(dofs, dofs.size))
        vals.append(Kn.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * n, 3 * n))
    return K.tocsr()
