"""FS-FEM-T4 in plain FP64 numpy: geometry, faces, Eq. 7 smoothing, Eq. 9 stiffness.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): never imported by the
product path.  Loops are vectorised over tets or faces only where every tet
or face runs the same formula; nothing is blocked, fused or reordered.

Conventions
  * node and tet ids are 0-based (the paper notes TetGen is 0-based, Sec. 3.2);
  * DOF numbering is 3*node + component (x, y, z);
  * strains are in the Voigt order of Eq. 4 and Eq. 6: (xx, yy, zz, yz, zx, xy)
    with engineering shears, i.e. row 4 of B_I is (0, b_z, b_y), row 5 is
    (b_z, 0, b_x) and row 6 is (b_y, b_x, 0).
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# O1: input validation
# ---------------------------------------------------------------------------

def validate(xyz: np.ndarray, tets: np.ndarray) -> None:
    """Node ids in range, at least one tet, finite coordinates."""
    if tets.ndim != 2 or tets.shape[1] != 4 or tets.shape[0] < 1:
        raise ValueError("tets must be (n_tets>=1, 4)")
    if tets.min() < 0 or tets.max() >= xyz.shape[0]:
        raise ValueError("tet node id out of range")
    if not np.all(np.isfinite(xyz)):
        raise ValueError("non-finite coordinates")


# ---------------------------------------------------------------------------
# O2: per-tet geometry (Eq. 10, Eq. 11, face normals of Fig. 9)
# ---------------------------------------------------------------------------

def tet_volume_eq10(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Eq. 10: V = (1/6) det [[x_A y_A z_A 1], ..., [x_D y_D z_D 1]] (signed).

    With this row layout a right-handed tet (det[B-A, C-A, D-A] > 0) gives a
    negative value; the volume is its absolute value."""
    M = np.ones((tets.shape[0], 4, 4))
    M[:, :, :3] = xyz[tets]
    return np.linalg.det(M) / 6.0


def tet_volumes(xyz, tets) -> np.ndarray:
    """|V_e| of every tet (Eq. 10 without the orientation sign)."""
    return np.abs(tet_volume_eq10(xyz, tets))


def tri_area_eq11(A, B, C) -> np.ndarray:
    """Eq. 11: S = |AB x AC| / 2 (vectorised over leading axes)."""
    return 0.5 * np.linalg.norm(np.cross(B - A, C - A), axis=-1)


def tri_unit_normal(A, B, C) -> np.ndarray:
    """Unit normal AB x AC / |AB x AC| (Fig. 9, vectorin)."""
    n = np.cross(B - A, C - A)
    return n / np.linalg.norm(n, axis=-1, keepdims=True)


def outward_normal(P, Q, R, O) -> np.ndarray:
    """Unit normal of triangle PQR pointing away from the point O."""
    n = tri_unit_normal(P, Q, R)
    s = np.sign(np.einsum("...i,...i->...", n, O - P))
    return -n * s[..., None]


def tet_gradients_jacobian(xyz, tets) -> np.ndarray:
    """Shape-function gradients (n_tets, 4, 3) of the linear T4 (Eq. 1).

    x = x_0 + J xi with J = [x1-x0, x2-x0, x3-x0]; N_a = xi_a for a = 1..3, so
    grad N_a is row a of inv(J), and grad N_0 = -sum of the others."""
    X = xyz[tets]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    Ji = np.linalg.inv(J)
    G = np.empty((tets.shape[0], 4, 3))
    G[:, 1:] = Ji
    G[:, 0] = -Ji.sum(axis=1)
    return G


def tet_gradients_normals(xyz, tets) -> np.ndarray:
    """Same gradients a second way: grad N_a = -A_a n_a / (3 V), with A_a the
    area (Eq. 11) and n_a the outward unit normal of the face opposite vertex a
    (N_a falls linearly from 1 at vertex a to 0 on that face)."""
    X = xyz[tets]
    V = tet_volumes(xyz, tets)
    G = np.empty((tets.shape[0], 4, 3))
    for a in range(4):
        o = [b for b in range(4) if b != a]
        P, Q, R = X[:, o[0]], X[:, o[1]], X[:, o[2]]
        n = outward_normal(P, Q, R, X[:, a])
        G[:, a] = -(tri_area_eq11(P, Q, R) / (3.0 * V))[:, None] * n
    return G


def sliver_quality(xyz, tets) -> np.ndarray:
    """q = 6*sqrt(2)*V / l_rms^3 (1 for a regular tet, -> 0 for slivers)."""
    X = xyz[tets]
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    l2 = sum(np.sum((X[:, i] - X[:, j]) ** 2, axis=1) for i, j in pairs) / 6.0
    return 6.0 * np.sqrt(2.0) * tet_volumes(xyz, tets) / l2 ** 1.5


# ---------------------------------------------------------------------------
# O3: faces (Section 3.2, Fig. 7, Algorithm 1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Faces:
    tri: np.ndarray   # (N_f, 3) sorted node triple (the face ABC)
    tet: np.ndarray   # (N_f, 2) adjacent tets; tet[:,1] = -1 on the exterior
    opp: np.ndarray   # (N_f, 2) node of each adjacent tet not on the face; -1
    # Face_in / Face_out of Fig. 7 are tri|tet|opp restricted to interior / exterior

    @property
    def n(self) -> int:
        return self.tri.shape[0]

    @property
    def interior(self) -> np.ndarray:
        return self.tet[:, 1] >= 0

    @property
    def n_interior(self) -> int:
        return int(self.interior.sum())

    @property
    def n_boundary(self) -> int:
        return self.n - self.n_interior


def build_faces(tets: np.ndarray) -> Faces:
    """Group the four faces of every tet by their sorted node triple.

    A triple seen once is an exterior face (Face_out: face + tet + opposite
    node), one seen twice an interior face (Face_in: face + 2 tets + 2
    opposite nodes), as in Fig. 7.  Seen more than twice is a mesh error.
    Faces are returned in lexicographic order of their triples."""
    owners: dict = {}
    for e in range(tets.shape[0]):
        t = [int(v) for v in tets[e]]
        for a in range(4):
            key = tuple(sorted(t[:a] + t[a + 1:]))
            owners.setdefault(key, []).append((e, t[a]))
    keys = sorted(owners)
    nf = len(keys)
    tri = np.array(keys, dtype=np.int64).reshape(nf, 3)
    tet = -np.ones((nf, 2), dtype=np.int64)
    opp = -np.ones((nf, 2), dtype=np.int64)
    for f, k in enumerate(keys):
        lst = owners[k]
        if len(lst) > 2:
            raise ValueError(f"face {k} shared by {len(lst)} tets")
        for s, (e, o) in enumerate(lst):
            tet[f, s] = e
            opp[f, s] = o
    return Faces(tri, tet, opp)


# ---------------------------------------------------------------------------
# O4: smoothing domains and Eq. 7 with the Gauss-point values of Table 1
# ---------------------------------------------------------------------------

def gauss_point_shape_values() -> dict:
    """Table 1 from first principles, in exact rationals.

    Stencil of interior face ABC with tets ABCD (centroid F) and ABCE
    (centroid G).  N_I is 1 at its own field node, 1/4 at the centroid of a
    tet containing I; being linear on each boundary triangle, its value at the
    triangle's centroid (the Gauss point) is the mean of its three vertex
    values.  Returns {site: [N_A, N_B, N_C, N_D, N_E]}."""
    q = Fraction(1, 4)
    site = {s: [Fraction(int(s == n)) for n in "ABCDE"] for s in "ABCDE"}
    site["F"] = [q, q, q, q, Fraction(0)]
    site["G"] = [q, q, q, Fraction(0), q]
    # The six triangles of Gamma^k (two sub-tets ABCF and ABCG, three
    # triangles each, Fig. 1), named g1..g6 in the order of Table 1.
    tris = {"g1": "ACF", "g2": "ACG", "g3": "BCG", "g4": "BCF", "g5": "ABF", "g6": "ABG"}
    for g, (p, r, s) in tris.items():
        site[g] = [(site[p][i] + site[r][i] + site[s][i]) / 3 for i in range(5)]
    return site


@dataclasses.dataclass
class SmoothingDomains:
    nodes: np.ndarray  # (N_f, 5) stencil nodes [a, b, c, d0, d1]; d1 = -1 on the exterior
    Bbar: np.ndarray   # (N_f, 5, 3) smoothed gradients b_I of Eq. 5/7 (row 5 zero if exterior)
    Vk: np.ndarray     # (N_f,) smoothing-domain volumes V_k^s


def smoothing_domains_eq7(xyz, tets, faces: Faces) -> SmoothingDomains:
    """Eq. 7: b_Ih = (1/V_k) sum_{i=1..P} n_ih N_I(x_i^G) A_i for every face.

    The domain of face ABC is the union of the sub-tets ABC+centroid of each
    adjacent tet (Fig. 1, STEP 2).  Its boundary Gamma^k is made of the
    triangles (a,b,g), (b,c,g), (c,a,g) of each sub-tet, plus the face ABC
    itself when the face is exterior: P = 6 interior, P = 4 exterior.  Each
    triangle's outer normal (Fig. 9) points away from the sub-tet vertex not on
    it; its area is Eq. 11; its Gauss point is its centroid, where N_I is the
    mean of the vertex values (Table 1).  V_k is the sum of the sub-tet
    volumes, each by Eq. 10."""
    nf = faces.n
    interior = faces.interior
    nodes = np.concatenate([faces.tri, faces.opp], axis=1)          # (N_f, 5)
    P = {s: xyz[faces.tri[:, s]] for s in range(3)}                   # face vertices a, b, c
    gpos = [xyz[tets[np.maximum(faces.tet[:, s], 0)]].mean(axis=1) for s in range(2)]
    # shape values of the 5 stencil nodes at each point type
    val = {0: np.eye(5)[0], 1: np.eye(5)[1], 2: np.eye(5)[2],
           "g0": np.array([.25, .25, .25, .25, 0.]), "g1": np.array([.25, .25, .25, 0., .25])}
    Bbar = np.zeros((nf, 5, 3))
    Vk = np.zeros(nf)
    for s in range(2):
        m = np.ones(nf, bool) if s == 0 else interior
        g = gpos[s]
        # sub-tet volume by Eq. 10 on (a, b, c, g)
        sub = np.ones((nf, 4, 4))
        sub[:, 0, :3], sub[:, 1, :3], sub[:, 2, :3], sub[:, 3, :3] = P[0], P[1], P[2], g
        Vk += np.where(m, np.abs(np.linalg.det(sub)) / 6.0, 0.0)
        gv = val["g0" if s == 0 else "g1"]
        for (i, j), o in (((0, 1), 2), ((1, 2), 0), ((2, 0), 1)):
            n = outward_normal(P[i], P[j], g, P[o])
            A = tri_area_eq11(P[i], P[j], g)
            NG = (val[i] + val[j] + gv) / 3.0                       # (5,) Gauss-point values
            contrib = (n * A[:, None])[:, None, :] * NG[None, :, None]
            Bbar += np.where(m[:, None, None], contrib, 0.0)
    # the exterior face ABC itself closes Gamma^k of a boundary domain (P = 4)
    ext = ~interior
    n = outward_normal(P[0], P[1], P[2], gpos[0])
    A = tri_area_eq11(P[0], P[1], P[2])
    NG = (val[0] + val[1] + val[2]) / 3.0
    Bbar += np.where(ext[:, None, None], (n * A[:, None])[:, None, :] * NG[None, :, None], 0.0)
    Bbar /= Vk[:, None, None]
    return SmoothingDomains(nodes, Bbar, Vk)


def smoothing_domains_average(xyz, tets, faces: Faces) -> SmoothingDomains:
    """Cross-check of Eq. 2-3: the smoothed gradient is the volume average of
    the compatible gradient over Omega_k.  The gradient is constant in each tet
    and each sub-tet holds a quarter of its tet's volume (the centroid lies at a
    quarter of the height), so b_I = sum_e (V_e/4) grad N_I^e / V_k with
    V_k = sum_e V_e/4."""
    V = tet_volumes(xyz, tets)
    G = tet_gradients_jacobian(xyz, tets)
    nodes = np.concatenate([faces.tri, faces.opp], axis=1)
    nf = faces.n
    Bbar = np.zeros((nf, 5, 3))
    Vk = np.zeros(nf)
    for s in range(2):
        e = faces.tet[:, s]
        m = e >= 0
        ee = np.maximum(e, 0)
        w = np.where(m, V[ee] / 4.0, 0.0)
        Vk += w
        for slot in range(5):
            node = nodes[:, slot]
            # local index of this stencil node inside tet e (or absent)
            hit = tets[ee] == node[:, None]                          # (N_f, 4)
            present = hit.any(axis=1) & m & (node >= 0)
            loc = hit.argmax(axis=1)
            g = G[ee, loc]
            Bbar[:, slot] += np.where(present[:, None], w[:, None] * g, 0.0)
    Bbar /= Vk[:, None, None]
    return SmoothingDomains(nodes, Bbar, Vk)


# ---------------------------------------------------------------------------
# O5: material matrix (Eq. 9's c, isotropic; Voigt order of Eq. 4)
# ---------------------------------------------------------------------------

def lame(E: float, nu: float):
    """Lame parameters (lambda, mu) of Young's modulus E and Poisson ratio nu
    (isotropic linear elasticity, the material of Sec. 4)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def material_D(E: float, nu: float) -> np.ndarray:
    """6x6 isotropic elasticity matrix, Voigt (xx, yy, zz, yz, zx, xy),
    engineering shear strains."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] = lam + 2.0 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    return D


def strain_matrix(b: np.ndarray) -> np.ndarray:
    """Eq. 4: the 6x3 matrix B_I of a gradient vector b = (b_x, b_y, b_z)
    (vectorised over leading axes)."""
    B = np.zeros(b.shape[:-1] + (6, 3))
    B[..., 0, 0] = b[..., 0]
    B[..., 1, 1] = b[..., 1]
    B[..., 2, 2] = b[..., 2]
    B[..., 3, 1], B[..., 3, 2] = b[..., 2], b[..., 1]
    B[..., 4, 0], B[..., 4, 2] = b[..., 2], b[..., 0]
    B[..., 5, 0], B[..., 5, 1] = b[..., 1], b[..., 0]
    return B


# ---------------------------------------------------------------------------
# O6: smoothed stiffness (Eq. 9), COO of Eq. 12, CSR
# ---------------------------------------------------------------------------

def face_stiffness(dom: SmoothingDomains, D: np.ndarray) -> np.ndarray:
    """K_k = V_k B_k^T c B_k over the 5-node stencil (Eq. 9), (N_f, 15, 15).
    Exterior faces use the leading 12x12 block (4 nodes)."""
    B = strain_matrix(dom.Bbar)                       # (N_f, 5, 6, 3)
    Bk = np.concatenate([B[:, i] for i in range(5)], axis=2)   # (N_f, 6, 15)
    return dom.Vk[:, None, None] * (np.transpose(Bk, (0, 2, 1)) @ (D @ Bk))


def assemble_coo(dom: SmoothingDomains, Kloc: np.ndarray):
    """Triplets (IK, JK, VK) in face order, 144 per exterior face and 225 per
    interior face (Eq. 12), plus the face id of each triplet."""
    IK, JK, VK, FID = [], [], [], []
    for f in range(dom.nodes.shape[0]):
        nn = 5 if dom.nodes[f, 4] >= 0 else 4
        dof = (3 * dom.nodes[f, :nn, None] + np.arange(3)[None, :]).ravel()
        m = 3 * nn
        IK.append(np.repeat(dof, m))
        JK.append(np.tile(dof, m))
        VK.append(Kloc[f, :m, :m].ravel())
        FID.append(np.full(m * m, f))
    return (np.concatenate(IK), np.concatenate(JK), np.concatenate(VK), np.concatenate(FID))


def assemble_coo_vectorised(dom: SmoothingDomains, Kloc: np.ndarray):
    """The same triplets as assemble_coo, in the same order (face, then row
    slot, then column slot), built without the Python loop over faces: all
    15x15 slots are laid out and those beyond 12x12 of exterior faces dropped."""
    nf = dom.nodes.shape[0]
    m = np.where(dom.nodes[:, 4] >= 0, 15, 12)
    dof = (3 * np.maximum(dom.nodes, 0)[:, :, None] + np.arange(3)[None, None, :]).reshape(nf, 15)
    I = np.repeat(dof, 15, axis=1)
    J = np.tile(dof, (1, 15))
    slot_i = np.repeat(np.arange(15), 15)[None, :]
    slot_j = np.tile(np.arange(15), 15)[None, :]
    keep = ((slot_i < m[:, None]) & (slot_j < m[:, None])).ravel()
    fid = np.repeat(np.arange(nf), 225)
    return I.ravel()[keep], J.ravel()[keep], Kloc.reshape(nf, 225).ravel()[keep], fid[keep]


def coo_to_csr(ndof: int, IK, JK, VK):
    """Sum duplicates of a triplet list into canonical CSR (row-major, column
    indices ascending within a row), as Julia's sparse() does for COO input
    (Section 3.3, STEP 5).  Duplicates are summed in triplet (face) order."""
    order = np.lexsort((JK, IK))                  # stable: ties keep face order
    r, c, v = IK[order], JK[order], VK[order]
    new = np.ones(r.shape[0], bool)
    new[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    starts = np.nonzero(new)[0]
    data = np.add.reduceat(v, starts) if starts.size else np.zeros(0)
    rows, cols = r[starts], c[starts]
    indptr = np.zeros(ndof + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, cols.astype(np.int32), data


@dataclasses.dataclass
class Assembly:
    ndof: int
    faces: Faces
    dom: SmoothingDomains
    D: np.ndarray
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray
    n_triplets: int

    def matrix(self) -> sp.csr_matrix:
        """The assembled stiffness as a scipy CSR matrix (3 n_nodes square)."""
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.ndof, self.ndof))


def assemble(xyz, tets, E, nu, vectorised=True, chunk=None) -> Assembly:
    """Section 3.3 end to end: faces, Eq. 7 domains, Eq. 9 face matrices,
    Eq. 12 triplets, summed into CSR (the unconstrained K).

    With chunk=n the faces are processed n at a time to bound memory: each
    chunk's triplets are summed into a CSR matrix and the chunk matrices are
    added; the sparsity structure is the same, only the order in which
    duplicate entries are added differs."""
    validate(xyz, tets)
    faces = build_faces(tets)
    dom = smoothing_domains_eq7(xyz, tets, faces)
    D = material_D(E, nu)
    ndof = 3 * xyz.shape[0]
    if chunk is None:
        Kloc = face_stiffness(dom, D)
        IK, JK, VK, _ = (assemble_coo_vectorised if vectorised else assemble_coo)(dom, Kloc)
        indptr, indices, data = coo_to_csr(ndof, IK, JK, VK)
        return Assembly(ndof, faces, dom, D, indptr, indices, data, IK.shape[0])
    rows, cols, vals = [], [], []
    n_trip = 0
    for s in range(0, faces.n, chunk):
        sub = SmoothingDomains(dom.nodes[s:s + chunk], dom.Bbar[s:s + chunk], dom.Vk[s:s + chunk])
        IK, JK, VK, _ = assemble_coo_vectorised(sub, face_stiffness(sub, D))
        n_trip += IK.shape[0]
        ip, ix, dv = coo_to_csr(ndof, IK, JK, VK)
        rows.append(np.repeat(np.arange(ndof, dtype=np.int64), np.diff(ip)))
        cols.append(ix.astype(np.int64))
        vals.append(dv)
    # merge the chunk sums with the same duplicate-summing rule (explicit
    # zeros are kept: the structure is every pair of nodes sharing a stencil)
    indptr, indices, data = coo_to_csr(ndof, np.concatenate(rows), np.concatenate(cols),
                                       np.concatenate(vals))
    return Assembly(ndof, faces, dom, D, indptr, indices, data, n_trip)


# ---------------------------------------------------------------------------
# Brute-force dense matrices for tiny meshes (independent of Eq. 7 and COO)
# ---------------------------------------------------------------------------

def fem_strain_operator(xyz, tets) -> np.ndarray:
    """Dense compatible-strain operators (n_tets, 6, ndof): eps_e = B_e u."""
    ndof = 3 * xyz.shape[0]
    G = tet_gradients_jacobian(xyz, tets)
    S = np.zeros((tets.shape[0], 6, ndof))
    B = strain_matrix(G)                                          # (n, 4, 6, 3)
    for e in range(tets.shape[0]):
        for a in range(4):
            S[e, :, 3 * tets[e, a]:3 * tets[e, a] + 3] += B[e, a]
    return S


def dense_K_bruteforce(xyz, tets, E, nu) -> np.ndarray:
    """K as the Hessian of the smoothed strain energy
    Pi(u) = 1/2 sum_k V_k eps_k(u)^T c eps_k(u), with eps_k(u) the average of
    the compatible strain over Omega_k (Eq. 2-3): eps_k = sum_e (V_e/4) B_e u / V_k.
    Built densely as S^T W S (no Eq. 7, no triplets)."""
    faces = build_faces(tets)
    V = tet_volumes(xyz, tets)
    Se = fem_strain_operator(xyz, tets)
    D = material_D(E, nu)
    ndof = 3 * xyz.shape[0]
    K = np.zeros((ndof, ndof))
    for f in range(faces.n):
        es = [e for e in faces.tet[f] if e >= 0]
        Vk = sum(V[e] / 4.0 for e in es)
        Ek = sum((V[e] / 4.0) * Se[e] for e in es) / Vk
        K += Vk * Ek.T @ D @ Ek
    return K


def dense_K_fem(xyz, tets, E, nu) -> np.ndarray:
    """Standard FEM-T4 stiffness sum_e V_e B_e^T c B_e (dense)."""
    V = tet_volumes(xyz, tets)
    Se = fem_strain_operator(xyz, tets)
    D = material_D(E, nu)
    return np.einsum("e,eri,rs,esj->ij", V, Se, D, Se)


def fem_K_csr(xyz, tets, E, nu) -> sp.csr_matrix:
    """Sparse FEM-T4 stiffness sum_e V_e B_e^T c B_e (for larger meshes)."""
    V = tet_volumes(xyz, tets)
    G = tet_gradients_jacobian(xyz, tets)
    B = strain_matrix(G)                                          # (n, 4, 6, 3)
    Be = np.concatenate([B[:, a] for a in range(4)], axis=2)      # (n, 6, 12)
    Ke = V[:, None, None] * np.einsum("eri,rs,esj->eij", Be, material_D(E, nu), Be)
    dof = (3 * tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
    ndof = 3 * xyz.shape[0]
    rows = np.repeat(dof, 12, axis=1).ravel()
    cols = np.tile(dof, (1, 12)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(ndof, ndof))


def smoothed_strains(dom: SmoothingDomains, u: np.ndarray) -> np.ndarray:
    """eps_k = B_k u on every face (N_f, 6), Voigt order of Eq. 4."""
    B = strain_matrix(dom.Bbar)                                   # (N_f, 5, 6, 3)
    uu = np.where((dom.nodes >= 0)[:, :, None], u.reshape(-1, 3)[np.maximum(dom.nodes, 0)], 0.0)
    return np.einsum("fnri,fni->fr", B, uu)


# ---------------------------------------------------------------------------
# O7: loads and essential boundary conditions (STEP 5, Section 3.3 STEP 5)
# ---------------------------------------------------------------------------

def traction_load(n_nodes: int, xyz, tris, trac) -> np.ndarray:
    """Nodal loads of piecewise-constant tractions on boundary triangles: each
    triangle gives t*A/3 to each of its three nodes (A by Eq. 11).
    trac is (nrhs, n_tri, 3); returns (nrhs, 3*n_nodes)."""
    trac = np.asarray(trac, dtype=np.float64)
    if trac.ndim == 2:
        trac = trac[None]
    A = tri_area_eq11(xyz[tris[:, 0]], xyz[tris[:, 1]], xyz[tris[:, 2]])
    f = np.zeros((trac.shape[0], n_nodes, 3))
    for r in range(trac.shape[0]):
        for v in range(3):
            np.add.at(f[r], tris[:, v], trac[r] * (A / 3.0)[:, None])
    return f.reshape(trac.shape[0], 3 * n_nodes)


def dirichlet_system(K: sp.spmatrix, f: np.ndarray, dir_dofs, dir_vals):
    """Essential conditions by elimination (STEP 5, read as masking):
    A = P K P + (I - P),  b = P (f - K g) + (I - P) g, with P the diagonal
    0/1 mask of free DOFs and g the prescribed values (zero elsewhere)."""
    n = K.shape[0]
    free = np.ones(n)
    free[dir_dofs] = 0.0
    g = np.zeros(n)
    g[dir_dofs] = dir_vals
    P = sp.diags(free)
    A = (P @ K @ P + sp.diags(1.0 - free)).tocsr()
    b = free * (f - K @ g) + (1.0 - free) * g
    return A, b, free, g


def penalty_system(K: sp.spmatrix, f: np.ndarray, dir_dofs, dir_vals, alpha: float):
    """The penalty method of STEP 5 (Section 3.3): A = K + alpha S and
    b = f + alpha S g, S the diagonal selector of the prescribed DOFs and g
    their values; no row or column is removed, and u tends to the masked
    elimination's solution as alpha grows (error of order 1/alpha)."""
    n = K.shape[0]
    s = np.zeros(n)
    s[np.asarray(dir_dofs)] = 1.0
    g = np.zeros(n)
    g[np.asarray(dir_dofs)] = np.asarray(dir_vals, dtype=np.float64)
    A = (sp.csr_matrix(K) + alpha * sp.diags(s)).tocsr()
    return A, np.asarray(f, dtype=np.float64) + alpha * s * g


def true_relative_residual(A, b, x) -> float:
    """||b - A x||_2 / ||b||_2 in FP64."""
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# Sampled rows of K for very large meshes (same arithmetic on a sub-mesh)
# ---------------------------------------------------------------------------

def K_rows_submesh(xyz, tets, E, nu, node: int):
    """Rows 3*node..3*node+2 of the global K, computed by running the full
    oracle on the sub-mesh of tets that share a node with any tet containing
    `node`.  Every face whose stencil holds `node` is a face of a tet that
    contains it, and all its neighbours lie in that sub-mesh, so its
    interior/exterior status and its smoothing domain are the global ones.
    Returns (cols, vals) with cols ascending, vals (3, n_cols)."""
    ring1 = np.nonzero((tets == node).any(axis=1))[0]
    ring_nodes = np.unique(tets[ring1])
    ring2 = np.nonzero(np.isin(tets, ring_nodes).any(axis=1))[0]
    sub = tets[ring2]
    used, inv = np.unique(sub, return_inverse=True)
    sub_local = inv.reshape(sub.shape)
    asm = assemble(xyz[used], sub_local, E, nu)
    loc = int(np.searchsorted(used, node))
    Ksub = asm.matrix()
    rows = Ksub[3 * loc:3 * loc + 3]
    coo = rows.tocoo()
    gcols = 3 * used[coo.col // 3] + coo.col % 3
    cols = np.unique(gcols)
    vals = np.zeros((3, cols.shape[0]))
    vals[coo.row, np.searchsorted(cols, gcols)] = coo.data
    return cols, vals
