"""Seeded synthetic cantilever meshes and load sets for FS-FEM-T4 workloads.

This module only generates inputs: node coordinates, tet connectivity, the
clamped degrees of freedom and traction triangles.  It holds none of the
method's arithmetic (no volumes, gradients, smoothing domains or stiffness),
so both the CPU oracle and the CUDA path can consume what it produces.

Meshes follow the test problems of Section 4: a box cantilever meshed with
4-node tetrahedra.  The paper's TetGen meshes are not available, so a box of
nx*ny*nz hexahedral cells is split into six tets per cell (Kuhn/Freudenthal
split along the cell's main diagonal, one tet per permutation of the axes),
and interior nodes are jittered uniformly by up to +/- jitter*h per axis.

Numbering (0-based, as in TetGen output, Section 3.2):
  node(i, j, k) = (i*(ny+1) + j)*(nz+1) + k      (k fastest)
  cell(i, j, k) = (i*ny + j)*nz + k;  tets 6*cell .. 6*cell+5
Every tet of the undistorted grid is positively oriented (det[x1-x0, x2-x0,
x3-x0] > 0): even axis permutations keep the order (v0, v1, v2, v3), odd ones
swap v1 and v2.  A jitter of at most 0.1h per axis cannot invert a Kuhn tet.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Corner offsets (di, dj, dk) of the four vertices of each Kuhn tet.  Tet p
# walks (0,0,0) -> +e_a -> +e_a+e_b -> (1,1,1) for the axis permutation (a,b,c).
_PERMS = [(0, 1, 2), (1, 2, 0), (2, 0, 1),   # even permutations
          (0, 2, 1), (2, 1, 0), (1, 0, 2)]   # odd permutations


def _kuhn_offsets() -> np.ndarray:
    offs = np.zeros((6, 4, 3), dtype=np.int64)
    for p, (a, b, c) in enumerate(_PERMS):
        v = [np.zeros(3, np.int64)]
        for ax in (a, b, c):
            nxt = v[-1].copy()
            nxt[ax] = 1
            v.append(nxt)
        if p >= 3:  # odd permutation: swap v1 and v2 to keep a positive orientation
            v[1], v[2] = v[2], v[1]
        offs[p] = np.stack(v)
    return offs


KUHN_OFFSETS = _kuhn_offsets()


@dataclasses.dataclass
class BeamMesh:
    nx: int
    ny: int
    nz: int
    dims: tuple          # (Lx, Ly, Lz) in metres; the box is [0,Lx]x[0,Ly]x[0,Lz]
    xyz: np.ndarray      # (n_nodes, 3) float64
    tets: np.ndarray     # (n_tets, 4) int32

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]

    @property
    def ndof(self) -> int:
        return 3 * self.n_nodes

    def node_id(self, i, j, k):
        return (np.asarray(i) * (self.ny + 1) + np.asarray(j)) * (self.nz + 1) + np.asarray(k)

    def lattice(self) -> np.ndarray:
        """(n_nodes, 3) integer lattice indices (i, j, k) of every node."""
        i, j, k = np.meshgrid(np.arange(self.nx + 1), np.arange(self.ny + 1),
                              np.arange(self.nz + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


def kuhn_beam(nx: int, ny: int, nz: int, dims=(10.0, 1.0, 1.0),
              jitter: float = 0.1, seed: int = 1) -> BeamMesh:
    """Kuhn-split box mesh with seeded uniform jitter of interior nodes.

    The jitter draws rng.uniform(-1, 1, (n_nodes, 3)) from
    numpy.random.default_rng(seed) for all nodes in node order, scales axis a
    by jitter*h_a (h_a = dims[a]/n_a) and zeroes it on boundary nodes, so the
    six box faces stay planar and boundary-condition sets stay exact.
    """
    dims = tuple(float(d) for d in dims)
    h = np.array([dims[0] / nx, dims[1] / ny, dims[2] / nz])
    lat = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    xyz = lat.astype(np.float64) * h
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-1.0, 1.0, size=xyz.shape) * (jitter * h)
        interior = ((lat[:, 0] > 0) & (lat[:, 0] < nx) & (lat[:, 1] > 0) & (lat[:, 1] < ny)
                    & (lat[:, 2] > 0) & (lat[:, 2] < nz))
        xyz = xyz + d * interior[:, None]
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)       # (n_cells, 3)
    corner = cells[:, None, None, :] + KUHN_OFFSETS[None, :, :, :]        # (n_cells, 6, 4, 3)
    tets = (corner[..., 0] * (ny + 1) + corner[..., 1]) * (nz + 1) + corner[..., 2]
    tets = tets.reshape(-1, 4).astype(np.int32)
    return BeamMesh(nx, ny, nz, dims, xyz, tets)


# ---------------------------------------------------------------------------
# Boundary sets
# ---------------------------------------------------------------------------

def face_nodes(mesh: BeamMesh, axis: int, side: int) -> np.ndarray:
    """Node ids on the box face axis=0 (side 0) or axis=n_axis (side 1)."""
    lat = mesh.lattice()
    n = (mesh.nx, mesh.ny, mesh.nz)[axis]
    return np.nonzero(lat[:, axis] == (n if side else 0))[0].astype(np.int32)


def clamp_dofs(mesh: BeamMesh, axis: int = 0, side: int = 0):
    """All three DOFs (DOF = 3*node + component) of the nodes on one box face,
    with zero prescribed values."""
    nodes = face_nodes(mesh, axis, side)
    dofs = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel().astype(np.int32)
    return dofs, np.zeros(dofs.shape[0], dtype=np.float64)


def face_triangles(mesh: BeamMesh, axis: int, side: int) -> np.ndarray:
    """Triangles (n_tri, 3) tiling one box face, matching the faces of the
    Kuhn tets: each boundary quad is cut along its (0,0)-(1,1) diagonal in the
    two tangential lattice axes taken in increasing order."""
    n = [mesh.nx, mesh.ny, mesh.nz]
    t1, t2 = [a for a in range(3) if a != axis]
    a_idx, b_idx = np.meshgrid(np.arange(n[t1]), np.arange(n[t2]), indexing="ij")
    a_idx, b_idx = a_idx.ravel(), b_idx.ravel()

    def nid(da, db):
        ijk = [None, None, None]
        ijk[axis] = np.full(a_idx.shape, n[axis] if side else 0)
        ijk[t1] = a_idx + da
        ijk[t2] = b_idx + db
        return mesh.node_id(*ijk)

    n00, n10, n01, n11 = nid(0, 0), nid(1, 0), nid(0, 1), nid(1, 1)
    tris = np.concatenate([np.stack([n00, n10, n11], 1), np.stack([n00, n01, n11], 1)])
    return tris.astype(np.int32)


def uniform_traction(tris: np.ndarray, t) -> np.ndarray:
    """Per-triangle traction vectors (n_tri, 3), all equal to t (Pa)."""
    return np.tile(np.asarray(t, dtype=np.float64)[None, :], (tris.shape[0], 1))


def torsion_traction(mesh: BeamMesh, tris: np.ndarray, magnitude: float = 1e6) -> np.ndarray:
    """Torsional couple on an x-normal face: t = m*(0, -(z-zc), (y-yc))/r_max,
    evaluated at each triangle's vertex mean and held constant on it."""
    c = mesh.xyz[tris].mean(axis=1)
    yc, zc = 0.5 * mesh.dims[1], 0.5 * mesh.dims[2]
    rmax = np.hypot(0.5 * mesh.dims[1], 0.5 * mesh.dims[2])
    t = np.zeros_like(c)
    t[:, 1] = -(c[:, 2] - zc)
    t[:, 2] = c[:, 1] - yc
    return magnitude * t / rmax


@dataclasses.dataclass
class Problem:
    """A complete FS-FEM input set: mesh, material, clamps, tractions.

    trac has shape (nrhs, n_tri, 3): one traction field per load case."""
    mesh: BeamMesh
    E: float
    nu: float
    dir_dofs: np.ndarray   # (n_dir,) int32
    dir_vals: np.ndarray   # (n_dir,) float64
    trac_tris: np.ndarray  # (n_tri, 3) int32
    trac: np.ndarray       # (nrhs, n_tri, 3) float64

    @property
    def nrhs(self) -> int:
        return self.trac.shape[0]


def cantilever(nx, ny, nz, dims=(10.0, 1.0, 1.0), seed=1, E=210e9, nu=0.3,
               traction=(0.0, 0.0, -1e6), jitter=0.1) -> Problem:
    """The cantilever workload: x=0 face clamped, uniform traction on x=Lx."""
    mesh = kuhn_beam(nx, ny, nz, dims, jitter, seed)
    dofs, vals = clamp_dofs(mesh, 0, 0)
    tris = face_triangles(mesh, 0, 1)
    return Problem(mesh, E, nu, dofs, vals, tris, uniform_traction(tris, traction)[None])


def four_load_cases(mesh: BeamMesh, magnitude: float = 1e6) -> tuple:
    """Traction triangles on x=Lx and the four load cases used for batching:
    z-bending, y-bending, torsional couple, axial pull (in that order)."""
    tris = face_triangles(mesh, 0, 1)
    cases = [uniform_traction(tris, (0.0, 0.0, -magnitude)),
             uniform_traction(tris, (0.0, -magnitude, 0.0)),
             torsion_traction(mesh, tris, magnitude),
             uniform_traction(tris, (magnitude, 0.0, 0.0))]
    return tris, np.stack(cases)


def batch_beams(n_beams: int = 64, seed: int = 5, min_cells=(20, 4, 4),
                max_cells=(120, 24, 24)) -> list:
    """Uneven batch of cantilevers: nx ~ U{20..120}, ny, nz ~ U{4..24}, length
    ~ U[5, 20] m on a 1x1 m section, E ~ U[50, 300] GPa, nu ~ U[0.2, 0.45];
    four load cases each.  Mesh jitter seeds are seed*1000 + beam index."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_beams):
        nx = int(rng.integers(min_cells[0], max_cells[0] + 1))
        ny = int(rng.integers(min_cells[1], max_cells[1] + 1))
        nz = int(rng.integers(min_cells[2], max_cells[2] + 1))
        L = float(rng.uniform(5.0, 20.0))
        E = float(rng.uniform(50e9, 300e9))
        nu = float(rng.uniform(0.2, 0.45))
        mesh = kuhn_beam(nx, ny, nz, (L, 1.0, 1.0), 0.1, seed * 1000 + b)
        dofs, vals = clamp_dofs(mesh, 0, 0)
        tris, trac = four_load_cases(mesh)
        out.append(Problem(mesh, E, nu, dofs, vals, tris, trac))
    return out


def random_loads(mesh: BeamMesh, seed: int, n_patches: int = 3, magnitude: float = 1e6):
    """Randomised traction loads for training data: a few random patches of
    boundary triangles on the free faces (x=Lx, y=0/Ly, z=0/Lz), each with a
    random traction vector of norm <= magnitude.  Returns (tris, trac[1])."""
    rng = np.random.default_rng(seed)
    faces = [(0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]
    all_tris, all_t = [], []
    for _ in range(n_patches):
        axis, side = faces[int(rng.integers(len(faces)))]
        tris = face_triangles(mesh, axis, side)
        c = mesh.xyz[tris].mean(axis=1)
        centre = c[int(rng.integers(c.shape[0]))]
        radius = float(rng.uniform(0.1, 0.5)) * max(mesh.dims)
        sel = np.linalg.norm(c - centre, axis=1) <= radius
        tvec = rng.normal(size=3)
        tvec *= magnitude * float(rng.uniform(0.2, 1.0)) / np.linalg.norm(tvec)
        all_tris.append(tris[sel])
        all_t.append(np.tile(tvec, (int(sel.sum()), 1)))
    return np.concatenate(all_tris).astype(np.int32), np.concatenate(all_t)[None]


def multi_load_cantilever(nx, ny, nz, load_seeds, dims=(10.0, 1.0, 1.0), seed=2, E=210e9, nu=0.3,
                          jitter=0.1) -> Problem:
    """The cantilever with one load case per entry of load_seeds: the
    random_loads patches of that seed, each case given on the union of the
    free-face triangles (zero traction elsewhere)."""
    base = cantilever(nx, ny, nz, dims, seed, E, nu, jitter=jitter)
    m = base.mesh
    faces = [(0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]
    tris = np.concatenate([face_triangles(m, a, s) for a, s in faces]).astype(np.int32)
    key = {tuple(sorted(t)): i for i, t in enumerate(tris.tolist())}
    trac = np.zeros((len(load_seeds), len(tris), 3))
    for k, sd in enumerate(load_seeds):
        st, sv = random_loads(m, sd)
        for t, v in zip(st.tolist(), sv[0]):
            trac[k, key[tuple(sorted(t))]] += v
    return Problem(m, E, nu, base.dir_dofs, base.dir_vals, tris, trac)
