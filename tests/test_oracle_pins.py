"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/), closed forms, invariants of linear elasticity,
an independent dense construction, textbook special cases and beam theory.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from inputs.kuhn_beam import cantilever, clamp_dofs, face_nodes, face_triangles, kuhn_beam, uniform_traction
from oracle import fsfem as F
from oracle import solve as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _rigid_modes(xyz):
    n = xyz.shape[0]
    modes = []
    for a in range(3):
        t = np.zeros((n, 3))
        t[:, a] = 1.0
        modes.append(t.ravel())
    for w in np.eye(3):
        modes.append(np.cross(w[None, :], xyz).ravel())
    return np.stack(modes, 1)


# --------------------------------------------------------------------------
# Paper-printed values
# --------------------------------------------------------------------------

def test_table1_gauss_point_values():
    """Table 1: the shape values at field nodes, centroids and Gauss points."""
    got = F.gauss_point_shape_values()
    for row in _read_golden("table1_shape_values.txt"):
        site, vals = row[0], [Fraction(v) for v in row[1:]]
        assert got[site] == vals, site


def test_table5_dense_size_is_3n_squared_fp64():
    """Table 5: an uncompressed K holds (3 N_n)^2 FP64 entries (ndof = 3 N_n)."""
    for n, gb in _read_golden("table5_dense_memory.txt"):
        ndof = 3 * int(n)
        assert abs(ndof ** 2 * 8 / 2 ** 30 - float(gb)) < 0.01


def test_eq12_triplet_count_and_face_counts():
    """Eq. 12: 144 triplets per exterior face and 225 per interior face; the
    face counts of a Kuhn box follow from 4 N_e = 2 N_i + N_b with two
    boundary triangles per boundary quad."""
    p = cantilever(20, 4, 4, seed=1)
    asm = F.assemble(p.mesh.xyz, p.mesh.tets, p.E, p.nu)
    nx, ny, nz = 20, 4, 4
    nb = 4 * (nx * ny + ny * nz + nz * nx)
    ni = (4 * p.mesh.n_tets - nb) // 2
    assert asm.faces.n_boundary == nb == 704
    assert asm.faces.n_interior == ni == 3488
    assert asm.n_triplets == nb * 144 + ni * 225
    # loop and vectorised triplet builders agree exactly
    small = cantilever(3, 2, 2, seed=3)
    a1 = F.assemble(small.mesh.xyz, small.mesh.tets, small.E, small.nu, vectorised=False)
    a2 = F.assemble(small.mesh.xyz, small.mesh.tets, small.E, small.nu, vectorised=True)
    assert np.array_equal(a1.indptr, a2.indptr) and np.array_equal(a1.indices, a2.indices)
    assert np.array_equal(a1.data, a2.data)


def test_table4_direction_on_paper_beam():
    """Table 4 / Section 5.1.1: on the same mesh FS-FEM-T4 deflects more than
    FEM-T4 and less than the converged beam value (~0.0122 m by Timoshenko
    theory for the 1 x 0.2 x 0.2 beam under 12500 Pa)."""
    rows = _read_golden("table4_deflections.txt")
    tip = [float(v) for v in rows[-1][1:]]
    assert abs(tip[0]) < abs(tip[1]) < abs(tip[2])        # the paper's own ordering
    mesh = kuhn_beam(16, 4, 4, (1.0, 0.2, 0.2), 0.1, seed=7)
    dofs, vals = clamp_dofs(mesh, 0, 0)
    tris = face_triangles(mesh, 2, 1)
    f = F.traction_load(mesh.n_nodes, mesh.xyz, tris, uniform_traction(tris, (0, 0, -12500.0)))[0]
    E, nu = 2e8, 0.3
    Kfs = F.assemble(mesh.xyz, mesh.tets, E, nu).matrix()
    Kfem = F.fem_K_csr(mesh.xyz, mesh.tets, E, nu)
    tipn = face_nodes(mesh, 0, 1)
    d = []
    for K in (Kfem, Kfs):
        A, b, _, _ = F.dirichlet_system(K, f, dofs, vals)
        x = S.jacobi_pcg(A, b, 1e-10).x
        d.append(-x.reshape(-1, 3)[tipn, 2].mean())
    q, L, bw, h = 12500 * 0.2, 1.0, 0.2, 0.2
    I, Aa = bw * h ** 3 / 12, bw * h
    G = E / (2 * (1 + nu))
    kap = 10 * (1 + nu) / (12 + 11 * nu)
    d_beam = q * L ** 4 / (8 * E * I) + q * L ** 2 / (2 * kap * G * Aa)
    assert 0 < d[0] < d[1] < d_beam


# --------------------------------------------------------------------------
# Geometry closed forms
# --------------------------------------------------------------------------

REF_TET = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])


def test_eq10_volume_and_eq11_area():
    tets = np.array([[0, 1, 2, 3]])
    assert np.isclose(F.tet_volumes(REF_TET, tets)[0], 1 / 6, rtol=1e-15)
    M = np.array([[2., 0.3, 0], [0, 3, 0.1], [0.2, 0, 5]])
    X = REF_TET @ M.T + np.array([4., -1, 7])
    assert np.isclose(F.tet_volumes(X, tets)[0], abs(np.linalg.det(M)) / 6, rtol=1e-13)
    # orientation flip leaves |V| unchanged and flips the sign of Eq. 10
    flipped = np.array([[0, 2, 1, 3]])
    assert np.isclose(F.tet_volume_eq10(X, flipped)[0], -F.tet_volume_eq10(X, tets)[0], rtol=1e-13)
    A = F.tri_area_eq11(np.array([0., 0, 0]), np.array([3., 0, 0]), np.array([0., 4, 0]))
    assert A == 6.0
    s = 2.0
    A = F.tri_area_eq11(np.array([0., 0, 0]), np.array([s, 0, 0]), np.array([s / 2, s * np.sqrt(3) / 2, 0]))
    assert np.isclose(A, np.sqrt(3) / 4 * s * s, rtol=1e-15)


def test_gradients_reference_tet_and_two_routes():
    tets = np.array([[0, 1, 2, 3]])
    G = F.tet_gradients_jacobian(REF_TET, tets)[0]
    assert np.allclose(G, [[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], atol=1e-15)
    m = kuhn_beam(3, 3, 3, (1.0, 2.0, 1.5), 0.1, seed=11)
    G1 = F.tet_gradients_jacobian(m.xyz, m.tets)
    G2 = F.tet_gradients_normals(m.xyz, m.tets)
    assert np.abs(G1 - G2).max() <= 1e-13 * np.abs(G1).max()
    # partition of unity and linear completeness: sum_a grad N_a = 0, sum_a x_a grad N_a^T = I
    X = m.xyz[m.tets]
    assert np.abs(G1.sum(axis=1)).max() <= 1e-12 * np.abs(G1).max()
    eye = np.einsum("eai,eaj->eij", X, G1)
    assert np.abs(eye - np.eye(3)).max() <= 1e-12


def test_kuhn_tets_positive_and_sub_tet_quarter():
    m = kuhn_beam(4, 3, 5, (2.0, 1.0, 1.5), 0.1, seed=2)
    X = m.xyz[m.tets]
    det = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 2))
    assert (det > 0).all()
    faces = F.build_faces(m.tets)
    dom = F.smoothing_domains_eq7(m.xyz, m.tets, faces)
    V = F.tet_volumes(m.xyz, m.tets)
    Vk = np.where(faces.interior, (V[faces.tet[:, 0]] + V[np.maximum(faces.tet[:, 1], 0)]) / 4,
                  V[faces.tet[:, 0]] / 4)
    assert np.abs(dom.Vk - Vk).max() <= 1e-14 * Vk.max()
    assert np.isclose(dom.Vk.sum(), 2.0 * 1.0 * 1.5, rtol=1e-13)      # domains tile the box


def test_eq7_equals_volume_average():
    """Eq. 7 by boundary triangles equals the average of grad N over Omega_k."""
    m = kuhn_beam(5, 3, 4, (3.0, 1.0, 1.2), 0.1, seed=4)
    faces = F.build_faces(m.tets)
    d1 = F.smoothing_domains_eq7(m.xyz, m.tets, faces)
    d2 = F.smoothing_domains_average(m.xyz, m.tets, faces)
    assert np.abs(d1.Bbar - d2.Bbar).max() <= 1e-13 * np.abs(d1.Bbar).max()
    assert np.abs(d1.Vk - d2.Vk).max() <= 1e-14 * d1.Vk.max()
    assert np.array_equal(d1.nodes, d2.nodes)
    # the five rows of each face sum to zero (constant fields give no strain)
    assert np.abs(d1.Bbar.sum(axis=1)).max() <= 1e-12 * np.abs(d1.Bbar).max()


def test_faces_shared_by_three_tets_rejected():
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]])
    with pytest.raises(ValueError):
        F.build_faces(tets)


# --------------------------------------------------------------------------
# Material and strain layout: textbook special cases
# --------------------------------------------------------------------------

def test_material_matrix_textbook():
    E, nu = 210e9, 0.3
    D = F.material_D(E, nu)
    eps = np.array([1e-3, 0, 0, 0, 0, 0])
    s = D @ eps
    assert np.isclose(s[0], E * (1 - nu) / ((1 + nu) * (1 - 2 * nu)) * 1e-3, rtol=1e-14)
    assert np.isclose(s[1], E * nu / ((1 + nu) * (1 - 2 * nu)) * 1e-3, rtol=1e-14)
    for r in (3, 4, 5):
        g = np.zeros(6)
        g[r] = 2e-3
        assert np.isclose((D @ g)[r], E / (2 * (1 + nu)) * 2e-3, rtol=1e-14)
    # uniaxial stress: sigma = (s, 0, 0) gives eps_xx = s/E, eps_yy = -nu s/E
    e = np.linalg.solve(D, np.array([1e6, 0, 0, 0, 0, 0]))
    assert np.isclose(e[0], 1e6 / E, rtol=1e-13) and np.isclose(e[1], -nu * 1e6 / E, rtol=1e-13)


def test_voigt_rows_engineering_shear():
    """Eq. 4 rows 4-6: u_y = g z gives gamma_yz = g, u_z = g x gives gamma_zx,
    u_x = g y gives gamma_xy."""
    m = kuhn_beam(3, 2, 2, (1.0, 1.0, 1.0), 0.1, seed=5)
    faces = F.build_faces(m.tets)
    dom = F.smoothing_domains_eq7(m.xyz, m.tets, faces)
    x, y, z = m.xyz.T
    g = 1e-3
    for comp, coord, row in ((1, z, 3), (2, x, 4), (0, y, 5)):
        u = np.zeros_like(m.xyz)
        u[:, comp] = g * coord
        eps = F.smoothed_strains(dom, u.ravel())
        want = np.zeros(6)
        want[row] = g
        assert np.abs(eps - want).max() <= 1e-13


# --------------------------------------------------------------------------
# Stiffness invariants
# --------------------------------------------------------------------------

def test_single_tet_fs_equals_fem():
    """One tet: four exterior faces, each domain a quarter of the tet with
    b = grad N, so K_FS is the textbook linear-tet stiffness V B^T c B."""
    X = np.array([[0.1, 0.0, 0.2], [1.3, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.2, 1.1]])
    tets = np.array([[0, 1, 2, 3]])
    asm = F.assemble(X, tets, 1e9, 0.25)
    Kfs = asm.matrix().toarray()
    Kfem = F.dense_K_fem(X, tets, 1e9, 0.25)
    assert np.abs(Kfs - Kfem).max() <= 1e-13 * np.abs(Kfem).max()
    # and the uniaxial strain energy: u = (e x, 0, 0) stores V (lam + 2 mu) e^2 / 2
    e = 1e-3
    u = np.zeros((4, 3))
    u[:, 0] = e * X[:, 0]
    lam, mu = F.lame(1e9, 0.25)
    V = F.tet_volumes(X, tets)[0]
    assert np.isclose(u.ravel() @ Kfs @ u.ravel(), V * (lam + 2 * mu) * e * e, rtol=1e-12)


def test_bruteforce_dense_K_equals_csr():
    """Dense K from the energy of volume-averaged strains equals the Eq. 7 ->
    Eq. 9 -> Eq. 12 -> CSR route, entry by entry, including its structure."""
    m = kuhn_beam(3, 2, 2, (2.0, 1.0, 1.0), 0.1, seed=9)
    E, nu = 70e9, 0.33
    asm = F.assemble(m.xyz, m.tets, E, nu)
    Kd = F.dense_K_bruteforce(m.xyz, m.tets, E, nu)
    Kc = asm.matrix().toarray()
    assert np.abs(Kd - Kc).max() <= 1e-12 * np.abs(Kd).max()
    # structure: exactly the node pairs sharing a face stencil, x 3 x 3
    pairs = set()
    for f in range(asm.faces.n):
        nn = [v for v in asm.dom.nodes[f] if v >= 0]
        pairs.update((a, b) for a in nn for b in nn)
    nnz_expected = 9 * len(pairs)
    assert asm.indices.size == nnz_expected
    rows = np.repeat(np.arange(asm.ndof), np.diff(asm.indptr))
    got = set(zip((rows // 3).tolist(), (asm.indices // 3).tolist()))
    assert got == pairs
    for r in range(asm.ndof):
        seg = asm.indices[asm.indptr[r]:asm.indptr[r + 1]]
        assert np.all(np.diff(seg) > 0)


def test_rigid_modes_symmetry_spd():
    m = kuhn_beam(3, 2, 2, (2.0, 1.0, 1.0), 0.1, seed=13)
    asm = F.assemble(m.xyz, m.tets, 210e9, 0.3)
    K = asm.matrix().toarray()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    R = _rigid_modes(m.xyz)
    assert np.abs(K @ R).max() <= 1e-12 * np.abs(K).max() * np.abs(R).max()
    w = np.linalg.eigvalsh(K)
    assert int((np.abs(w) < 1e-10 * w.max()).sum()) == 6
    assert w[6] > 1e-8 * w.max()
    dofs, vals = clamp_dofs(m, 0, 0)
    A, _, _, _ = F.dirichlet_system(asm.matrix(), np.zeros(asm.ndof), dofs, vals)
    S.cholesky(A.toarray())                      # raises if not SPD


def test_fs_softer_than_fem():
    """K_FEM - K_FS is positive semidefinite (Jensen on each sub-tet), so for
    any load the FS-FEM compliance is at least the FEM one (Section 5.1.1)."""
    m = kuhn_beam(3, 2, 2, (2.0, 1.0, 1.0), 0.1, seed=17)
    E, nu = 210e9, 0.3
    Kfs = F.assemble(m.xyz, m.tets, E, nu).matrix().toarray()
    Kfem = F.dense_K_fem(m.xyz, m.tets, E, nu)
    w = np.linalg.eigvalsh(Kfem - Kfs)
    assert w.min() >= -1e-12 * np.abs(Kfem).max()
    assert w.max() > 1e-3 * np.abs(Kfem).max()


def test_patch_test_linear_field():
    """A linear field prescribed on all boundary nodes is reproduced inside to
    1e-12, and every smoothed strain equals sym(H) exactly."""
    m = kuhn_beam(4, 3, 5, (2.0, 1.0, 1.5), 0.1, seed=21)
    rng = np.random.default_rng(0)
    a = rng.normal(size=3) * 1e-3
    H = rng.normal(size=(3, 3)) * 1e-3
    u_lin = (a[None, :] + m.xyz @ H.T).ravel()
    lat = m.lattice()
    bnd = ((lat == 0) | (lat == np.array([m.nx, m.ny, m.nz]))).any(axis=1)
    dofs = (3 * np.nonzero(bnd)[0][:, None] + np.arange(3)).ravel()
    E, nu = 210e9, 0.3
    asm = F.assemble(m.xyz, m.tets, E, nu)
    A, b, free, g = F.dirichlet_system(asm.matrix(), np.zeros(asm.ndof), dofs, u_lin[dofs])
    x = S.cholesky_solve(A.toarray(), b)
    assert np.abs(x - u_lin).max() <= 1e-12 * np.abs(u_lin).max()
    eps = F.smoothed_strains(asm.dom, u_lin)
    Hs = 0.5 * (H + H.T)
    want = np.array([Hs[0, 0], Hs[1, 1], Hs[2, 2], 2 * Hs[1, 2], 2 * Hs[2, 0], 2 * Hs[0, 1]])
    assert np.abs(eps - want[None]).max() <= 1e-12 * np.abs(want).max()
    # interior rows of K carry no force for a linear field
    Ku = asm.matrix() @ u_lin
    assert np.abs(Ku[free > 0]).max() <= 1e-10 * np.abs(asm.data).max() * np.abs(u_lin).max()


def test_orientation_and_node_order_invariance():
    p = cantilever(4, 2, 2, seed=3)
    t2 = p.mesh.tets.copy()
    t2[::2] = t2[::2][:, [0, 2, 1, 3]]        # flip every other tet
    t2[1::3] = t2[1::3][:, [3, 1, 2, 0]]
    K1 = F.assemble(p.mesh.xyz, p.mesh.tets, p.E, p.nu).matrix().toarray()
    K2 = F.assemble(p.mesh.xyz, t2, p.E, p.nu).matrix().toarray()
    assert np.abs(K1 - K2).max() <= 1e-13 * np.abs(K1).max()


def test_chunked_assembly_and_submesh_rows():
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    a1 = F.assemble(m.xyz, m.tets, p.E, p.nu)
    a2 = F.assemble(m.xyz, m.tets, p.E, p.nu, chunk=777)
    assert np.array_equal(a1.indptr, a2.indptr) and np.array_equal(a1.indices, a2.indices)
    assert np.abs(a1.data - a2.data).max() <= 1e-14 * np.abs(a1.data).max()
    K = a1.matrix()
    for node in (0, 137, 262, m.n_nodes - 1):
        cols, vals = F.K_rows_submesh(m.xyz, m.tets, p.E, p.nu, node)
        for c in range(3):
            row = K[3 * node + c]
            assert np.array_equal(np.sort(row.indices), cols)
            ref = row.toarray()[0, cols]
            assert np.abs(ref - vals[c]).max() <= 1e-13 * np.abs(ref).max()


# --------------------------------------------------------------------------
# Loads, solvers
# --------------------------------------------------------------------------

def test_traction_resultant():
    p = cantilever(6, 3, 2, dims=(3.0, 0.7, 0.4), seed=2, traction=(1.0, -2.0, 3.0))
    f = F.traction_load(p.mesh.n_nodes, p.mesh.xyz, p.trac_tris, p.trac)[0]
    assert np.allclose(f.reshape(-1, 3).sum(0), np.array([1.0, -2.0, 3.0]) * 0.7 * 0.4, rtol=1e-14)


def test_cholesky_and_pcg():
    p = cantilever(10, 2, 2, seed=1)
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, _, _ = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    Ad = A.toarray()
    L = S.cholesky(Ad)
    Lnp = np.linalg.cholesky(Ad)
    assert np.abs(L - Lnp).max() <= 1e-12 * np.abs(Lnp).max()
    x_ch = S.cholesky_solve(Ad, b)
    x_np = np.linalg.solve(Ad, b)
    assert np.linalg.norm(x_ch - x_np) <= 1e-10 * np.linalg.norm(x_np)
    r = S.jacobi_pcg(A, b, 1e-10)
    assert r.true_relres <= 1e-10
    assert np.linalg.norm(r.x - x_np) <= 1e-6 * np.linalg.norm(x_np)


def test_cantilever_converges_to_timoshenko():
    """Tip deflection of the 10 x 1 x 1 m cantilever (P = 1e6 N on x = 10)
    approaches the Timoshenko value PL^3/(3EI) + PL/(kGA) under refinement;
    FEM-T4 stays stiffer than FS-FEM at every level, and the Richardson
    limit of three FS-FEM levels lies within 2% of the beam value."""
    E, nu = 210e9, 0.3
    P, L, I, A = 1e6, 10.0, 1.0 / 12.0, 1.0
    G = E / (2 * (1 + nu))
    kap = 10 * (1 + nu) / (12 + 11 * nu)
    dT = P * L ** 3 / (3 * E * I) + P * L / (kap * G * A)
    d_fs = []
    for n in ((20, 4, 4), (40, 8, 8), (80, 16, 16)):
        p = cantilever(*n, seed=1)
        m = p.mesh
        f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
        tip = face_nodes(m, 0, 1)
        out = []
        for K in (F.fem_K_csr(m.xyz, m.tets, E, nu), F.assemble(m.xyz, m.tets, E, nu).matrix()):
            Am, b, _, _ = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
            x = S.jacobi_pcg(Am, b, 1e-9).x
            out.append(-x.reshape(-1, 3)[tip, 2].mean())
        assert out[0] < out[1] < dT
        d_fs.append(out[1])
    err = [dT - d for d in d_fs]
    assert err[0] > err[1] > err[2] > 0
    rho = (d_fs[1] - d_fs[0]) / (d_fs[2] - d_fs[1])
    d_inf = d_fs[2] + (d_fs[2] - d_fs[1]) / (rho - 1)
    assert abs(d_inf - dT) / dT < 0.02


def test_penalty_converges_to_elimination():
    """STEP 5's penalty method: the solution of (K + alpha S) u = f + alpha S g
    tends to the masked elimination's solution with an error of order 1/alpha
    (100x smaller for a 100x larger alpha), and the prescribed values to g."""
    m = kuhn_beam(4, 1, 1, (4.0, 1.0, 1.0), 0.1, seed=3)
    dofs, vals = clamp_dofs(m, 0, 0)
    vals = np.random.default_rng(2).standard_normal(dofs.shape[0]) * 1e-4  # nonzero prescribed values
    tris = face_triangles(m, 0, 1)
    f = F.traction_load(m.n_nodes, m.xyz, tris, uniform_traction(tris, (0, 0, -1e6)))[0]
    K = F.assemble(m.xyz, m.tets, 210e9, 0.3).matrix()
    A, b, _, _ = F.dirichlet_system(K, f, dofs, vals)
    u0 = np.linalg.solve(A.toarray(), b)
    kmax = K.diagonal().max()
    errs = []
    for a in (1e4, 1e6):
        Ap, bp = F.penalty_system(K, f, dofs, vals, a * kmax)
        up = np.linalg.solve(Ap.toarray(), bp)
        errs.append(np.linalg.norm(up - u0) / np.linalg.norm(u0))
        assert np.abs(up[dofs] - vals).max() <= 1e3 / a * np.abs(u0).max()
    assert 30 < errs[0] / errs[1] < 300, errs


def test_sliver_quality_and_mesh_validation():
    """Sliver quality: 1 for the regular tet, invariant under scaling,
    rotation and node order, 0 for a flat tet, 6 sqrt(2) V / l_rms^3 on the
    unit right tet (V = 1/6, three unit edges and three sqrt(2) edges).  Mesh
    validation rejects out-of-range ids, non-finite coordinates and a
    malformed connectivity."""
    reg = np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    t = np.array([[0, 1, 2, 3]])
    assert abs(F.sliver_quality(reg, t)[0] - 1.0) < 1e-14
    c, s = np.cos(0.7), np.sin(0.7)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    moved = 3.5 * reg @ R.T + np.array([2.0, -1.0, 0.5])
    assert abs(F.sliver_quality(moved, np.array([[2, 0, 3, 1]]))[0] - 1.0) < 1e-13
    flat = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, 1.0, 0.0]])
    assert F.sliver_quality(flat, t)[0] == 0.0
    right = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    l_rms = np.sqrt((3 * 1.0 + 3 * 2.0) / 6.0)
    assert abs(F.sliver_quality(right, t)[0] - 6 * np.sqrt(2) / 6 / l_rms ** 3) < 1e-14
    F.validate(right, t)
    with pytest.raises(ValueError):
        F.validate(right, np.array([[0, 1, 2, 4]]))
    with pytest.raises(ValueError):
        F.validate(np.where(np.arange(12).reshape(4, 3) == 5, np.nan, right), t)
    with pytest.raises(ValueError):
        F.validate(right, np.array([[0, 1, 2]]))
