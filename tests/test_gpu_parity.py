"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (stated once, used below):
  * integers (neighbours, faces, CSR structure): bit-exact;
  * FP64 geometry and K entries: |dK_ij| <= 1e-12 max(|K_ij|, sqrt(K_ii K_jj));
  * FP64 operator: |dy_i| <= 1e-12 (|K| |u|)_i + tiny;
  * FP32 operator: the operator data is FP64 rounded once to FP32 and the
    apply sums O(100) FP32 terms per entry, so
    |dy|_inf <= 2e-5 || |K||u| ||_inf and ||dy||_2 <= 1e-5 ||y||_2;
  * FP32 operator, row by row (sampled rows at full size, FP32 input u):
    |dy_i| <= 64 * 2^-24 * (|K| (|u| + ||u||_inf))_i.  Each output entry
    passes through fewer than 32 FP32 roundings along its longest chain
    (operator data rounded from FP64, the tile's reference displacement
    subtracted, 4-term strain sums, the face average of two strains, the
    6-term stress, the 3-term nodal force, the compensated nodal sum); the
    subtracted reference is at most ||u||_inf in size; c = 64 doubles the
    rounding count;
  * displacements of reduced-precision solves: relative L2 <= 1e-6 against
    the oracle's exact (Cholesky) solution;
  * FP64 Jacobi-PCG iteration counts within 10% of the oracle's: finite-
    precision CG is sensitive to rounding near a tight tolerance; on the
    20x4x4 beam at 1e-10, perturbing b by 1e-15 (relative) already moves the
    oracle's own count between 567 and 605.
"""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever, clamp_dofs, face_nodes, kuhn_beam
from oracle import fsfem as F
from oracle import solve as OS
from tolerances import MF32_ROW_C, mf32_row_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem
    return sfem


@pytest.fixture(scope="module")
def cfg1():
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    asm = F.assemble(m.xyz, m.tets, p.E, p.nu)
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, free, g = F.dirichlet_system(asm.matrix(), f, p.dir_dofs, p.dir_vals)
    return p, asm, A, b


def _k_close(got, ref_data, indptr, indices, ndof):
    rows = np.repeat(np.arange(ndof), np.diff(indptr))
    diag = np.zeros(ndof)
    dmask = rows == indices
    diag[rows[dmask]] = ref_data[dmask]
    scale = np.maximum(np.abs(ref_data), np.sqrt(np.abs(diag[rows] * diag[indices])))
    return np.abs(got - ref_data) <= 1e-12 * scale


def test_geometry_neighbors_faces(S, cfg1):
    p, asm, _, _ = cfg1
    m = p.mesh
    with S.FsFem(p) as ctx:
        info = ctx.info
        assert info["n_faces"] == asm.faces.n
        assert info["n_interior"] == asm.faces.n_interior and info["n_boundary"] == asm.faces.n_boundary
        assert info["n_bad_tets"] == 0 and info["n_bad_faces"] == 0
        vol, grad = S.sfem_get_geometry(ctx.h, m.n_tets)
        Vr = F.tet_volumes(m.xyz, m.tets)
        Gr = F.tet_gradients_jacobian(m.xyz, m.tets)
        assert np.abs(vol - Vr).max() <= 1e-13 * Vr.max()
        assert np.abs(grad - Gr).max() <= 1e-12 * np.abs(Gr).max()
        assert np.isclose(info["min_volume"], Vr.min(), rtol=1e-13)
        # neighbours, bit-exact
        nbr = S.sfem_get_neighbors(ctx.h, m.n_tets)
        want = -np.ones((m.n_tets, 4), np.int64)
        fc = asm.faces
        for s_ in range(2):
            t = fc.tet[:, s_]
            o = fc.opp[:, s_]
            other = fc.tet[:, 1 - s_]
            ok = t >= 0
            slot = np.argmax(m.tets[t[ok]] == o[ok][:, None], axis=1)
            want[t[ok], slot] = other[ok]
        assert np.array_equal(nbr, want)
        # faces: same set of (triple, tets, opposite nodes); V_k to 1e-13
        nodes, ftets, Vk = S.sfem_get_faces(ctx.h, info["n_faces"])
        order = np.lexsort((nodes[:, 2], nodes[:, 1], nodes[:, 0]))
        assert np.array_equal(nodes[order, :3], fc.tri)
        gtet = np.sort(ftets[order], axis=1)
        otet = np.sort(np.where(fc.tet < 0, -1, fc.tet), axis=1)
        assert np.array_equal(gtet, otet)
        gopp = np.sort(nodes[order, 3:], axis=1)
        assert np.array_equal(gopp, np.sort(fc.opp, axis=1))
        assert np.abs(Vk[order] - asm.dom.Vk).max() <= 1e-13 * asm.dom.Vk.max()


def test_csr_structure_and_values(S, cfg1):
    p, asm, A, _ = cfg1
    with S.FsFem(p) as ctx:
        rp, col, val = S.sfem_assemble(ctx.h)
        assert S.sfem_get_info(ctx.h)["nnz"] == asm.indices.size
        assert np.array_equal(rp.cpu().numpy(), asm.indptr)
        assert np.array_equal(col.cpu().numpy(), asm.indices)
        ok = _k_close(val.cpu().numpy(), asm.data, asm.indptr, asm.indices, asm.ndof)
        assert ok.all(), f"{(~ok).sum()} entries off"
        diag = S.sfem_get_diag(ctx.h, asm.ndof)
        assert np.abs(diag - A.diagonal()).max() <= 1e-12 * A.diagonal().max()


def test_rhs_and_operators(S, cfg1):
    import torch
    p, asm, A, b = cfg1
    rng = np.random.default_rng(3)
    with S.FsFem(p) as ctx:
        bg = S.sfem_get_rhs(ctx.h, asm.ndof)
        assert np.abs(bg - b).max() <= 1e-12 * np.abs(b).max()
        S.sfem_assemble(ctx.h)
        absK = asm.matrix().copy()
        absK.data = np.abs(absK.data)
        for nrhs in (1, 2):
            u = rng.standard_normal((nrhs, asm.ndof))
            y_ref = np.stack([A @ u[r] for r in range(nrhs)])
            maj = np.stack([absK @ np.abs(u[r]) for r in range(nrhs)])
            ud = torch.from_numpy(u).cuda()
            for op in (S.SFEM_OP_MF64, S.SFEM_OP_CSR64):
                y = torch.empty_like(ud)
                S.sfem_apply(ctx.h, ud, y, op, nrhs)
                err = np.abs(y.cpu().numpy() - y_ref)
                assert (err <= 1e-12 * maj + 1e-300).all(), (op, (err / maj).max())
            u32 = ud.float()
            y32 = torch.empty_like(u32)
            S.sfem_apply(ctx.h, u32, y32, S.SFEM_OP_MF32, nrhs)
            # reference on the FP32-rounded input
            y_ref32 = np.stack([A @ u32.double().cpu().numpy()[r] for r in range(nrhs)])
            d = y32.double().cpu().numpy() - y_ref32
            assert np.abs(d).max() <= 2e-5 * maj.max()
            assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(y_ref32)
            # FP32 arithmetic on FP64 vectors (inner operator of the mixed solve)
            y64 = torch.empty_like(ud)
            S.sfem_apply(ctx.h, ud, y64, S.SFEM_OP_MF32_F64, nrhs)
            d = y64.cpu().numpy() - y_ref
            assert np.abs(d).max() <= 2e-5 * maj.max()
            assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(y_ref)


def test_pcg64_matches_oracle(S, cfg1):
    p, asm, A, b = cfg1
    x_ref = OS.cholesky_solve(A.toarray(), b)
    ref_its = OS.jacobi_pcg(A, b, 1e-10).iterations
    with S.FsFem(p) as ctx:
        S.sfem_assemble(ctx.h)
        for op in (S.SFEM_OP_CSR64, S.SFEM_OP_MF64):
            x = np.zeros(asm.ndof)
            info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=op, tol=1e-10))
            assert info["true_relres"] <= 1e-10
            assert abs(info["iterations"] - ref_its) <= 0.10 * ref_its, (info, ref_its)
            rel = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
            assert rel <= 1e-7, rel
            # the oracle's own true residual of the GPU solution
            assert OS.np.linalg.norm(b - A @ x) <= 2e-10 * np.linalg.norm(b)


def test_ir32_64_matches_oracle(S, cfg1):
    p, asm, A, b = cfg1
    x_ref = OS.cholesky_solve(A.toarray(), b)
    with S.FsFem(p) as ctx:
        for op in (S.SFEM_OP_MF64,):
            x = np.zeros(asm.ndof)
            info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, op64=op, tol=1e-10))
            assert info["true_relres"] <= 1e-10
            assert info["outer_iterations"] >= 2
            rel = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
            assert rel <= 1e-6, rel


def test_device_inputs_and_warm_start(S, cfg1):
    import torch
    p, asm, A, b = cfg1
    x_ref = OS.cholesky_solve(A.toarray(), b)
    with S.FsFem(p, on_device=True) as ctx:
        x = torch.zeros(asm.ndof, dtype=torch.float64, device="cuda")
        info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10, u_on_device=True))
        assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
        # warm start from the solution converges at once
        info2 = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10, u_on_device=True,
                                                    warm_start=True))
        assert info2["iterations"] <= 2 and info2["true_relres"] <= 1e-10


def test_f_extra_body_force(S, cfg1):
    p, asm, A, b = cfg1
    rng = np.random.default_rng(9)
    fx = rng.standard_normal(asm.ndof) * 1e3
    _, b2, _, _ = F.dirichlet_system(asm.matrix(), F.traction_load(p.mesh.n_nodes, p.mesh.xyz, p.trac_tris,
                                                                   p.trac)[0] + fx, p.dir_dofs, p.dir_vals)
    x_ref = OS.cholesky_solve(A.toarray(), b2)
    with S.FsFem(p) as ctx:
        x = np.zeros(asm.ndof)
        info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10), f_extra=fx)
        assert np.isclose(info["bnorm"], np.linalg.norm(b2), rtol=1e-12)
        assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

class _P:
    """Minimal problem record for hand-made meshes."""

    def __init__(self, xyz, tets, E=1e9, nu=0.25, dofs=None, vals=None, tris=None, trac=None):
        self.mesh = type("M", (), {"xyz": np.asarray(xyz, float), "tets": np.asarray(tets, np.int32)})()
        self.E, self.nu = E, nu
        self.dir_dofs = np.zeros(0, np.int32) if dofs is None else np.asarray(dofs, np.int32)
        self.dir_vals = np.zeros(0) if vals is None else np.asarray(vals, float)
        self.trac_tris = np.zeros((0, 3), np.int32) if tris is None else np.asarray(tris, np.int32)
        self.trac = np.zeros((1, 0, 3)) if trac is None else np.asarray(trac, float)


def test_single_tet_equals_fem(S):
    X = np.array([[0.1, 0.0, 0.2], [1.3, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.2, 1.1]])
    T = np.array([[0, 1, 2, 3]])
    with S.FsFem(_P(X, T)) as ctx:
        assert ctx.info["n_faces"] == 4 and ctx.info["n_boundary"] == 4
        rp, col, val = S.sfem_assemble(ctx.h)
        K = np.zeros((12, 12))
        rpn, cn, vn = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        for r in range(12):
            K[r, cn[rpn[r]:rpn[r + 1]]] = vn[rpn[r]:rpn[r + 1]]
        Kf = F.dense_K_fem(X, T, 1e9, 0.25)
        assert np.abs(K - Kf).max() <= 1e-12 * np.abs(Kf).max()


def test_orientation_and_ragged_sizes(S):
    import torch
    m = kuhn_beam(3, 2, 1, (1.5, 1.0, 0.5), 0.1, seed=4)     # 36 tets: a ragged tail of one block
    t2 = m.tets.copy()
    t2[::2] = t2[::2][:, [0, 2, 1, 3]]
    dofs, vals = clamp_dofs(m, 0, 0)
    K_ref = F.assemble(m.xyz, m.tets, 70e9, 0.3).matrix()
    for tets in (m.tets, t2):
        with S.FsFem(_P(m.xyz, tets, 70e9, 0.3, dofs, vals)) as ctx:
            _, _, val = S.sfem_assemble(ctx.h)
            assert np.abs(val.cpu().numpy() - K_ref.data).max() <= 1e-12 * np.abs(K_ref.data).max()
            u = torch.randn(ctx.ndof, dtype=torch.float64, device="cuda")
            y = torch.empty_like(u)
            S.sfem_apply(ctx.h, u, y, S.SFEM_OP_MF64)
            A, _, _, _ = F.dirichlet_system(K_ref, np.zeros(ctx.ndof), dofs, vals)
            yr = A @ u.cpu().numpy()
            assert np.abs(y.cpu().numpy() - yr).max() <= 1e-11 * np.abs(yr).max()


def test_patch_test_on_gpu(S):
    """Nonzero prescribed values: the linear field on all boundary nodes is
    reproduced inside (STEP 5 with g != 0)."""
    m = kuhn_beam(4, 3, 5, (2.0, 1.0, 1.5), 0.1, seed=21)
    rng = np.random.default_rng(0)
    a = rng.normal(size=3) * 1e-3
    H = rng.normal(size=(3, 3)) * 1e-3
    u_lin = (a[None, :] + m.xyz @ H.T).ravel()
    lat = m.lattice()
    bnd = ((lat == 0) | (lat == np.array([m.nx, m.ny, m.nz]))).any(axis=1)
    dofs = (3 * np.nonzero(bnd)[0][:, None] + np.arange(3)).ravel().astype(np.int32)
    with S.FsFem(_P(m.xyz, m.tets, 210e9, 0.3, dofs, u_lin[dofs])) as ctx:
        for kind in (S.SFEM_SOLVE_PCG64, S.SFEM_SOLVE_IR32_64):
            x = np.zeros(ctx.ndof)
            S.sfem_solve(ctx.h, x, S.solve_opts(kind=kind, tol=1e-12 if kind == 0 else 1e-10))
            assert np.abs(x - u_lin).max() <= 1e-9 * np.abs(u_lin).max()


@pytest.mark.parametrize("case", ["degenerate", "index", "three_tets_one_face", "nan", "bad_dof"])
def test_invalid_meshes_rejected(S, case):
    X = np.array([[0., 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]])
    T = np.array([[0, 1, 2, 3], [0, 2, 1, 4]])
    dofs = None
    if case == "degenerate":
        X = X.copy()
        X[3] = [0.3, 0.3, 0.0]               # coplanar with 0,1,2
    elif case == "index":
        T = np.array([[0, 1, 2, 3], [0, 2, 1, 9]])
    elif case == "three_tets_one_face":
        T = np.array([[0, 1, 2, 3], [0, 2, 1, 4], [0, 1, 2, 5]])
    elif case == "nan":
        X = X.copy()
        X[1, 0] = np.nan
    elif case == "bad_dof":
        dofs = [0, 1, 999]
    P = _P(X, T, dofs=dofs, vals=None if dofs is None else [0.0, 0.0, 0.0])
    with pytest.raises(S.SfemError) as ei:
        S.FsFem(P)
    assert ei.value.status == S.SFEM_EMESH


def test_breakdown_and_iteration_cap(S, cfg1):
    p, asm, _, _ = cfg1
    with S.FsFem(p) as ctx:
        x = np.zeros(asm.ndof)
        info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10, max_iter=5),
                            check=False)
        assert info["status"] == S.SFEM_ENOCONV and info["iterations"] <= 5 + 1
        assert info["true_relres"] > 1e-10
    # unconstrained K is singular: CG must end with a status, not a hang
    P = _P(p.mesh.xyz, p.mesh.tets, p.E, p.nu, tris=p.trac_tris, trac=p.trac)
    with S.FsFem(P) as ctx:
        x = np.zeros(asm.ndof)
        info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-12, max_iter=3000),
                            check=False)
        assert info["status"] in (S.SFEM_ENOCONV, S.SFEM_EBREAKDOWN, S.SFEM_OK)


# ---------------------------------------------------------------------------
# the 2M-tet beam (200 x 40 x 42 cells): sampled rows and properties
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg2():
    return cantilever(200, 40, 42, seed=2)


def test_full_size_sampled_rows_and_solve(S, cfg2):
    import torch
    p = cfg2
    m = p.mesh
    assert m.n_tets == 2_016_000
    rng = np.random.default_rng(5)
    with S.FsFem(p, on_device=True) as ctx:
        info = ctx.info
        nb = 4 * (200 * 40 + 40 * 42 + 42 * 200)
        assert info["n_boundary"] == nb and info["n_interior"] == (4 * m.n_tets - nb) // 2
        rp, col, val = S.sfem_assemble(ctx.h)
        rp, col, val = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        u = torch.randn(ctx.ndof, dtype=torch.float64, device="cuda") * 1e-3
        free = np.ones(ctx.ndof)
        free[p.dir_dofs] = 0
        um = u.cpu().numpy() * free
        y64 = torch.empty_like(u)
        S.sfem_apply(ctx.h, u, y64, S.SFEM_OP_MF64)
        y64 = y64.cpu().numpy()
        # the FP32 tiled operator (4928 tiles of <= 512 tets, 16-bit local
        # ids, halo tets) on the FP32-rounded input, as the mixed solve runs it
        u32 = u.float()
        y32 = torch.empty_like(u32)
        S.sfem_apply(ctx.h, u32, y32, S.SFEM_OP_MF32)
        y32 = y32.double().cpu().numpy()
        um32 = u32.double().cpu().numpy() * free
        u32_inf = np.abs(um32).max()
        worst32 = 0.0
        nodes = np.concatenate([[0, m.n_nodes - 1], rng.integers(0, m.n_nodes, 24)])
        for node in nodes:
            cols, vals = F.K_rows_submesh(m.xyz, m.tets, p.E, p.nu, int(node))
            for c in range(3):
                r = 3 * node + c
                g = slice(rp[r], rp[r + 1])
                assert np.array_equal(col[g], cols)
                ref = vals[c]
                # |dK_ij| <= 1e-12 max(|K_ij|, sqrt(K_ii K_jj)), with K_jj taken
                # as K_ii (the sampled row's diagonal) at this size
                kii = abs(ref[np.searchsorted(cols, r)])
                bad = np.abs(val[g] - ref) > 1e-12 * np.maximum(np.abs(ref), kii)
                assert not bad.any(), (node, c, (np.abs(val[g] - ref) / kii).max())
                if free[r]:
                    yr = ref @ um[cols]
                    assert abs(y64[r] - yr) <= 1e-11 * (np.abs(ref) @ np.abs(um[cols]))
                    bound = mf32_row_bound(ref, um32[cols], u32_inf)
                    d32 = abs(y32[r] - ref @ um32[cols])
                    worst32 = max(worst32, d32 / bound * MF32_ROW_C)
                    assert d32 <= bound, (node, c, d32, bound)
        print(f"\nMF32 sampled rows: max |dy_i| / (2^-24 (|K|(|u|+|u|_inf))_i) = {worst32:.2f} (bound {MF32_ROW_C:.0f})")
        # mixed-precision solve to 1e-8; global equilibrium: reactions balance the load
        x = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        si = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=1e-8, u_on_device=True))
        assert si["true_relres"] <= 1e-8
        # global equilibrium with the GPU's own K: the clamp reactions balance
        # the 1e6 N load (rigid translations lie in the null space of K)
        import scipy.sparse as sp
        K = sp.csr_matrix((val, col, rp), shape=(ctx.ndof, ctx.ndof))
        xr = x.cpu().numpy()
        Kx = K @ xr
        clamp = np.zeros(ctx.ndof, bool)
        clamp[p.dir_dofs] = True
        Rz = Kx[2::3][clamp[2::3]].sum()
        assert abs(Rz - 1e6) <= 1e-5 * 1e6, Rz
        tip = face_nodes(m, 0, 1)
        d = -xr.reshape(-1, 3)[tip, 2].mean()
        # between the 80x16x16 oracle level (0.01872 m) and the Timoshenko value
        assert 0.0187 < d < 0.01920, d
