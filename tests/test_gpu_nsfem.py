"""NS-FEM-T4 and ES-FEM-T4 on the GPU (SFEM_OP_NS64 / SFEM_OP_ES64 through the
C ABI) against the oracle's node-by-node and edge-by-edge assemblies
(oracle/nsfem.py, oracle/esfem.py): the operator on random vectors, the PCG64
solve, and the stiffness ordering of the T4 models on the cantilever
(FEM-T4 stiffest, NS-FEM softest)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from inputs.kuhn_beam import cantilever, face_nodes
from oracle import esfem as ES
from oracle import fsfem as F
from oracle import nsfem as N

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem
    return sfem


@pytest.mark.parametrize("model", ["ns", "es"])
def test_ns_es_operator_and_solve(S, model):
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    K = (N.assemble_ns if model == "ns" else ES.assemble_es)(m.xyz, m.tets, p.E, p.nu)
    OP = S.SFEM_OP_NS64 if model == "ns" else S.SFEM_OP_ES64
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, free, _ = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    rng = np.random.default_rng(9)
    with S.FsFem(p) as fe:
        u = rng.standard_normal((2, fe.ndof))
        ud = torch.from_numpy(u).cuda()
        y = torch.empty_like(ud)
        S.sfem_apply(fe.h, ud, y, OP, 2)
        y = y.cpu().numpy()
        for k in range(2):
            ref = A @ u[k]
            assert np.abs(y[k] - ref).max() <= 1e-12 * np.abs(ref).max()
        x = np.zeros(fe.ndof)
        info = S.sfem_solve(fe.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=OP, tol=1e-10))
        assert info["status"] == 0 and info["true_relres"] <= 1e-10
        ref = spla.spsolve(A.tocsc(), b)
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
        x_fs = np.zeros(fe.ndof)
        S.sfem_solve(fe.h, x_fs, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_MF64, tol=1e-10))
        for kw in ({"kind": S.SFEM_SOLVE_IR32_64, "op64": OP},
                   {"kind": S.SFEM_SOLVE_PCG64, "op64": OP, "bc": 1}):
            with pytest.raises(S.SfemError):
                S.sfem_solve(fe.h, np.zeros(fe.ndof), S.solve_opts(**kw))
    Kfem = F.fem_K_csr(m.xyz, m.tets, p.E, p.nu)
    Af, bf, _, _ = F.dirichlet_system(Kfem, f, p.dir_dofs, p.dir_vals)
    x_fem = spla.spsolve(Af.tocsc(), bf)
    tip = face_nodes(m, 0, 1)
    d = [-v.reshape(-1, 3)[tip, 2].mean() for v in (x_fem, x_fs, x)]
    print(f"\ntip deflection (m), 20x4x4 cantilever: FEM-T4 {d[0]:.5e}  FS-FEM-T4 {d[1]:.5e}  "
          f"{model.upper()}-FEM-T4 {d[2]:.5e}; PCG64 {info['iterations']} iterations")
    assert d[0] < d[1] and d[0] < d[2]
