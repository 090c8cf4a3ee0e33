"""The penalty method of STEP 5 (sfem_solve_opts.bc = 1) on the GPU against
the oracle's penalty system (oracle/fsfem.py penalty_system), with the CSR
and the matrix-free FP64 operators, and its effect on the solve: the
iteration count next to the masked elimination's.  Tolerance 1e-9: the
penalty rows (alpha ~ 1e8 max K_ii) cancel in the recursive residual, so FP64
CG does not reach the 1e-12 that the elimination reaches on this beam."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from inputs.kuhn_beam import cantilever
from oracle import fsfem as F

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


def test_penalty_matches_oracle(S):
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    alpha = 1e8 * K.diagonal().max()
    Ap, bp = F.penalty_system(K, f, p.dir_dofs, p.dir_vals, alpha)
    u_pen = spla.spsolve(Ap.tocsc(), bp)
    A, b, _, _ = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    u_el = spla.spsolve(A.tocsc(), b)
    with S.FsFem(p) as fe:
        S.sfem_assemble(fe.h)
        its = {}
        for name, op in (("csr", S.SFEM_OP_CSR64), ("mf", S.SFEM_OP_MF64)):
            u = np.zeros(fe.ndof)
            info = S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=op, tol=1e-9, bc=1))
            assert info["status"] == 0 and info["true_relres"] <= 1e-9
            err = np.linalg.norm(u - u_pen) / np.linalg.norm(u_pen)
            assert err <= 1e-6, (name, err)
            its[name] = info["iterations"]
        u = np.zeros(fe.ndof)
        el = S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, tol=1e-9))
        d = np.linalg.norm(u_pen - u_el) / np.linalg.norm(u_el)
        print(f"\npenalty (alpha = 1e8 max K_ii): {its['csr']} / {its['mf']} iterations (CSR / matrix-free) vs "
              f"{el['iterations']} with elimination; |u_pen - u_elim| / |u_elim| = {d:.1e}")
        assert d <= 1e-5
        # options the penalty path does not take
        for kw in ({"kind": S.SFEM_SOLVE_IR32_64, "bc": 1}, {"bc": 2}, {"bc": 1, "penalty_exp": 16}):
            with pytest.raises(S.SfemError):
                S.sfem_solve(fe.h, np.zeros(fe.ndof), S.solve_opts(**kw))
