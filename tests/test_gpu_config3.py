"""The mixed-precision solve on the large cantilever (400 x 80 x 64 cells x 6 =
12,288,000 tets, 6.33M DOF) at nu = 0.3 and at the near-incompressible
nu = 0.49, with the two-level preconditioner: FP32 matrix-free operator and
FP32 inner vectors, FP64 true residual and correction.

The oracle cannot solve at this size, so the checks are sampled:
- rows of K computed by the oracle on the sub-mesh around sampled nodes
  (oracle/fsfem.py K_rows_submesh) against the GPU's FP64 operator;
- the residual b - K u of the mixed solution at sampled free rows, formed
  with those oracle rows and the oracle's traction load b: bounded by the
  solve's own stopping test, |r_i| <= ||r|| <= 1e-8 ||b||;
- the mixed solution against the FP64 two-level PCG solution of the same
  system at the same tolerance (relative L2 difference, printed);
- the FP32 tiled operator (the inner operator of the mixed solve: 16-bit
  tile-local ids and halo tables at their full-size extent) on an FP32
  input at the same sampled rows, with the row-wise FP32 bound of
  tests/test_gpu_parity.py.
"""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever
from oracle import fsfem as F
from tolerances import mf32_row_bound

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


# relative L2 distance between the mixed solution and the FP64 PCG solution,
# both at 1e-8 (FP64 CG does not get much below 1e-8 on these beams: the
# element forces cancel to loads of about 1e-9 of their size): bounded by
# about cond(A) x 1e-8, larger at nu = 0.49 (lambda / mu = 49)
@pytest.mark.parametrize("nu,max_diff", [(0.3, 1e-6), (0.49, 1e-5)])
def test_large_beam_mixed_solve(S, nu, max_diff):
    p = cantilever(400, 80, 64, seed=4, nu=nu)
    m = p.mesh
    assert m.n_tets == 12_288_000 and 3 * m.n_nodes == 6_333_795
    rng = np.random.default_rng(11)
    with S.FsFem(p, on_device=True) as fe:
        info = S.sfem_coarse_setup(fe.h, patch_dims=(41, 9, 7))
        assert info["n_coarse"] == 7749
        u = torch.zeros(fe.ndof, dtype=torch.float64, device="cuda")
        si = S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=1e-8, u_on_device=True,
                                                precond=1, fp32_vectors=3, inner_tol=0.03))
        assert si["status"] == 0 and si["true_relres"] <= 1e-8
        print(f"\nnu={nu}: mixed solve {si['iterations']} inner iterations, {si['outer_iterations']} outer, "
              f"{si['fallbacks']} fallbacks, {si['solve_ms']:.0f} ms, true relres {si['true_relres']:.2e}")
        # the FP64 form of the same solve
        u64 = torch.zeros_like(u)
        s64 = S.sfem_solve(fe.h, u64, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_MF64, tol=1e-8,
                                                   u_on_device=True, precond=1))
        assert s64["status"] == 0 and s64["true_relres"] <= 1e-8
        diff = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))
        print(f"nu={nu}: FP64 PCG {s64['iterations']} iterations; mixed vs FP64 relative L2 {diff:.2e}")
        assert diff <= max_diff
        # oracle rows at sampled nodes: K rows against the GPU's FP64 operator
        # on a random vector, and the residual of the mixed solution
        free = np.ones(fe.ndof, bool)
        free[p.dir_dofs] = False
        v = torch.randn(fe.ndof, dtype=torch.float64, device="cuda") * 1e-3
        vm = v.cpu().numpy() * free
        yv = torch.empty_like(v)
        S.sfem_apply(fe.h, v, yv, S.SFEM_OP_MF64)
        yv = yv.cpu().numpy()
        v32 = v.float()
        yv32 = torch.empty_like(v32)
        S.sfem_apply(fe.h, v32, yv32, S.SFEM_OP_MF32)
        yv32 = yv32.double().cpu().numpy()
        vm32 = v32.double().cpu().numpy() * free
        v32_inf = np.abs(vm32).max()
        x = u.cpu().numpy()
        f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
        bnorm = np.linalg.norm(f * free)
        nodes = [int(n) for n in rng.integers(0, m.n_nodes, 10)]
        worst = 0.0
        for node in nodes:
            cols, vals = F.K_rows_submesh(m.xyz, m.tets, p.E, p.nu, node)
            for c in range(3):
                r = 3 * node + c
                if not free[r]:
                    continue
                ref = vals[c] @ vm[cols]
                assert abs(yv[r] - ref) <= 1e-11 * (np.abs(vals[c]) @ np.abs(vm[cols])), (node, c)
                d32 = abs(yv32[r] - vals[c] @ vm32[cols])
                assert d32 <= mf32_row_bound(vals[c], vm32[cols], v32_inf), (node, c, d32)
                res = abs(f[r] - vals[c] @ x[cols])
                worst = max(worst, res / bnorm)
        print(f"nu={nu}: sampled residual rows (oracle K) max |r_i| / ||b|| = {worst:.2e}")
        assert worst <= 1e-8
