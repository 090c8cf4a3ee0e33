"""Batched solve (many beams x four load cases in persistent launches)
against the FP64 oracle and against the single-system solver.

Tolerance: each system reaches a FP64 true relative residual <= tol, and
its displacements match the oracle's exact (Cholesky) solution to 1e-6
relative L2, the bar for reduced-precision forms."""
import numpy as np
import pytest

from inputs.kuhn_beam import batch_beams, clamp_dofs, four_load_cases, kuhn_beam, Problem
from oracle import fsfem as F
from oracle import solve as OS

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


def _small_batch():
    out = []
    rng = np.random.default_rng(77)
    for b, cells in enumerate([(6, 2, 2), (9, 3, 2), (12, 2, 3), (5, 3, 3), (8, 4, 2)]):
        mesh = kuhn_beam(*cells, dims=(float(rng.uniform(2, 6)), 1.0, 1.0), jitter=0.1, seed=300 + b)
        dofs, vals = clamp_dofs(mesh, 0, 0)
        tris, trac = four_load_cases(mesh)
        out.append(Problem(mesh, float(rng.uniform(50e9, 300e9)), float(rng.uniform(0.2, 0.45)), dofs, vals,
                           tris, trac))
    return out


def _oracle_solutions(p):
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    fs = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)
    sols = []
    for r in range(p.nrhs):
        A, b, _, _ = F.dirichlet_system(K, fs[r], p.dir_dofs, p.dir_vals)
        sols.append(OS.cholesky_solve(A.toarray(), b))
    return np.stack(sols)


@pytest.mark.parametrize("graph,precond", [(True, 0), (False, 0), (True, 2), (False, 2)])
def test_batch_matches_oracle(S, graph, precond):
    """precond 0: Jacobi; precond 2: the two-level preconditioner inside the
    persistent launch (these small beams get one or two patch centres per
    axis, so the clamped interpolation cells of the coarse space are
    exercised)."""
    probs = _small_batch()
    ctxs = [S.FsFem(p) for p in probs]
    try:
        us = [np.zeros((p.nrhs, c.ndof)) for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        infos, stats = S.sfem_batch_solve([c.h for c in ctxs], us,
                                          S.batch_opts(tol=1e-10, use_graph=graph, precond=precond), n_sys)
        assert stats["n_systems"] == n_sys == 20
        assert stats["rounds"] >= 2 and stats["ctas_per_sm"] >= 1
        k = 0
        for p, u in zip(probs, us):
            ref = _oracle_solutions(p)
            for r in range(p.nrhs):
                assert infos[k]["status"] == S.SFEM_OK and infos[k]["true_relres"] <= 1e-10, infos[k]
                rel = np.linalg.norm(u[r] - ref[r]) / np.linalg.norm(ref[r])
                assert rel <= 1e-6, (k, rel)
                k += 1
    finally:
        for c in ctxs:
            c.close()


def test_batch_single_system_equals_single_solve(S):
    p = _small_batch()[1]
    p1 = Problem(p.mesh, p.E, p.nu, p.dir_dofs, p.dir_vals, p.trac_tris, p.trac[2:3])   # torsion case only
    with S.FsFem(p1) as ctx:
        u = np.zeros((1, ctx.ndof))
        infos, stats = S.sfem_batch_solve([ctx.h], [u], S.batch_opts(tol=1e-10), 1)
        x = np.zeros(ctx.ndof)
        info = S.sfem_solve(ctx.h, x, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=1e-10))
        assert np.linalg.norm(u[0] - x) <= 1e-7 * np.linalg.norm(x)
        assert infos[0]["true_relres"] <= 1e-10


def test_batch_uneven_beams_device_vectors(S):
    """Eight beams of the uneven batch family (seeded grids, lengths and
    materials), device vectors: every system reaches 1e-8."""
    import torch
    probs = [p for p in batch_beams(64, seed=5) if p.mesh.n_tets < 60000][:8]
    ctxs = [S.FsFem(p) for p in probs]
    try:
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        infos, stats = S.sfem_batch_solve([c.h for c in ctxs], us, S.batch_opts(tol=1e-8, u_on_device=True), n_sys)
        assert all(i["status"] == S.SFEM_OK and i["true_relres"] <= 1e-8 for i in infos)
        # single-system solves of the first beam agree
        c0 = ctxs[0]
        for r in range(probs[0].nrhs):
            x = np.zeros(c0.ndof)
            S.sfem_solve(c0.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=r, tol=1e-9), check=False)
            assert np.linalg.norm(us[0][r].cpu().numpy() - x) <= 1e-5 * np.linalg.norm(x)
    finally:
        for c in ctxs:
            c.close()


def test_batch_two_level_uneven_beams(S):
    """The per-system two-level mode (precond = 1) on eight beams of the
    uneven batch family: every system reaches 1e-8 and agrees with FP64 PCG
    of the same context."""
    import torch
    probs = [p for p in batch_beams(64, seed=5) if p.mesh.n_tets < 60000][:8]
    ctxs = [S.FsFem(p) for p in probs]
    try:
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        infos, stats = S.sfem_batch_solve([c.h for c in ctxs], us, S.batch_opts(tol=1e-8, u_on_device=True,
                                                                                  precond=1), n_sys)
        assert stats["n_systems"] == n_sys
        assert all(i["status"] == S.SFEM_OK and i["true_relres"] <= 1e-8 for i in infos)
        for k in (0, 3):
            c = ctxs[k]
            for r in range(probs[k].nrhs):
                x = np.zeros(c.ndof)
                S.sfem_solve(c.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=r, tol=1e-9), check=False)
                assert np.linalg.norm(us[k][r].cpu().numpy() - x) <= 1e-5 * np.linalg.norm(x)
        with pytest.raises(S.SfemError):
            S.sfem_batch_solve([c.h for c in ctxs], us, S.batch_opts(precond=3, u_on_device=True), n_sys)
    finally:
        for c in ctxs:
            c.close()


def test_batch_persistent_two_level_uneven_beams(S):
    """precond = 2 (the two-level preconditioner as phases of the persistent
    launch) on eight beams of the uneven batch family, one of them with a
    user-chosen coarse grid kept by its context: every system reaches 1e-8,
    agrees with FP64 PCG of its context, and the batch needs a fraction of
    the persistent Jacobi solve's iterations."""
    import torch
    probs = [p for p in batch_beams(64, seed=5) if p.mesh.n_tets < 60000][:8]
    ctxs = [S.FsFem(p) for p in probs]
    try:
        S.sfem_coarse_setup(ctxs[2].h, patch_dims=(3, 2, 2))
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        _, st0 = S.sfem_batch_solve([c.h for c in ctxs], us, S.batch_opts(tol=1e-8, u_on_device=True), n_sys)
        for u in us:
            u.zero_()
        infos, st2 = S.sfem_batch_solve([c.h for c in ctxs], us,
                                        S.batch_opts(tol=1e-8, u_on_device=True, precond=2), n_sys)
        print(f"\npersistent batch, 8 beams x 4 loads: Jacobi {st0['total_iterations']} iterations "
              f"({st0['launch_iterations']} launch iterations, {st0['fallback_systems']} fallbacks, "
              f"{st0['ms']:.1f} ms); two-level {st2['total_iterations']} ({st2['launch_iterations']}, "
              f"{st2['fallback_systems']}, {st2['ms']:.1f} ms)")
        assert S.sfem_coarse_info(ctxs[2].h)["patch_dims"] == (3, 2, 2)
        assert all(i["status"] == S.SFEM_OK and i["true_relres"] <= 1e-8 for i in infos), infos
        assert st2["n_systems"] == n_sys and st2["launch_iterations"] > 0
        assert st2["fallback_systems"] <= 1
        assert 3 * st2["total_iterations"] < st0["total_iterations"]
        for k in (0, 2, 5):
            c = ctxs[k]
            for r in range(probs[k].nrhs):
                x = np.zeros(c.ndof)
                S.sfem_solve(c.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=r, tol=1e-9), check=False)
                assert np.linalg.norm(us[k][r].cpu().numpy() - x) <= 1e-5 * np.linalg.norm(x)
    finally:
        for c in ctxs:
            c.close()


def test_batch_in_launch_two_level_with_jacobi_beams(S):
    """precond = 2 with patch_nodes = -1: only the contexts that have a coarse
    space (three of six here) use the two-level preconditioner, the others
    run Jacobi inside the same persistent launch; every system reaches 1e-8
    and agrees with FP64 PCG of its context, and no coarse space is built."""
    import torch
    probs = [p for p in batch_beams(64, seed=5) if p.mesh.n_tets < 60000][:6]
    ctxs = [S.FsFem(p) for p in probs]
    try:
        for k in (0, 2, 4):
            S.sfem_coarse_setup(ctxs[k].h)
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        infos, st = S.sfem_batch_solve([c.h for c in ctxs], us,
                                       S.batch_opts(tol=1e-8, u_on_device=True, precond=2, patch_nodes=-1), n_sys)
        assert all(i["status"] == S.SFEM_OK and i["true_relres"] <= 1e-8 for i in infos), infos
        for k in (1, 3, 5):  # still without a coarse space
            with pytest.raises(S.SfemError):
                S.sfem_coarse_info(ctxs[k].h)
        # two-level beams need far fewer iterations than the Jacobi beams of similar size
        its = [sum(i["iterations"] for i in infos[4 * k:4 * k + 4]) for k in range(len(probs))]
        print("\nper-beam iterations (two-level on beams 0, 2, 4):", its)
        for k in (0, 1):
            c = ctxs[k]
            for r in range(probs[k].nrhs):
                x = np.zeros(c.ndof)
                S.sfem_solve(c.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=r, tol=1e-9), check=False)
                assert np.linalg.norm(us[k][r].cpu().numpy() - x) <= 1e-5 * np.linalg.norm(x)
        with pytest.raises(S.SfemError):
            S.sfem_batch_solve([c.h for c in ctxs], us, S.batch_opts(precond=2, patch_nodes=-2, u_on_device=True),
                               n_sys)
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("precond", [0, 2])
def test_batch_many_systems_mixed_load_cases(S, precond):
    """110 small beams with 1 to 4 load cases each (273 systems: more than one
    block-wide pass of the kernel's per-system loops and work lists): every
    system reaches 1e-8, and a sample agrees with single-system FP64 PCG."""
    import torch
    rng = np.random.default_rng(11)
    probs = []
    for b in range(110):
        cells = (int(rng.integers(4, 9)), int(rng.integers(2, 4)), int(rng.integers(2, 4)))
        mesh = kuhn_beam(*cells, dims=(float(rng.uniform(2, 5)), 1.0, 1.0), jitter=0.1, seed=500 + b)
        dofs, vals = clamp_dofs(mesh, 0, 0)
        tris, trac = four_load_cases(mesh)
        k = 1 + b % 4
        probs.append(Problem(mesh, float(rng.uniform(50e9, 300e9)), float(rng.uniform(0.2, 0.45)), dofs, vals,
                             tris, trac[:k]))
    ctxs = [S.FsFem(p) for p in probs]
    try:
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        assert n_sys == 273
        infos, st = S.sfem_batch_solve([c.h for c in ctxs], us,
                                       S.batch_opts(tol=1e-8, u_on_device=True, precond=precond), n_sys)
        assert st["n_systems"] == n_sys
        assert all(i["status"] == S.SFEM_OK and i["true_relres"] <= 1e-8 for i in infos)
        for k in (0, 37, 74, 109):
            c = ctxs[k]
            for r in range(probs[k].nrhs):
                x = np.zeros(c.ndof)
                S.sfem_solve(c.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=r, tol=1e-9), check=False)
                assert np.linalg.norm(us[k][r].cpu().numpy() - x) <= 1e-5 * np.linalg.norm(x)
    finally:
        for c in ctxs:
            c.close()
