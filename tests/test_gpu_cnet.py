"""The learned coarse solve (sfem_cnet_*) through the C ABI against the oracle
(oracle/cnet.py, oracle/mlp.py, oracle/coarse.py).

Tolerances (FP32 arithmetic on the GPU, FP64 in the oracle):
  * forward (BF16 weights, rounded the same way on both sides, FP32
    accumulation): ||dy|| <= 1e-4 ||y|| per row;
  * loss and gradient (FP32 master weights and GEMMs): loss relative 1e-5,
    gradient |dg| <= 1e-4 max|g| per parameter block;
  * correction (FP32 restriction, network and A_c, FP64 vectors): alpha
    relative 1e-4, ||dz|| <= 1e-4 ||z||;
  * solves: the true FP64 residual decides (1e-8); displacements within
    1e-6 relative of the oracle's Cholesky solution.
"""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever, multi_load_cantilever
from oracle import cnet as CN
from oracle import coarse as OC
from oracle import fsfem as F
from oracle import mlp as M
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


DIMS = (4, 2, 2)


@pytest.fixture(scope="module")
def beam(S):
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, free, g = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    A = A.tocsr()
    freef = np.ones(A.shape[0])
    freef[p.dir_dofs] = 0
    Pi = OC.prolongation(m.xyz, DIMS, freef)
    Ac = OC.galerkin(A, Pi)
    return p, A, b, freef, Pi, Ac


def _ctx(S, p):
    ctx = S.FsFem(p, on_device=True)
    S.sfem_assemble(ctx.h)
    S.sfem_coarse_setup(ctx.h, patch_dims=DIMS)
    return ctx


def test_forward_matches_oracle_bf16(S, beam):
    import torch
    p, A, b, freef, Pi, Ac = beam
    with _ctx(S, p) as ctx:
        for hid in (32, 128):
            net = S.CNet(ctx.h, hidden=hid, seed=7, keepalive=ctx._keep)
            nc = net.n_coarse
            assert nc == 3 * int(np.prod(DIMS)) and net.n_params == CN.n_params(nc, hid)
            rng = np.random.default_rng(hid)
            theta = (rng.normal(size=net.n_params) * 0.3).astype(np.float32)
            net.set_params(theta)
            X = rng.normal(size=(5, nc)).astype(np.float32)
            Y = torch.zeros((5, nc), dtype=torch.float32, device="cuda")
            net.forward(ctx.h, torch.from_numpy(X).cuda(), Y)
            f = CN.network(theta.astype(np.float64), nc, hid, bf16=True)
            for r in range(5):
                x = X[r].astype(np.float64)
                want = f(x / np.sqrt(np.mean(x * x)))
                got = Y[r].double().cpu().numpy()
                assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want), (hid, r)
            net.close()


def test_loss_and_gradient_match_oracle(S, beam):
    import torch
    p, A, b, freef, Pi, Ac = beam
    with _ctx(S, p) as ctx:
        net = S.CNet(ctx.h, hidden=64, seed=3, keepalive=ctx._keep)
        nc, hid = net.n_coarse, net.hidden
        rng = np.random.default_rng(5)
        theta = (rng.normal(size=net.n_params) * 0.2).astype(np.float32)
        net.set_params(theta)
        for rows in (3, 700):
            X = rng.normal(size=(rows, nc)).astype(np.float32)
            T = rng.normal(size=(rows, nc)).astype(np.float32)
            g = torch.zeros(net.n_params, dtype=torch.float32, device="cuda")
            loss = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), g)
            lo, go = M.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                                     CN.dims(nc, hid))
            assert abs(loss - lo) <= 1e-5 * abs(lo), (rows, loss, lo)
            gg = g.double().cpu().numpy()
            W1, b1, W2, b2, W3, b3 = M.unpack(go, nc, hid, nc)
            k = 0
            for blk in (W1, b1, W2, b2, W3, b3):
                ref = blk.ravel()
                d = np.abs(gg[k:k + ref.size] - ref)
                assert d.max() <= 1e-4 * np.abs(ref).max() + 1e-12, (rows, k, d.max(), np.abs(ref).max())
                k += ref.size
        net.close()


def test_correction_matches_oracle(S, beam):
    import torch
    p, A, b, freef, Pi, Ac = beam
    dinv = 1.0 / A.diagonal()
    with _ctx(S, p) as ctx:
        net = S.CNet(ctx.h, hidden=64, seed=11, keepalive=ctx._keep)
        rng = np.random.default_rng(8)
        theta = (rng.normal(size=net.n_params) * 0.2).astype(np.float32)
        net.set_params(theta)
        f = CN.network(theta.astype(np.float64), net.n_coarse, net.hidden, bf16=True)
        for k in range(3):
            r = rng.normal(size=A.shape[0]) * freef
            z = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            alpha = net.correction(ctx.h, torch.from_numpy(r).cuda(), z)
            zo, ao = CN.correction(f, r, Pi, Ac, dinv)
            assert ao != 0.0 and abs(alpha - ao) <= 1e-4 * abs(ao), (k, alpha, ao)
            assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-4 * np.linalg.norm(zo), k
        net.close()


def test_jacobi_fcg_and_untrained_model_solve(S, beam):
    """FCG(m) with the Jacobi preconditioner alone is Jacobi-PCG (iteration
    count within 10% of PCG64's, the same solution); with an untrained model
    the solve still converges to the oracle solution (the true residual
    decides; bad corrections cost iterations, not accuracy)."""
    import torch
    p, A, b, freef, Pi, Ac = beam
    x_ref = OS.cholesky_solve(A.toarray(), b)
    with _ctx(S, p) as ctx:
        o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, tol=1e-10, u_on_device=True)
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        pcg = S.sfem_solve(ctx.h, u, o)
        for window in (1, 5):
            u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
            info, _ = S.cnet_solve(None, ctx.h, u, o, window=window)
            assert info["status"] == 0 and info["true_relres"] <= 1e-10
            assert abs(info["iterations"] - pcg["iterations"]) <= 0.1 * pcg["iterations"], (window, info, pcg)
            err = np.linalg.norm(u.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
            assert err <= 1e-6, (window, err)
        net = S.CNet(ctx.h, seed=1, keepalive=ctx._keep)
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        info, _ = S.cnet_solve(net, ctx.h, u, o, window=5)
        assert info["status"] == 0 and info["true_relres"] <= 1e-10
        err = np.linalg.norm(u.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
        assert err <= 1e-6, err
        print(f"\nJacobi-PCG {pcg['iterations']}, FCG(5) with an untrained network {info['iterations']} iterations "
              f"network ({info['fallbacks']} fallbacks)")
        net.close()


def test_collected_rows_are_features_and_galerkin_targets(S, beam):
    """Rows collected from a Jacobi-PCG solve: unit-RMS inputs, and targets
    that solve the oracle's coarse system for their input up to a scale:
    A_c (s t) = x (FP32 restriction and C: relative 1e-3)."""
    import torch
    p, A, b, freef, Pi, Ac = beam
    with _ctx(S, p) as ctx:
        nc = 3 * int(np.prod(DIMS))
        X = torch.zeros((100, nc), dtype=torch.float32, device="cuda")
        T = torch.zeros_like(X)
        o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, tol=1e-8, u_on_device=True)
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        info, rows = S.cnet_solve(None, ctx.h, u, o, snap_every=7, X=X, T=T)
        assert info["status"] == 0
        assert rows >= min(100, (info["iterations"] + 6) // 7), (rows, info["iterations"])
        Xn, Tn = X[:rows].double().cpu().numpy(), T[:rows].double().cpu().numpy()
        assert np.abs(np.sqrt((Xn ** 2).mean(1)) - 1).max() < 1e-5
        for k in (0, rows // 2, rows - 1):
            x, t = Xn[k], Tn[k]
            At = Ac @ t
            s = (At @ x) / (At @ At)
            assert np.linalg.norm(s * At - x) <= 1e-3 * np.linalg.norm(x), k


def train_coarse_net(S, ctx, net, train_rhs, cap=80000, n_random=20000, rounds=4, seed=1, max_iter=3000):
    """The training protocol: round 0 on the rows of Jacobi-PCG solves of the
    training loads (a row every 3 iterations) and n_random random coarse rows
    (the coarse solve in every direction); then `rounds` on-policy rounds on
    the rows of the learned solver's own solves (a row every 2 iterations,
    solves capped at max_iter).  Returns (rows, loss after round 0, final loss)."""
    import torch
    nc = net.n_coarse
    X = torch.zeros((cap, nc), dtype=torch.float32, device="cuda")
    T = torch.zeros_like(X)
    rows = 0
    for k in train_rhs:
        o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, rhs=k, tol=1e-8, u_on_device=True)
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        _, rows = S.cnet_solve(None, ctx.h, u, o, snap_every=3, X=X, T=T, rows=rows)
    n_rand = min(n_random, cap - rows)
    net.random_rows(ctx.h, X, T, rows, n_rand, seed=seed)
    rows += n_rand
    loss0 = loss = net.train(X, T, rows=rows, batch_rows=256, epochs=80, lr=1e-3, seed=seed)
    for rnd in range(rounds):
        for k in train_rhs:
            o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, rhs=k, tol=1e-8, u_on_device=True,
                             max_iter=max_iter)
            u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
            _, rows = S.cnet_solve(net, ctx.h, u, o, window=5, snap_every=2, X=X, T=T, rows=rows, check=False)
        loss = net.train(X, T, rows=rows, batch_rows=256, epochs=30, lr=1e-3, seed=seed + 1 + rnd)
    return rows, loss0, loss


def test_training_gains_over_jacobi(S):
    """The spec claim, on the 40x8x8 cantilever (15,360 tets) with an
    11x3x3 coarse grid: train by train_coarse_net on 8 random load cases,
    then solve 2 held-out load cases.  The learned FCG(5) must take fewer
    iterations than Jacobi-PCG (both to a true residual of 1e-8): the gain
    is asserted and printed."""
    import torch
    train_seeds, test_seeds = list(range(100, 108)), [200, 201]
    p = multi_load_cantilever(40, 8, 8, train_seeds + test_seeds, seed=3)
    with S.FsFem(p, on_device=True) as ctx:
        S.sfem_assemble(ctx.h)
        S.sfem_coarse_setup(ctx.h, patch_dims=(11, 3, 3))
        net = S.CNet(ctx.h, seed=1, keepalive=ctx._keep)
        rows, loss0, loss = train_coarse_net(S, ctx, net, range(len(train_seeds)))
        gains = []
        for k in range(len(train_seeds), len(train_seeds) + len(test_seeds)):
            o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, rhs=k, tol=1e-8, u_on_device=True)
            u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
            jac = S.sfem_solve(ctx.h, u, o)
            u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
            lrn, _ = S.cnet_solve(net, ctx.h, u, o, window=5)
            assert lrn["status"] == 0 and lrn["true_relres"] <= 1e-8
            gains.append(jac["iterations"] / lrn["iterations"])
            print(f"\nheld-out load {k}: Jacobi-PCG {jac['iterations']}, learned FCG(5) {lrn['iterations']} "
                  f"iterations ({lrn['fallbacks']} fallbacks); rows {rows}, loss {loss0:.4f} -> {loss:.4f}")
        assert min(gains) > 1.3, gains
        net.close()
