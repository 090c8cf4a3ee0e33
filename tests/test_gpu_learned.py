"""Learned coarse correction: GPU kernels against the oracle (oracle/mlp.py),
flexible PCG behaviour, training on the library's own CG snapshots, and the
measured iteration gain on a slender beam (reported as measured, not
assumed)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from inputs.kuhn_beam import cantilever, multi_load_cantilever
from oracle import fsfem, mlp

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


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _random_theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for (i, o) in [(84, 128), (128, 128), (128, 3)]:
        parts += [rng.normal(size=(i, o)) * scale * math.sqrt(2.0 / i), rng.normal(size=o) * 0.1]
    return mlp.pack(parts).astype(np.float32)


def _bf16_weights(theta32):
    """Parameters as the inference path uses them: BF16 weights, FP32 biases."""
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta32.astype(np.float64))
    return mlp.pack([mlp.to_bf16(W1), b1, mlp.to_bf16(W2), b2, mlp.to_bf16(W3), b3])


@pytest.fixture(scope="module")
def beam(S):
    p = cantilever(12, 3, 3, seed=4)
    fe = S.FsFem(p)
    yield p, fe
    fe.close()


def _model(S, fe, dims, seed=0):
    return S.Learned(fe.h, patch_dims=dims, seed=seed, keepalive=fe._keep)


def test_forward_matches_oracle_bf16(S, beam):
    _, fe = beam
    m = _model(S, fe, (4, 2, 2))
    theta = _random_theta(1)
    m.set_params(theta)
    assert np.array_equal(m.get_params(), theta)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(37, 84)).astype(np.float32)      # 37 rows: ragged against 8-row blocks
    Y = torch.zeros(37, 3, dtype=torch.float32, device="cuda")
    m.forward(_cuda(X), Y)
    ref, _ = mlp.forward(_bf16_weights(theta), X.astype(np.float64))
    err = np.abs(Y.cpu().numpy() - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), err
    # the BF16 rounding of the weights is visible at this tolerance
    full, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.abs(full - ref).max() > 10 * err
    m.close()


def test_loss_and_gradient_match_oracle(S, beam):
    _, fe = beam
    m = _model(S, fe, (4, 2, 2))
    theta = _random_theta(3)
    m.set_params(theta)
    rng = np.random.default_rng(4)
    for rows in (5, 300, 1100):        # 1100 rows: the split-K weight-gradient path
        X = rng.normal(size=(rows, 84)).astype(np.float32)
        T = rng.normal(size=(rows, 3)).astype(np.float32)
        g = torch.zeros(S.N_PARAMS, dtype=torch.float32, device="cuda")
        loss = m.loss_grad(_cuda(X), _cuda(T), g)
        loss_ref, g_ref = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
        assert abs(loss - loss_ref) <= 1e-5 * loss_ref
        gg = g.cpu().numpy().astype(np.float64)
        for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), mlp.unpack(gg), mlp.unpack(g_ref)):
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel < 2e-4, (rows, name, rel)
    m.close()


def test_adam_matches_oracle(S, beam):
    _, fe = beam
    m = _model(S, fe, (4, 2, 2))
    theta = _random_theta(5)
    m.set_params(theta)
    rng = np.random.default_rng(6)
    X = _cuda(rng.normal(size=(64, 84)).astype(np.float32))
    T = _cuda(rng.normal(size=(64, 3)).astype(np.float32))
    g = torch.zeros(S.N_PARAMS, dtype=torch.float32, device="cuda")
    m.loss_grad(X, T, g)
    grad = g.cpu().numpy().astype(np.float64)
    th = theta.astype(np.float64)
    mo = np.zeros_like(th)
    ve = np.zeros_like(th)
    for step in (1, 2):
        m.adam(g, lr=1e-3)
        th, mo, ve = mlp.adam(th, grad, mo, ve, step, 1e-3)
        got = m.get_params().astype(np.float64)
        assert np.abs(got - th).max() <= 2e-6 * max(1.0, np.abs(th).max()), step
    m.close()


def test_sample_matches_oracle(S, beam):
    p, fe = beam
    dims = (4, 2, 3)
    m = _model(S, fe, dims)
    assert m.patch_dims == dims and m.n_patches == 24
    rng = np.random.default_rng(7)
    r = rng.normal(size=fe.ndof)
    e = rng.normal(size=fe.ndof) * 1e-3
    X = torch.zeros(m.n_patches, 84, dtype=torch.float32, device="cuda")
    T = torch.zeros(m.n_patches, 3, dtype=torch.float32, device="cuda")
    m.sample(fe.h, _cuda(r), X, _cuda(e), T)
    pid, _, lo, ext = mlp.patch_grid(p.mesh.xyz, dims)
    Xr = mlp.features(mlp.pool(r, pid, m.n_patches), dims)
    pe = mlp.pool(e, pid, m.n_patches)
    Tr = pe / math.sqrt(float(np.mean(pe ** 2)))
    assert np.abs(X.cpu().numpy() - Xr).max() <= 1e-6 * np.abs(Xr).max()
    assert np.abs(T.cpu().numpy() - Tr).max() <= 1e-6 * np.abs(Tr).max()
    m.close()


def _oracle_system(p, rhs=0):
    m = p.mesh
    asm = fsfem.assemble(m.xyz, m.tets, p.E, p.nu)
    K = sp.csr_matrix((asm.data, asm.indices, asm.indptr), shape=(asm.ndof, asm.ndof))
    f = fsfem.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[rhs]
    A, b, free, g = fsfem.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    return A, b, free


def test_correction_matches_oracle(S, beam):
    p, fe = beam
    dims = (4, 2, 2)
    m = _model(S, fe, dims)
    theta = _random_theta(8)
    m.set_params(theta)
    A, b, free = _oracle_system(p)
    rng = np.random.default_rng(9)
    r = rng.normal(size=fe.ndof) * free
    z = torch.zeros(fe.ndof, dtype=torch.float64, device="cuda")
    alpha = m.correction(fe.h, _cuda(r), z)
    pid, _, lo, ext = mlp.patch_grid(p.mesh.xyz, dims)
    dinv = free / A.diagonal()
    z_ref, a_ref = mlp.correction(_bf16_weights(theta), r, dims, pid, p.mesh.xyz, lo, ext, free,
                                  lambda c: A @ c, dinv)
    assert a_ref != 0.0
    assert abs(alpha - a_ref) <= 1e-4 * abs(a_ref)          # c.A c from the FP32 operator
    zz = z.cpu().numpy()
    assert np.linalg.norm(zz - z_ref) <= 1e-5 * np.linalg.norm(z_ref)
    m.close()


def test_flexible_cg_without_model_is_jacobi_pcg(S, beam):
    _, fe = beam
    u1 = np.zeros(fe.ndof)
    u2 = np.zeros(fe.ndof)
    i1 = S.sfem_solve(fe.h, u1, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-9))
    i2 = S.sfem_solve(fe.h, u2, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, tol=1e-9))
    assert i2["status"] == 0 and i2["true_relres"] <= 1e-9
    assert abs(i2["iterations"] - i1["iterations"]) <= max(3, 0.03 * i1["iterations"])
    assert i2["learned_iterations"] == 0 and i2["fallbacks"] == 0
    assert np.linalg.norm(u2 - u1) <= 1e-7 * np.linalg.norm(u1)


def test_flexible_cg_with_model_reaches_the_oracle_solution(S, beam):
    p, fe = beam
    m = _model(S, fe, (4, 2, 2), seed=11)
    A, b, free = _oracle_system(p)
    u_ref = spla.spsolve(A.tocsc(), b)
    u = np.zeros(fe.ndof)
    info = S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, tol=1e-9, learned=m))
    assert info["status"] == 0 and info["true_relres"] <= 1e-9
    assert info["learned_iterations"] > 0
    assert np.linalg.norm(u - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    m.close()


@pytest.mark.parametrize("kind", ["nan", "huge"])
def test_bad_network_falls_back_to_jacobi(S, beam, kind):
    """A network that returns NaN gives z = D^-1 r at every iteration; a
    wildly scaled one is cut off by the stagnation guard.  Either way the
    solve converges with a bounded number of iterations."""
    _, fe = beam
    m = _model(S, fe, (4, 2, 2))
    theta = _random_theta(12, scale=30.0)
    if kind == "nan":
        theta[: 84 * 128] = np.nan
    m.set_params(theta)
    uj = np.zeros(fe.ndof)
    ij = S.sfem_solve(fe.h, uj, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, tol=1e-9))
    u = np.zeros(fe.ndof)
    info = S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, tol=1e-9, learned=m,
                                              learned_window=40, learned_pace=ij["iterations"]))
    assert info["status"] == 0 and info["true_relres"] <= 1e-9, info
    if kind == "nan":
        assert info["fallbacks"] == info["learned_iterations"], info
        assert abs(info["iterations"] - ij["iterations"]) <= max(3, 0.03 * ij["iterations"]), info
    else:
        # switched off by a guard; the pace guard bounds the cost
        assert info["learned_iterations"] < info["iterations"], info
        assert info["iterations"] <= 1.35 * ij["iterations"] + 40, (info, ij["iterations"])
    assert np.linalg.norm(u - uj) <= 1e-6 * np.linalg.norm(uj)
    m.close()


def test_export_import_roundtrip(S, beam):
    _, fe = beam
    m1 = _model(S, fe, (4, 2, 2), seed=21)
    blob = m1.export_blob()
    assert len(blob) == 32 + 4 * S.N_PARAMS
    m2 = _model(S, fe, (4, 2, 2), seed=22)
    assert not np.array_equal(m1.get_params(), m2.get_params())
    m2.import_blob(blob)
    assert np.array_equal(m1.get_params(), m2.get_params())
    m3 = _model(S, fe, (3, 2, 2))
    with pytest.raises(S.SfemError):
        m3.import_blob(blob)
    for m in (m1, m2, m3):
        m.close()


def test_model_of_another_mesh_is_rejected(S, beam):
    _, fe = beam
    other = S.FsFem(cantilever(6, 2, 2, seed=1))
    m = _model(S, other, (2, 1, 1))
    with pytest.raises(S.SfemError):
        S.sfem_solve(fe.h, np.zeros(fe.ndof), S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, learned=m))
    m.close()
    other.close()


# ---- training on the solver's own snapshots, and the measured gain ----------

def test_training_reduces_loss_and_gain_is_reported(S, record_property):
    train_seeds = list(range(100, 112))
    test_seeds = [200, 201, 202, 203]
    p = multi_load_cantilever(40, 8, 8, train_seeds + test_seeds)
    fe = S.FsFem(p)
    dims = (6, 2, 2)
    m = _model(S, fe, dims, seed=1)
    n = fe.ndof
    every = 4
    cap = 400 * m.n_patches * len(train_seeds)
    X = torch.zeros(cap, 84, dtype=torch.float32, device="cuda")
    T = torch.zeros(cap, 3, dtype=torch.float32, device="cuda")
    rows = 0
    jac_train = []
    for k in range(len(train_seeds)):
        us = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.sfem_solve(fe.h, us, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, rhs=k, tol=1e-10, u_on_device=True),
                     check=False)
        got, info = m.collect(fe.h, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, rhs=k, tol=1e-8,
                                                 check_every=every), us, X, T, rows)
        assert info["status"] == 0
        jac_train.append(info["iterations"])
        rows += got
    assert rows > 0
    before = m.loss_grad(X[:rows], T[:rows])
    after = m.train(X, T, rows=rows, batch_rows=2048, epochs=12, lr=1e-3, seed=3)
    assert after < before, (before, after)
    # held-out loads: iterations of Jacobi-PCG (flexible form, no model) and
    # of flexible PCG with the trained correction, paced by the Jacobi
    # iterations seen on the training loads
    pace = int(np.mean(jac_train))
    it_j, it_l, fb = [], [], []
    for k in range(len(train_seeds), len(train_seeds) + len(test_seeds)):
        uj = np.zeros(n)
        ij = S.sfem_solve(fe.h, uj, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, rhs=k, tol=1e-8))
        ul = np.zeros(n)
        il = S.sfem_solve(fe.h, ul, S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, rhs=k, tol=1e-8, learned=m,
                                                  learned_pace=pace))
        assert ij["status"] == 0 and il["status"] == 0
        assert np.linalg.norm(ul - uj) <= 1e-6 * np.linalg.norm(uj)
        # robustness bound: the pace guard caps the cost of an unhelpful network
        assert il["iterations"] <= 1.35 * ij["iterations"] + 100, (il, ij["iterations"])
        it_j.append(ij["iterations"])
        it_l.append(il["iterations"])
        fb.append(il["learned_iterations"])
    gain = float(np.mean(it_j)) / float(np.mean(it_l))
    record_property("learned_gain", gain)
    print(f"\nlearned correction: loss {before:.4f} -> {after:.4f}; held-out iterations "
          f"Jacobi {it_j} vs learned {it_l} (learned phase {fb}); gain x{gain:.3f}")
    m.close()
    fe.close()
