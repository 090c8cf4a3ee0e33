"""Pins of the two-level preconditioner oracle (oracle/coarse.py): the coarse
space reproduces constants and linear fields, the unconstrained Galerkin
matrix annihilates rigid translations, the coarse correction is the
A-orthogonal projection onto the coarse space, the preconditioner is
symmetric, and two-level PCG reaches the direct solution in fewer iterations
than Jacobi-PCG."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from inputs.kuhn_beam import cantilever
from oracle import coarse as C
from oracle import fsfem as F
from oracle import mlp
from oracle import solve as OS


def _system(cells=(12, 3, 3)):
    p = cantilever(*cells, seed=4)
    m = p.mesh
    asm = F.assemble(m.xyz, m.tets, p.E, p.nu)
    K = asm.matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, free, g = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)
    return p, K, A, b, free


def test_coarse_space_reproduces_constants_and_linear_fields():
    p, K, A, b, free = _system()
    xyz = p.mesh.xyz
    dims = (4, 2, 3)
    ones = np.ones(3 * p.mesh.n_nodes)
    Pi = C.prolongation(xyz, dims, ones)
    P = int(np.prod(dims))
    # partition of unity per component
    for c in range(3):
        y = np.zeros((P, 3))
        y[:, c] = 1.0
        v = (Pi @ y.ravel()).reshape(-1, 3)
        assert np.allclose(v[:, c], 1.0, atol=1e-13) and np.allclose(np.delete(v, c, axis=1), 0.0)
    # a linear field sampled at the centres is reproduced inside their hull
    _, cent, lo, ext = mlp.patch_grid(xyz, dims)
    a0, G = np.array([0.3, -1.0, 2.0]), np.array([[1.0, 2.0, -1.0], [0.5, -0.2, 3.0], [-2.0, 1.0, 0.7]])
    yc = (a0 + cent.reshape(-1, 3) @ G.T).ravel()
    v = (Pi @ yc).reshape(-1, 3)
    cmin, cmax = cent.reshape(-1, 3).min(0), cent.reshape(-1, 3).max(0)
    inside = np.all((xyz >= cmin - 1e-12) & (xyz <= cmax + 1e-12), axis=1)
    assert inside.sum() > 20
    assert np.abs(v[inside] - (a0 + xyz[inside] @ G.T)).max() < 1e-12


def test_unconstrained_galerkin_matrix_annihilates_translations():
    p, K, A, b, free = _system()
    dims = (4, 2, 2)
    Pi = C.prolongation(p.mesh.xyz, dims, np.ones(K.shape[0]))
    Kc = C.galerkin(K, Pi)
    assert np.allclose(Kc, Kc.T, rtol=0, atol=1e-9 * np.abs(Kc).max())
    P = int(np.prod(dims))
    for c in range(3):
        t = np.zeros((P, 3))
        t[:, c] = 1.0
        assert np.abs(Kc @ t.ravel()).max() <= 1e-9 * np.abs(Kc).max()


def test_coarse_correction_is_the_A_orthogonal_projection():
    p, K, A, b, free = _system()
    dims = (4, 2, 2)
    Pi = C.prolongation(p.mesh.xyz, dims, free)
    Ac = C.galerkin(A, Pi)
    assert np.all(np.linalg.eigvalsh(Ac) > 0)
    rng = np.random.default_rng(1)
    y = rng.normal(size=Ac.shape[0])
    r = A @ (Pi @ y)                      # a residual whose error lies in the coarse space
    zero = np.zeros(A.shape[0])
    corr = C.apply_two_level(r, zero, Pi, Ac)
    assert np.linalg.norm(corr - Pi @ y) <= 1e-10 * np.linalg.norm(Pi @ y)
    # symmetric preconditioner: w^T M^-1 v = v^T M^-1 w
    dinv = free / A.diagonal()
    v, w = rng.normal(size=A.shape[0]) * free, rng.normal(size=A.shape[0]) * free
    mv, mw = C.apply_two_level(v, dinv, Pi, Ac), C.apply_two_level(w, dinv, Pi, Ac)
    assert abs(w @ mv - v @ mw) <= 1e-10 * abs(w @ mv)


def test_two_level_pcg_reaches_the_direct_solution_faster_than_jacobi():
    p, K, A, b, free = _system((24, 4, 4))
    dims = (7, 2, 2)
    Pi = C.prolongation(p.mesh.xyz, dims, free)
    Ac = C.galerkin(A, Pi)
    dinv = free / A.diagonal()
    x, it2 = C.two_level_pcg(A, b, dinv, Pi, Ac, tol=1e-10)
    x_ref = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    itj = OS.jacobi_pcg(A, b, tol=1e-10).iterations
    assert it2 < itj / 2, (it2, itj)


def test_galerkin_matrix_equals_the_per_tet_gradient_form():
    """A second derivation of A_c = Pi^T P K P Pi, from the definition of K
    rather than from the assembled matrix: K = sum_k V_k Bbar_k^T D Bbar_k with
    V_k Bbar_k = sum over the tets e of face k of (V_e / 4) B_e (Eq. 2-3, Eq. 9),
    hence K = sum_e (V_e / 4) B_e^T D sum_{faces k of e} Bbar_k.  For the coarse
    functions w_I e_a (hat weights w_I masked by the clamp) the tet gradient is
    x_I = sum_nodes w_I grad N and the face-smoothed one of face k is
    (V_e x_I^e + V_n x_I^n) / (V_e + V_n) (x_I^e on the exterior).  With
    isotropic D (Lame lambda, mu) the 3x3 block of centres I, J is then
    sum_e (V_e / 4) [lambda x_I y_J^T + mu y_J x_I^T + mu (x_I . y_J) I]
    with y_J the sum of tet e's four face-smoothed gradients.  A wrong shear
    factor, a transposed block or a dropped face fails this."""
    p, K, A, b, free = _system((10, 3, 3))
    m = p.mesh
    xyz, tets = m.xyz, m.tets.astype(np.int64)
    dims = (4, 2, 2)
    Pi = C.prolongation(xyz, dims, free)
    Ac_ref = C.galerkin(A, Pi)
    P = int(np.prod(dims))
    # hat weights per node and centre; the clamp prescribes whole nodes, so
    # the three components carry the same masked weight
    Pd = Pi.toarray()
    W = Pd[0::3, 0::3]
    assert np.array_equal(W, Pd[1::3, 1::3]) and np.array_equal(W, Pd[2::3, 2::3])
    # tet volumes and shape-function gradients from the vertex coordinates
    X4 = xyz[tets]                                     # (ne, 4, 3)
    J = (X4[:, 1:] - X4[:, :1])                        # rows: edge vectors
    V = np.abs(np.linalg.det(J)) / 6.0
    Ginv = np.linalg.inv(J)                            # columns: grad N_1..3
    grad = np.concatenate([-Ginv.sum(axis=2, keepdims=True), Ginv], axis=2).transpose(0, 2, 1)  # (ne, 4, 3)
    X = np.einsum("eaj,eai->eji", W[tets], grad)       # (ne, P, 3): x_I of every tet
    faces = F.build_faces(m.tets)
    Y = np.zeros_like(X)
    e0, e1 = faces.tet[:, 0], faces.tet[:, 1]
    inner = e1 >= 0
    gbar = X[e0].copy()
    ve, vn = V[e0[inner]], V[e1[inner]]
    gbar[inner] = (ve[:, None, None] * X[e0[inner]] + vn[:, None, None] * X[e1[inner]]) / (ve + vn)[:, None, None]
    np.add.at(Y, e0, gbar)
    np.add.at(Y, e1[inner], gbar[inner])
    E, nu = p.E, p.nu
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    w = V / 4.0
    T1 = np.einsum("e,eia,ejc->iajc", w, X, Y)
    T2 = np.einsum("e,eic,eja->iajc", w, X, Y)
    T3 = np.einsum("e,eib,ejb->ij", w, X, Y)
    Ac = lam * T1 + mu * T2 + mu * np.einsum("ij,ac->iajc", T3, np.eye(3))
    Ac = Ac.reshape(3 * P, 3 * P)
    scale = np.abs(Ac_ref).max()
    assert scale > 0
    assert np.abs(Ac - Ac_ref).max() <= 1e-10 * scale, np.abs(Ac - Ac_ref).max() / scale
