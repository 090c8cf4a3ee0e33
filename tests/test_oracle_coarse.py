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
