"""Strain and stress recovery on the GPU (sfem_recover, through the C ABI)
against the oracle (oracle/recover.py), and the VTU output of a solution.

The library forms each face's smoothed gradients from the adjacent tets'
gradients (the volume-average identity); the oracle uses the Gauss-point
route of Eq. 7.  Both are FP64: faces and nodes agree to rounding."""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever
from oracle import fsfem as F
from oracle import recover as R

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


def _face_index(S, h, n_faces, faces):
    """library face f -> oracle face index (by the sorted node triple)"""
    nodes, _, _ = S.sfem_get_faces(h, n_faces)
    where = {tuple(t): i for i, t in enumerate(faces.tri.tolist())}
    return np.array([where[tuple(sorted(r[:3]))] for r in nodes.tolist()])


def _close(got, want, rtol):
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= rtol * scale, (np.abs(got - want).max(), scale)


def test_recover_matches_oracle(S):
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    u = np.random.default_rng(7).standard_normal(3 * m.n_nodes) * 1e-3
    ref = R.recover(m.xyz, m.tets, p.E, p.nu, u)
    with S.FsFem(p) as fe:
        ud = torch.from_numpy(u).cuda()
        out = S.sfem_recover(fe.h, ud)
        idx = _face_index(S, fe.h, fe.info["n_faces"], ref.faces)
        _close(out["face_strain"].cpu().numpy(), ref.face_strain[idx], 1e-12)
        _close(out["face_stress"].cpu().numpy(), ref.face_stress[idx], 1e-12)
        _close(out["node_strain"].cpu().numpy(), ref.node_strain, 1e-12)
        _close(out["node_stress"].cpu().numpy(), ref.node_stress, 1e-12)
        _close(out["node_vm"].cpu().numpy(), ref.node_vm, 1e-12)
        # outputs may be requested separately
        only = S.sfem_recover(fe.h, ud, faces=False, nodes=True)
        _close(only["node_vm"].cpu().numpy(), ref.node_vm, 1e-12)
        # a NULL displacement is an argument error, not a fault
        assert S.lib.sfem_recover(fe.h, None, None, None, None, None, None) == S.SFEM_EINVAL


def test_recover_linear_field_on_gpu(S):
    prob = cantilever(3, 3, 3, dims=(1.0, 2.0, 1.5), seed=11)
    m = prob.mesh
    H = np.random.default_rng(3).standard_normal((3, 3)) * 1e-3
    u = (np.array([0.1, -0.2, 0.3])[None, :] + m.xyz @ H.T).ravel()
    with S.FsFem(prob) as fe:
        out = S.sfem_recover(fe.h, torch.from_numpy(u).cuda())
    e = 0.5 * (H + H.T)
    want = np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[2, 0], 2 * e[0, 1]])
    tol = 1e-12 * np.abs(u).max()
    assert np.abs(out["face_strain"].cpu().numpy() - want).max() <= tol
    assert np.abs(out["node_strain"].cpu().numpy() - want).max() <= tol


def test_recover_full_size_sampled_faces(S):
    """The 2M-tet beam, solved: sampled faces against the oracle on the
    sub-mesh of the face's adjacent tets (a face's smoothed strain depends
    only on them)."""
    p = cantilever(200, 40, 42, seed=2)
    m = p.mesh
    rng = np.random.default_rng(8)
    with S.FsFem(p, on_device=True) as fe:
        S.sfem_coarse_setup(fe.h)
        u = torch.zeros(fe.ndof, dtype=torch.float64, device="cuda")
        S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=1e-8, u_on_device=True, precond=1,
                                           fp32_vectors=3, inner_tol=0.03))
        out = S.sfem_recover(fe.h, u)
        nf = fe.info["n_faces"]
        nodes, ftets, _ = S.sfem_get_faces(fe.h, nf)
        fs = out["face_strain"].cpu().numpy()
        vm = out["node_vm"].cpu().numpy()
        x = u.cpu().numpy()
    assert np.isfinite(fs).all() and np.isfinite(vm).all()
    for f in rng.integers(0, nf, 24):
        ts = [t for t in ftets[f] if t >= 0]
        sub = m.tets[ts]
        used, inv = np.unique(sub, return_inverse=True)
        xs, ts_loc, us = m.xyz[used], inv.reshape(sub.shape), x.reshape(-1, 3)[used]
        r = R.recover(xs, ts_loc, p.E, p.nu, us.ravel())
        tri = tuple(sorted(np.searchsorted(used, nodes[f, :3]).tolist()))
        k = [tuple(t) for t in r.faces.tri.tolist()].index(tri)
        want = r.face_strain[k]
        # FP64 rounding bound: the strain sums terms b_I u_I far larger than
        # itself (the displacement, not its variation over the face)
        dom = F.smoothing_domains_eq7(xs, ts_loc, r.faces)
        st = dom.nodes[k] >= 0
        scale = (np.abs(dom.Bbar[k][st]).sum(1) * np.abs(us[dom.nodes[k][st]]).max(1)).sum()
        assert np.abs(fs[f] - want).max() <= 1e-13 * scale, (f, fs[f], want, scale)


def test_write_solution_vtu(S, tmp_path):
    from paper_2001_08849_gb300 import vtu
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    with S.FsFem(p) as fe:
        u = torch.zeros(3 * m.n_nodes, dtype=torch.float64, device="cuda")
        S.sfem_solve(fe.h, u, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10, u_on_device=True))
        path = tmp_path / "cantilever.vtu"
        pd = vtu.write_solution(str(path), fe.h, m.xyz, m.tets, u)
    got = vtu.read_vtu_arrays(str(path))
    assert got["NumberOfPoints"] == m.n_nodes and got["NumberOfCells"] == m.n_tets
    for k in ("displacement", "strain", "stress", "von_mises"):
        assert np.array_equal(got[k], pd[k]), k
    # the clamp face carries the largest bending stress; the tip is nearly free
    tip = m.xyz[:, 0] > 9.99
    root = m.xyz[:, 0] < 0.01
    assert pd["von_mises"][root].mean() > 10 * pd["von_mises"][tip].mean()
