"""The allocation-free operator entry point (sfem_apply_noalloc) against the
ordinary one (sfem_apply, FP64 matrix-free) through the C ABI.

It serves callers that must not allocate device memory per call (a host
application whose pool already owns the GPU memory, or a loop applying the
operator thousands of times where allocations would synchronise the
device).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process, where the first call sets up the scratch address.
"""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever
from oracle import fsfem as F

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


def test_noalloc_matches_apply_on_two_calls(S):
    import torch
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    absK = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    absK.data = np.abs(absK.data)
    rng = np.random.default_rng(11)
    with S.FsFem(p) as ctx:
        for _ in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
            u = torch.from_numpy(rng.standard_normal(ctx.ndof)).cuda()
            y_ref = torch.empty_like(u)
            y = torch.full_like(u, np.nan)
            S.sfem_apply(ctx.h, u, y_ref, S.SFEM_OP_MF64, 1)
            S.sfem_apply_noalloc(ctx.h, u, y)
            torch.cuda.synchronize()
            maj = absK @ np.abs(u.cpu().numpy())
            err = np.abs(y.cpu().numpy() - y_ref.cpu().numpy())
            # the FP64 operator tolerance of the parity tests: 1e-12 (|K||u|)_i
            assert np.isfinite(y.cpu().numpy()).all()
            assert (err <= 1e-12 * maj + 1e-300).all(), (err / maj).max()


def test_noalloc_rejects_meshes_above_the_limit(S):
    import torch
    p = cantilever(60, 20, 20, seed=3)          # 144000 tets > 131072
    with S.FsFem(p) as ctx:
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(u)
        with pytest.raises(S.SfemError) as ei:
            S.sfem_apply_noalloc(ctx.h, u, y)
        assert ei.value.status == S.SFEM_EINVAL
        assert "131072" in str(ei.value)
