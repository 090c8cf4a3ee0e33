"""The allocation-free operator entry point (sfem_apply_noalloc) through the
C ABI: against the oracle's y = A u, against the ordinary entry point
(sfem_apply, FP64 matrix-free), and with no device allocation.

It serves callers that must not allocate device memory per call (a host
application whose pool already owns the GPU memory, or a loop applying the
operator thousands of times where allocations would synchronise the
device).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process, where the first call sets up the scratch address.
"""
import os
import re

import numpy as np
import pytest

from inputs.kuhn_beam import cantilever
from oracle import fsfem as F

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_2001_08849_gb300", "csrc", "noalloc.cu")


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem
    return sfem


def test_noalloc_source_calls_no_allocator():
    """The entry point's source names no allocation routine: no cudaMalloc or
    cudaFree of any kind and none of the context allocator's calls."""
    src = open(SRC).read()
    code = re.sub(r"//[^\n]*", "", src)           # comments may name them
    for pat in (r"cudaMalloc", r"cudaFree", r"\bmem\.get\b", r"\bmem\.drop\b", r"\bscratch_get\b", r"\bnew\b",
                r"\bmalloc\b"):
        assert not re.search(pat, code), pat


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_apply_on_two_calls(S):
    import torch
    p = cantilever(20, 4, 4, seed=1)
    m = p.mesh
    K = F.assemble(m.xyz, m.tets, p.E, p.nu).matrix()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, _, _, _ = F.dirichlet_system(K, f, p.dir_dofs, p.dir_vals)   # A = P K P + (I - P)
    absA = abs(A).tocsr()
    rng = np.random.default_rng(11)
    with S.FsFem(p) as ctx:
        u0 = torch.from_numpy(rng.standard_normal(ctx.ndof)).cuda()
        y0 = torch.empty_like(u0)
        S.sfem_apply_noalloc(ctx.h, u0, y0)          # first call on the device: scratch address set-up
        torch.cuda.synchronize()
        for call in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
            un = rng.standard_normal(ctx.ndof)
            u = torch.from_numpy(un).cuda()
            y_ref = torch.empty_like(u)
            y = torch.full_like(u, np.nan)
            S.sfem_apply(ctx.h, u, y_ref, S.SFEM_OP_MF64, 1)
            torch.cuda.synchronize()
            n_alloc = torch.cuda.memory_stats()["allocation.all.allocated"]
            S.sfem_apply_noalloc(ctx.h, u, y)
            torch.cuda.synchronize()
            # the library's device allocations go through torch's caching
            # allocator (the context's hooks): none happened during the call
            assert torch.cuda.memory_stats()["allocation.all.allocated"] == n_alloc, call
            yn = y.cpu().numpy()
            assert np.isfinite(yn).all()
            maj = absA @ np.abs(un)
            # the FP64 operator tolerance of the parity tests: 1e-12 (|A||u|)_i
            err_oracle = np.abs(yn - A @ un)
            assert (err_oracle <= 1e-12 * maj + 1e-300).all(), (err_oracle / maj).max()
            err_apply = np.abs(yn - y_ref.cpu().numpy())
            assert (err_apply <= 1e-12 * maj + 1e-300).all(), (err_apply / maj).max()


@pytest.mark.gpu
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
