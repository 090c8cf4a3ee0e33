"""The tensor-core FP32 GEMM that trains both learned corrections (tcgen05,
3xTF32 split, FP32 accumulation in tensor memory), called alone through the
C ABI and compared with an FP64 product on the CPU: every transposition,
ragged shapes that leave partial 128 x 128 tiles and partial K chunks, the
split over K, and the training shapes of the coarse network."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem
    torch.cuda.set_device(0)
    return sfem


def _operand(rows, cols, gen):
    return torch.randn(rows, cols, generator=gen, dtype=torch.float32)


SHAPES = [(1, 1, 1), (7, 5, 0), (128, 128, 32), (129, 130, 33), (1000, 77, 64), (300, 200, 5000),
          (256, 128, 3150), (256, 3150, 128), (128, 3150, 256), (3150, 128, 256)]


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
def test_gemm_matches_fp64_product(S, ta, tb):
    gen = torch.Generator().manual_seed(11 + 2 * ta + tb)
    for M, N, K in SHAPES:
        A = _operand(K, M, gen) if ta else _operand(M, K, gen)
        B = _operand(N, K, gen) if tb else _operand(K, N, gen)
        C, _ = S.sfem_gemm_f32(A.cuda(), B.cuda(), ta=ta, tb=tb)
        opA = (A.T if ta else A).double().numpy()
        opB = (B.T if tb else B).double().numpy()
        ref = opA @ opB
        bound = np.abs(opA) @ np.abs(opB)
        got = C.cpu().double().numpy()
        assert got.shape == (M, N)
        err = np.abs(got - ref)
        # 3xTF32 with FP32 accumulation: FP32-level error.  Plain TF32 (one
        # product of the truncated operands) is ~1e-4 relative and fails.
        assert (err <= 2e-5 * bound + 1e-30).all(), (M, N, K, ta, tb, float((err / (bound + 1e-30)).max()))
        if K > 0:
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= 1e-5, (M, N, K, ta, tb, rel)
        else:
            assert not got.any()


def test_gemm_writes_only_m_by_n_of_a_wider_c(S):
    """C with a leading dimension wider than N: columns beyond N keep their values."""
    gen = torch.Generator().manual_seed(5)
    A, B = _operand(130, 40, gen).cuda(), _operand(40, 70, gen).cuda()
    wide = torch.full((130, 96), 7.0, device="cuda")
    st = S.lib.sfem_gemm_f32(130, 70, 40, A.data_ptr(), 40, 0, B.data_ptr(), 70, 0, wide.data_ptr(), 96, None)
    assert st == 0
    torch.cuda.synchronize()
    ref = (A.double() @ B.double()).cpu()
    assert torch.allclose(wide[:, :70].cpu().double(), ref, rtol=0, atol=1e-4)
    assert (wide[:, 70:] == 7.0).all()


def test_gemm_throughput_report(S):
    """Device time of a large square product (reported, not asserted)."""
    gen = torch.Generator().manual_seed(3)
    n = 4096
    A, B = _operand(n, n, gen).cuda(), _operand(n, n, gen).cuda()
    S.sfem_gemm_f32(A, B)
    ms = min(S.sfem_gemm_f32(A, B)[1] for _ in range(5))
    print(f"tensor-core 3xTF32 GEMM {n}^3: {ms:.3f} ms, {2 * n ** 3 / ms / 1e9:.1f} TFLOP/s")
    for M, N, K in ((256, 128, 3150), (128, 3150, 256), (3150, 128, 256)):
        A, B = _operand(M, K, gen).cuda(), _operand(K, N, gen).cuda()
        S.sfem_gemm_f32(A, B)
        ms = min(S.sfem_gemm_f32(A, B)[1] for _ in range(5))
        print(f"  {M}x{N}x{K}: {ms * 1e3:.1f} us, {2 * M * N * K / ms / 1e9:.2f} TFLOP/s")
