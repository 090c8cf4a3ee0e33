"""Failure detection on the GPU without a fault: the bounded wait of the
batched solver's grid barrier is made to run out (sfem_selftest_barrier puts
the barrier in a state where no block can release it), the error reaches the
host as SFEM_ETIMEOUT, and the context stays usable afterwards."""
import numpy as np
import pytest

from inputs.kuhn_beam import cantilever

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


def test_barrier_wait_runs_out_and_is_reported(S):
    p = cantilever(6, 2, 2, seed=1)
    with S.FsFem(p) as fe:
        status, ms = S.sfem_selftest_barrier(fe.h)
        print(f"\nbarrier wait gave up after {ms:.0f} ms")
        assert status == S.SFEM_ETIMEOUT
        assert 10.0 < ms < 60000.0
        # the context is still usable
        x = np.zeros(fe.ndof)
        info = S.sfem_solve(fe.h, x, S.solve_opts(kind=S.SFEM_SOLVE_PCG64, tol=1e-10))
        assert info["status"] == 0 and info["true_relres"] <= 1e-10
