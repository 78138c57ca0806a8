"""Failure detection without a GPU fault: the bounded grid barrier of the
cooperative kernels, run with a block that never arrives, gives up after its
spin limit, records DMRG_ETIMEOUT in the context's status word and returns;
the context stays usable.  With both blocks arriving it passes."""
import pytest
import torch

pytestmark = pytest.mark.gpu

DMRG_OK, DMRG_ETIMEOUT = 0, 5


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


def test_barrier_passes_when_all_arrive(G):
    ctx = G.Context(0)
    assert ctx.wait_selftest(2_000_000, absent=False) == DMRG_OK
    ctx.close()


def test_barrier_times_out_and_context_survives(G):
    ctx = G.Context(0)
    assert ctx.wait_selftest(200_000, absent=True) == DMRG_ETIMEOUT
    # the status word was read and cleared; later work runs normally
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(64, 48, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(48, 32, dtype=torch.float64, device="cuda", generator=g)
    C = ctx.gemm(A, B, prec=G.PREC_FP64)
    assert torch.allclose(C, A @ B, rtol=1e-12, atol=1e-12)
    assert ctx.wait_selftest(2_000_000, absent=False) == DMRG_OK
    ctx.close()
