"""Independent chains advanced together (batched bond steps): every chain's
results are those of the same chain swept alone -- the same kernels on the
same inputs, so bit-identical energies and bond-dimension schedules -- while
the chains' kernels are interleaved on the device.  One chain is also checked
against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

CHAINS = [(12, 0.5), (16, 1.0), (20, 1.5), (14, 0.0)]


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


def make(G, N, Delta, prec, seed, **kw):
    ctx = G.Context(0, stream=torch.cuda.Stream())
    p = G.make_params(prec=prec, **kw)
    W = ctx.build_mpo(G.XXZ, N, 1.0, Delta)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(4, seed), N, p.chi_init)).cuda()
    torch.cuda.synchronize()
    st = G.State(ctx, W, m0, p, 1.0, Delta)
    return ctx, st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chains_match_single_runs(G, prec):
    pr = G.PREC_FP64 if prec == "fp64" else G.PREC_3XTF32
    kw = dict(ctrl=G.CTRL_PID, chi_max=32, chi_init=4)
    pairs = [make(G, N, D, pr, i, **kw) for i, (N, D) in enumerate(CHAINS)]
    recs, secs = G.sweep_chains([st for _, st in pairs], 3)
    assert secs > 0
    chis = [st.chi() for _, st in pairs]
    for ctx, st in pairs:
        st.close(); ctx.close()
    for i, (N, D) in enumerate(CHAINS):
        ctx, st = make(G, N, D, pr, i, **kw)
        r1, _ = st.sweep(3)
        assert [r.E for r in r1] == [r.E for r in recs[i]], (N, D)
        assert [r.mean_chi for r in r1] == [r.mean_chi for r in recs[i]]
        assert st.chi() == chis[i]
        st.close(); ctx.close()


def test_chain_matches_oracle(G):
    N, Delta = CHAINS[0]
    kw = dict(ctrl=G.CTRL_THRESHOLD, chi_max=32, chi_init=4)
    pairs = [make(G, N, D, G.PREC_FP64, i, **kw) for i, (N, D) in enumerate(CHAINS[:2])]
    recs, _ = G.sweep_chains([st for _, st in pairs], 2)
    for ctx, st in pairs:
        st.close(); ctx.close()
    m0 = synth.initial_mps_entries(synth.workload_seed(4, 0), N, 4)
    ref = O.dmrg_run(O.mpo(O.MODEL_XXZ, N, 1.0, Delta), m0, O.make_params(**kw), 2)
    assert np.all(np.abs(np.array([r.E for r in recs[0]]) - ref["E"]) / N <= 1e-10)


def test_chains_reject_shared_context(G):
    ctx = G.Context(0, stream=torch.cuda.Stream())
    p = G.make_params(chi_max=8)
    W = ctx.build_mpo(G.XXZ, 8, 1.0, 1.0)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(4, 9), 8, p.chi_init)).cuda()
    torch.cuda.synchronize()
    a = G.State(ctx, W, m0, p, 1.0, 1.0)
    b = G.State(ctx, W, m0, p, 1.0, 1.0)
    with pytest.raises(RuntimeError):
        G.sweep_chains([a, b], 1)
    a.close(); b.close(); ctx.close()
