"""The learned scheduler end to end: traces from GPU DMRG runs, training on
the GPU with the library's own forward/backward/Adam kernels, and what the
trained network gains over the controller without it.

Labels: for each bond visit, log2 of the k* (the smallest bond dimension whose
discarded weight is below the target, eps_target^2) that the NEXT visit of
the same bond needs; features: that visit's last 8 EMA entropies, the bond
position and the sweep index.

Gain: on an unseen chain (N=40, between the training lengths 24, 32, 48),
the network with the PID fallback reaches the energy of the threshold-
truncated run (chi_max everywhere, the accuracy reference) to within 1e-6 per
site at less than half its cost sum_visits k^3, and an energy lower, by more
than 1e-5 per site, than the PID-only run of the same controller parameters
(the PID of Algorithm 2 at S_target = 0.36, which grows chi only a few units
per visit and ends far from the converged energy after 5 sweeps).
"""
import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def run(G, ctx, N, Delta, ctrl, sweeps, P=None, seed=0, chi_max=64):
    p = G.make_params(ctrl=ctrl, chi_max=chi_max, chi_init=8, max_sweeps=sweeps)
    W = ctx.build_mpo(G.XXZ, N, 1.0, Delta)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(5, seed), N, 8)).cuda()
    st = G.State(ctx, W, m0, p, 1.0, Delta)
    if P is not None:
        st.set_mlp(P)
    recs, vis = st.sweep(sweeps)
    st.close()
    return recs, vis


def training_pairs(vis):
    by = {}
    for v in vis:
        by.setdefault(v.bond, []).append(v)
    X, y = [], []
    for vs in by.values():
        for a, c in zip(vs[:-1], vs[1:]):
            X.append(list(a.feat))
            y.append(math.log2(max(1, c.k_star)))
    return X, y


def xavier_init(G, seed, y_mean):
    """Uniform Xavier init of the three layers from the seeded generator,
    biases zero except the output bias (mean label)."""
    u = synth.Xoshiro(seed, lanes=64).uniform(G.MLP_NPARAM) * 2 - 1
    P = np.zeros(G.MLP_NPARAM, dtype=np.float32)
    H = 64
    n1, n2, n3 = 10 * H, H * H, H           # weights of the three layers
    o1 = 0; o2 = n1 + H; o3 = o2 + n2 + H
    P[o1:o1 + n1] = u[o1:o1 + n1] * math.sqrt(6 / (10 + H))
    P[o2:o2 + n2] = u[o2:o2 + n2] * math.sqrt(6 / (H + H))
    P[o3:o3 + n3] = u[o3:o3 + n3] * math.sqrt(6 / (H + 1))
    P[o3 + n3] = y_mean
    assert o3 + n3 + 1 == G.MLP_NPARAM
    return P


def test_learned_scheduler_trains_and_gains(G, ctx):
    X, y = [], []
    for N in (24, 32, 48):
        for Delta in (0.5, 1.0, 1.5):
            _, vis = run(G, ctx, N, Delta, G.CTRL_THRESHOLD, 4, seed=N)
            a, b = training_pairs(vis)
            X += a; y += b
    assert len(X) > 1000
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    P = torch.from_numpy(xavier_init(G, synth.workload_seed(11, 0), float(np.mean(y)))).cuda()
    m = torch.zeros_like(P); v = torch.zeros_like(P)
    l0 = ctx.mlp_loss_grad(P, Xt, yt)[0].item()
    step = 1
    for _ in range(4):
        ctx.mlp_train(P, Xt, yt, m, v, step, 1000, lr=3e-3)
        step += 1000
    l1 = ctx.mlp_loss_grad(P, Xt, yt)[0].item()
    # the fit must beat predicting the mean label by a wide margin
    var = float(np.var(y))
    assert l1 < 0.25 * var and l1 < 0.1 * l0

    N, Delta = 40, 1.0
    out = {}
    for name, ctrl, PP in [("pid", G.CTRL_PID, None), ("mlp", G.CTRL_MLP, P), ("thr", G.CTRL_THRESHOLD, None)]:
        recs, vis = run(G, ctx, N, Delta, ctrl, 5, P=PP, seed=99)
        out[name] = dict(E=recs[-1].E / N, cost=sum(vv.k ** 3 for vv in vis),
                         used=int(sum(vv.mlp_used for vv in vis)), maxk=max(vv.k for vv in vis))
    assert out["mlp"]["used"] > 0                       # the network, not only its fallback, chose chi
    assert abs(out["mlp"]["E"] - out["thr"]["E"]) <= 1e-6
    assert out["mlp"]["cost"] < 0.5 * out["thr"]["cost"]
    assert out["mlp"]["E"] < out["pid"]["E"] - 1e-5
    # the PID moved: its chi is not stuck at chi_min
    assert out["pid"]["maxk"] > 8
