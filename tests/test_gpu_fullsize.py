"""Sampled-bond parity at the benchmark's full size.

The N = 200 Heisenberg chain of the benchmark is grown on the GPU (mixed
form, threshold truncation under chi_max = 1024) until its bulk bonds carry
chi ~ 200-290; the orthogonality centre is then moved to a bulk bond and the
inputs of that bond's local update -- L_k, W_k, W_{k+1}, R_{k+2} and theta --
are read back.  The oracle recomputes each step of the update (Eq. 19 by
Lanczos, Eq. 20 SVD, Eqs. 4-5 entropy and truncation error, the left
environment update) on exactly these inputs, and each GPU building block, in
the FP64 and in the mixed form, is compared with it on the same inputs.

Tolerances:
  * Ritz value: FP64 1e-10 relative; mixed 2e-6 relative (first order in
    the FP32-accumulated contractions), and the FP64 Rayleigh quotient of the
    mixed Ritz vector within 1e-8 per site of the chain (|dE| <= 1e-8 N);
  * Ritz vector: overlap 1 - 1e-10 (FP64), 1 - 1e-7 (mixed);
  * singular values of the oracle's Ritz vector: FP64 |s - s_ref| <= 1e-10 s_ref
    + 8 n eps s_1; mixed 1e-7 s_ref + 8 sqrt(r) 2^-24 |theta|_F (the bounds of
    the isolated-SVD tests); entropy 1e-12 (FP64) / 1e-6 (mixed); the FP64
    retained k equal to the oracle's;
  * environment update: 1e-12 relative to its largest entry (FP64).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


@pytest.fixture(scope="module")
def bulk_bond(G):
    """Inputs of the local update at bond k = 99 of the grown N = 200 chain."""
    N, k = 200, 99
    ctx = G.Context(0)
    p = G.make_params(prec=G.PREC_3XTF32, ctrl=G.CTRL_THRESHOLD, chi_max=1024, chi_init=16, eps_trunc=1e-10)
    W = ctx.build_mpo(G.XXZ, N, 1.0, 1.0)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(2, 0), N, 16)).cuda()
    st = G.State(ctx, W, m0, p, 1.0, 1.0)
    st.sweep(3, visits=False)
    for b in range(k):                      # centre from bond 0 to bond k
        st.bond_update(b, 1)
    chi = st.chi()
    L = st.env(True, k).cpu().numpy()
    R = st.env(False, k + 2).cpu().numpy()
    A1 = st.site(k).cpu().numpy()
    A2 = st.site(k + 1).cpu().numpy()
    th = np.tensordot(A1, A2, axes=([2], [0]))          # chi_k x 2 x 2 x chi_{k+2}
    Wn = W.cpu().numpy()
    st.close()
    ctx.close()
    assert chi[k] >= 150 and chi[k + 2] >= 150, chi[k - 2:k + 4]
    return dict(N=N, k=k, L=L, R=R, th=th, W1=Wn[k], W2=Wn[k + 1])


@pytest.fixture(scope="module")
def oracle_update(bulk_bond):
    b = bulk_bond
    E, th, steps, _, _ = O.lanczos(b["L"], b["W1"], b["W2"], b["R"], b["th"], K=20)
    cl, cr = th.shape[0], th.shape[3]
    U, s, Vt = O.svd(th.reshape(2 * cl, 2 * cr))
    S, eps = O.entropy(s)
    return dict(E=E, th=th, steps=steps, U=U, s=s, Vt=Vt, S=S, eps=eps)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_fullsize_lanczos(G, bulk_bond, oracle_update, form):
    b, ref = bulk_bond, oracle_update
    ctx = G.Context(0)
    prec = G.PREC_FP64 if form == "fp64" else G.PREC_3XTF32
    E, th, steps = ctx.lanczos(dev(b["L"]), dev(b["W1"]), dev(b["W2"]), dev(b["R"]), dev(b["th"]), K=20, prec=prec)
    ctx.close()
    ov = abs(float(np.dot(th.cpu().numpy().ravel(), ref["th"].ravel())))
    if form == "fp64":
        assert steps == ref["steps"]
        assert abs(E - ref["E"]) <= 1e-10 * abs(ref["E"])
        assert ov >= 1.0 - 1e-10
    else:
        # the mixed Ritz value is first order in the contractions' rounding
        # (E = <y|H~|y> with H~ the FP32-accumulated operator): stated bar 2e-6
        # relative; the state's energy, the FP64 Rayleigh quotient of the mixed
        # Ritz vector, is second order and meets the mixed forms' 1e-8 per site
        assert abs(E - ref["E"]) <= 2e-6 * abs(ref["E"])
        y = th.cpu().numpy()
        Hy = O.heff_apply(b["L"], b["W1"], b["W2"], b["R"], y)
        E_rq = float(np.dot(y.ravel(), Hy.ravel()) / np.dot(y.ravel(), y.ravel()))
        assert abs(E_rq - ref["E"]) <= 1e-8 * b["N"]
        assert ov >= 1.0 - 1e-7                     # angle to the FP64 Ritz vector below 4.5e-4


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_fullsize_svd_entropy_truncation(G, bulk_bond, oracle_update, form):
    ref = oracle_update
    th = ref["th"]
    cl, cr = th.shape[0], th.shape[3]
    A = th.reshape(2 * cl, 2 * cr)
    ctx = G.Context(0)
    ctx.set_option("svd_prec", 0 if form == "fp64" else 1)
    U, s, Vt, k, S, err = ctx.svd_truncate(dev(A), 1024, 1e-10)
    s = s.cpu().numpy()
    ctx.close()
    s_ref = ref["s"]
    n = max(A.shape)
    if form == "fp64":
        assert np.all(np.abs(s - s_ref) <= 1e-10 * s_ref + 8 * n * EPS * s_ref[0])
        assert abs(S - ref["S"]) <= 1e-12
        assert k == O.trunc_k(s_ref, 1024, 1e-10, multiplet_guard=0)
        assert abs(err - ref["eps"][k]) <= 1e-12
        Un = U.cpu().numpy()
        assert np.linalg.norm(Un[:, :k] * s[:k] @ Vt.cpu().numpy()[:k] - A) <= ref["eps"][k] * np.linalg.norm(A) \
            + 20 * n * EPS * np.linalg.norm(A)
    else:
        fro = np.sqrt(np.sum(s_ref ** 2))
        kk = min(k, len(s_ref))
        assert np.all(np.abs(s[:kk] - s_ref[:kk]) <= 1e-7 * s_ref[:kk] + 8 * np.sqrt(len(s_ref)) * 2.0 ** -24 * fro)
        assert abs(S - ref["S"]) <= 1e-6
        assert k <= O.trunc_k(s_ref, 1024, 1e-10, multiplet_guard=0)


def test_fullsize_env_update(G, bulk_bond, oracle_update):
    b, ref = bulk_bond, oracle_update
    cl = b["L"].shape[1]
    k = O.trunc_k(ref["s"], 1024, 1e-10, multiplet_guard=0)
    A = np.ascontiguousarray(ref["U"][:, :k]).reshape(cl, 2, k)
    Lref = O.env_left(b["L"], b["W1"], A)
    ctx = G.Context(0)
    Lg = ctx.env_left(dev(b["L"]), dev(b["W1"]), dev(A)).cpu().numpy()
    ctx.close()
    assert np.max(np.abs(Lg - Lref)) <= 1e-12 * np.max(np.abs(Lref))
