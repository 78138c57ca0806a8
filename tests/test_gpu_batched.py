"""Batched SVD + entropy + truncation of many independent, unevenly sized
matrices in one launch (the uneven isolated-SVD batch), checked matrix by
matrix against the oracle's two-sided Jacobi SVD, entropy and truncation rule,
and replayed through a captured CUDA graph.

Bars.  FP64: singular values within 1e-10 relative + 8 l eps s_0, factors
orthogonal and reconstructing to 20 l eps (one-sided Jacobi stops when every
pair's cosine is below l eps), k exact, entropy and truncation error to 1e-12.
FP32 form: the Jacobi runs in FP32 to cosines below 1e-5; the factor built
from the accumulated rotations takes up to about 2 u per rotation applied to
each vector (u = 2^-24), i.e. 2 u r per sweep, so its orthogonality bar is
20 r u (10 sweeps, worst-case linear growth) and at least 1e-4; the values
carry the FP32 rounding of the rotations (bar 1e-5 s_0 + 1e-4 relative).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

EPS = 2.220446049250313e-16


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


def make_batch(seed, shapes, kind="exp"):
    mats = []
    for b, (m, n) in enumerate(shapes):
        r = min(m, n)
        chi = max(1, max(m, n) // 2)
        s = synth.spectrum(kind, r, chi)
        mats.append(synth.svd_test_matrix(synth.workload_seed(seed, b), m, n, s))
    return mats


def check_fp64(packed, mats, chi_max, eps):
    U = packed["U"].cpu().numpy(); s = packed["s"].cpu().numpy(); Vt = packed["Vt"].cpu().numpy()
    k = packed["k"].cpu().numpy(); S = packed["S"].cpu().numpy(); err = packed["err"].cpu().numpy()
    for b, A in enumerate(mats):
        m, n = A.shape
        r = min(m, n); l = max(m, n)
        Ub = U[packed["oU"][b]: packed["oU"][b] + m * r].reshape(m, r)
        sb = s[packed["os"][b]: packed["os"][b] + r]
        Vb = Vt[packed["oV"][b]: packed["oV"][b] + r * n].reshape(r, n)
        _, s_ref, _ = O.svd(A)
        assert np.all(np.abs(sb - s_ref) <= 1e-10 * s_ref + 8 * l * EPS * s_ref[0]), (b, m, n)
        tol = 20 * l * EPS
        assert np.linalg.norm(Ub * sb @ Vb - A) <= tol * np.linalg.norm(A), (b, m, n)
        assert np.abs(Ub.T @ Ub - np.eye(r)).max() <= tol, (b, m, n)
        assert np.abs(Vb @ Vb.T - np.eye(r)).max() <= tol, (b, m, n)
        S_ref, eps_ref = O.entropy(s_ref)
        k_ref = O.trunc_k(s_ref, chi_max, eps, multiplet_guard=0)
        assert k[b] == k_ref, (b, m, n, k[b], k_ref)
        assert abs(S[b] - S_ref) <= 1e-12
        assert abs(err[b] - eps_ref[k_ref]) <= 1e-12


def test_batched_fp64_uneven(G, ctx):
    # ragged shapes: 1x1, a row, a column, tall, wide, square, odd sizes
    sizes = synth.uneven_sizes(synth.workload_seed(40, 0), 24, 2, 120)
    shapes = [(1, 1), (1, 7), (9, 1), (3, 70), (70, 3), (33, 33)]
    shapes += [(int(a), int(b)) for a, b in zip(sizes[:12], sizes[12:])]
    mats = make_batch(41, shapes)
    dev = [torch.from_numpy(A).cuda() for A in mats]
    p = ctx.svd_batched(dev, chi_max=40, eps=1e-8, prec=G.PREC_FP64)
    torch.cuda.synchronize()
    assert (p["sweeps"].cpu().numpy() > 0).all()
    check_fp64(p, mats, 40, 1e-8)


def test_batched_matches_single_call(G, ctx):
    """Same matrices through svd_truncate one by one: same values, k, S."""
    shapes = [(64, 64), (48, 96), (96, 48), (130, 130)]
    mats = make_batch(42, shapes, kind="pow")
    dev = [torch.from_numpy(A).cuda() for A in mats]
    p = ctx.svd_batched(dev, chi_max=50, eps=1e-6, prec=G.PREC_FP64)
    s = p["s"].cpu().numpy(); kk = p["k"].cpu().numpy(); SS = p["S"].cpu().numpy()
    for b, A in enumerate(dev):
        U1, s1, Vt1, k1, S1, e1 = ctx.svd_truncate(A, 50, 1e-6)
        r = min(A.shape)
        sb = s[p["os"][b]: p["os"][b] + r]
        assert np.allclose(sb, s1.cpu().numpy(), rtol=1e-12, atol=1e-13 * sb[0])
        assert kk[b] == k1
        assert abs(SS[b] - S1) <= 1e-12


def test_batched_fp32_form(G, ctx):
    sizes = synth.uneven_sizes(synth.workload_seed(43, 0), 16, 32, 200)
    shapes = [(int(2 * c), int(2 * c)) for c in sizes[:8]] + [(5, 300), (300, 5)]
    mats = make_batch(44, shapes)
    dev = [torch.from_numpy(A).cuda() for A in mats]
    p = ctx.svd_batched(dev, chi_max=512, eps=1e-6, prec=G.PREC_3XTF32)
    assert (p["sweeps"].cpu().numpy() > 0).all()
    U = p["U"].cpu().numpy(); s = p["s"].cpu().numpy(); Vt = p["Vt"].cpu().numpy()
    S = p["S"].cpu().numpy(); k = p["k"].cpu().numpy()
    for b, A in enumerate(mats):
        m, n = A.shape
        r = min(m, n)
        Ub = U[p["oU"][b]: p["oU"][b] + m * r].reshape(m, r)
        sb = s[p["os"][b]: p["os"][b] + r]
        Vb = Vt[p["oV"][b]: p["oV"][b] + r * n].reshape(r, n)
        _, s_ref, _ = O.svd(A)
        assert np.all(np.abs(sb - s_ref) <= 1e-4 * s_ref + 1e-5 * s_ref[0]), b
        # orthogonality on the resolved part (values above the 2^-22 floor)
        kk = int(np.sum(s_ref > 2.0 ** -20 * s_ref[0]))
        bar = max(1e-4, 20 * r * 2.0 ** -24)
        assert np.abs(Ub[:, :kk].T @ Ub[:, :kk] - np.eye(kk)).max() <= bar, b
        assert np.abs(Vb[:kk] @ Vb[:kk].T - np.eye(kk)).max() <= bar, b
        assert np.linalg.norm(Ub * sb @ Vb - A) <= bar * np.linalg.norm(A), b
        S_ref, _ = O.entropy(s_ref)
        assert abs(S[b] - S_ref) <= 1e-5
        k_ref = O.trunc_k(s_ref, 512, 1e-6, multiplet_guard=0)
        assert abs(int(k[b]) - k_ref) <= 1


def test_batched_graph_replay(G):
    """A captured launch sequence replayed on new inputs gives the results of
    a direct call on those inputs."""
    stream = torch.cuda.Stream()
    ctx = G.Context(0, stream=stream)      # capture needs a stream other than the legacy default
    shapes = [(40, 40), (17, 90), (128, 64), (2, 2)]
    mats1 = make_batch(45, shapes)
    mats2 = make_batch(46, shapes)
    dev1 = [torch.from_numpy(A).cuda() for A in mats1]
    dev2 = [torch.from_numpy(A).cuda() for A in mats2]
    torch.cuda.synchronize()
    p = ctx.svd_batched(dev1, chi_max=30, eps=1e-9, prec=G.PREC_FP64)   # sizes the workspace
    stream.synchronize()
    ctx.graph_begin()
    ctx.svd_batched(None, chi_max=30, eps=1e-9, prec=G.PREC_FP64, packed=p)
    g = ctx.graph_end()
    try:
        with torch.cuda.stream(stream):
            for A, o in zip(dev2, p["oin"]):
                p["theta"][int(o): int(o) + A.numel()].copy_(A.reshape(-1))
        ctx.graph_launch(g)
        stream.synchronize()
        check_fp64(p, mats2, 30, 1e-9)
        # and a second replay on the first inputs
        with torch.cuda.stream(stream):
            for A, o in zip(dev1, p["oin"]):
                p["theta"][int(o): int(o) + A.numel()].copy_(A.reshape(-1))
        ctx.graph_launch(g)
        stream.synchronize()
        check_fp64(p, mats1, 30, 1e-9)
    finally:
        G.lib().dmrg_graph_destroy(g)
        ctx.close()


def test_batched_rejects_bad_input(G, ctx):
    import ctypes as C
    m = (C.c_int * 1)(0); n = (C.c_int * 1)(4); off = (C.c_longlong * 1)(0)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    ki = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = G.lib().svd_truncate_batched(ctx.h, G.PREC_FP64, 1, m, n, buf.data_ptr(), off, buf.data_ptr(), off,
                                      buf.data_ptr(), off, buf.data_ptr(), off, 4, 0.0, ki.data_ptr(),
                                      buf.data_ptr(), buf.data_ptr(), None)
    assert st != 0
