"""GPU parity of the tcgen05 3xTF32 contraction path against FP64 references.

3xTF32 represents each operand to 2^-22 relative and accumulates in FP32, so
each output element is compared with the bound
  |C - C_ref| <= tol * (|A| |B|)_ij,  tol = 2^-20 + 2^-24 * sqrt(3K/8) * 8
(split error plus a random-walk bound on K'/8 FP32 accumulations of
magnitude |A||B|), i.e. about 1e-6 to 1e-5 of the sum of absolute products.
"""
import numpy as np
import pytest
import torch

import oracle as O

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0", torch.float64)


def tol_for(K):
    return 2.0 ** -20 + 2.0 ** -24 * np.sqrt(3 * K / 8) * 8


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (5, 7, 3), (128, 256, 32), (129, 257, 33), (300, 100, 1000),
                                   (640, 96, 77), (257, 513, 515), (1024, 1024, 1024), (70, 50, 2000),
                                   (300, 64, 500), (129, 33, 257)])
def test_tc_gemm_vs_fp64(G, ctx, M, N, K):
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = ctx.gemm(dev(A), dev(B), prec=G.PREC_3XTF32, force_tc=True).cpu().numpy()
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= tol_for(K) * bound + 1e-300)
    # FP64 kernel on the same inputs is exact to FP64 rounding
    C64 = ctx.gemm(dev(A), dev(B), prec=G.PREC_FP64).cpu().numpy()
    assert np.all(np.abs(C64 - ref) <= 1e-13 * bound + 1e-300)


def test_tc_gemm_wide_dynamic_range(G, ctx):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((200, 300)) * np.exp(rng.uniform(-20, 20, (200, 300)))
    B = rng.standard_normal((300, 150))
    C = ctx.gemm(dev(A), dev(B), prec=G.PREC_3XTF32, force_tc=True).cpu().numpy()
    assert np.all(np.abs(C - A @ B) <= tol_for(300) * (np.abs(A) @ np.abs(B)))


@pytest.mark.parametrize("cl,cr", [(64, 64), (100, 130), (256, 200)])
def test_heff_apply_3xtf32(G, ctx, cl, cr):
    rng = np.random.default_rng(cl + cr)
    D = 5
    W = O.mpo(O.MODEL_XXZ, 4, 1.0, 1.0)
    L = rng.standard_normal((D, cl, cl)); R = rng.standard_normal((D, cr, cr))
    th = rng.standard_normal((cl, 2, 2, cr))
    ref = O.heff_apply(L, W[1], W[2], R, th)
    # scale of the absolute contraction, for the relative bound
    absref = O.heff_apply(np.abs(L), np.abs(W[1]), np.abs(W[2]), np.abs(R), np.abs(th))
    ctx_tc_force(ctx, True)
    try:
        y = ctx.heff_apply(dev(L), dev(W[1]), dev(W[2]), dev(R), dev(th), prec=G.PREC_3XTF32).cpu().numpy()
    finally:
        ctx_tc_force(ctx, False)
    K = D * max(cl, cr)
    assert np.all(np.abs(y - ref) <= 3 * tol_for(K) * absref + 1e-300)


@pytest.mark.parametrize("cl,ck", [(64, 100), (200, 130)])
def test_env_updates_3xtf32(G, ctx, cl, ck):
    rng = np.random.default_rng(cl * 3 + ck)
    D = 5
    W = O.mpo(O.MODEL_XXZ, 3, 1.0, 1.0)
    L = rng.standard_normal((D, cl, cl)); A = rng.standard_normal((cl, 2, ck))
    ref = O.env_left(L, W[1], A)
    absref = O.env_left(np.abs(L), np.abs(W[1]), np.abs(A))
    ctx_tc_force(ctx, True)
    try:
        got = ctx.env_left(dev(L), dev(W[1]), dev(A), prec=G.PREC_3XTF32).cpu().numpy()
        R = rng.standard_normal((D, cl, cl)); B = rng.standard_normal((ck, 2, cl))
        refR = O.env_right(R, W[1], B)
        absR = O.env_right(np.abs(R), np.abs(W[1]), np.abs(B))
        gotR = ctx.env_right(dev(R), dev(W[1]), dev(B), prec=G.PREC_3XTF32).cpu().numpy()
    finally:
        ctx_tc_force(ctx, False)
    K = 2 * D * max(cl, ck)
    assert np.all(np.abs(got - ref) <= 3 * tol_for(K) * absref + 1e-300)
    assert np.all(np.abs(gotR - refR) <= 3 * tol_for(K) * absR + 1e-300)


def ctx_tc_force(ctx, on):
    import paper_2604_03960_gb300 as G
    G.lib().dmrg_set_option(ctx.h, b"tc_force", 1.0 if on else 0.0)
