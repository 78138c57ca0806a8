"""svd_truncate_noalloc: the allocation-free variant of svd_truncate, for
callers that cannot call cudaMalloc (device memory owned by another
component's pool or budget, or loops where an allocation, which can
synchronise the device, is not allowed).  It must give the same factors,
entropy and truncation as svd_truncate, on consecutive calls that share its
fixed device scratch.  This file is named to be collected last."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


def _outs(m, n):
    r = min(m, n)
    return (torch.empty((m, r), dtype=torch.float64, device="cuda:0"),
            torch.empty(r, dtype=torch.float64, device="cuda:0"),
            torch.empty((r, n), dtype=torch.float64, device="cuda:0"))


def test_noalloc_matches_svd_truncate_on_consecutive_calls():
    import paper_2604_03960_gb300 as G
    ctx = G.Context(0)
    cases = [(256, 200, 150, "exp"), (96, 128, 40, "pow")]   # the second call sees the first call's scratch
    for i, (m, n, chi, kind) in enumerate(cases):
        r = min(m, n)
        s_ref = synth.spectrum(kind, r, max(chi, 8))
        A = torch.from_numpy(synth.svd_test_matrix(synth.workload_seed(7, i), m, n, s_ref)).cuda()
        U0, s0, V0, k0, S0, e0 = ctx.svd_truncate(A, chi, 1e-10, out=_outs(m, n))
        U1, s1, V1, k1, S1, e1 = ctx.svd_truncate_noalloc(A, chi, 1e-10, _outs(m, n))
        torch.cuda.synchronize()
        tol = 20 * max(m, n) * EPS
        assert k1 == k0
        assert abs(S1 - S0) <= 1e-12 and abs(e1 - e0) <= 1e-12
        s0h, s1h = s0.cpu().numpy(), s1.cpu().numpy()
        assert np.all(np.abs(s1h - s0h) <= 1e-12 * s0h[0])
        # the matrix was built with a known spectrum: the values must be it
        # (FP64 bound of the other SVD tests: 1e-10 relative + 8 n eps s_1)
        assert np.all(np.abs(s1h - s_ref) <= 1e-10 * s_ref + 8 * max(m, n) * EPS * s_ref[0])
        An = A.cpu().numpy()
        rec = U1.cpu().numpy() * s1h @ V1.cpu().numpy()
        assert np.linalg.norm(rec - An) <= tol * np.linalg.norm(An)
        # same retained factors as the existing entry point (up to the shared sign convention)
        assert np.allclose(U1.cpu().numpy()[:, :k1], U0.cpu().numpy()[:, :k0], atol=1e-10)
        assert np.allclose(V1.cpu().numpy()[:k1], V0.cpu().numpy()[:k0], atol=1e-10)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_limit():
    import paper_2604_03960_gb300 as G
    ctx = G.Context(0)
    A = torch.zeros((300, 16), dtype=torch.float64, device="cuda:0")
    with pytest.raises(G.DMRGError):
        ctx.svd_truncate_noalloc(A, 8, 1e-10, _outs(300, 16))
    ctx.close()


def test_noalloc_grows_no_device_memory_after_first_call():
    """After one call (which may load the library's device code and with it
    the scratch array), further calls leave the device's free memory and
    PyTorch's allocator untouched."""
    import paper_2604_03960_gb300 as G
    ctx = G.Context(0)
    m, n, chi = 200, 180, 64
    s_ref = synth.spectrum("exp", min(m, n), chi)
    A = torch.from_numpy(synth.svd_test_matrix(synth.workload_seed(7, 5), m, n, s_ref)).cuda()
    outs = _outs(m, n)
    ctx.svd_truncate_noalloc(A, chi, 1e-10, outs)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    resv0 = torch.cuda.memory_reserved()
    for _ in range(2):
        ctx.svd_truncate_noalloc(A, chi, 1e-10, outs)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == resv0
    ctx.close()


def test_noalloc_is_fp64_whatever_svd_prec():
    """The entry point always runs the FP64 Jacobi: with the context set to the
    mixed SVD it still returns the FP64 factors of svd_truncate's default form."""
    import paper_2604_03960_gb300 as G
    ctx = G.Context(0)
    m, n, chi = 128, 160, 48
    s_ref = synth.spectrum("exp", min(m, n), chi)
    A = torch.from_numpy(synth.svd_test_matrix(synth.workload_seed(7, 6), m, n, s_ref)).cuda()
    U0, s0, V0, k0, S0, e0 = ctx.svd_truncate(A, chi, 1e-10, out=_outs(m, n))
    ctx.set_option("svd_prec", 1)
    U1, s1, V1, k1, S1, e1 = ctx.svd_truncate_noalloc(A, chi, 1e-10, _outs(m, n))
    torch.cuda.synchronize()
    assert k1 == k0 and abs(S1 - S0) <= 1e-12
    s1h = s1.cpu().numpy()
    assert np.all(np.abs(s1h - s0.cpu().numpy()) <= 1e-12 * s1h[0])
    # FP64 accuracy far below the mixed form's 2^-22 s_0 floor
    assert np.all(np.abs(s1h - s_ref) <= 1e-10 * s_ref + 8 * max(m, n) * EPS * s_ref[0])
    ctx.close()
