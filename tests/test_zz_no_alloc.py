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
