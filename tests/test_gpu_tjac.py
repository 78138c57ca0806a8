"""The blocked one-sided Jacobi whose Gram blocks and block rotations are
tcgen05 GEMMs (option tjac = 64 or 128 vectors per block pair; Eq. 20's SVD
as block pairs: Gram block G = P P^T, one cyclic Jacobi sweep on G, P <- Q^T P).

It is held to the bars of the other FP32 Jacobi kernels of the mixed form:
  * singular values: |s - s_ref| <= 1e-7 s_ref + 8 sqrt(r) u |A|_F, u = 2^-24
    (FP64 norms of the FP64 projection on the re-orthonormalised isometry);
  * isometry orthonormal within (3/4) k tol^2 after its Newton-Schulz step;
  * truncated reconstruction within the discarded weight plus 1e-6 |A|;
  * entropy within 1e-6;
  * a mixed DMRG sweep with every SVD on this kernel within 1e-8 per site of
    the FP64 form and of exact diagonalisation.
That the tensor-core form ran is checked by its launches: a round is five
launches (split, Gram product, slice sum, in-CTA sweep, rotation product),
nb rounds an outer sweep.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


def mixed_svd(G, A, k_max, opts):
    c = G.Context(0)
    c.set_option("svd_prec", 1)
    for name, val in opts:
        c.set_option(name, val)
    n0 = G.launch_count()
    U, s, Vt, k, S, err = c.svd_truncate(torch.from_numpy(A).cuda(), k_max, 1e-10)
    torch.cuda.synchronize()
    launches = G.launch_count() - n0
    out = tuple(x.cpu().numpy() for x in (U, s, Vt))
    c.status()
    c.close()
    return out + (k, S, launches)


def check(A, s_ref, U, s, Vt, k, S, m, n):
    r = len(s_ref)
    fro = np.sqrt(np.sum(s_ref ** 2))
    assert np.all(np.abs(s[:k] - s_ref[:k]) <= 1e-7 * s_ref[:k] + 8 * np.sqrt(r) * 2.0 ** -24 * fro)
    iso = U[:, :k] if n <= m else Vt[:k].T
    assert np.abs(iso.T @ iso - np.eye(k)).max() <= 0.75 * k * 1e-10
    Ak = (U[:, :k] * s[:k]) @ Vt[:k]
    tail = np.sqrt(np.sum(s_ref[k:] ** 2))
    assert np.linalg.norm(Ak - A) <= tail + 1e-6 * np.linalg.norm(A)
    S_ref, _ = O.entropy(s_ref)
    assert abs(S - S_ref) <= 1e-6


@pytest.mark.parametrize("tb", [64, 128])
@pytest.mark.parametrize("m,n", [(66, 70), (130, 94), (94, 130), (300, 200), (450, 450), (512, 512), (700, 650),
                                 (1024, 1024)])
def test_tjac_exact_spectrum(G, tb, m, n):
    """Ragged and rectangular shapes (a padded last block, an odd block count
    padded to even, lengths not a multiple of 32), exponential spectra: the
    bars above, and the round structure of the tensor-core form in the launch
    count."""
    r = min(m, n)
    s_ref = synth.spectrum("exp", r, max(2, r // 2))
    A = synth.svd_test_matrix(synth.workload_seed(5, m * 1000 + n), m, n, s_ref)
    U, s, Vt, k, S, nl = mixed_svd(G, A, r, [("tjac", tb), ("tjac_min_r", 2)])
    check(A, s_ref, U, s, Vt, k, S, m, n)
    *_, nl0 = mixed_svd(G, A, r, [])
    nb = -(-r // (tb // 2))                  # blocks of the r vectors (length max(m, n))
    nb += nb & 1
    rounds = nb if nb >= 4 else 1            # rounds with at least one block pair
    assert nl >= nl0 + 4 * rounds            # at least one outer sweep of rounds


@pytest.mark.parametrize("tb", [64, 128])
@pytest.mark.parametrize("chi", [256, 1024])
def test_tjac_isolated_svd_workload(G, tb, chi):
    """The isolated-SVD workload (2 chi x 2 chi, Haar factors, s_k =
    exp(-k / (0.1 chi))) at the sizes where the other kernels leave one
    cluster: the same bars."""
    n = 2 * chi
    s_ref = synth.spectrum("exp", n, chi)
    A = synth.svd_test_matrix(synth.workload_seed(1, chi), n, n, s_ref)
    U, s, Vt, k, S, _ = mixed_svd(G, A, n, [("tjac", tb), ("tjac_min_r", 2)])
    check(A, s_ref, U, s, Vt, k, S, n, n)


@pytest.mark.parametrize("tb", [64, 128])
def test_tjac_dmrg_sweep_energy(G, tb):
    """Every SVD of a mixed sweep (16 sites, chi <= 64, tensor cores on every
    contraction) on the tensor-core Jacobi: the energy within 1e-8 per site
    of the FP64 form and of exact diagonalisation, the isometries
    orthonormal."""
    N = 16
    ctx = G.Context(0)
    ctx.set_option("tc_force", 1)
    kw = dict(ctrl=G.CTRL_THRESHOLD, chi_max=64, chi_init=8)
    W = ctx.build_mpo(O.MODEL_XXZ, N, 1.0, 1.0, 0.0)
    out = {}
    for prec in (G.PREC_FP64, G.PREC_3XTF32):
        if prec == G.PREC_3XTF32:
            ctx.set_option("tjac", tb)
            ctx.set_option("tjac_min_r", 2)
        p = G.make_params(prec=prec, **kw)
        m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(0, 0), N, p.chi_init)).cuda()
        st = G.State(ctx, W, m0, p, 1.0, 1.0, 0.0)
        recs, _ = st.sweep(4)
        out[prec] = (st, recs[-1].E)
    E64, Em = out[G.PREC_FP64][1], out[G.PREC_3XTF32][1]
    assert abs(Em - E64) / N <= 1e-8
    assert abs(Em - O.ed_ground(O.MODEL_XXZ, N)) / N <= 1e-8
    stm = out[G.PREC_3XTF32][0]
    chi = stm.chi()
    for i in range(1, N):
        B = stm.site(i).cpu().numpy().reshape(chi[i], 2 * chi[i + 1])
        assert np.abs(B @ B.T - np.eye(chi[i])).max() <= 2 * chi[i] * 1e-10
    ctx.status()
    for st, _ in out.values():
        st.close()
    ctx.close()
