"""Autotuner: decisions are timed on the device, kept per context, saved to
and loaded from JSON, and change only the launch configuration -- a tuned
GEMM gives the same bits as a fixed launch of the tile width and split depth
it chose, and a tuned SVD meets the mixed form's accuracy against the oracle."""
import json

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

SHAPES = [(2048, 1024, 512), (640, 4096, 256)]


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


def clog2(v):
    b = 0
    while (1 << b) < v:
        b += 1
    return b


def test_gemm_tuning_roundtrip_and_bits(G, tmp_path):
    ctx = G.Context(0)
    ctx.autotune_gemm(SHAPES, reps=2)
    assert ctx.autotune_entries() == (2, 0)
    path = str(tmp_path / "tune.json")
    ctx.autotune_save(path)
    doc = json.load(open(path))
    assert doc["format"] == "dmrg-autotune-4" and len(doc["gemm"]) == 2
    for e in doc["gemm"]:
        assert e["bn"] in (64, 128, 256) and e["kb"] in (4, 8)
        assert e["ms64"] > 0 and e["ms128"] > 0 and e["ms256"] > 0
    ctx2 = G.Context(0)
    ctx2.autotune_load(path)
    assert ctx2.autotune_entries() == (2, 0)
    g = torch.Generator(device="cuda").manual_seed(3)
    for M, N, K in SHAPES:
        e = next(x for x in doc["gemm"] if (x["lm"], x["ln"], x["lk"]) == (clog2(M), clog2(N), clog2(K)))
        A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g)
        tuned = ctx2.gemm(A, B, prec=G.PREC_3XTF32, force_tc=True)
        # the same launch fixed by options gives the same bits
        ctx.set_option("tc_bn", e["bn"])
        ctx.set_option("tc_split_kb", e["kb"])
        fixed = ctx.gemm(A, B, prec=G.PREC_3XTF32, force_tc=True)
        assert torch.equal(tuned, fixed)
        # any tile width at that depth gives the same bits too
        for bn in (64, 128, 256):
            ctx.set_option("tc_bn", bn)
            assert torch.equal(tuned, ctx.gemm(A, B, prec=G.PREC_3XTF32, force_tc=True))
        ctx.set_option("tc_bn", 0)
        ctx.set_option("tc_split_kb", 8)
        ref = (A @ B).cpu().numpy()
        bound = (A.abs() @ B.abs()).cpu().numpy()
        assert np.all(np.abs(tuned.cpu().numpy() - ref) <= (2.0 ** -20 + 2.0 ** -24 * np.sqrt(3 * K / 8) * 8) * bound)
    ctx.close(); ctx2.close()


def test_svd_tuning_keeps_accuracy(G, tmp_path):
    ctx = G.Context(0)
    ctx.set_option("gjac32", 1)
    n = 600
    # n = 200 takes the grouped Jacobi (one CTA's shared memory), n = 600 the blocked kernel
    ctx.autotune_svd([200, n], reps=1)
    assert ctx.autotune_entries()[1] == 2
    path = str(tmp_path / "tune_svd.json")
    ctx.autotune_save(path)
    small, big = json.load(open(path))["svd"]
    # n = 200: the cluster kernel (8 or 16 CTAs) or the grouped kernel;
    # n = 600: beyond a cluster's length limit, the blocked kernel or the
    # tensor-core block form (pairs of 64 or 128 vectors)
    assert small["cj"] in (0, 8, 16) and small["tj"] == 0
    if small["cj"] == 0:
        assert small["nv"] in (16, 32) and small["groups"] in (1, 2, 4)
    assert big["cj"] == 0 and big["nv"] == 0 and big["pairs"] in (24, 48, 96, 152) and big["inner"] in (1, 2)
    assert big["tj"] in (0, 64, 128)
    ctx.autotune_load(path)
    assert ctx.autotune_entries()[1] == 2
    ctx.set_option("svd_prec", 1)
    chi = n // 2
    A = synth.svd_test_matrix(synth.workload_seed(2, 5), n, n, synth.spectrum("exp", n, chi))
    U, s, Vt, k, S, err = ctx.svd_truncate(torch.from_numpy(A).cuda(), chi, 1e-10)
    s = s.cpu().numpy()
    s_ref = synth.spectrum("exp", n, chi)          # exact by construction
    # values of the retained part: FP64 norms of the FP64 projection on the
    # re-orthonormalised isometry
    fro = np.sqrt(np.sum(s_ref ** 2))
    assert np.all(np.abs(s[:k] - s_ref[:k]) <= 1e-7 * s_ref[:k] + 8 * np.sqrt(len(s_ref)) * 2.0 ** -24 * fro)
    S_ref, _ = O.entropy(s_ref)
    assert abs(S - S_ref) <= 1e-5
    ctx.close()


def test_load_rejects_other_files(G, tmp_path):
    ctx = G.Context(0)
    bad = tmp_path / "bad.json"
    bad.write_text('{"something": 1}\n')
    with pytest.raises(RuntimeError):
        ctx.autotune_load(str(bad))
    with pytest.raises(RuntimeError):
        ctx.autotune_load(str(tmp_path / "missing.json"))
    ctx.close()
