"""Mixed-precision form of the local update (3xTF32 tcgen05 contractions,
FP32 Jacobi + FP64 re-orthonormalised isometry, FP64 Lanczos and entropy)
against the FP64 path, the oracle and exact diagonalisation.

Bar (from the mixed forms' target): |E_mixed - E_ref| / N <= 1e-8 per site.
The isometries must stay orthonormal to FP64 level (<= 1e-10), since a
non-orthonormal basis would bias every later Ritz value.
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


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(0)
    c.set_option("tc_force", 1)       # tensor cores even for these small bonds
    yield c
    c.close()


def run(G, ctx, N, sweeps, prec, model=O.MODEL_XXZ, Delta=1.0, J2=0.0, **kw):
    p = G.make_params(prec=prec, **kw)
    W = ctx.build_mpo(model, N, 1.0, Delta, J2)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(0, 0), N, p.chi_init)).cuda()
    st = G.State(ctx, W, m0, p, 1.0, Delta, J2)
    recs, vis = st.sweep(sweeps)
    return st, recs, vis


# chi_max = 128: theta up to 256 x 256 takes the blocked FP32 Jacobi (block
# width 4, Gram-form inner sweep); smaller bonds take the single-CTA kernel
@pytest.mark.parametrize("N,chi_max,gbj", [(16, 64, 0), (24, 48, 0), (16, 64, 16), (16, 128, 0)])
def test_mixed_energy_matches_fp64_and_ed(G, ctx, N, chi_max, gbj):
    ctx.set_option("gbj_min_r", gbj)
    kw = dict(ctrl=G.CTRL_THRESHOLD, chi_max=chi_max, chi_init=8)
    st64, r64, _ = run(G, ctx, N, 4, G.PREC_FP64, **kw)
    stm, rm, vm = run(G, ctx, N, 4, G.PREC_3XTF32, **kw)
    E64 = r64[-1].E
    Em = rm[-1].E
    assert abs(Em - E64) / N <= 1e-8
    E0 = O.ed_ground(O.MODEL_XXZ, N) if N <= 20 else None
    if E0 is not None:
        assert abs(Em - E0) / N <= 1e-8
    # after the closing right-to-left half-sweep, sites 1..N-1 are right-orthonormal
    # isometries (B B^T = I): the FP32 Jacobi leaves cosines below tol <= 1e-5 and
    # one Newton-Schulz step maps them to about (3/4) chi tol^2
    chi = stm.chi()
    for i in range(1, N):
        B = stm.site(i).cpu().numpy().reshape(chi[i], 2 * chi[i + 1])
        assert np.abs(B @ B.T - np.eye(chi[i])).max() <= 2 * chi[i] * 1e-10
    st64.close(); stm.close()
    ctx.set_option("gbj_min_r", 0)


def test_mixed_pid_schedule_matches_fp64(G, ctx):
    """The paper's controller (Algorithm 2 with Eqs. 8, 16) live on both forms,
    20-site chain, 4 sweeps: the mixed form takes the same integer chi at
    every visit as the FP64 form (its entropies differ by far less than the
    distance of the PID output from a rounding tie) and the same energy to
    the mixed forms' bar of 1e-8 per site."""
    kw = dict(ctrl=G.CTRL_PID, chi_max=32, chi_init=4)
    st64, r64, v64 = run(G, ctx, 20, 4, G.PREC_FP64, **kw)
    stm, rm, vm = run(G, ctx, 20, 4, G.PREC_3XTF32, **kw)
    chi64 = np.array([v.chi_ctrl for v in v64])
    chim = np.array([v.chi_ctrl for v in vm])
    assert len(set(chi64.tolist())) > 2          # the controller moves
    assert np.array_equal(chi64, chim)
    assert np.array_equal(np.array([v.k for v in v64]), np.array([v.k for v in vm]))
    assert np.max(np.abs(np.array([v.S for v in v64]) - np.array([v.S for v in vm]))) <= 1e-5
    for a, b in zip(r64, rm):
        assert abs(a.E - b.E) / 20 <= 1e-8
    st64.close(); stm.close()


def test_checkpoint_roundtrip(G, ctx):
    st, recs, _ = run(G, ctx, 16, 2, G.PREC_FP64, ctrl=G.CTRL_THRESHOLD, chi_max=32, chi_init=8)
    n = st.mps_size()
    host = torch.empty(n, dtype=torch.float64)
    st.get_mps(host)
    st.put_mps(host)
    r2, _ = st.sweep(1)
    assert abs(r2[0].E - recs[-1].E) / 16 <= 1e-10
    st.close()


@pytest.mark.parametrize("chi,opt", [(64, None), (150, None), (256, None), (512, None), (1024, None),
                                     (256, ("gbj_min_r", 32)),
                                     (512, ("gbj_min_r", 32)), (256, ("bjac_gram", 0)), (512, ("bjac_gram", 0))])
def test_mixed_svd_exact_spectrum(G, chi, opt):
    """Standalone mixed SVD (svd_prec = 1) on U diag(s) V^T with s known:
    retained values within 1e-7 relative (FP64 norms of the FP64 projection
    on the re-orthonormalised isometry: second order in its direction errors,
    which the FP32 Jacobi leaves below its cosine tolerance, <= 1e-5) plus
    8 sqrt(r) u |A|_F absolute, u = 2^-24: a vector near the FP32 rank floor
    carries the rounding of its rotations against all r others, each up to
    u times their norm, and its projection picks those components up (the
    values there are overestimated); the isometry orthonormal within
    (3/4) k tol^2 after its Newton-Schulz step, and the truncated
    reconstruction within the discarded weight plus 1e-6 |A|."""
    c = G.Context(0)
    c.set_option("svd_prec", 1)
    if opt:                                 # gbj_min_r: the Gram-block cooperative Jacobi;
        c.set_option(*opt)                  # bjac_gram = 0: blocked Jacobi, inner sweep over vectors
    n = 2 * chi
    s_ref = synth.spectrum("exp", n, chi)
    A = synth.svd_test_matrix(synth.workload_seed(1, chi), n, n, s_ref)
    U, s, Vt, k, S, err = c.svd_truncate(torch.from_numpy(A).cuda(), n, 1e-10)
    U, s, Vt = (x.cpu().numpy() for x in (U, s, Vt))
    fro = np.sqrt(np.sum(s_ref ** 2))
    assert np.all(np.abs(s[:k] - s_ref[:k]) <= 1e-7 * s_ref[:k] + 8 * np.sqrt(len(s_ref)) * 2.0 ** -24 * fro)
    # the Jacobi leaves pairwise cosines up to tol <= 1e-5; one Newton-Schulz
    # step maps the error E of Q Q^T - I to about (3/4) E^2, |(E^2)_ij| <= k tol^2
    assert np.abs(U[:, :k].T @ U[:, :k] - np.eye(k)).max() <= 0.75 * k * 1e-10
    Ak = (U[:, :k] * s[:k]) @ Vt[:k]
    tail = np.sqrt(np.sum(s_ref[k:] ** 2))
    assert np.linalg.norm(Ak - A) <= tail + 1e-6 * np.linalg.norm(A)
    S_ref, _ = O.entropy(s_ref)
    assert abs(S - S_ref) <= 1e-6
    c.close()


@pytest.mark.parametrize("m,n", [(64, 64), (66, 70), (94, 130), (130, 94), (201, 199), (256, 256), (300, 300),
                                 (40, 500), (450, 450), (500, 500), (512, 512)])
@pytest.mark.parametrize("cj", [1, 0])
def test_mixed_svd_cluster_kernel(G, m, n, cj):
    """The FP32 Jacobi on one thread-block cluster (option cjac32 = 1: blocks
    of vectors in the shared memory of 8 CTAs, or 16 for 500 and 512 vectors,
    moved through distributed shared memory) and the single-CTA / grid
    kernels it replaces (cjac32 = 0) on ragged and rectangular shapes (blocks
    of 2..32 vectors, padded blocks, lengths not a multiple of 32): both meet
    the exact-spectrum bar of the mixed SVD, and both converge (status word
    clean)."""
    c = G.Context(0)
    c.set_option("svd_prec", 1)
    c.set_option("cjac32", cj)
    r = min(m, n)
    s_ref = synth.spectrum("exp", r, max(2, r // 2))
    A = synth.svd_test_matrix(synth.workload_seed(4, m * 1000 + n), m, n, s_ref)
    U, s, Vt, k, S, err = c.svd_truncate(torch.from_numpy(A).cuda(), r, 1e-10)
    U, s, Vt = (x.cpu().numpy() for x in (U, s, Vt))
    fro = np.sqrt(np.sum(s_ref ** 2))
    assert np.all(np.abs(s[:k] - s_ref[:k]) <= 1e-7 * s_ref[:k] + 8 * np.sqrt(r) * 2.0 ** -24 * fro)
    # the Jacobi's vectors lie along the longer side and become the isometry
    # (U if n <= m, else V); the other factor is the projection scaled by 1/s
    iso = U[:, :k] if n <= m else Vt[:k].T
    assert np.abs(iso.T @ iso - np.eye(k)).max() <= 0.75 * k * 1e-10
    Ak = (U[:, :k] * s[:k]) @ Vt[:k]
    tail = np.sqrt(np.sum(s_ref[k:] ** 2))
    assert np.linalg.norm(Ak - A) <= tail + 1e-6 * np.linalg.norm(A)
    S_ref, _ = O.entropy(s_ref)
    assert abs(S - S_ref) <= 1e-6
    c.status()
    c.close()


def test_presplit_matvec_is_bit_identical(G):
    """Option tc_presplit: L and R split into TF32 parts once per local
    update, the Lanczos vector and the mix output split by the kernels that
    produce them.  Same parts, same products, same order: the sweep must give
    the same bits as splitting every operand before every product."""
    out = []
    for ps in (1, 0):
        c = G.Context(0)
        c.set_option("tc_force", 1)
        c.set_option("tc_presplit", ps)
        st, recs, vis = run(G, c, 16, 3, G.PREC_3XTF32, ctrl=G.CTRL_THRESHOLD, chi_max=64, chi_init=8)
        n = st.mps_size()
        host = torch.empty(n, dtype=torch.float64)
        st.get_mps(host)
        out.append((np.array([r.E for r in recs]), np.array([v.k for v in vis]), host.numpy().copy()))
        st.close()
        c.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_long_chain_state_stays_finite(G, prec):
    """A random initial MPS on N = 400 sites carries a norm of about 2^N
    through its right-canonicalisation; the state must come out normalised
    and finite, and one sweep must give a Heisenberg energy per site in the
    physical range (bound -ln 2 + 1/4 = -0.4431 below, and well below 0)."""
    c = G.Context(0)
    N = 400
    p = G.make_params(prec=G.PREC_3XTF32 if prec == "mixed" else G.PREC_FP64, ctrl=G.CTRL_PID, chi_max=16,
                      chi_init=4)
    W = c.build_mpo(G.XXZ, N, 1.0, 1.0)
    m0 = torch.from_numpy(synth.initial_mps_entries(synth.workload_seed(52, N), N, 4)).cuda()
    st = G.State(c, W, m0, p, 1.0, 1.0)
    recs, _ = st.sweep(1)
    E = recs[0].E / N
    assert np.isfinite(E) and -0.4432 < E < -0.3
    st.close()
    c.close()


def test_hold_mode_freezes_the_schedule(G, ctx):
    """DMRG_CTRL_HOLD set between sweeps keeps every bond at the chi its PID
    reached: the controller chi of the held sweeps equals the last PID sweep's
    chi at the same visit, and at a fixed schedule the energy does not rise."""
    N = 20
    st, recs, vis = run(G, ctx, N, 3, G.PREC_FP64, ctrl=G.CTRL_PID, chi_max=32, chi_init=4)
    held = {}
    for v in vis:                      # each bond's chi after its last PID step
        held[v.bond] = v.chi_ctrl
    assert len(set(held.values())) > 1
    p = G.make_params(prec=G.PREC_FP64, ctrl=G.CTRL_HOLD, chi_max=32, chi_init=4)
    st.set_params(p)
    r2, v2 = st.sweep(3)
    assert all(v.chi_ctrl == held[v.bond] for v in v2)
    # at a frozen schedule the run settles: the held sweeps' energies agree to
    # well within the truncation's effect (two-site sweep energies are Ritz
    # values before truncation, so they need not fall monotonically)
    E = [r.E for r in r2]
    assert max(E) - min(E) <= 1e-6 * N
    with pytest.raises(G.DMRGError):
        st.set_params(G.make_params(prec=G.PREC_FP64, ctrl=G.CTRL_HOLD, chi_max=64, chi_init=4))
    st.close()


def test_replay_reproduces_a_run_and_compares_precisions(G, ctx):
    """DMRG_CTRL_REPLAY: an FP64 run that replays, sweep by sweep, the retained
    k of an FP64 PID run reproduces it bit for bit (same kernels, same k), and
    the mixed form replaying the same k ends within the mixed forms' 1e-8 per
    site of it."""
    N, sweeps = 20, 4
    kw = dict(ctrl=G.CTRL_PID, chi_max=32, chi_init=4)
    st, recs, vis = run(G, ctx, N, sweeps, G.PREC_FP64, **kw)
    st.close()
    V = 2 * N - 3
    sched = [[v.k for v in vis[i * V:(i + 1) * V]] for i in range(sweeps)]
    for prec in (G.PREC_FP64, G.PREC_3XTF32):
        st2, _, _ = run(G, ctx, N, 0, prec, ctrl=G.CTRL_REPLAY, chi_max=32, chi_init=4)
        E = []
        for t in range(sweeps):
            st2.set_schedule(sched[t])
            r, v = st2.sweep(1)
            assert [x.k for x in v] == sched[t]
            E.append(r[0].E)
        st2.close()
        if prec == G.PREC_FP64:
            assert E == [r.E for r in recs]
        else:
            assert all(abs(a - b.E) / N <= 1e-8 for a, b in zip(E, recs))
