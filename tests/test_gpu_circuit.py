"""Circuit-level bond dimension maps (Section 8) on the GPU against the
oracle: the same layers of two-qubit gates on the same MPS, the same per-bond
controllers; the chi map must be identical, the entropies of the gated bonds
equal to 1e-10 and the final states equal to 1e-10.  Without truncation the
state is the exact statevector; a warm start from a recorded map
reproduces the run."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_2604_03960_gb300 as G
    G.lib()
    return G


def run_gpu(G, N, layers, params, warm=None):
    ctx = G.Context(0)
    c = G.Circuit(ctx, N, params)
    chi, S = [], []
    for l, (pos, gates) in enumerate(layers):
        row, srow = c.apply_layer(pos, gates, None if warm is None else warm[l])
        chi.append(row)
        S.append(srow)
    psi = c.state().cpu().numpy()
    c.close()
    ctx.close()
    return np.array(chi), np.array(S), psi


def test_circuit_untruncated_is_exact(G):
    N, L = 12, 8
    layers = synth.brickwork_circuit(synth.workload_seed(60, 4), N, L)
    kw = dict(chi_max=64, chi_min=64, ctrl=G.CTRL_FIXED, chi_fixed=64)
    chi, S, psi = run_gpu(G, N, layers, G.make_params(**kw))
    exact = O.statevector(N, layers)
    assert np.max(np.abs(psi - exact)) < 1e-12
    chi_ref, S_ref, _ = O.circuit_run(N, layers, O.make_params(**kw))
    assert np.array_equal(chi, chi_ref)
    # the last layer's map is the exact state's Schmidt ranks (values above
    # the eps_trunc = 1e-10 threshold of the normalised spectrum)
    for b in range(N - 1):
        sv = np.linalg.svd(exact.reshape(2 ** (b + 1), -1), compute_uv=False)
        assert chi[-1, b] == int(np.sum(sv / np.linalg.norm(sv) > 1e-10))


@pytest.mark.parametrize("N,L,chi_max", [(12, 10, 16), (16, 12, 24)])
def test_circuit_pid_map_matches_oracle(G, N, L, chi_max):
    layers = synth.brickwork_circuit(synth.workload_seed(60, N), N, L)
    kw = dict(chi_max=chi_max, chi_min=2)
    chi, S, psi = run_gpu(G, N, layers, G.make_params(**kw))
    chi_ref, S_ref, psi_ref = O.circuit_run(N, layers, O.make_params(**kw))
    assert np.array_equal(chi, chi_ref)
    assert np.max(np.abs(S - S_ref)) <= 1e-10
    assert np.max(np.abs(psi - psi_ref)) <= 1e-10
    assert chi.min() >= 1 and chi.max() <= chi_max
    assert len(set(chi[-1].tolist())) > 2                       # the map varies along the chain
    # warm start from the recorded map: same map, same state, no controller transient
    chi2, _, psi2 = run_gpu(G, N, layers, G.make_params(**kw), warm=chi)
    assert np.array_equal(chi2, chi)
    assert np.max(np.abs(psi2 - psi)) <= 1e-12


def test_circuit_rejects_overlapping_pairs(G):
    ctx = G.Context(0)
    c = G.Circuit(ctx, 6, G.make_params(chi_max=8))
    eye = np.eye(4)[None].repeat(2, axis=0)
    with pytest.raises(G.DMRGError):
        c.apply_layer([1, 2], eye)
    c.close()
    ctx.close()
