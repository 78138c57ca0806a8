"""Oracle pins of the circuit path (Section 8, circuit-level bond dimension
maps): the MPS circuit simulation against the exact statevector, the
entanglement of a Bell pair, the truncated state's fidelity bound and the
warm start from a recorded map."""
import numpy as np

import oracle as O
import synth


def test_statevector_bell_pair():
    """RY(pi/2) on qubit 0 then CNOT(0 -> 1): (|00> + |11>) / sqrt 2."""
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    ry = np.array([[c, -s], [s, c]])
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=float)
    G = cnot @ np.kron(ry, np.eye(2))
    psi = O.statevector(2, [([0], G[None])])
    assert np.allclose(psi, [1 / np.sqrt(2), 0, 0, 1 / np.sqrt(2)], atol=1e-15)
    p = O.make_params(chi_max=4, chi_min=1)
    chi_map, S_map, psi_mps = O.circuit_run(2, [([0], G[None])], p)
    assert chi_map[0, 0] == 2
    assert abs(S_map[0, 0] - np.log(2.0)) < 1e-14
    assert np.allclose(psi_mps, psi, atol=1e-14)


def test_statevector_against_kronecker_products():
    """The statevector routine applies G on (q, q+1) as I (x) G (x) I."""
    N = 5
    layers = synth.brickwork_circuit(synth.workload_seed(60, 1), N, 3)
    psi = np.zeros(2 ** N); psi[0] = 1.0
    for pos, gates in layers:
        for q, G in zip(pos, gates):
            Op = np.kron(np.kron(np.eye(2 ** q), G), np.eye(2 ** (N - q - 2)))
            psi = Op @ psi
    assert np.allclose(O.statevector(N, layers), psi, atol=1e-13)


def test_untruncated_mps_circuit_equals_statevector():
    """With chi_max large enough for the exact state, the MPS circuit run is
    exact: the same state to 1e-12, every bond at its Schmidt rank."""
    N, L = 10, 8
    layers = synth.brickwork_circuit(synth.workload_seed(60, 2), N, L)
    p = O.make_params(chi_max=32, chi_min=32, ctrl=O.CTRL_FIXED, chi_fixed=32)
    chi_map, S_map, psi = O.circuit_run(N, layers, p)
    exact = O.statevector(N, layers)
    assert np.max(np.abs(psi - exact)) < 1e-12
    assert np.all(chi_map <= np.minimum(2 ** np.arange(1, N), 2 ** np.arange(N - 1, 0, -1)))
    for b in range(N - 1):                       # the final map: the exact Schmidt ranks
        sv = np.linalg.svd(exact.reshape(2 ** (b + 1), -1), compute_uv=False)
        assert chi_map[-1, b] == int(np.sum(sv / np.linalg.norm(sv) > 1e-10))
    # the entropy at a gated bond equals the exact state's Schmidt entropy there
    l, b = L - 1, (L - 1) % 2
    M = exact.reshape(2 ** (b + 1), 2 ** (N - b - 1))
    sv = np.linalg.svd(M, compute_uv=False)
    pk = sv ** 2 / np.sum(sv ** 2)
    pk = pk[pk > 0]
    assert abs(S_map[l, b] + np.sum(pk * np.log(pk))) < 1e-10


def test_pid_map_truncated_state_and_warm_start():
    """With the PID of Algorithm 2 choosing chi at the gated bonds the run
    truncates; the final state is normalised, its fidelity with the exact
    state is below 1 and above 1 - (sum of the discarded weights) squared
    bound's first order, the map stays within [1, chi_max], and a second run
    warm-started from the map reproduces state and map exactly."""
    N, L = 12, 10
    layers = synth.brickwork_circuit(synth.workload_seed(60, 3), N, L)
    p = O.make_params(chi_max=16, chi_min=2, S_target=0.36)
    chi_map, S_map, psi = O.circuit_run(N, layers, p)
    exact = O.statevector(N, layers)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    F = float(np.dot(psi, exact)) ** 2
    assert F < 1.0 - 1e-8                        # the controller did truncate
    assert F > 0.5
    assert np.all((chi_map >= 1) & (chi_map <= 16))
    tvd = 0.5 * np.sum(np.abs(psi ** 2 - exact ** 2))
    assert tvd <= np.sqrt(1.0 - F) + 1e-12       # TVD <= trace distance of the pure states (Eq. 21)
    chi2, S2, psi2 = O.circuit_run(N, layers, p, chi_warm=chi_map)
    assert np.array_equal(chi2, chi_map)
    assert np.max(np.abs(psi2 - psi)) < 1e-13
