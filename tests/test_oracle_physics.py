"""Pins of the oracle's MPOs, exact diagonalisation and DMRG driver against
values the paper prints, closed forms and independently built Hamiltonians."""
import functools
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

SX = np.array([[0, 0.5], [0.5, 0]]); SZ = np.diag([0.5, -0.5]); SY2 = None
SP = np.array([[0, 1.0], [0, 0]]); SM = SP.T.copy(); I2 = np.eye(2)
PX = 2 * SX; PZ = 2 * SZ


@functools.lru_cache(maxsize=None)
def ed_heisenberg(N):
    """Oracle ED ground energy of the open Heisenberg chain (J = Delta = 1), cached."""
    return O.ed_ground(O.MODEL_XXZ, N, 1.0, 1.0)


def kron_op(ops):
    out = np.ones((1, 1))
    for o in ops:
        out = np.kron(out, o)
    return out


def two_site(N, i, j, a, b):
    ops = [I2] * N
    ops[i], ops[j] = a, b
    return kron_op(ops)


def heis_pair(N, i, j, Delta=1.0):
    return 0.5 * (two_site(N, i, j, SP, SM) + two_site(N, i, j, SM, SP)) + Delta * two_site(N, i, j, SZ, SZ)


def dense_model(model, N, J, Delta, J2):
    H = np.zeros((2 ** N, 2 ** N))
    if model == O.MODEL_TFIM:
        for i in range(N - 1):
            H -= J * two_site(N, i, i + 1, PZ, PZ)
        for i in range(N):
            ops = [I2] * N; ops[i] = PX
            H -= Delta * kron_op(ops)
        return H
    for i in range(N - 1):
        H += J * heis_pair(N, i, i + 1, Delta)
    if model == O.MODEL_J1J2:
        for i in range(N - 2):
            H += J2 * heis_pair(N, i, i + 2, Delta)
    return H


@pytest.mark.parametrize("model,J,Delta,J2", [(O.MODEL_XXZ, 1.3, 0.7, 0.0), (O.MODEL_XXZ, 1.0, 1.0, 0.0),
                                              (O.MODEL_J1J2, 1.0, 1.0, 0.24), (O.MODEL_TFIM, 1.0, 0.6, 0.0)])
def test_mpo_contracts_to_hamiltonian(model, J, Delta, J2):
    N = 6
    W = O.mpo(model, N, J, Delta, J2)
    H = O.mpo_to_dense(W)
    assert np.allclose(H, dense_model(model, N, J, Delta, J2), atol=1e-14)


@pytest.mark.parametrize("model,J,Delta,J2", [(O.MODEL_XXZ, 1.0, 0.5, 0.0), (O.MODEL_J1J2, 1.0, 1.0, 0.4),
                                              (O.MODEL_TFIM, 1.0, 1.0, 0.0)])
def test_ed_matches_library_eigensolver(model, J, Delta, J2):
    N = 8
    ev = np.linalg.eigvalsh(dense_model(model, N, J, Delta, J2))
    n_up = -1 if model == O.MODEL_TFIM else None
    # the ground state of these even-N chains lies in the S^z = 0 sector
    assert abs(O.ed_ground(model, N, J, Delta, J2, n_up=n_up) - ev[0]) < 1e-11
    assert abs(O.ed_dense(model, N, J, Delta, J2)[0] - ev[0]) < 1e-11


def test_xx_chain_free_fermion_closed_form():
    """Delta = 0: Jordan-Wigner gives hopping J/2, single-particle energies J cos(pi k/(N+1))."""
    N, J = 12, 1.0
    eps = J * np.cos(np.pi * np.arange(1, N + 1) / (N + 1))
    assert abs(O.ed_ground(O.MODEL_XXZ, N, J, 0.0, n_up=-1) - eps[eps < 0].sum()) < 1e-11


def test_majumdar_ghosh_dimer_energy():
    """J2/J1 = 1/2, open chain, even N: the dimer product state is exact, E0 = -3 J1 N / 8."""
    for N in (8, 12):
        assert abs(O.ed_ground(O.MODEL_J1J2, N, 1.0, 1.0, 0.5) - (-3 * N / 8)) < 1e-11


def test_paper_table4_heisenberg_N20():
    """Table 4: E/N = -1.73649 for the 20-site Heisenberg chain in the Pauli convention (= 4 E0/N)."""
    g = GOLD["heisenberg_N20_pauli_E_per_site"]
    E0 = ed_heisenberg(20)
    assert round(4 * E0 / 20, g["decimals"]) == g["value"]


def test_paper_table5_critical_ising_N20():
    """Table 5 / Section 13.2: E/N = -1.25539 for the critical Ising chain, N = 20,
    and the open-chain free-fermion closed form E0 = 1 - 1/sin(pi / (2 (2N+1)))."""
    g = GOLD["ising_critical_N20_E_per_site"]
    N = 20
    closed = 1.0 - 1.0 / np.sin(np.pi / (2 * (2 * N + 1)))
    assert round(closed / N, g["decimals"]) == g["value"]
    E0 = O.ed_ground(O.MODEL_TFIM, 16, 1.0, 1.0)   # ED at a size the CPU finishes quickly
    assert abs(E0 - (1.0 - 1.0 / np.sin(np.pi / (2 * (2 * 16 + 1))))) < 1e-10


def _run(N, model=O.MODEL_XXZ, J=1.0, Delta=1.0, J2=0.0, sweeps=4, seed_inst=0, **kw):
    p = O.make_params(**kw)
    W = O.mpo(model, N, J, Delta, J2)
    m0 = synth.initial_mps_entries(synth.workload_seed(0, seed_inst), N, p.chi_init)
    return O.dmrg_run(W, m0, p, sweeps), p


def test_dmrg_reaches_ed_energy_N12():
    r, p = _run(12, chi_max=64, ctrl=O.CTRL_THRESHOLD)
    E0 = O.ed_ground(O.MODEL_XXZ, 12)
    assert abs(r["E"][-1] - E0) / 12 < 1e-10
    assert np.all(np.diff(r["E"]) <= 1e-12)          # variational, monotone at fixed cap
    # after the closing right-to-left half-sweep site 0 is the orthogonality
    # centre, so |A_0| = <psi|psi>^(1/2) = 1 (renormalised retained spectrum)
    assert abs(r["norm"] - 1.0) < 1e-13


def test_dmrg_xxz_and_j1j2_against_ed():
    r, _ = _run(10, Delta=1.5, chi_max=32, ctrl=O.CTRL_THRESHOLD)
    assert abs(r["E"][-1] - O.ed_ground(O.MODEL_XXZ, 10, 1.0, 1.5)) < 1e-9
    r, _ = _run(10, model=O.MODEL_J1J2, J2=0.24, chi_max=32, ctrl=O.CTRL_THRESHOLD)
    assert abs(r["E"][-1] - O.ed_ground(O.MODEL_J1J2, 10, 1.0, 1.0, 0.24)) < 1e-9


def test_dmrg_majumdar_ghosh_entropies():
    """At J2 = J1/2 the exact ground state is a dimer product: bond entropies alternate ln 2 / 0."""
    N = 10
    r, _ = _run(N, model=O.MODEL_J1J2, J2=0.5, chi_max=16, ctrl=O.CTRL_THRESHOLD, sweeps=4)
    assert abs(r["E"][-1] + 3 * N / 8) < 1e-10
    V = r["visits_per_sweep"]
    last = slice((r["sweeps"] - 1) * V, r["sweeps"] * V)
    for b, S in zip(r["bond"][last], r["S"][last]):
        assert abs(S - (np.log(2) if b % 2 == 0 else 0.0)) < 1e-8


def test_dmrg_pid_is_variational_and_records_schedule():
    r, p = _run(12, chi_max=16, ctrl=O.CTRL_PID)
    E0 = O.ed_ground(O.MODEL_XXZ, 12)
    assert np.all(r["E"] >= E0 - 1e-12)
    assert np.all((r["chi"] >= p.chi_min) & (r["chi"] <= p.chi_max))
    assert np.all(r["k"] <= r["chi"])
    # the first visit of every bond starts from chi_min plus the proportional/integral kick
    assert np.all(r["k"] >= 1)


def test_bulk_energy_approaches_bethe_ansatz():
    """Section 10: the spin-1/2 Heisenberg chain's energy per site tends to
    1/4 - ln 2.  Differences of open-chain ground energies cancel the two
    ends, e(N1, N2) = (E0(N2) - E0(N1)) / (N2 - N1); from the oracle's
    exact diagonalisation at N = 12, 16, 20 they approach the Bethe value
    from above, within 1e-3 at (16, 20) and closer than at (12, 16)."""
    e_inf = GOLD["bethe_ansatz_E_per_site"]["value"]
    assert abs(e_inf - (0.25 - np.log(2.0))) < 1e-15
    E = {N: ed_heisenberg(N) for N in (12, 16, 20)}
    e1 = (E[16] - E[12]) / 4.0
    e2 = (E[20] - E[16]) / 4.0
    assert e2 > e_inf and e1 > e_inf
    assert abs(e2 - e_inf) < abs(e1 - e_inf)
    assert abs(e2 - e_inf) < 1e-3


def test_pid_target_reading_reproduces_table4_mean_chi():
    """The paper gives no S_target.  The reading S_target = 0.36 nats (the
    default of make_params) is the value at which Algorithm 2 with the
    paper's gains, run in Table 4's ablation setting (20-site Heisenberg
    chain, chi_max = 64, 5 sweeps, chi = chi_min = 4 at the start), ends with
    the table's mean bond dimension 7.6.  The PID run stays variational and
    below the fixed-chi accuracy: its energy lies between the exact ground
    energy and Table 4's PID value plus 3e-4 (Pauli units per site)."""
    g_chi = GOLD["table4_pid_mean_chi"]["value"]
    g_E = GOLD["table4_pid_E_per_site_pauli"]["value"]
    N = 20
    p = O.make_params(chi_max=64, chi_init=4, max_sweeps=5, ctrl=O.CTRL_PID)
    assert p.S_target == 0.36
    W = O.mpo(O.MODEL_XXZ, N, 1.0, 1.0)
    m0 = synth.initial_mps_entries(synth.workload_seed(1, 20), N, 4)
    r = O.dmrg_run(W, m0, p, 5)
    V = r["visits_per_sweep"]
    mean_chi = float(np.mean(r["k"][-V:]))
    assert abs(mean_chi - g_chi) <= 0.25
    E_pauli = 4 * r["E"][-1] / N
    E0_pauli = GOLD["heisenberg_N20_pauli_E_per_site"]["value"]
    assert E0_pauli - 1e-5 <= E_pauli <= g_E + 3e-4
