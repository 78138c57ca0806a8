"""FP64 CPU oracle for the adaptive two-site DMRG local update (arXiv 2604.03960).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  The product path (``paper_2604_03960_gb300``) never
imports it, and it never imports the product package.

The arithmetic lives in ``dmrg_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmrg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CTRL_PID, CTRL_DIRECT, CTRL_FIXED, CTRL_THRESHOLD, CTRL_MLP, CTRL_GLOBAL = range(6)
MODEL_XXZ, MODEL_J1J2, MODEL_TFIM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Oracle parameter block (same meaning as the library's; declared separately)."""
    _fields_ = [
        ("alpha_ema", C.c_double), ("gamma", C.c_double), ("S_target", C.c_double),
        ("Kp", C.c_double), ("Ki", C.c_double), ("Kd", C.c_double), ("beta", C.c_double),
        ("eps_trunc", C.c_double), ("eps_conv", C.c_double),
        ("chi_min", C.c_int), ("chi_max", C.c_int), ("lanczos_steps", C.c_int),
        ("max_sweeps", C.c_int), ("jacobi_max_sweeps", C.c_int), ("prec", C.c_int),
        ("ctrl", C.c_int), ("ema_init_zero", C.c_int), ("multiplet_guard", C.c_int),
        ("pid_steps_per_sweep", C.c_int), ("chi_init", C.c_int), ("chi_fixed", C.c_int),
        ("second_order", C.c_int),
    ]


class CtrlState(C.Structure):
    _fields_ = [
        ("Sbar", C.c_double), ("Sbar_prev", C.c_double), ("Sbar_prev2", C.c_double),
        ("e_prev", C.c_double), ("I", C.c_double), ("hist", C.c_double * 8),
        ("chi", C.c_int), ("initialized", C.c_int), ("nhist", C.c_int), ("pad", C.c_int),
    ]


def make_params(**kw) -> Params:
    """Defaults: the paper's gains K_p=2, K_i=0.1, K_d=0.5 (Section 13.2),
    beta=0.4 (Section 13.2), eps_trunc=1e-10 (Table 4), eps_conv=1e-8
    (Section 10); alpha, gamma, chi_min and S_target are not given by the
    paper.  S_target = 0.36 nats is the value at which the PID run of Table 4's
    ablation setting (20-site Heisenberg chain, chi_max = 64, 5 sweeps)
    reaches Table 4's mean bond dimension 7.6; the rest are design choices."""
    chi_max = kw.get("chi_max", 32)
    gamma = kw.get("gamma", 1.5)
    d = dict(alpha_ema=0.3, gamma=gamma, S_target=0.36, Kp=2.0, Ki=0.1, Kd=0.5,
             beta=0.4, eps_trunc=1e-10, eps_conv=1e-8, chi_min=4, chi_max=chi_max, lanczos_steps=20,
             max_sweeps=8, jacobi_max_sweeps=60, prec=0, ctrl=CTRL_PID, ema_init_zero=0,
             multiplet_guard=1, pid_steps_per_sweep=2, chi_init=4, chi_fixed=chi_max, second_order=0)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.ref_build_mpo.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
            L.ref_mpo_dim.argtypes = [C.c_int]
            L.ref_mpo_to_dense.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ref_qr.argtypes = [C.c_int, C.c_int] + [C.POINTER(C.c_double)] * 3
            L.ref_sym_eig.argtypes = [C.c_int] + [C.POINTER(C.c_double)] * 3
            L.ref_svd.argtypes = [C.c_int, C.c_int] + [C.POINTER(C.c_double)] * 4 + [C.c_int]
            L.ref_entropy.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ref_entropy.restype = C.c_double
            L.ref_ctrl_step.argtypes = [C.POINTER(CtrlState), C.c_double, C.POINTER(Params), C.POINTER(C.c_int)]
            L.ref_ctrl_replay.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(Params),
                                          C.POINTER(CtrlState), C.POINTER(C.c_int)]
            L.ref_ctrl_step_real.argtypes = [C.POINTER(CtrlState), C.c_double, C.POINTER(Params),
                                             C.POINTER(C.c_double)]
            L.ref_mlp_nparam.restype = C.c_int
            L.ref_mlp_forward.argtypes = [C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ref_mlp_loss_grad.argtypes = [C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ref_adam_step.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            L.ref_statevector_apply.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int),
                                                C.POINTER(C.c_double)]
            L.ref_circuit_run.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_double), C.POINTER(Params), C.POINTER(C.c_int),
                                          C.POINTER(CtrlState), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]
            L.ref_heff_apply.argtypes = [C.c_int] * 4 + [C.POINTER(C.c_double)] * 6
            L.ref_env_left.argtypes = [C.c_int] * 4 + [C.POINTER(C.c_double)] * 4
            L.ref_env_right.argtypes = [C.c_int] * 4 + [C.POINTER(C.c_double)] * 4
            L.ref_lanczos.argtypes = ([C.c_int] * 4 + [C.POINTER(C.c_double)] * 5 + [C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)])
            L.ref_trunc_k.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int]
            L.ref_dmrg_run.argtypes = ([C.c_int] * 3 + [C.POINTER(C.c_double)] * 2 + [C.POINTER(Params), C.c_int, C.c_int,
                                       C.POINTER(CtrlState), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_double)])
            L.ref_ed_ground.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                        C.POINTER(C.c_double)]
            L.ref_ed_dense.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
            L.ref_round_half_even.argtypes = [C.c_double]
            L.ref_round_half_even.restype = C.c_double
        return _lib


# --------------------------------------------------------------------------
# numpy-level wrappers
# --------------------------------------------------------------------------
def mpo(model: int, N: int, J: float = 1.0, Delta: float = 1.0, J2: float = 0.0) -> np.ndarray:
    """MPO tensors W[i][wl][wr][s][s'] (Section 10's H; Eq. 18 for XXX)."""
    D = lib().ref_mpo_dim(model)
    W = np.zeros((N, D, D, 2, 2))
    lib().ref_build_mpo(model, N, J, Delta, J2, _dp(W))
    return W


def mpo_to_dense(W: np.ndarray) -> np.ndarray:
    N, D = W.shape[0], W.shape[1]
    W = np.ascontiguousarray(W, dtype=np.float64)
    H = np.zeros((2 ** N, 2 ** N))
    lib().ref_mpo_to_dense(N, D, _dp(W), _dp(H))
    return H


def qr(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    Q = np.zeros((m, n)); R = np.zeros((n, n))
    st = lib().ref_qr(m, n, _dp(A), _dp(Q), _dp(R))
    assert st == 0
    return Q, R


def sym_eig(A: np.ndarray):
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    n = A.shape[0]
    w = np.zeros(n); Z = np.zeros((n, n))
    lib().ref_sym_eig(n, _dp(A), _dp(w), _dp(Z))
    return w, Z


def svd(A: np.ndarray, max_sweeps: int = 60):
    """Two-sided Jacobi SVD (Golub & Van Loan 8.6.4): A = U diag(s) Vt."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    r = min(m, n)
    U = np.zeros((m, r)); s = np.zeros(r); Vt = np.zeros((r, n))
    st = lib().ref_svd(m, n, _dp(A), _dp(U), _dp(s), _dp(Vt), max_sweeps)
    if st != 0:
        raise RuntimeError(f"oracle svd status {st}")
    return U, s, Vt


def entropy(s: np.ndarray):
    """Eq. (5) entropy and the Eq. (4) truncation errors eps[k] for keeping k values."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    eps = np.zeros(len(s) + 1)
    S = lib().ref_entropy(len(s), _dp(s), _dp(eps))
    return S, eps


def new_ctrl_states(n: int, chi0: int) -> "C.Array":
    arr = (CtrlState * n)()
    for i in range(n):
        arr[i].chi = chi0
    return arr


def ctrl_replay(S_seq: np.ndarray, params: Params, chi0: int | None = None, states=None):
    """Feed a recorded (steps x bonds) entropy sequence through per-bond controllers."""
    S_seq = np.ascontiguousarray(S_seq, dtype=np.float64)
    T, B = S_seq.shape
    if states is None:
        states = new_ctrl_states(B, params.chi_min if chi0 is None else chi0)
    out = np.zeros((T, B), dtype=np.int32)
    lib().ref_ctrl_replay(T, B, _dp(S_seq), C.byref(params), states, _ip(out))
    return out, states


def ctrl_closed_loop_real(params: Params, g: float, S_star: float, chi_star: float, chi0: float,
                          n_steps: int) -> np.ndarray:
    """chi(0..n_steps) of one real-valued controller (rounding and clamp off)
    driving the linear plant S(t) = S_star + g (chi(t) - chi_star)."""
    st = CtrlState()
    chi = C.c_double(chi0)
    out = [chi0]
    for _ in range(n_steps):
        S = S_star + g * (chi.value - chi_star)
        lib().ref_ctrl_step_real(C.byref(st), S, C.byref(params), C.byref(chi))
        out.append(chi.value)
    return np.array(out)


def mlp_nparam() -> int:
    return lib().ref_mlp_nparam()


def mlp_forward(P: np.ndarray, X: np.ndarray) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64); X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.zeros(X.shape[0])
    lib().ref_mlp_forward(_dp(P), X.shape[0], _dp(X), _dp(y))
    return y


def mlp_loss_grad(P: np.ndarray, X: np.ndarray, t: np.ndarray):
    P = np.ascontiguousarray(P, dtype=np.float64); X = np.ascontiguousarray(X, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros_like(P); loss = np.zeros(1)
    lib().ref_mlp_loss_grad(_dp(P), X.shape[0], _dp(X), _dp(t), _dp(loss), _dp(g))
    return float(loss[0]), g


def adam_step(P, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    for a in (P, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().ref_adam_step(len(P), _dp(P), _dp(g), _dp(m), _dp(v), step, lr, b1, b2, eps)


def heff_apply(L, W1, W2, R, theta):
    """y = H_eff theta (Eq. 19) with L[w][a'][a], R[u][b'][b], theta[a][s1][s2][b]."""
    L, W1, W2, R, theta = (np.ascontiguousarray(x, dtype=np.float64) for x in (L, W1, W2, R, theta))
    D, cl = L.shape[0], L.shape[1]
    cr = R.shape[1]
    y = np.zeros_like(theta)
    lib().ref_heff_apply(cl, cr, 2, D, _dp(L), _dp(W1), _dp(W2), _dp(R), _dp(theta), _dp(y))
    return y


def env_left(L, W, A):
    L, W, A = (np.ascontiguousarray(x, dtype=np.float64) for x in (L, W, A))
    D, cl = L.shape[0], L.shape[1]
    ck = A.shape[2]
    out = np.zeros((D, ck, ck))
    lib().ref_env_left(cl, ck, 2, D, _dp(L), _dp(W), _dp(A), _dp(out))
    return out


def env_right(R, W, B):
    R, W, B = (np.ascontiguousarray(x, dtype=np.float64) for x in (R, W, B))
    D, cr = R.shape[0], R.shape[1]
    ck = B.shape[0]
    out = np.zeros((D, ck, ck))
    lib().ref_env_right(ck, cr, 2, D, _dp(R), _dp(W), _dp(B), _dp(out))
    return out


def lanczos(L, W1, W2, R, theta, K=20):
    """Returns (E, theta', steps, alpha, beta) of the K-step Lanczos of Section 10's eigenproblem."""
    L, W1, W2, R = (np.ascontiguousarray(x, dtype=np.float64) for x in (L, W1, W2, R))
    th = np.array(theta, dtype=np.float64, copy=True, order="C")
    D, cl = L.shape[0], L.shape[1]
    cr = R.shape[1]
    E = np.zeros(1); ku = np.zeros(1, dtype=np.int32)
    al = np.zeros(max(K, 1)); be = np.zeros(max(K, 1))
    lib().ref_lanczos(cl, cr, 2, D, _dp(L), _dp(W1), _dp(W2), _dp(R), _dp(th), K, _dp(E), _ip(ku), _dp(al), _dp(be))
    k = int(ku[0])
    return float(E[0]), th, k, al[:k].copy(), be[:k].copy()


def trunc_k(s, chi_ctrl, eps_trunc, multiplet_guard=1):
    s = np.ascontiguousarray(s, dtype=np.float64)
    return lib().ref_trunc_k(len(s), _dp(s), int(chi_ctrl), float(eps_trunc), int(multiplet_guard))


def init_chi(N: int, chi_init: int, d: int = 2):
    return [min(chi_init, d ** i, d ** (N - i)) for i in range(N + 1)]


def mps_size(N: int, chi_init: int, d: int = 2) -> int:
    c = init_chi(N, chi_init, d)
    return sum(c[i] * d * c[i + 1] for i in range(N))


def dmrg_run(W, mps_init, params: Params, n_sweeps: int, stop_on_conv: bool = False,
             ctrl_states=None, mlp_params=None):
    """Adaptive two-site DMRG (Section 10) from a Gaussian initial MPS.

    Returns a dict with the per-sweep energies and per-visit records."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    N, D = W.shape[0], W.shape[1]
    mps_init = np.ascontiguousarray(mps_init, dtype=np.float64)
    assert mps_init.size == mps_size(N, params.chi_init)
    V = 2 * N - 3
    E_sweep = np.zeros(n_sweeps)
    rb = np.zeros(n_sweeps * V, dtype=np.int32); rE = np.zeros(n_sweeps * V); rS = np.zeros(n_sweeps * V)
    reps = np.zeros(n_sweeps * V); rk = np.zeros(n_sweeps * V, dtype=np.int32); rchi = np.zeros(n_sweeps * V, dtype=np.int32)
    chi_f = np.zeros(N + 1, dtype=np.int32)
    nrm = np.zeros(1)
    if mlp_params is not None:
        mlp_params = np.ascontiguousarray(mlp_params, dtype=np.float64)
    ret = lib().ref_dmrg_run(N, 2, D, _dp(W), _dp(mps_init), C.byref(params), n_sweeps, int(stop_on_conv),
                             ctrl_states, _dp(mlp_params) if mlp_params is not None else None,
                             _dp(E_sweep), _ip(rb), _dp(rE), _dp(rS), _dp(reps), _ip(rk), _ip(rchi), _ip(chi_f), _dp(nrm))
    if ret < 0:
        raise RuntimeError(f"oracle dmrg status {-ret}")
    n = ret
    sl = slice(0, n * V)
    return dict(sweeps=n, E=E_sweep[:n], bond=rb[sl], E_visit=rE[sl], S=rS[sl], eps=reps[sl], k=rk[sl],
                chi=rchi[sl], chi_final=chi_f, visits_per_sweep=V, norm=float(nrm[0]))


def ed_ground(model: int, N: int, J=1.0, Delta=1.0, J2=0.0, n_up=None, max_iter=400) -> float:
    """Lowest eigenvalue by sparse Lanczos in a bit-string basis (independent of the MPO)."""
    if n_up is None:
        n_up = N // 2 if model != MODEL_TFIM else -1
    E = np.zeros(1)
    st = lib().ref_ed_ground(model, N, J, Delta, J2, n_up, max_iter, _dp(E))
    assert st == 0
    return float(E[0])


def ed_dense(model: int, N: int, J=1.0, Delta=1.0, J2=0.0) -> np.ndarray:
    ev = np.zeros(2 ** N)
    lib().ref_ed_dense(model, N, J, Delta, J2, _dp(ev))
    return ev


def statevector(N: int, layers):
    """Exact state of the circuit `layers` (list of (positions, gates)) on
    |0...0>, qubit 0 the most significant bit of the index."""
    psi = np.zeros(2 ** N)
    psi[0] = 1.0
    for pos, gates in layers:
        pos = np.ascontiguousarray(pos, dtype=np.int32)
        gates = np.ascontiguousarray(gates, dtype=np.float64)
        assert lib().ref_statevector_apply(N, _dp(psi), len(pos), _ip(pos), _dp(gates)) == 0
    return psi


def circuit_run(N: int, layers, params: Params, chi_warm=None, want_state: bool = True):
    """MPS circuit run with per-bond chi control (Section 8); returns the chi
    map (layers x (N-1)), the entropy map and the final state (N <= 24)."""
    nl = len(layers)
    ng = np.array([len(p) for p, _ in layers], dtype=np.int32)
    pos = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.int32) for p, _ in layers])
                               if nl else np.zeros(0, np.int32), dtype=np.int32)
    gates = np.ascontiguousarray(np.concatenate([np.asarray(g, dtype=np.float64).reshape(-1) for _, g in layers])
                                 if nl else np.zeros(0), dtype=np.float64)
    chi_map = np.zeros((nl, N - 1), dtype=np.int32)
    S_map = np.zeros((nl, N - 1))
    psi = np.zeros(2 ** N) if want_state and N <= 24 else None
    warm = None
    if chi_warm is not None:
        warm = np.ascontiguousarray(chi_warm, dtype=np.int32)
    st = lib().ref_circuit_run(N, nl, _ip(ng), _ip(pos), _dp(gates), C.byref(params),
                               _ip(warm) if warm is not None else None, None, _ip(chi_map), _dp(S_map),
                               _dp(psi) if psi is not None else None)
    if st != 0:
        raise RuntimeError(f"oracle circuit status {-st}")
    return chi_map, S_map, psi
