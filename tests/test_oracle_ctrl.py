"""Pins of the oracle's controller (Eq. 8 EMA, Eq. 16 predictor, Algorithm 2
PID with rounding, clamping and anti-windup, Algorithm 1 direct map) and of
the learned scheduler's network (forward, gradient, Adam).  Expected integer
sequences below are worked out by hand in the comments."""
import math

import numpy as np
import pytest
from scipy.stats import norm

import oracle as O
import synth


def P(**kw):
    base = dict(alpha_ema=1.0, beta=0.0, Kp=2.0, Ki=0.1, Kd=0.5, chi_min=4, chi_max=1000, S_target=1.0)
    base.update(kw)
    return O.make_params(**base)


def run_single(S_seq, p, chi0=None):
    out, st = O.ctrl_replay(np.asarray(S_seq, dtype=float)[:, None], p, chi0=chi0)
    return out[:, 0].tolist(), st[0]


def test_ema_step_response():
    """Eq. (8) on a step S0 -> S1: Sbar(t) = S1 - (S1 - S0)(1 - alpha)^t."""
    a, S0, S1 = 0.3, 0.2, 1.7
    p = P(alpha_ema=a, ctrl=O.CTRL_FIXED, chi_fixed=8)
    st = O.new_ctrl_states(1, 8)
    chi = np.zeros(1, dtype=np.int32)
    O.lib().ref_ctrl_step(st, S0, p, chi.ctypes.data_as(O.C.POINTER(O.C.c_int)))
    assert st[0].Sbar == S0                       # initialised to the first measurement (Section 4)
    for t in range(1, 30):
        O.lib().ref_ctrl_step(st, S1, p, chi.ctypes.data_as(O.C.POINTER(O.C.c_int)))
        assert abs(st[0].Sbar - (S1 - (S1 - S0) * (1 - a) ** t)) < 1e-14


def test_ema_init_zero_variant():
    p = P(alpha_ema=0.25, ema_init_zero=1, ctrl=O.CTRL_FIXED, chi_fixed=8)
    _, st = run_single([2.0], p, chi0=8)
    assert st.Sbar == 0.5                         # Section 10 initialisation: Sbar(0) = 0, then one EMA step


def test_pid_constant_error_by_hand():
    """alpha=1, beta=0, e = 1 every step: u_t = 2*1 + 0.1*t + 0.5*0
       t=1: 2.1->2 (6)  t=2: 2.2->2 (8)  t=3: 2.3->2 (10) t=4: 2.4->2 (12)
       t=5: 2.5->2 (half to even, 14)  t=6: 2.6->3 (17) t=7: 2.7->3 (20)."""
    chi, _ = run_single([2.0] * 7, P(S_target=1.0))
    # 0.1 summed in binary floating point stays on the same side of each .5 boundary
    assert chi == [6, 8, 10, 12, 14, 17, 20]


def test_pid_half_even_exact():
    """Exactly representable gains: Kp=1, Ki=0.25, Kd=0, e=2:
       u = 2 + 0.5 = 2.5 -> 2; u = 2 + 1.0 = 3 -> 3; u = 2 + 1.5 = 3.5 -> 4; u = 4.0 -> 4; 4.5 -> 4."""
    chi, _ = run_single([3.0] * 5, P(Kp=1.0, Ki=0.25, Kd=0.0, S_target=1.0))
    assert chi == [4 + 2, 6 + 3, 9 + 4, 13 + 4, 17 + 4]


def test_pid_negative_error_and_clamp_antiwindup():
    """Kp=1, Ki=0.5, Kd=0, chi0 = 10, e = -1.5:
       t=1: I=-0.75, u=-2.25 -> -2, chi 8
       t=2: I=-1.5,  u=-3.0  -> -3, chi 5
       t=3: I=-2.25, u=-3.75 -> -4, raw 1 -> clamp 4, I undone -> -1.5
       t=4: I=-2.25 again, raw 0 -> clamp 4, I undone -> -1.5."""
    chi, st = run_single([0.5] * 4, P(Kp=1.0, Ki=0.5, Kd=0.0, S_target=2.0), chi0=10)
    assert chi == [8, 5, 4, 4]
    assert st.I == -1.5


def test_pid_upper_clamp_freezes_integral():
    """Kp=1, Ki=1, Kd=0, e = 1, chi0 = 4, chi_max = 9:
       t=1: I=1, u=2 -> 6;  t=2: I=2, u=3 -> 9;  t=3: I=3, u=4 -> 13 -> clamp 9, I back to 2
       t=4: same as t=3 -> 9, I stays 2."""
    chi, st = run_single([2.0] * 4, P(Kp=1.0, Ki=1.0, Kd=0.0, chi_max=9, S_target=1.0))
    assert chi == [6, 9, 9, 9]
    assert st.I == 2.0


def test_pid_derivative_term():
    """Kp=0, Ki=0, Kd=2: D = 2 (e_t - e_{t-1}); e = 1, 3, 2 ->
       t=1: D=0 (e_prev := e) -> 4;  t=2: D=4 -> 8;  t=3: D=-2 -> 6."""
    chi, _ = run_single([2.0, 4.0, 3.0], P(Kp=0.0, Ki=0.0, Kd=2.0, S_target=1.0))
    assert chi == [4, 8, 6]


def test_predictor_on_ramp():
    """Eq. (16) with alpha = 1: Sbar follows S; on S_t = 1 + 0.5 t the prediction is
    Sbar + beta*0.5.  Kp=1, Ki=Kd=0, S_target = 0, beta = 1:
       t=0 (S=1):   Shat = 1 (no history) -> u=1   -> 5
       t=1 (S=1.5): Shat = 2              -> u=2   -> 7
       t=2 (S=2):   Shat = 2.5            -> u=2.5 -> 2 -> 9."""
    chi, _ = run_single([1.0, 1.5, 2.0], P(Kp=1.0, Ki=0.0, Kd=0.0, S_target=0.0, beta=1.0))
    assert chi == [5, 7, 9]


def test_second_order_predictor_curvature():
    """Section 7 second-order variant adds beta*(Sbar - 2 Sbar_prev + Sbar_prev2).
    S = 0, 1, 4 (alpha = 1), beta = 1, Kp = 1: t=2: linear 4 + 3 = 7, curvature 4 - 2 + 0 = 2 -> 9."""
    p = P(Kp=1.0, Ki=0.0, Kd=0.0, S_target=0.0, beta=1.0, second_order=1, chi_max=10000)
    chi, _ = run_single([0.0, 1.0, 4.0], p, chi0=100)
    # t=0: Shat = 0 -> 100; t=1: linear 1 + 1 = 2, curvature 1 - 0 + 0 = 1 -> 3 -> 103; t=2: 9 -> 112
    assert chi == [100, 103, 112]


def test_direct_map_algorithm1():
    """Algorithm 1: chi = clamp(ceil(gamma exp(Sbar)), chi_min, chi_max).  With gamma = 1.5 and
    Sbar = ln m for odd m, gamma*m is a half-integer so the ceiling is (3m+1)/2 exactly."""
    for m in [3, 5, 21, 101]:
        p = P(ctrl=O.CTRL_DIRECT, gamma=1.5, chi_min=2, chi_max=1000)
        chi, _ = run_single([math.log(m)], p)
        assert chi == [(3 * m + 1) // 2]
    p = P(ctrl=O.CTRL_DIRECT, gamma=1.5, chi_min=2, chi_max=10)
    assert run_single([math.log(101)], p)[0] == [10]
    p = P(ctrl=O.CTRL_DIRECT, gamma=1.0, chi_min=6, chi_max=10)
    assert run_single([0.0], p)[0] == [6]


def test_replay_is_per_bond_independent():
    rng = np.random.default_rng(3)
    S = rng.random((12, 5)) * 3
    p = P(alpha_ema=0.3, beta=0.4)
    allb, _ = O.ctrl_replay(S, p)
    for b in range(5):
        single, _ = O.ctrl_replay(S[:, b:b + 1].copy(), p)
        assert np.array_equal(single[:, 0], allb[:, b])


# ---------------------------------------------------------------------------
# learned scheduler network
# ---------------------------------------------------------------------------
NP = 4929


def test_mlp_param_count():
    assert O.mlp_nparam() == NP == 64 * 10 + 64 + 64 * 64 + 64 + 64 + 1


def _split(Pv):
    W1 = Pv[:640].reshape(64, 10); b1 = Pv[640:704]; W2 = Pv[704:4800].reshape(64, 64)
    b2 = Pv[4800:4864]; W3 = Pv[4864:4928]; b3 = Pv[4928:]
    return W1, b1, W2, b2, W3, b3


def test_mlp_forward_hand_case():
    """One active path: y = w3 * gelu(w2 * gelu(w1 x0)) + b3 with gelu(x) = x Phi(x) (scipy's normal cdf)."""
    Pv = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = _split(Pv)
    W1[0, 0] = 1.3; W2[0, 0] = -0.7; W3[0] = 2.0; b3[0] = 0.25
    X = np.array([[0.9] + [5.0] * 9, [-1.2] + [0.0] * 9])
    g = lambda x: x * norm.cdf(x)
    ref = 2.0 * g(-0.7 * g(1.3 * X[:, 0])) + 0.25
    assert np.allclose(O.mlp_forward(Pv, X), ref, rtol=1e-14, atol=1e-15)


def test_mlp_gelu_odd_part_identity():
    """gelu(x) - gelu(-x) = x for the exact-erf GELU."""
    Pv = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = _split(Pv)
    W1[0, 0] = 1.0; W2[0, 0] = 1.0; W3[0] = 1.0
    # second layer sees gelu(x); use a unit second layer on the raw GELU via W2 = identity-like path
    x = np.linspace(-3, 3, 13)
    X = np.zeros((13, 10)); X[:, 0] = x
    Xn = X.copy(); Xn[:, 0] = -x
    # y(x) = gelu(gelu(x)); check on the inner layer with a linear read-out instead
    Pv2 = np.zeros(NP); W1b, b1b, W2b, b2b, W3b, b3b = _split(Pv2)
    W1b[0, 0] = 1.0; W2b[0, 0] = 1e-6; W3b[0] = 1e6      # gelu(1e-6 h) ~ 0.5e-6 h (+O(1e-12))
    y = O.mlp_forward(Pv2, X) - O.mlp_forward(Pv2, Xn)
    assert np.allclose(y, 0.5 * x, atol=1e-5)


def test_mlp_gradient_central_differences():
    rng = np.random.default_rng(5)
    Pv = rng.standard_normal(NP) * 0.2
    X = rng.standard_normal((7, 10)); t = rng.standard_normal(7)
    L0, g = O.mlp_loss_grad(Pv, X, t)
    h = 1e-6
    idx = rng.choice(NP, 60, replace=False)
    for i in list(idx) + [0, 639, 640, 4863, 4864, 4928]:
        e = np.zeros(NP); e[i] = h
        fd = (O.mlp_loss_grad(Pv + e, X, t)[0] - O.mlp_loss_grad(Pv - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-8


def test_adam_first_step_is_signed_lr():
    """Kingma & Ba: with m = v = 0, the bias-corrected first step is -lr g/(|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    Pv = np.zeros(4); m = np.zeros(4); v = np.zeros(4)
    O.adam_step(Pv, g.copy(), m, v, 1, lr=1e-3)
    assert np.allclose(Pv, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_adam_training_reduces_loss():
    rng = np.random.default_rng(9)
    lim1 = np.sqrt(6 / (10 + 64)); lim2 = np.sqrt(6 / 128); lim3 = np.sqrt(6 / 65)
    Pv = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = _split(Pv)
    W1[:] = rng.uniform(-lim1, lim1, W1.shape); W2[:] = rng.uniform(-lim2, lim2, W2.shape)
    W3[:] = rng.uniform(-lim3, lim3, W3.shape)
    X = rng.standard_normal((32, 10)); t = X[:, 0] * 2 + np.sin(X[:, 1])
    m = np.zeros(NP); v = np.zeros(NP)
    L_first = O.mlp_loss_grad(Pv, X, t)[0]
    for step in range(1, 301):
        L, g = O.mlp_loss_grad(Pv, X, t)
        O.adam_step(Pv, g, m, v, step, lr=3e-3)
    assert O.mlp_loss_grad(Pv, X, t)[0] < 0.1 * L_first


def test_global_adaptive_chi_closed_form():
    """Global adaptive chi (Section 6): one controller on the mean of the
    per-bond filtered entropies, stepped once per sweep, chi uniform over the
    bonds.  With alpha = 1 (S-bar_i = the bond's latest entropy), beta = 0,
    K_p = 1, K_i = K_d = 0 the law is chi(t+1) = clamp(chi(t) +
    round_half_even(mean_i S_last(i, t) - S_target)), written out here from
    the recorded per-visit entropies."""
    N, chi_min, chi_max, sweeps = 10, 2, 24, 4
    kw = dict(ctrl=O.CTRL_GLOBAL, alpha_ema=1.0, beta=0.0, Kp=1.0, Ki=0.0, Kd=0.0, S_target=-3.0,
              chi_min=chi_min, chi_max=chi_max, chi_init=chi_min, eps_trunc=1e-10)
    p = O.make_params(**kw)
    m0 = synth.initial_mps_entries(synth.workload_seed(0, 7), N, chi_min)
    ref = O.dmrg_run(O.mpo(O.MODEL_XXZ, N, 1.0, 1.0), m0, p, sweeps)
    V = ref["visits_per_sweep"]
    g = chi_min
    for t in range(sweeps):
        chi_t = ref["chi"][t * V:(t + 1) * V]
        assert np.all(chi_t == g), (t, chi_t, g)          # uniform over the bonds, set before the sweep
        last = {}
        for b, S in zip(ref["bond"][t * V:(t + 1) * V], ref["S"][t * V:(t + 1) * V]):
            last[int(b)] = S                              # the bond's latest visit in this sweep
        mean = sum(last[b] for b in range(N - 1)) / (N - 1)
        g = int(min(max(g + round(mean - kw["S_target"]), chi_min), chi_max))
    assert g > chi_min                                    # the law did move chi


# ---------------------------------------------------------------------------
# Closed loop with rounding and clamping off (the linear loop that Section 5's
# stability analysis reasons about).  Plant S(t) = S* + g (chi(t) - chi*),
# target S_target = S*, so with x = chi - chi*:
#   EMA (Eq. 8)        s(t) = alpha g x(t) + (1 - alpha) s(t-1)
#   predictor (Eq. 16) e(t) = s(t) + beta (s(t) - s(t-1))
#   PID (Algorithm 2)  u(t) = Kp e(t) + I(t) + Kd (e(t) - e(t-1)),
#                      I(t) = I(t-1) + Ki e(t)
#   update             x(t+1) = x(t) + u(t).
# In z: (z - 1) X = C(z) F(z) g X with C = Kp + Ki z/(z-1) + Kd (z-1)/z and
# F = alpha ((1+beta) z - beta) / (z - (1-alpha)); cleared of denominators,
#   z (z-1)^2 (z-(1-alpha)) - g alpha ((1+beta) z - beta)
#       [Kp z (z-1) + Ki z^2 + Kd (z-1)^2] = 0.
# (Eqs. 14-15 omit the integrating update of chi, so the paper's quadratic is
# not this loop's polynomial.)  The first visit's initialisation (S-bar = S,
# S-bar_prev = S-bar, e_prev = e, I = Ki e) is the linear state extended
# backwards, so the whole trajectory from t = 0 obeys the recurrence.


def _char_poly(alpha, beta, Kp, Ki, Kd, g):
    """Coefficients (highest power first) of the closed loop's polynomial."""
    P_ = np.polynomial.polynomial
    z = [0.0, 1.0]
    zm1 = [-1.0, 1.0]
    lhs = P_.polymul(P_.polymul(z, P_.polymul(zm1, zm1)), [-(1.0 - alpha), 1.0])
    ctrl = P_.polyadd(P_.polyadd(Kp * P_.polymul(z, zm1), Ki * P_.polymul(z, z)), Kd * P_.polymul(zm1, zm1))
    rhs = g * alpha * P_.polymul([-beta, 1.0 + beta], ctrl)
    return P_.polysub(lhs, rhs)[::-1]


@pytest.mark.parametrize("alpha,beta,g", [(0.3, 0.4, -0.2), (0.5, 0.8, -0.05), (0.3, 0.0, 0.02), (0.9, 0.4, -0.6)])
def test_closed_loop_real_valued_obeys_characteristic_recurrence(alpha, beta, g):
    Kp, Ki, Kd = 2.0, 0.1, 0.5
    p = P(alpha_ema=alpha, beta=beta, Kp=Kp, Ki=Ki, Kd=Kd, S_target=1.3)
    chi = O.ctrl_closed_loop_real(p, g, S_star=1.3, chi_star=100.0, chi0=40.0, n_steps=40)
    x = chi - 100.0
    c = _char_poly(alpha, beta, Kp, Ki, Kd, g)
    assert len(c) == 5
    scale = np.max(np.abs(x)) * np.sum(np.abs(c))
    for t in range(len(x) - 4):
        r = sum(c[k] * x[t + 4 - k] for k in range(5))
        assert abs(r) <= 1e-13 * scale, (t, r)
    # a plausible slip changes the polynomial and breaks the recurrence
    wrong = _char_poly(alpha, beta, Kp, Ki, -Kd, g)
    res = max(abs(sum(wrong[k] * x[t + 4 - k] for k in range(5))) for t in range(len(x) - 4))
    assert res > 1e-6 * scale


def test_closed_loop_pure_pid_closed_form():
    """alpha = 1, beta = 0: the state is (x(t), I(t-1), e(t-1)) and the loop's
    polynomial is the cubic z (z-1)^2 - g [Kp z(z-1) + Ki z^2 + Kd (z-1)^2]
    = z^3 - (2 + g(Kp+Ki+Kd)) z^2 + (1 + g(Kp+2Kd)) z - g Kd.  So x(t) =
    sum_i c_i r_i^t, with c fixed by x(0), x(1), x(2) worked out by hand from
    the first visit's rules."""
    Kp, Ki, Kd, g, x0 = 2.0, 0.1, 0.5, -0.3, -60.0
    p = P(alpha_ema=1.0, beta=0.0, Kp=Kp, Ki=Ki, Kd=Kd, S_target=0.7)
    chi = O.ctrl_closed_loop_real(p, g, S_star=0.7, chi_star=100.0, chi0=100.0 + x0, n_steps=40)
    x = chi - 100.0
    e0 = g * x0
    I0 = Ki * e0
    x1 = x0 + Kp * e0 + I0                    # e_prev = e on the first visit: no D term
    e1 = g * x1
    I1 = I0 + Ki * e1
    x2 = x1 + Kp * e1 + I1 + Kd * (e1 - e0)
    r = np.roots([1.0, -(2.0 + g * (Kp + Ki + Kd)), 1.0 + g * (Kp + 2.0 * Kd), -g * Kd])
    V = np.vander(r, 3, increasing=True).T    # V[k][i] = r_i^k
    c = np.linalg.solve(V, np.array([x0, x1, x2], dtype=complex))
    t = np.arange(len(x))
    closed = np.real((c[None, :] * r[None, :] ** t[:, None]).sum(axis=1))
    assert np.max(np.abs(closed - x)) <= 1e-12 * np.max(np.abs(x))
    # the loop settles (|r| < 1 for these gains), towards chi* = 100
    assert np.max(np.abs(r)) < 1.0 and abs(x[-1]) < abs(x0)
