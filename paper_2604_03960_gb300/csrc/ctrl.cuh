// ctrl.cuh -- device-side entropy monitor, controller and truncation rule.
#pragma once
#include "common.cuh"

namespace dmrg {

constexpr int MLP_IN = 10, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;   // 4929

// Result of the per-bond decision, written by the decide kernel.
struct BondResult {
    double S;        // Eq. (5) entropy of the full spectrum
    double eps;      // Eq. (4) truncation error of the retained k
    double znorm;    // sqrt(sum_{j<k} s_j^2), for renormalisation
    double E;        // Ritz value of the visit (copied from the Lanczos state)
    int k;           // retained bond dimension
    int chi_ctrl;    // controller output
    int mlp_fallback;
    int pad;
};

// Controller step of Algorithms 1-2 (Eqs. 8, 9-11, 16) for one bond, in
// FP64 with every product and sum rounded separately (no FMA) and in the
// same order as the plain C oracle, so a recorded entropy sequence gives
// the same integer schedule.
__device__ __forceinline__ int clamp_chi(double x, int lo, int hi)
{
    if (x < (double)lo) return lo;
    if (x > (double)hi) return hi;
    return (int)x;
}

__device__ __forceinline__ int ctrl_step_dev(dmrg_ctrl_state *st, double S, const dmrg_params &p)
{
    const double a = p.alpha_ema;
    if (!st->initialized) {
        double sb = p.ema_init_zero ? __dmul_rn(a, S) : S;
        st->Sbar = sb;
        st->Sbar_prev = sb;
        st->Sbar_prev2 = sb;
    } else {
        double nb = __dadd_rn(__dmul_rn(a, S), __dmul_rn(__dsub_rn(1.0, a), st->Sbar));
        st->Sbar_prev2 = st->Sbar_prev;
        st->Sbar_prev = st->Sbar;
        st->Sbar = nb;
    }
    if (st->nhist < 8) {
        st->hist[st->nhist++] = st->Sbar;
    } else {
        for (int i = 0; i < 7; ++i) st->hist[i] = st->hist[i + 1];
        st->hist[7] = st->Sbar;
    }
    double Shat = __dadd_rn(st->Sbar, __dmul_rn(p.beta, __dsub_rn(st->Sbar, st->Sbar_prev)));
    if (p.second_order)
        Shat = __dadd_rn(Shat, __dmul_rn(p.beta, __dadd_rn(__dsub_rn(st->Sbar, __dmul_rn(2.0, st->Sbar_prev)),
                                                          st->Sbar_prev2)));
    int chi_new;
    if (p.ctrl == DMRG_CTRL_DIRECT) {
        double tgt = ceil(__dmul_rn(p.gamma, exp(st->Sbar)));
        chi_new = clamp_chi(tgt, p.chi_min, p.chi_max);
    } else if (p.ctrl == DMRG_CTRL_FIXED) {
        chi_new = p.chi_fixed;
    } else if (p.ctrl == DMRG_CTRL_THRESHOLD) {
        chi_new = p.chi_max;
    } else {
        double e = __dsub_rn(Shat, p.S_target);
        if (!st->initialized) st->e_prev = e;
        double P = __dmul_rn(p.Kp, e);
        st->I = __dadd_rn(st->I, __dmul_rn(p.Ki, e));
        double Dt = __dmul_rn(p.Kd, __dsub_rn(e, st->e_prev));
        double u = __dadd_rn(__dadd_rn(P, st->I), Dt);
        double delta = rint(u);                     // round half to even
        double raw = __dadd_rn((double)st->chi, delta);
        chi_new = clamp_chi(raw, p.chi_min, p.chi_max);
        if ((double)chi_new != raw) st->I = __dsub_rn(st->I, __dmul_rn(p.Ki, e));   // anti-windup
        st->e_prev = e;
    }
    st->chi = chi_new;
    st->initialized = 1;
    return chi_new;
}

// Launchers (ctrl.cu)
// rank_floor: singular values <= rank_floor * s_0 count as zero (r eps for the
// FP64 SVD; the FP32 Jacobi of the mixed form resolves about 2^-22).
dmrg_status launch_global_step(dmrg_ctx *ctx, const dmrg_ctrl_state *bonds, int n_bonds, dmrg_ctrl_state *g,
                               const dmrg_params &p);
dmrg_status launch_decide(dmrg_ctx *ctx, const double *s, int r, dmrg_ctrl_state *st_bond, const dmrg_params &p,
                          int do_ctrl, int chi_override, const float *mlp, int bond, int N, int sweep,
                          const void *lz_state, BondResult *res, dmrg_visit_record *visit, int direction,
                          double rank_floor, const int *jac_info = nullptr);
dmrg_status launch_ctrl_steps(dmrg_ctx *ctx, int n, const double *S, dmrg_ctrl_state *st, const dmrg_params &p,
                              int *chi_out);
dmrg_status launch_entropy(dmrg_ctx *ctx, int n, const double *s, double *S, double *eps);

}  // namespace dmrg
