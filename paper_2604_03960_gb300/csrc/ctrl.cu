// ctrl.cu -- entropy monitor (Eq. 5), truncation error (Eq. 4), controller
// (Algorithms 1-2 with Eqs. 8 and 16), learned-scheduler inference and the
// truncation rule of Section 10, fused into one small kernel per bond visit
// so that chi never leaves the device inside a sweep.
#include "ctrl.cuh"
#include "lanczos.cuh"

namespace dmrg {
namespace {

constexpr int DB = 256;

struct Neum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
};

// Compensated block sum: each thread's (s, c) are summed separately.
__device__ double block_sum_neum(const Neum &n, double *sh)
{
    double a = block_sum(n.s, sh);
    double b = block_sum(n.c, sh);
    return a + b;
}

__device__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// Forward of the learned scheduler for one feature vector, by one block
// (>= 64 threads).  Returns y in every thread.
__device__ float mlp_forward_block(const float *P, const float *x, float *h1, float *h2, float *red)
{
    const float *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const float *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    const int t = threadIdx.x;
    if (t < MLP_H) {
        float acc = b1[t];
        for (int i = 0; i < MLP_IN; ++i) acc = fmaf(W1[t * MLP_IN + i], x[i], acc);
        h1[t] = gelu_f(acc);
    }
    __syncthreads();
    if (t < MLP_H) {
        float acc = b2[t];
        for (int i = 0; i < MLP_H; ++i) acc = fmaf(W2[t * MLP_H + i], h1[i], acc);
        h2[t] = gelu_f(acc);
    }
    __syncthreads();
    if (t == 0) {
        float acc = b3[0];
        for (int i = 0; i < MLP_H; ++i) acc = fmaf(W3[i], h2[i], acc);
        red[0] = acc;
    }
    __syncthreads();
    float y = red[0];
    __syncthreads();
    return y;
}

// k = min(chi, rank, above), >= 1, then the multiplet guard.
__device__ int trunc_k_dev(const double *s, int r, int chi, int rank, int above, int guard)
{
    int k = chi;
    if (rank < k) k = rank;
    if (above < k) k = above;
    if (k < 1) k = 1;
    if (guard && k < r) {
        while (k > 1 && fabs(s[k - 1] - s[k]) <= 1e-10 * s[k - 1]) k--;
    }
    return k;
}

// spectra up to this length are staged in shared memory first, so that the
// serial scans below (multiplet guard, label tail) read shared memory
constexpr int kDecideSmem = 4096;

__global__ void __launch_bounds__(DB) k_decide(const double *__restrict__ s_g, int r, dmrg_ctrl_state *st,
                                               dmrg_params p, int do_ctrl, int chi_override, const float *mlp,
                                               int bond, int N, int sweep, const LzState *lz, BondResult *res,
                                               dmrg_visit_record *visit, int direction, double rank_floor,
                                               const int *jac_info, double eps_target, int *status)
{
    extern __shared__ double s_sm[];
    const double *s = s_g;
    if (r <= kDecideSmem) {
        for (int j = threadIdx.x; j < r; j += DB) s_sm[j] = s_g[j];
        __syncthreads();
        s = s_sm;
    }
    __shared__ double sh[32];
    __shared__ float h1[MLP_H], h2[MLP_H], xin[MLP_IN], red[2];
    __shared__ int sh_chi, sh_k, sh_kp, sh_fb, sh_mlp_ok, sh_chim;
    const int t = threadIdx.x;
    // 1. norm of the spectrum
    Neum z;
    for (int j = t; j < r; j += DB) z.add(s[j] * s[j]);
    const double Z = block_sum_neum(z, sh);
    // 2. entropy of the full spectrum (0 ln 0 := 0)
    Neum en;
    if (Z > 0.0)
        for (int j = t; j < r; j += DB) {
            double pj = s[j] * s[j] / Z;
            if (pj > 0.0) en.add(-pj * log(pj));
        }
    const double S = block_sum_neum(en, sh);
    // 3. numerical rank and the count above the threshold on the normalised spectrum
    const double nz = sqrt(Z);
    const double rank_tol = rank_floor * (r > 0 ? s[0] : 0.0);
    double cr = 0.0, ca = 0.0;
    for (int j = t; j < r; j += DB) {
        if (s[j] > rank_tol) cr += 1.0;
        if (nz > 0.0 && s[j] / nz > p.eps_trunc) ca += 1.0;
    }
    const int rank = (int)block_sum(cr, sh);
    const int above = (int)block_sum(ca, sh);
    // 4. controller
    if (t == 0) {
        int c;
        if (p.ctrl == DMRG_CTRL_GLOBAL && st) {
            // global adaptive chi: the bond's filter advances, the uniform chi
            // of this sweep (chi_override) truncates
            if (do_ctrl) (void)ctrl_step_dev(st, S, p);
            c = chi_override > 0 ? chi_override : st->chi;
        } else if (chi_override > 0) c = chi_override;
        else if (do_ctrl) c = ctrl_step_dev(st, S, p);
        else c = st->chi;
        sh_chi = c;
        sh_fb = 0;
        sh_mlp_ok = 0;
        if (p.ctrl == DMRG_CTRL_MLP && mlp && do_ctrl && chi_override <= 0) {
            const int h = st->nhist;
            for (int j = 0; j < 8; ++j) {
                int idx = h - 8 + j;
                if (idx < 0) idx = 0;
                xin[j] = (h > 0) ? (float)st->hist[idx] : 0.0f;
            }
            xin[8] = (float)(bond + 1) / (float)N;
            xin[9] = (float)sweep / (float)(p.max_sweeps > 0 ? p.max_sweeps : 1);
            sh_mlp_ok = 1;
        }
    }
    __syncthreads();
    if (sh_mlp_ok) {
        float y = mlp_forward_block(mlp, xin, h1, h2, red);
        if (t == 0) {
            // a finite output is clamped to [chi_min, chi_max]; a non-finite one falls back
            double c = rint(exp2((double)y));
            c = c < (double)p.chi_min ? (double)p.chi_min : (c > (double)p.chi_max ? (double)p.chi_max : c);
            sh_fb = 1;
            sh_chim = isfinite(y) ? (int)c : -1;
        }
        __syncthreads();
        if (sh_chim > 0) {
            if (t == 0) {
                sh_k = trunc_k_dev(s, r, sh_chim, rank, above, p.multiplet_guard);
                sh_kp = trunc_k_dev(s, r, sh_chi, rank, above, p.multiplet_guard);
            }
            __syncthreads();
            double tm = 0.0, tp = 0.0;
            for (int j = t; j < r; j += DB) {
                double pj = (Z > 0.0) ? s[j] * s[j] / Z : 0.0;
                if (j >= sh_k) tm += pj;
                if (j >= sh_kp) tp += pj;
            }
            double em = sqrt(fmax(block_sum(tm, sh), 0.0));
            double ep = sqrt(fmax(block_sum(tp, sh), 0.0));
            if (t == 0 && !(em > 10.0 * ep + 1e-10)) {
                sh_chi = sh_chim;
                sh_fb = 0;
            }
            __syncthreads();
        }
    }
    // 5. truncation
    if (t == 0) sh_k = trunc_k_dev(s, r, sh_chi, rank, above, p.multiplet_guard);
    __syncthreads();
    const int k = sh_k;
    Neum tail, head;
    for (int j = t; j < r; j += DB) {
        if (j >= k) tail.add((Z > 0.0) ? s[j] * s[j] / Z : 0.0);
        else head.add(s[j] * s[j]);
    }
    const double T = block_sum_neum(tail, sh);
    const double H = block_sum_neum(head, sh);
    if (t == 0) {
        BondResult br;
        br.S = S;
        br.eps = sqrt(fmax(T, 0.0));
        br.znorm = sqrt(H);
        br.E = lz ? lz->E : 0.0;
        br.k = k;
        br.chi_ctrl = sh_chi;
        br.mlp_fallback = sh_fb;
        br.pad = 0;
        *res = br;
        if (visit) {
            visit->bond = bond;
            visit->k = k;
            visit->chi_ctrl = sh_chi;
            visit->direction = direction;
            visit->E = br.E;
            visit->S = S;
            visit->trunc_err = br.eps;
            visit->jacobi_sweeps = jac_info ? jac_info[0] : 0;
            visit->lanczos_steps = lz ? lz->m : 0;
            visit->mlp_used = sh_mlp_ok && !sh_fb;
            // learned-scheduler features after this step (same recipe as its inference)
            if (st) {
                const int h = st->nhist;
                for (int j = 0; j < 8; ++j) {
                    int idx = h - 8 + j;
                    if (idx < 0) idx = 0;
                    visit->feat[j] = (h > 0) ? (float)st->hist[idx] : 0.0f;
                }
            } else {
                for (int j = 0; j < 8; ++j) visit->feat[j] = 0.0f;
            }
            visit->feat[8] = (float)(bond + 1) / (float)N;
            visit->feat[9] = (float)sweep / (float)(p.max_sweeps > 0 ? p.max_sweeps : 1);
            // label source: smallest k whose discarded weight is <= eps_target^2
            int ks = r;
            if (Z > 0.0) {
                double tail = 0.0;
                const double lim = eps_target * eps_target, iz = 1.0 / Z;
                for (int j = r - 1; j >= 1; --j) {
                    tail += s[j] * s[j] * iz;
                    if (tail > lim) break;
                    ks = j;
                }
            }
            visit->k_star = ks;
        }
        if (!isfinite(S) || !isfinite(br.znorm) || br.znorm == 0.0) atomicOr(status, ST_NAN);
    }
}

__global__ void k_ctrl_steps(int n, const double *__restrict__ S, dmrg_ctrl_state *st, dmrg_params p, int *chi_out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    chi_out[i] = ctrl_step_dev(&st[i], S[i], p);
}

__global__ void k_entropy(int n, const double *__restrict__ s, double *S_out, double *eps)
{
    __shared__ double sh[32];
    Neum z;
    for (int j = threadIdx.x; j < n; j += blockDim.x) z.add(s[j] * s[j]);
    const double Z = block_sum_neum(z, sh);
    Neum en;
    if (Z > 0.0)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double pj = s[j] * s[j] / Z;
            if (pj > 0.0) en.add(-pj * log(pj));
        }
    const double S = block_sum_neum(en, sh);
    if (threadIdx.x == 0) {
        S_out[0] = S;
        if (eps) {
            Neum tail;
            eps[n] = 0.0;
            for (int k = n - 1; k >= 0; --k) {
                tail.add(Z > 0.0 ? s[k] * s[k] / Z : 0.0);
                eps[k] = sqrt(fmax(tail.s + tail.c, 0.0));
            }
        }
    }
}

}  // namespace

// Global adaptive chi: S-bar(t) = (N-1)^-1 sum_i S-bar_i(t) over the bonds'
// filtered entropies (summed in bond order), then one controller step with
// alpha = 1 (the inputs are already filtered).  Same arithmetic as the oracle.
__global__ void k_global_step(const dmrg_ctrl_state *__restrict__ bonds, int n_bonds, dmrg_ctrl_state *g,
                              dmrg_params p)
{
    double sum = 0.0;
    for (int b = 0; b < n_bonds; ++b) sum = __dadd_rn(sum, bonds[b].Sbar);
    const double mean = __ddiv_rn(sum, (double)n_bonds);
    p.alpha_ema = 1.0;
    (void)ctrl_step_dev(g, mean, p);
}

dmrg_status launch_global_step(dmrg_ctx *ctx, const dmrg_ctrl_state *bonds, int n_bonds, dmrg_ctrl_state *g,
                               const dmrg_params &p)
{
    k_global_step<<<1, 1, 0, ctx->stream>>>(bonds, n_bonds, g, p); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status launch_decide(dmrg_ctx *ctx, const double *s, int r, dmrg_ctrl_state *st_bond, const dmrg_params &p,
                          int do_ctrl, int chi_override, const float *mlp, int bond, int N, int sweep,
                          const void *lz_state, BondResult *res, dmrg_visit_record *visit, int direction,
                          double rank_floor, const int *jac_info)
{
    prof_mark(ctx, PROF_DECIDE);
    const size_t smem = r <= kDecideSmem ? sizeof(double) * (size_t)r : 0;
    static bool attr = false;
    if (!attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_decide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * kDecideSmem)));
        attr = true;
    }
    k_decide<<<1, DB, smem, ctx->stream>>>(s, r, st_bond, p, do_ctrl, chi_override, mlp, bond, N, sweep,
                                        static_cast<const LzState *>(lz_state), res, visit, direction, rank_floor,
                                        jac_info, ctx->mlp_eps_target, ctx->d_status); DMRG_COUNT_LAUNCH();
    prof_mark(ctx, PROF_DECIDE);
    prof_count(ctx, PROF_DECIDE, 0.0, 0.0);
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status launch_ctrl_steps(dmrg_ctx *ctx, int n, const double *S, dmrg_ctrl_state *st, const dmrg_params &p,
                              int *chi_out)
{
    if (n <= 0) return DMRG_OK;
    k_ctrl_steps<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, S, st, p, chi_out); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status launch_entropy(dmrg_ctx *ctx, int n, const double *s, double *S, double *eps)
{
    if (n <= 0) return DMRG_EINVAL;
    k_entropy<<<1, 256, 0, ctx->stream>>>(n, s, S, eps); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg
