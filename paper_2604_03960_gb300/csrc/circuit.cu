// circuit.cu -- circuit simulation with per-bond chi control: the
// circuit-level bond dimension maps of Section 8.
//
// The state is an MPS on N qubits, |0...0> at the start (every bond
// dimension 1).  A layer of two-qubit gates on disjoint neighbouring pairs is
// applied in one pass over the bonds that moves the orthogonality centre
// across every bond (left to right on even layers, right to left on odd):
// at bond k the two-site tensor theta = A_k A_{k+1} takes the layer's gate on
// (k, k+1) if there is one, then the SVD (the FP64 Jacobi of Eq. 20), the
// entropy of the full spectrum (Eq. 5), the truncation and the split with the
// centre moving on.  At a gated bond the bond's controller (EMA -> predictor
// -> PID, Algorithms 1-2 with Eqs. 8 and 16) takes a step and its chi bounds
// the retained dimension; a bond without a gate only moves the centre (its
// spectrum is that of the previous layer, so nothing is cut but values below
// the eps_trunc threshold).  The bond dimensions after each layer form the
// map chi_i^(l); a map recorded by one run can be replayed by the next (warm
// start), which then skips the controller's transient.
#include "common.cuh"
#include "ctrl.cuh"

#include <algorithm>
#include <vector>

namespace dmrg {
namespace {

// theta2[a][q'][b] = sum_q G[q'][q] theta[a][q][b], q = 2 s1 + s2
__global__ void k_gate4(const double *__restrict__ theta, const double *__restrict__ G, int cl, int cr,
                        double *__restrict__ out)
{
    __shared__ double g[16];
    if (threadIdx.x < 16) g[threadIdx.x] = G[threadIdx.x];
    __syncthreads();
    const long long total = (long long)cl * cr;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long a = e / cr, b = e % cr;
        double in[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) in[q] = theta[(a * 4 + q) * cr + b];
#pragma unroll
        for (int qo = 0; qo < 4; ++qo) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc = fma(g[4 * qo + q], in[q], acc);
            out[(a * 4 + qo) * cr + b] = acc;
        }
    }
}

// |0> on every site: A_i[0][0][0] = 1 (bond dimensions 1)
__global__ void k_zero_state(double *const *A, int N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        A[i][0] = 1.0;
        A[i][1] = 0.0;
    }
}

int grid_for(long long n, int num_sms)
{
    long long b = (n + 255) / 256;
    if (b > 4LL * num_sms) b = 4LL * num_sms;
    return (int)(b < 1 ? 1 : b);
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace dmrg

using namespace dmrg;

struct dmrg_circ {
    dmrg_ctx *ctx = nullptr;
    int N = 0;
    dmrg_params p{};
    std::vector<int> chi, cap;
    DevBuf arena;
    std::vector<double *> A;
    double **A_dev = nullptr;       // device copy of the site pointers
    dmrg_ctrl_state *ctrl = nullptr;
    double *theta = nullptr, *theta2 = nullptr, *U = nullptr, *s = nullptr, *Vt = nullptr, *G = nullptr;
    void *svdw = nullptr;
    BondResult *d_res = nullptr, *h_res = nullptr;
    int *d_info = nullptr;
    int layers = 0;
};

extern "C" {

dmrg_status dmrg_circ_create(dmrg_ctx *ctx, int N, const dmrg_params *p, dmrg_circ **out)
{
    if (!ctx || !p || !out || N < 2 || N > 62 || p->chi_max < 1 || p->chi_min < 1 || p->chi_min > p->chi_max)
        return DMRG_EINVAL;
    // the per-bond rules of Algorithms 1-2 and the fixed / threshold rules
    if (p->ctrl != DMRG_CTRL_PID && p->ctrl != DMRG_CTRL_DIRECT && p->ctrl != DMRG_CTRL_FIXED &&
        p->ctrl != DMRG_CTRL_THRESHOLD)
        return DMRG_EINVAL;
    *out = nullptr;
    dmrg_circ *c = new (std::nothrow) dmrg_circ();
    if (!c) return DMRG_ENOMEM;
    c->ctx = ctx;
    c->N = N;
    c->p = *p;
    if (c->p.jacobi_max_sweeps <= 0) c->p.jacobi_max_sweeps = 60;
    c->chi.assign(N + 1, 1);
    c->cap.resize(N + 1);
    for (int i = 0; i <= N; ++i) {
        long long v = p->chi_max;
        v = std::min(v, i < 40 ? (1LL << i) : v);
        v = std::min(v, N - i < 40 ? (1LL << (N - i)) : v);
        c->cap[i] = (int)v;
    }
    size_t total = 0, th = 1, um = 1, vm = 1, sm = 1, sw = 1;
    std::vector<size_t> off(N);
    for (int i = 0; i < N; ++i) { off[i] = total; total += al(sizeof(double) * (size_t)c->cap[i] * 2 * c->cap[i + 1]); }
    for (int k = 0; k + 1 < N; ++k) {
        const size_t m = 2 * (size_t)c->cap[k], n = 2 * (size_t)c->cap[k + 2];
        const size_t r = std::min(m, n), l = std::max(m, n);
        th = std::max(th, m * n);
        um = std::max(um, m * r);
        vm = std::max(vm, r * n);
        sm = std::max(sm, r);
        sw = std::max(sw, svd_work_bytes((int)r, (int)l));
    }
    const size_t o_ptr = total; total += al(sizeof(double *) * N);
    const size_t o_ctrl = total; total += al(sizeof(dmrg_ctrl_state) * (N - 1));
    const size_t o_th = total; total += al(sizeof(double) * th);
    const size_t o_th2 = total; total += al(sizeof(double) * th);
    const size_t o_u = total; total += al(sizeof(double) * um);
    const size_t o_s = total; total += al(sizeof(double) * sm);
    const size_t o_vt = total; total += al(sizeof(double) * vm);
    const size_t o_g = total; total += al(sizeof(double) * 16 * (size_t)N);
    const size_t o_sw = total; total += al(sw);
    const size_t o_res = total; total += al(sizeof(BondResult));
    const size_t o_info = total; total += al(sizeof(int) * 4);
    if (c->arena.ensure(total) != DMRG_OK) { delete c; return DMRG_ENOMEM; }
    char *b = c->arena.as<char>();
    c->A.resize(N);
    for (int i = 0; i < N; ++i) c->A[i] = reinterpret_cast<double *>(b + off[i]);
    c->A_dev = reinterpret_cast<double **>(b + o_ptr);
    c->ctrl = reinterpret_cast<dmrg_ctrl_state *>(b + o_ctrl);
    c->theta = reinterpret_cast<double *>(b + o_th);
    c->theta2 = reinterpret_cast<double *>(b + o_th2);
    c->U = reinterpret_cast<double *>(b + o_u);
    c->s = reinterpret_cast<double *>(b + o_s);
    c->Vt = reinterpret_cast<double *>(b + o_vt);
    c->G = reinterpret_cast<double *>(b + o_g);
    c->svdw = b + o_sw;
    c->d_res = reinterpret_cast<BondResult *>(b + o_res);
    c->d_info = reinterpret_cast<int *>(b + o_info);
    if (cudaMallocHost(&c->h_res, sizeof(BondResult)) != cudaSuccess) { c->arena.release(); delete c; return DMRG_ENOMEM; }
    cudaStream_t st = ctx->stream;
    auto fail = [&](dmrg_status e) {
        cudaStreamSynchronize(st);
        cudaFreeHost(c->h_res);
        c->arena.release();
        delete c;
        return e;
    };
    if (cudaMemcpyAsync(c->A_dev, c->A.data(), sizeof(double *) * N, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(DMRG_ECUDA);
    k_zero_state<<<(N + 127) / 128, 128, 0, st>>>(c->A_dev, N); DMRG_COUNT_LAUNCH();
    if (cudaGetLastError() != cudaSuccess) return fail(DMRG_ECUDA);
    dmrg_status e = launch_init_ctrl(ctx, c->ctrl, N - 1, p->chi_min);
    if (e != DMRG_OK) return fail(e);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(DMRG_ECUDA);
    *out = c;
    return DMRG_OK;
}

void dmrg_circ_destroy(dmrg_circ *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->ctx->stream);
    if (c->h_res) cudaFreeHost(c->h_res);
    c->arena.release();
    delete c;
}

dmrg_status dmrg_circ_apply_layer(dmrg_circ *c, int n_gates, const int *pos_host, const double *gates_host,
                                  const int *chi_warm_host, int *chi_row_host, double *S_row_host)
{
    if (!c || n_gates < 0 || (n_gates > 0 && (!pos_host || !gates_host))) return DMRG_EINVAL;
    const int N = c->N;
    if (n_gates > N / 2) return DMRG_EINVAL;
    std::vector<int> gate_at(N - 1, -1);
    for (int g = 0; g < n_gates; ++g) {
        const int q = pos_host[g];
        // disjoint neighbouring pairs only (a brickwork layer)
        if (q < 0 || q >= N - 1 || gate_at[q] >= 0 || (q > 0 && gate_at[q - 1] >= 0) ||
            (q + 1 < N - 1 && gate_at[q + 1] >= 0))
            return DMRG_EINVAL;
        gate_at[q] = g;
    }
    if (chi_warm_host)
        for (int b = 0; b < N - 1; ++b)
            if (chi_warm_host[b] < 1) return DMRG_EINVAL;
    dmrg_ctx *ctx = c->ctx;
    cudaStream_t st = ctx->stream;
    if (n_gates > 0)
        DMRG_CUDA(cudaMemcpyAsync(c->G, gates_host, sizeof(double) * 16 * (size_t)n_gates, cudaMemcpyHostToDevice, st));
    const int go_right = (c->layers % 2 == 0);
    for (int step = 0; step < N - 1; ++step) {
        const int k = go_right ? step : N - 2 - step;
        const int cl = c->chi[k], cm = c->chi[k + 1], cr = c->chi[k + 2];
        const int m = 2 * cl, n = 2 * cr, r = std::min(m, n);
        DMRG_TRY(gemm_f64(st, m, n, cm, 1.0, c->A[k], cm, 1, 0, c->A[k + 1], n, 1, 0, 0.0, c->theta, n, 1, 0, 1));
        const double *th = c->theta;
        const bool gated = gate_at[k] >= 0;
        if (gated) {
            k_gate4<<<grid_for((long long)cl * cr, ctx->num_sms), 256, 0, st>>>(c->theta, c->G + 16 * gate_at[k], cl,
                                                                                cr, c->theta2);
            DMRG_COUNT_LAUNCH();
            DMRG_CUDA(cudaGetLastError());
            th = c->theta2;
        }
        DMRG_TRY(svd_jacobi(ctx, th, m, n, c->U, c->s, c->Vt, c->svdw, c->p.jacobi_max_sweeps, c->d_info));
        // gated: the controller's step (or the warm map); ungated: a gauge move
        int override = 0, do_ctrl = 0;
        if (!gated) override = c->p.chi_max;
        else if (chi_warm_host) override = chi_warm_host[k];
        else do_ctrl = 1;
        DMRG_TRY(launch_decide(ctx, c->s, r, c->ctrl + k, c->p, do_ctrl, override, nullptr, k, N, c->layers, nullptr,
                               c->d_res, nullptr, go_right ? 1 : -1, (double)r * 2.220446049250313e-16, c->d_info));
        DMRG_CUDA(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(BondResult), cudaMemcpyDeviceToHost, st));
        DMRG_CUDA(cudaStreamSynchronize(st));
        const int kk = c->h_res->k;
        if (kk < 1 || kk > r || kk > c->cap[k + 1]) return DMRG_ENAN;
        DMRG_TRY(launch_split(ctx, c->U, c->s, c->Vt, m, n, r, c->d_res, go_right, c->A[k], c->A[k + 1], kk));
        c->chi[k + 1] = kk;
        if (S_row_host) S_row_host[k] = gated ? c->h_res->S : 0.0;
    }
    if (chi_row_host)
        for (int b = 0; b < N - 1; ++b) chi_row_host[b] = c->chi[b + 1];
    c->layers++;
    dmrg_status ds = dmrg_get_status(ctx);
    if (ds != DMRG_OK && ds != DMRG_ENOCONV) return ds;
    return DMRG_OK;
}

dmrg_status dmrg_circ_state(dmrg_circ *c, double *psi_dev)
{
    if (!c || !psi_dev || c->N > 22) return DMRG_EINVAL;
    const int N = c->N;
    dmrg_ctx *ctx = c->ctx;
    cudaStream_t st = ctx->stream;
    const size_t dim = (size_t)1 << N;
    DMRG_TRY(ctx->work3.ensure(sizeof(double) * dim));
    double *tmp = ctx->work3.as<double>();
    // T (rows x chi_i) <- T A_i viewed as (rows x chi_i) (chi_i x 2 chi_{i+1});
    // the buffers alternate so that the last product lands in psi_dev
    double *bufs[2] = {psi_dev, tmp};
    int cur = (N % 2 == 0) ? 1 : 0;           // buffer that receives step 0's product
    DMRG_CUDA(cudaMemcpyAsync(bufs[cur], c->A[0], sizeof(double) * 2 * c->chi[1], cudaMemcpyDeviceToDevice, st));
    size_t rows = 2;
    for (int i = 1; i < N; ++i) {
        const int ci = c->chi[i], cn = c->chi[i + 1];
        DMRG_TRY(gemm_f64(st, (int)rows, 2 * cn, ci, 1.0, bufs[cur], ci, 1, 0, c->A[i], 2LL * cn, 1, 0, 0.0,
                          bufs[cur ^ 1], 2LL * cn, 1, 0, 1));
        cur ^= 1;
        rows *= 2;
    }
    DMRG_CUDA(cudaStreamSynchronize(st));
    return cur == 0 ? DMRG_OK : DMRG_ECUDA;
}

}  // extern "C"
