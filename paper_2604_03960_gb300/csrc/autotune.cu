// autotune.cu -- on-device autotuner for the launch choices that the hot
// path otherwise takes from fixed heuristics:
//
//   * the tile width (64, 128 or 256 columns) of the 3xTF32 tensor-core GEMM
//     and its split depth (4 or 8 K blocks of 32 per FP32 accumulator, the
//     K extent of a slice), per shape bucket (ceil log2 of M, N and K);
//   * the FP32 Jacobi of the mixed SVD, per size bucket (ceil log2 of the
//     vector count and length): the cluster kernel on 8 or 16 CTAs (which
//     sets its block width b = ceil(r / 2C)), or else the other kernels with
//     their own choices (the grouped kernel's vectors per block pair and
//     groups per CTA; the blocked kernel's block pairs per round, which set
//     its block width, and inner sweeps).
//
// Each candidate is timed with CUDA events on the context's stream after a
// warm-up call; the fastest is kept in the context's table, which the GEMM
// and Jacobi launchers consult before their heuristics.  Tables are saved to
// and loaded from a small JSON file (one entry per line).  Only the launch
// configuration changes: at a given split depth a GEMM gives the same bits
// with any tile width (each output element accumulates its K terms in the
// same order); the split depths on offer bound the FP32 accumulation at or
// below the default's; and the Jacobi converges to the same tolerance.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <string>

namespace dmrg {
namespace {

int clog2(long long v)
{
    int b = 0;
    while ((1LL << b) < v) ++b;
    return b;
}

// uniform values in [-1, 1) from a counter-based hash (timing inputs only)
__global__ void k_fill_uniform(double *x, long long n, unsigned long long seed)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

struct DevScratch {
    void *p = nullptr;
    ~DevScratch() { if (p) cudaFree(p); }
};

}  // namespace

int tune_lookup_bn(const dmrg_ctx *ctx, int M, int N, int K, int *kb)
{
    if (ctx->tune_gemm.empty()) return 0;
    const int lm = clog2(M), ln = clog2(N), lk = clog2(K);
    for (const auto &e : ctx->tune_gemm)
        if (e.lm == lm && e.ln == ln && e.lk == lk) {
            if (kb) *kb = e.kb;
            return e.bn;
        }
    return 0;
}

int tune_lookup_cj(const dmrg_ctx *ctx, int r, int l)
{
    if (ctx->tune_svd.empty()) return -1;
    const int lr = clog2(r), ll = clog2(l);
    for (const auto &e : ctx->tune_svd)
        if (e.lr == lr && e.ll == ll) return e.cj;
    return -1;
}

int tune_lookup_tj(const dmrg_ctx *ctx, int r, int l)
{
    if (ctx->tune_svd.empty()) return -1;
    const int lr = clog2(r), ll = clog2(l);
    for (const auto &e : ctx->tune_svd)
        if (e.lr == lr && e.ll == ll) return e.tj;
    return -1;
}

bool tune_lookup_gjac(const dmrg_ctx *ctx, int r, int l, int *nv, int *groups)
{
    if (ctx->tune_svd.empty()) return false;
    const int lr = clog2(r), ll = clog2(l);
    for (const auto &e : ctx->tune_svd)
        if (e.lr == lr && e.ll == ll && e.nv > 0) {
            *nv = e.nv;
            *groups = e.groups;
            return true;
        }
    return false;
}

bool tune_lookup_svd(const dmrg_ctx *ctx, int r, int l, int *pairs, int *inner)
{
    if (ctx->tune_svd.empty()) return false;
    const int lr = clog2(r), ll = clog2(l);
    for (const auto &e : ctx->tune_svd)
        if (e.lr == lr && e.ll == ll) {
            *pairs = e.pairs;
            *inner = e.inner;
            return true;
        }
    return false;
}

}  // namespace dmrg

using namespace dmrg;

namespace {

template <typename F> dmrg_status time_ms(dmrg_ctx *ctx, int reps, F &&call, float *ms)
{
    DMRG_TRY(call());   // warm-up (and workspace sizing)
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaEvent_t a, b;
    DMRG_CUDA(cudaEventCreate(&a));
    DMRG_CUDA(cudaEventCreate(&b));
    DMRG_CUDA(cudaEventRecord(a, ctx->stream));
    dmrg_status st = DMRG_OK;
    for (int i = 0; i < reps && st == DMRG_OK; ++i) st = call();
    DMRG_CUDA(cudaEventRecord(b, ctx->stream));
    DMRG_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = t / (float)std::max(1, reps);
    return st;
}

}  // namespace

extern "C" dmrg_status dmrg_autotune_gemm(dmrg_ctx *ctx, int n_shapes, const int *M, const int *N, const int *K,
                                          int reps)
{
    if (!ctx || n_shapes < 0 || (n_shapes > 0 && (!M || !N || !K)) || reps < 1) return DMRG_EINVAL;
    for (int i = 0; i < n_shapes; ++i) {
        if (M[i] < 1 || N[i] < 1 || K[i] < 1) return DMRG_EINVAL;
        const size_t na = (size_t)M[i] * K[i], nb = (size_t)K[i] * N[i], nc = (size_t)M[i] * N[i];
        DevScratch buf;
        DMRG_CUDA(cudaMalloc(&buf.p, sizeof(double) * (na + nb + nc)));
        double *A = static_cast<double *>(buf.p), *B = A + na, *Cm = B + nb;
        k_fill_uniform<<<ctx->num_sms, 256, 0, ctx->stream>>>(A, (long long)(na + nb), 0x1234ULL + i); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        const int saved_bn = ctx->tc_bn_override, saved_force = ctx->tc_force, saved_kb = ctx->tc_split_kb;
        ctx->tc_force = 1;
        const int bns[3] = {64, 128, 256}, kbs[2] = {4, 8};
        float ms[2][3] = {};
        dmrg_status st = DMRG_OK;
        for (int b = 0; b < 2 && st == DMRG_OK; ++b)
            for (int c = 0; c < 3 && st == DMRG_OK; ++c) {
                ctx->tc_split_kb = kbs[b];
                ctx->tc_bn_override = bns[c];
                st = time_ms(ctx, reps, [&]() {
                    return gemm(ctx, DMRG_PREC_3XTF32, M[i], N[i], K[i], 1.0, A, K[i], 1, 0, B, N[i], 1, 0, 0.0, Cm,
                                N[i], 1, 0, 1);
                }, &ms[b][c]);
            }
        ctx->tc_bn_override = saved_bn;
        ctx->tc_force = saved_force;
        ctx->tc_split_kb = saved_kb;
        if (st != DMRG_OK) return st;
        int bb = 1, bc = 1;                  // default: 128 columns at depth 8
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 3; ++c)
                if (ms[b][c] < ms[bb][bc]) {
                    bb = b;
                    bc = c;
                }
        dmrg_ctx::TuneGemm e{clog2(M[i]), clog2(N[i]), clog2(K[i]), bns[bc], ms[bb][1], ms[bb][2], kbs[bb], ms[bb][0]};
        auto it = std::find_if(ctx->tune_gemm.begin(), ctx->tune_gemm.end(), [&](const dmrg_ctx::TuneGemm &x) {
            return x.lm == e.lm && x.ln == e.ln && x.lk == e.lk;
        });
        if (it != ctx->tune_gemm.end()) *it = e;
        else ctx->tune_gemm.push_back(e);
    }
    return dmrg_get_status(ctx);
}

extern "C" dmrg_status dmrg_autotune_svd(dmrg_ctx *ctx, int n_sizes, const int *n, int reps)
{
    if (!ctx || n_sizes < 0 || (n_sizes > 0 && !n) || reps < 1) return DMRG_EINVAL;
    static const int kPairs[] = {24, 48, 96, 152};
    static const int kInner[] = {1, 2};
    for (int i = 0; i < n_sizes; ++i) {
        const int m = n[i];
        if (m < 2) return DMRG_EINVAL;
        const size_t nm = (size_t)m * m;
        DevScratch buf;
        DMRG_CUDA(cudaMalloc(&buf.p, sizeof(double) * (4 * nm + m)));
        double *A = static_cast<double *>(buf.p), *U = A + nm, *Vt = U + nm, *s = Vt + nm;
        k_fill_uniform<<<ctx->num_sms, 256, 0, ctx->stream>>>(A, (long long)nm, 0x5678ULL + i); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        const int saved_prec = ctx->svd_prec, saved_pairs = ctx->bjac_pairs, saved_inner = ctx->bjac_inner;
        const int saved_nv = ctx->gjac_nv, saved_groups = ctx->gjac_groups;
        const int saved_cj = ctx->cjac32, saved_fc = ctx->cjac_force_c;
        const int saved_tj = ctx->tjac, saved_tjr = ctx->tjac_min_r;
        const auto saved_table = ctx->tune_svd;
        ctx->tune_svd.clear();   // time the candidates themselves, not an earlier decision
        ctx->svd_prec = 1;
        float best = 0.f;
        int best_p = saved_pairs, best_i = saved_inner, best_nv = 0, best_g = 0, best_cj = 0, best_tj = 0;
        ctx->tjac = 0;            // the candidates below without the tensor-core block form
        dmrg_status st = DMRG_OK;
        auto timed = [&](float *ms) {
            return time_ms(ctx, reps, [&]() {
                int k;
                double S, err;
                dmrg_status e = svd_truncate(ctx, A, m, m, m, 0.0, U, s, Vt, &k, &S, &err);
                return e == DMRG_ENOCONV ? DMRG_OK : e;
            }, ms);
        };
        // the cluster kernel on 8 and on 16 CTAs, where the vectors fit
        // (QR preconditioning leaves r = l = m here)
        if (saved_cj && m >= ctx->cjac_min_r) {
            for (int c : {8, 16}) {
                if (st != DMRG_OK || !cjac32_fits_c(m, m, c)) continue;
                ctx->cjac32 = 1;
                ctx->cjac_force_c = c;
                float ms = 0.f;
                st = timed(&ms);
                if (st == DMRG_OK && (best == 0.f || ms < best)) {
                    best = ms;
                    best_cj = c;
                }
            }
        }
        ctx->cjac32 = 0;          // the other kernels
        ctx->cjac_force_c = 0;
        if (ctx->gjac32 == 2 || (ctx->gjac32 == 1 && (long long)m * m <= kSmemJacFloats)) {
            // grouped kernel: vectors per block pair x groups per CTA
            static const int kNv[] = {16, 32};
            static const int kGroups[] = {1, 2, 4};
            for (int nvc : kNv)
                for (int gc : kGroups) {
                    if (st != DMRG_OK) break;
                    ctx->gjac_nv = nvc;
                    ctx->gjac_groups = gc;
                    float ms = 0.f;
                    st = timed(&ms);
                    if (st == DMRG_OK && (best == 0.f || ms < best)) {
                        best = ms;
                        best_nv = nvc;
                        best_g = gc;
                        best_cj = 0;
                    }
                }
        } else {
            for (int pi : kPairs)
                for (int ii : kInner) {
                    if (st != DMRG_OK) break;
                    ctx->bjac_pairs = pi;
                    ctx->bjac_inner = ii;
                    float ms = 0.f;
                    st = timed(&ms);
                    if (st == DMRG_OK && (best == 0.f || ms < best)) {
                        best = ms;
                        best_p = pi;
                        best_i = ii;
                        best_nv = 0;
                        best_g = 0;
                        best_cj = 0;
                    }
                }
        }
        // the tensor-core block form (Gram blocks and rotations on tcgen05),
        // pairs of 64 and 128 vectors, from 256 vectors on
        if (m >= 256 && tc_available(ctx)) {
            ctx->cjac32 = saved_cj;
            ctx->bjac_pairs = saved_pairs;
            ctx->bjac_inner = saved_inner;
            ctx->tjac_min_r = 2;
            for (int tb : {64, 128}) {
                if (st != DMRG_OK) break;
                ctx->tjac = tb;
                float ms = 0.f;
                st = timed(&ms);
                if (st == DMRG_OK && (best == 0.f || ms < best)) {
                    best = ms;
                    best_tj = tb;
                }
            }
        }
        ctx->tjac = saved_tj;
        ctx->tjac_min_r = saved_tjr;
        if (best_tj) {            // the other kernels' fields keep their defaults
            best_p = saved_pairs;
            best_i = saved_inner;
            best_nv = 0;
            best_g = 0;
            best_cj = 0;
        }
        ctx->svd_prec = saved_prec;
        ctx->bjac_pairs = saved_pairs;
        ctx->bjac_inner = saved_inner;
        ctx->gjac_nv = saved_nv;
        ctx->gjac_groups = saved_groups;
        ctx->cjac32 = saved_cj;
        ctx->cjac_force_c = saved_fc;
        ctx->tune_svd = saved_table;
        if (st != DMRG_OK) return st;
        dmrg_ctx::TuneSvd e{clog2(m), clog2(m), best_p, best_i, best, best_nv, best_g, best_cj, best_tj};
        auto it = std::find_if(ctx->tune_svd.begin(), ctx->tune_svd.end(), [&](const dmrg_ctx::TuneSvd &x) {
            return x.lr == e.lr && x.ll == e.ll;
        });
        if (it != ctx->tune_svd.end()) *it = e;
        else ctx->tune_svd.push_back(e);
    }
    return dmrg_get_status(ctx);
}

extern "C" dmrg_status dmrg_autotune_clear(dmrg_ctx *ctx)
{
    if (!ctx) return DMRG_EINVAL;
    ctx->tune_gemm.clear();
    ctx->tune_svd.clear();
    return DMRG_OK;
}

extern "C" int dmrg_autotune_entries(const dmrg_ctx *ctx, int which)
{
    if (!ctx) return -1;
    return which == 0 ? (int)ctx->tune_gemm.size() : (int)ctx->tune_svd.size();
}

extern "C" dmrg_status dmrg_autotune_save(const dmrg_ctx *ctx, const char *path)
{
    if (!ctx || !path) return DMRG_EINVAL;
    FILE *f = std::fopen(path, "w");
    if (!f) return DMRG_EINVAL;
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess ? prop.name : "unknown";
    for (auto &ch : dev)
        if (ch == '"' || ch == '\\') ch = ' ';
    std::fprintf(f, "{\"format\": \"dmrg-autotune-4\", \"device\": \"%s\",\n \"gemm\": [\n", dev.c_str());
    for (size_t i = 0; i < ctx->tune_gemm.size(); ++i) {
        const auto &e = ctx->tune_gemm[i];
        std::fprintf(f, "  {\"lm\": %d, \"ln\": %d, \"lk\": %d, \"bn\": %d, \"ms128\": %.6g, \"ms256\": %.6g, "
                        "\"kb\": %d, \"ms64\": %.6g}%s\n",
                     e.lm, e.ln, e.lk, e.bn, e.ms128, e.ms256, e.kb, e.ms64, i + 1 < ctx->tune_gemm.size() ? "," : "");
    }
    std::fprintf(f, " ],\n \"svd\": [\n");
    for (size_t i = 0; i < ctx->tune_svd.size(); ++i) {
        const auto &e = ctx->tune_svd[i];
        std::fprintf(f, "  {\"lr\": %d, \"ll\": %d, \"pairs\": %d, \"inner\": %d, \"ms\": %.6g, \"nv\": %d, \"groups\": %d, "
                        "\"cj\": %d, \"tj\": %d}%s\n",
                     e.lr, e.ll, e.pairs, e.inner, e.ms, e.nv, e.groups, e.cj, e.tj,
                     i + 1 < ctx->tune_svd.size() ? "," : "");
    }
    std::fprintf(f, " ]}\n");
    const bool ok = std::fclose(f) == 0;
    return ok ? DMRG_OK : DMRG_EINVAL;
}

extern "C" dmrg_status dmrg_autotune_load(dmrg_ctx *ctx, const char *path)
{
    if (!ctx || !path) return DMRG_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return DMRG_EINVAL;
    std::vector<dmrg_ctx::TuneGemm> g;
    std::vector<dmrg_ctx::TuneSvd> v;
    char line[512];
    bool format_ok = false;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strstr(line, "\"dmrg-autotune-1\"") || std::strstr(line, "\"dmrg-autotune-2\"") ||
            std::strstr(line, "\"dmrg-autotune-3\"") || std::strstr(line, "\"dmrg-autotune-4\""))
            format_ok = true;
        dmrg_ctx::TuneGemm e{};
        dmrg_ctx::TuneSvd t{};
        if (std::sscanf(line, " {\"lm\": %d, \"ln\": %d, \"lk\": %d, \"bn\": %d, \"ms128\": %f, \"ms256\": %f", &e.lm,
                        &e.ln, &e.lk, &e.bn, &e.ms128, &e.ms256) == 6) {
            // format 3 adds the split depth and the 64-column time (absent: the defaults)
            const char *q = std::strstr(line, "\"kb\":");
            if (q && std::sscanf(q, "\"kb\": %d, \"ms64\": %f", &e.kb, &e.ms64) != 2) { std::fclose(f); return DMRG_EINVAL; }
            if ((e.bn != 64 && e.bn != 128 && e.bn != 256) || (e.kb != 0 && e.kb != 4 && e.kb != 8)) {
                std::fclose(f);
                return DMRG_EINVAL;
            }
            g.push_back(e);
        } else if (std::sscanf(line, " {\"lr\": %d, \"ll\": %d, \"pairs\": %d, \"inner\": %d, \"ms\": %f", &t.lr, &t.ll,
                               &t.pairs, &t.inner, &t.ms) == 5) {
            if (t.pairs < 1 || t.inner < 1 || t.inner > 8) { std::fclose(f); return DMRG_EINVAL; }
            // format 2 adds the grouped kernel's choice (absent in format 1: none)
            const char *q = std::strstr(line, "\"nv\":");
            if (q && std::sscanf(q, "\"nv\": %d, \"groups\": %d", &t.nv, &t.groups) == 2) {
                if ((t.nv != 0 && t.nv != 16 && t.nv != 32) || t.groups < 0 || t.groups > 4) {
                    std::fclose(f);
                    return DMRG_EINVAL;
                }
            }
            const char *c = std::strstr(line, "\"cj\":");
            if (c && (std::sscanf(c, "\"cj\": %d", &t.cj) != 1 || (t.cj != -1 && t.cj != 0 && t.cj != 8 && t.cj != 16))) {
                std::fclose(f);
                return DMRG_EINVAL;
            }
            // format 4 adds the tensor-core block form's pair width (absent: not chosen)
            const char *tq = std::strstr(line, "\"tj\":");
            if (tq && (std::sscanf(tq, "\"tj\": %d", &t.tj) != 1 || (t.tj != 0 && t.tj != 64 && t.tj != 128))) {
                std::fclose(f);
                return DMRG_EINVAL;
            }
            v.push_back(t);
        }
    }
    std::fclose(f);
    if (!format_ok) return DMRG_EINVAL;
    ctx->tune_gemm = g;
    ctx->tune_svd = v;
    return DMRG_OK;
}
