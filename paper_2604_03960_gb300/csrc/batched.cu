// batched.cu -- many independent SVD + entropy + truncation problems in one
// launch (the uneven isolated-SVD batch): one CTA per matrix, each running the
// one-sided Jacobi iteration of jacobi.cu on its own matrix with only
// __syncthreads between rounds, so the batch fills the GPU without grid
// barriers.  FP64, or FP32 for the mixed form.  The call performs no host
// synchronisation, so once a first call has sized the workspace the launch
// sequence can be captured in a CUDA graph (dmrg_graph_*).
#include "common.cuh"

#include <algorithm>

namespace dmrg {
namespace {

struct BDesc {
    int m, n, r, l, tr, pad;
    long long off_in, off_U, off_s, off_Vt, off_X, off_V;
};

constexpr int kBT = 512;   // threads per matrix

template <typename T> __device__ __forceinline__ T wsum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kBT) k_svd_batched(const BDesc *__restrict__ desc, const double *__restrict__ theta,
                                                    T *__restrict__ work, double *__restrict__ U,
                                                    double *__restrict__ s, double *__restrict__ Vt, int max_sweeps,
                                                    double tol_unit, int tol_by_l, double small, int *info,
                                                    int *status)
{
    __shared__ BDesc d;
    __shared__ unsigned rot_count;
    __shared__ double red[32];
    if (threadIdx.x == 0) d = desc[blockIdx.x];
    __syncthreads();
    const int m = d.m, n = d.n, r = d.r, l = d.l, tr = d.tr;
    T *X = work + d.off_X, *V = work + d.off_V;
    const double *A = theta + d.off_in;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBT / 32;
    // rotate while the cosine exceeds l eps (FP64) or 1e-5 (FP32)
    const double tol = tol_by_l ? tol_unit * (double)(l > 16 ? l : 16) : tol_unit;
    // load: vectors are the columns (tr = 0) or the rows (tr = 1) of A
    double f2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)r * l; e += kBT) {
        const int i = (int)(e / l), t = (int)(e % l);
        const double v = tr ? A[(long long)i * n + t] : A[(long long)t * n + i];
        X[e] = (T)v;
        f2 += v * v;
    }
    for (long long e = threadIdx.x; e < (long long)r * r; e += kBT) V[e] = (e / r == e % r) ? (T)1 : (T)0;
    f2 = block_sum(f2, red);
    const double floor2 = small * small * f2;
    __syncthreads();
    const int rp = r + (r & 1), npairs = rp / 2;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rot_count = 0;
        __syncthreads();
        for (int t = 0; t < rp - 1; ++t) {
            for (int p = warp; p < npairs; p += nw) {
                int i, j;
                if (p == 0) { i = rp - 1; j = t; } else { i = (t + p) % (rp - 1); j = (t - p + rp - 1) % (rp - 1); }
                if (i >= r || j >= r) continue;
                T *xi = X + (long long)i * l, *xj = X + (long long)j * l;
                T a = 0, b = 0, g = 0;
                for (int k = lane; k < l; k += 32) {
                    const T u = xi[k], v = xj[k];
                    a = fma(u, u, a); b = fma(v, v, b); g = fma(u, v, g);
                }
                a = wsum(a); b = wsum(b); g = wsum(g);
                if (!((double)a > floor2 && (double)b > floor2)) continue;
                if (!(fabs((double)g) > tol * sqrt((double)a) * sqrt((double)b))) continue;
                T c, sn;
                {
                    const T zeta = (b - a) / (T(2) * g);
                    const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                    c = T(1) / sqrt(T(1) + tt * tt);
                    sn = c * tt;
                }
                for (int k = lane; k < l; k += 32) {
                    const T u = xi[k], v = xj[k];
                    xi[k] = c * u - sn * v;
                    xj[k] = sn * u + c * v;
                }
                T *vi = V + (long long)i * r, *vj = V + (long long)j * r;
                for (int k = lane; k < r; k += 32) {
                    const T u = vi[k], v = vj[k];
                    vi[k] = c * u - sn * v;
                    vj[k] = sn * u + c * v;
                }
                if (lane == 0) atomicAdd(&rot_count, 1u);
            }
            __syncthreads();
        }
        const unsigned tot = rot_count;
        __syncthreads();
        if (tot == 0u) {
            converged = true;
            ++sweep;
            break;
        }
    }
    if (threadIdx.x == 0) {
        info[blockIdx.x] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
    // norms into the s slot (unsorted), then rank and write the factors
    double *sb = s + d.off_s;
    for (int i = warp; i < r; i += nw) {
        const T *x = X + (long long)i * l;
        double a = 0.0;
        for (int k = lane; k < l; k += 32) a = fma((double)x[k], (double)x[k], a);
        a = wsum(a);
        if (lane == 0) sb[i] = sqrt(a);
    }
    __syncthreads();
    // rank by counting (descending, ties by index), one thread per vector;
    // the permutation is kept in the spare workspace after V
    int *perm = reinterpret_cast<int *>(V + (long long)r * r) + 2;
    for (int i = threadIdx.x; i < r; i += kBT) {
        const double v = sb[i];
        int rank = 0;
        for (int j = 0; j < r; ++j) {
            const double w = sb[j];
            rank += (w > v) || (w == v && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    double *Ub = U + d.off_U, *Vb = Vt + d.off_Vt;
    // one warp per output index: sign convention "largest |U[:, c]| positive"
    for (int c = warp; c < r; c += nw) {
        const int i = perm[c];
        const double sig = sb[i];
        const double inv = sig > 0.0 ? 1.0 / sig : 0.0;
        const T *usrc = tr ? (V + (long long)i * r) : (X + (long long)i * l);
        const double usc = tr ? 1.0 : inv;
        double best = -1.0;
        int bi = 0;
        for (int k = lane; k < m; k += 32) {
            const double a = fabs((double)usrc[k]);
            if (a > best) { best = a; bi = k; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const double sign = ((double)usrc[bi] < 0.0) ? -1.0 : 1.0;
        for (int k = lane; k < m; k += 32) Ub[(long long)k * r + c] = sign * usc * (double)usrc[k];
        const T *vsrc = tr ? (X + (long long)i * l) : (V + (long long)i * r);
        const double vsc = tr ? inv : 1.0;
        for (int k = lane; k < n; k += 32) Vb[(long long)c * n + k] = sign * vsc * (double)vsrc[k];
    }
    __syncthreads();
    // sorted singular values back into the s slot
    double *tmp = reinterpret_cast<double *>(X);   // X no longer needed
    for (int c = threadIdx.x; c < r; c += kBT) tmp[c] = sb[perm[c]];
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += kBT) sb[c] = tmp[c];
}

// entropy, truncation error and k for every matrix (one CTA each)
// (rank floor: floor_unit * r * s_0 when floor_by_r, else floor_unit * s_0)
__global__ void k_decide_batched(const BDesc *__restrict__ desc, const double *__restrict__ s, int chi_max, double eps,
                                 double floor_unit, int floor_by_r, int *k_out, double *S_out, double *err_out)
{
    __shared__ double sh[32];
    const BDesc d = desc[blockIdx.x];
    const double *sb = s + d.off_s;
    const int r = d.r;
    double z = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x) z += sb[j] * sb[j];
    const double Z = block_sum(z, sh);
    double en = 0.0, cr = 0.0, ca = 0.0;
    const double rank_floor = floor_by_r ? floor_unit * (double)r : floor_unit;
    const double nz = sqrt(Z), rtol = rank_floor * (r > 0 ? sb[0] : 0.0);
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double pj = Z > 0.0 ? sb[j] * sb[j] / Z : 0.0;
        if (pj > 0.0) en -= pj * log(pj);
        if (sb[j] > rtol) cr += 1.0;
        if (nz > 0.0 && sb[j] / nz > eps) ca += 1.0;
    }
    const double S = block_sum(en, sh);
    const int rank = (int)block_sum(cr, sh), above = (int)block_sum(ca, sh);
    int k = chi_max;
    if (rank < k) k = rank;
    if (above < k) k = above;
    if (k < 1) k = 1;
    double t = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x)
        if (j >= k) t += Z > 0.0 ? sb[j] * sb[j] / Z : 0.0;
    const double T = block_sum(t, sh);
    if (threadIdx.x == 0) {
        k_out[blockIdx.x] = k;
        S_out[blockIdx.x] = S;
        err_out[blockIdx.x] = sqrt(fmax(T, 0.0));
    }
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace dmrg

using namespace dmrg;

extern "C" dmrg_status svd_truncate_batched(dmrg_ctx *ctx, int prec, int batch, const int *m, const int *n,
                                            const double *theta_dev, const long long *off_in, double *U_dev,
                                            const long long *off_U, double *s_dev, const long long *off_s,
                                            double *Vt_dev, const long long *off_Vt, int chi_max, double eps,
                                            int *k_dev, double *S_dev, double *err_dev)
{
    if (!ctx || batch < 1 || !m || !n || !theta_dev || !off_in || !U_dev || !off_U || !s_dev || !off_s || !Vt_dev ||
        !off_Vt || chi_max < 1 || !(eps >= 0.0) || !k_dev || !S_dev || !err_dev)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && prec != DMRG_PREC_3XTF32) return DMRG_EUNSUPPORTED;
    const size_t esz = prec == DMRG_PREC_FP64 ? sizeof(double) : sizeof(float);
    std::vector<BDesc> h(batch);
    long long wo = 0;
    for (int b = 0; b < batch; ++b) {
        if (m[b] < 1 || n[b] < 1) return DMRG_EINVAL;
        BDesc &d = h[b];
        d.m = m[b];
        d.n = n[b];
        d.tr = m[b] < n[b];
        d.r = std::min(m[b], n[b]);
        d.l = std::max(m[b], n[b]);
        d.pad = 0;
        d.off_in = off_in[b];
        d.off_U = off_U[b];
        d.off_s = off_s[b];
        d.off_Vt = off_Vt[b];
        // X needs max(r*l, r) elements (it also holds the sorted values), V r*r plus the permutation
        const long long xs = std::max<long long>((long long)d.r * d.l, 2LL * d.r);
        d.off_X = wo;
        wo += (long long)(al256(esz * xs) / esz);
        d.off_V = wo;
        wo += (long long)(al256(esz * ((long long)d.r * d.r) + sizeof(int) * (d.r + 8) + 16) / esz);
    }
    const size_t need_desc = al256(sizeof(BDesc) * batch), need_info = al256(sizeof(int) * batch);
    const size_t need = need_desc + need_info + esz * (size_t)wo;
    DMRG_TRY(ctx->work4.ensure(need));
    if ((size_t)batch * sizeof(BDesc) > ctx->pinned_desc_bytes) {
        if (ctx->pinned_desc) cudaFreeHost(ctx->pinned_desc);
        ctx->pinned_desc = nullptr;
        ctx->pinned_desc_bytes = 0;
        DMRG_CUDA(cudaMallocHost(&ctx->pinned_desc, sizeof(BDesc) * batch));
        ctx->pinned_desc_bytes = sizeof(BDesc) * batch;
    }
    std::memcpy(ctx->pinned_desc, h.data(), sizeof(BDesc) * batch);
    char *base = ctx->work4.as<char>();
    BDesc *ddesc = reinterpret_cast<BDesc *>(base);
    int *info = reinterpret_cast<int *>(base + need_desc);
    void *work = base + need_desc + need_info;
    DMRG_CUDA(cudaMemcpyAsync(ddesc, ctx->pinned_desc, sizeof(BDesc) * batch, cudaMemcpyHostToDevice, ctx->stream));
    const int sweeps = ctx->jacobi_max_sweeps;
    if (prec == DMRG_PREC_FP64) {
        k_svd_batched<double><<<batch, kBT, 0, ctx->stream>>>(ddesc, theta_dev, static_cast<double *>(work), U_dev,
                                                              s_dev, Vt_dev, sweeps, 2.220446049250313e-16, 1,
                                                              16.0 * 2.220446049250313e-16, info, ctx->d_status); DMRG_COUNT_LAUNCH();
        k_decide_batched<<<batch, 256, 0, ctx->stream>>>(ddesc, s_dev, chi_max, eps, 2.220446049250313e-16, 1, k_dev,
                                                  S_dev, err_dev); DMRG_COUNT_LAUNCH();
    } else {
        k_svd_batched<float><<<batch, kBT, 0, ctx->stream>>>(ddesc, theta_dev, static_cast<float *>(work), U_dev, s_dev,
                                                             Vt_dev, sweeps, 1e-5, 0, 1.1920928955078125e-07, info,
                                                             ctx->d_status); DMRG_COUNT_LAUNCH();
        k_decide_batched<<<batch, 256, 0, ctx->stream>>>(ddesc, s_dev, chi_max, eps, 2.384185791015625e-07, 0, k_dev,
                                                         S_dev, err_dev); DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_begin(dmrg_ctx *ctx)
{
    if (!ctx || !ctx->stream) return DMRG_EINVAL;   // the legacy default stream cannot be captured
    DMRG_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_end(dmrg_ctx *ctx, void **graph_exec)
{
    if (!ctx || !graph_exec) return DMRG_EINVAL;
    cudaGraph_t g = nullptr;
    DMRG_CUDA(cudaStreamEndCapture(ctx->stream, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return DMRG_ECUDA;
    *graph_exec = ex;
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_launch(dmrg_ctx *ctx, void *graph_exec)
{
    if (!ctx || !graph_exec) return DMRG_EINVAL;
    DMRG_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), ctx->stream));
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_destroy(void *graph_exec)
{
    if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
    return DMRG_OK;
}
