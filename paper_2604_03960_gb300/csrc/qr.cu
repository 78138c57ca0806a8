// qr.cu -- QR preconditioning of the FP32 one-sided Jacobi.
//
// The Jacobi rotates c vectors of length l, the rows of X (c x l, row-major).
// Replacing X by the R factor of its QR decomposition, X = Q R (Householder
// reflectors acting on the row index), changes neither the singular values
// nor the left singular vectors of X^T -- the directions the Jacobi returns --
// because X^T = R^T Q^T with Q orthogonal.  One-sided Jacobi on the rows of
// R converges in a few sweeps where the rows of X need many: for
// U diag(s) V^T with Haar factors and a graded spectrum, 8 sweeps instead of
// 20-27 (Drmac and Veselic's preconditioned Jacobi SVD, LAPACK xGEJSV).
//
// Blocked Householder QR in FP32 (the Jacobi's own precision: the reflectors
// perturb X by O(u |X|), the size of the FP32 rounding it already carries):
//   panel   -- one CTA factors rows k..c-1 x columns k..k+b-1 in shared memory,
//              writes R's block, the reflectors V (rows x b) and the
//              compact-WY factor T (H_0 ... H_{b-1} = I - V T V^T);
//   trailing -- X[k:, k+b:] <- (I - V T^T V^T) X[k:, k+b:], 32 columns per CTA.
#include "common.cuh"

#include <algorithm>

namespace dmrg {
namespace {

constexpr int kQrB = 16;          // panel width
constexpr int kQrPanelThreads = 512;
constexpr int kQrTrailThreads = 256;

__device__ __forceinline__ float wsumf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kQrPanelThreads) k_qr_panel(float *__restrict__ X, int c, int l, int k, int bw,
                                                              float *__restrict__ V, float *__restrict__ T)
{
    extern __shared__ float P[];                   // rows x bw, row-major
    __shared__ double red[32];
    __shared__ float wv[kQrB], sbeta[kQrB], G[kQrB][kQrB + 1];
    __shared__ float sv0, salpha;
    const int rows = c - k, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kQrPanelThreads / 32;
    for (int e = tid; e < rows * bw; e += kQrPanelThreads) {
        const int i = e / bw, j = e % bw;
        P[e] = X[(long long)(k + i) * l + k + j];
    }
    // columns bw..kQrB-1 of V are unused by this panel: zero them (the
    // trailing update multiplies them by zero entries of T)
    for (int e = tid; e < rows * (kQrB - bw); e += kQrPanelThreads)
        V[(long long)(e / (kQrB - bw)) * kQrB + bw + e % (kQrB - bw)] = 0.f;
    __syncthreads();
    for (int j = 0; j < bw; ++j) {
        // |column j below the diagonal|^2, FP64 accumulation
        double a = 0.0;
        for (int i = j + tid; i < rows; i += kQrPanelThreads) {
            const double x = P[i * bw + j];
            a = fma(x, x, a);
        }
        a = block_sum(a, red);
        if (tid == 0) {
            const float x0 = P[j * bw + j];
            const double nrm = sqrt(a);
            float beta = 0.f, v0 = 1.f, alpha = x0;
            if (rows - j > 1 && nrm > 0.0 && a > (double)x0 * x0) {
                alpha = x0 >= 0.f ? (float)-nrm : (float)nrm;
                v0 = x0 - alpha;
                beta = -1.f / (alpha * v0);           // 2 / (v^T v)
            }
            sbeta[j] = beta;
            sv0 = v0;
            salpha = alpha;
        }
        __syncthreads();
        const float beta = sbeta[j], v0 = sv0;
        // reflector j: v = (v0, P[j+1:, j]); stored in column j of V
        for (int i = tid; i < rows; i += kQrPanelThreads)
            V[(long long)i * kQrB + j] = i < j ? 0.f : (i == j ? v0 : P[i * bw + j]);
        if (beta != 0.f) {
            // w_q = v^T P[j:, q] for the columns q > j of the panel (one warp per column)
            for (int q = j + 1 + warp; q < bw; q += nw) {
                float s = 0.f;
                for (int i = j + lane; i < rows; i += 32) s = fmaf(i == j ? v0 : P[i * bw + j], P[i * bw + q], s);
                s = wsumf(s);
                if (lane == 0) wv[q] = s;
            }
            __syncthreads();
            const int nq = bw - j - 1;
            for (int e = tid; e < (rows - j) * nq; e += kQrPanelThreads) {
                const int i = j + e / nq, q = j + 1 + e % nq;
                const float vi = i == j ? v0 : P[i * bw + j];
                P[i * bw + q] -= beta * vi * wv[q];
            }
        }
        __syncthreads();
        // column j of R: alpha on the diagonal, zeros below
        for (int i = j + tid; i < rows; i += kQrPanelThreads) P[i * bw + j] = (i == j) ? salpha : 0.f;
        __syncthreads();
    }
    // compact WY: T upper triangular, T[j][j] = beta_j,
    // T[0:j, j] = -beta_j T[0:j, 0:j] (V[:, 0:j]^T v_j)
    for (int pq = warp; pq < bw * bw; pq += nw) {
        const int p = pq / bw, q = pq % bw;
        if (p >= q) continue;
        float s = 0.f;
        for (int i = q + lane; i < rows; i += 32) s = fmaf(V[(long long)i * kQrB + p], V[(long long)i * kQrB + q], s);
        s = wsumf(s);
        if (lane == 0) G[p][q] = s;
    }
    __syncthreads();
    if (tid == 0) {
        float Tl[kQrB][kQrB];
        for (int p = 0; p < kQrB; ++p)
            for (int q = 0; q < kQrB; ++q) Tl[p][q] = 0.f;
        for (int j = 0; j < bw; ++j) {
            Tl[j][j] = sbeta[j];
            for (int p = 0; p < j; ++p) {
                float s = 0.f;
                for (int q = p; q < j; ++q) s = fmaf(Tl[p][q], G[q][j], s);
                Tl[p][j] = -sbeta[j] * s;
            }
        }
        for (int p = 0; p < kQrB; ++p)
            for (int q = 0; q < kQrB; ++q) T[p * kQrB + q] = Tl[p][q];
    }
    for (int e = tid; e < rows * bw; e += kQrPanelThreads) {
        const int i = e / bw, j = e % bw;
        X[(long long)(k + i) * l + k + j] = P[e];
    }
}

// X[k:, p] <- X[k:, p] - V (T^T (V^T X[k:, p])) for the 32 columns p of this CTA
__global__ void __launch_bounds__(kQrTrailThreads) k_qr_trail(float *__restrict__ X, int c, int l, int k, int bw,
                                                              const float *__restrict__ V, const float *__restrict__ T)
{
    constexpr int nw = kQrTrailThreads / 32;
    __shared__ float Ws[nw][kQrB][33];
    __shared__ float Z[kQrB][33];
    const int rows = c - k, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = k + bw + blockIdx.x * 32 + lane;
    const bool live = p < l;
    float acc[kQrB];
#pragma unroll
    for (int j = 0; j < kQrB; ++j) acc[j] = 0.f;
    for (int i = warp; i < rows; i += nw) {
        const float x = live ? X[(long long)(k + i) * l + p] : 0.f;
        const float *vi = V + (long long)i * kQrB;
#pragma unroll
        for (int j = 0; j < kQrB; ++j) acc[j] = fmaf(vi[j], x, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kQrB; ++j) Ws[warp][j][lane] = acc[j];
    __syncthreads();
    // W = sum over warps; Z = T^T W  (Z[j] = sum_{t <= j} T[t][j] W[t])
    if (warp == 0) {
        float w[kQrB];
#pragma unroll
        for (int j = 0; j < kQrB; ++j) {
            float s = 0.f;
            for (int q = 0; q < nw; ++q) s += Ws[q][j][lane];
            w[j] = s;
        }
#pragma unroll
        for (int j = 0; j < kQrB; ++j) {
            float s = 0.f;
#pragma unroll
            for (int t = 0; t <= j; ++t) s = fmaf(T[t * kQrB + j], w[t], s);
            Z[j][lane] = (j < bw) ? s : 0.f;
        }
    }
    __syncthreads();
    if (!live) return;
    for (int i = warp; i < rows; i += nw) {
        const float *vi = V + (long long)i * kQrB;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kQrB; ++j) s = fmaf(vi[j], Z[j][lane], s);
        X[(long long)(k + i) * l + p] -= s;
    }
}

}  // namespace

size_t qr32_work_bytes(int c)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(sizeof(float) * (size_t)c * kQrB) + al(sizeof(float) * kQrB * kQrB);
}

// In-place QR of X (c x l, row-major FP32): X <- R.  `work` holds
// qr32_work_bytes(c) bytes.  Serves c up to the panel's shared-memory limit
// (c * 16 floats <= 200 KB, c <= 3200); returns DMRG_EUNSUPPORTED beyond.
dmrg_status qr_precondition32(dmrg_ctx *ctx, float *X, int c, int l, void *work)
{
    if (c <= 1 || l <= 0) return DMRG_OK;
    const size_t smem_max = (size_t)c * kQrB * sizeof(float);
    if (smem_max > 200 * 1024) return DMRG_EUNSUPPORTED;
    static size_t attr = 0;
    if (attr < smem_max) {
        DMRG_CUDA(cudaFuncSetAttribute(k_qr_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = 200 * 1024;
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    float *V = static_cast<float *>(work);
    float *T = reinterpret_cast<float *>(static_cast<char *>(work) + al(sizeof(float) * (size_t)c * kQrB));
    const int kmax = std::min(c - 1, l);          // reflectors 0..kmax-1
    for (int k = 0; k < kmax; k += kQrB) {
        const int bw = std::min(kQrB, kmax - k);
        const size_t smem = (size_t)(c - k) * bw * sizeof(float);
        k_qr_panel<<<1, kQrPanelThreads, smem, ctx->stream>>>(X, c, l, k, bw, V, T); DMRG_COUNT_LAUNCH();
        const int ncols = l - (k + bw);
        if (ncols > 0) {
            k_qr_trail<<<(ncols + 31) / 32, kQrTrailThreads, 0, ctx->stream>>>(X, c, l, k, bw, V, T);
            DMRG_COUNT_LAUNCH();
        }
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg
