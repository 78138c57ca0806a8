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
// panel threads: one warp per trailing panel column in the reflector step
// (measured at 128 rows: 35 us a panel with 512 threads, 120 us with 32)
constexpr int kQrPanelThreads = 512;
inline int qr_panel_threads(int) { return kQrPanelThreads; }
constexpr int kQrTrailThreads = 256;

__device__ __forceinline__ float wsumf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row ownership: thread t owns panel rows t, t + 512, ...; it alone reads and
// writes them, so a column step needs only two block reductions -- the norm
// of the column (which also publishes its diagonal entry) and the products of
// the reflector with the columns to its right -- and every thread derives the
// reflector from the reduced norm itself.  Panel rows have stride ps = the
// panel width + 1 (odd: no bank conflicts between consecutive rows).

template <int PT>
__global__ void __launch_bounds__(PT) k_qr_panel(float *__restrict__ X, int c, int l, int k, int bw,
                                                              int kPS, float *__restrict__ V, float *__restrict__ T)
{
    extern __shared__ float P[];                   // rows x kPS
    constexpr int nw = PT / 32;
    __shared__ float part[nw][kQrB];
    __shared__ float npart[nw];
    __shared__ float sbeta[kQrB], G[kQrB][kQrB + 1];
    const int rows = c - k, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < rows; i += PT) {
        for (int j = 0; j < bw; ++j) P[i * kPS + j] = X[(long long)(k + i) * l + k + j];
        for (int j = 0; j < kQrB; ++j) V[(long long)i * kQrB + j] = 0.f;
    }
    for (int j = 0; j < bw; ++j) {
        // 1. |P[j:, j]|^2, which also publishes P[j][j] after the barrier.  FP32
        // (FP64 is scarce on this part, and every thread repeats the final sum):
        // with alpha = -+sqrt(a) rounded once, beta = -1/(alpha v0) = 2/(v^T v)
        // to FP32 rounding, so each reflector is orthogonal at FP32 level
        float a = 0.f;
        for (int i = tid; i < rows; i += PT)
            if (i >= j) { const float x = P[i * kPS + j]; a = fmaf(x, x, a); }
        a = wsumf(a);
        if (lane == 0) npart[warp] = a;
        __syncthreads();
        a = 0.f;
        for (int w = 0; w < nw; ++w) a += npart[w];
        const float x0 = P[j * kPS + j];
        const float nrm = sqrtf(a);
        float beta = 0.f, v0 = 1.f, alpha = x0;
        if (rows - j > 1 && nrm > 0.f && a > x0 * x0) {
            alpha = x0 >= 0.f ? -nrm : nrm;
            v0 = x0 - alpha;
            beta = -1.f / (alpha * v0);               // 2 / (v^T v)
        }
        if (tid == 0) sbeta[j] = beta;
        // 2. w_q = v^T P[j:, q] for q > j (one warp per column, all rows: no
        // row is written between the two barriers), then P[j:, q] -= beta v w_q
        // on the own rows
        if (beta != 0.f) {
            for (int q = j + 1 + warp; q < bw; q += nw) {
                float sacc = 0.f;
                for (int i = j + lane; i < rows; i += 32)
                    sacc = fmaf(i == j ? v0 : P[i * kPS + j], P[i * kPS + q], sacc);
                sacc = wsumf(sacc);
                if (lane == 0) part[0][q] = sacc;
            }
        }
        __syncthreads();
        for (int i = tid; i < rows; i += PT) {
            if (i < j) continue;
            const float vi = i == j ? v0 : P[i * kPS + j];
            V[(long long)i * kQrB + j] = vi;
            if (beta != 0.f) {
                for (int q = j + 1; q < bw; ++q) P[i * kPS + q] -= beta * vi * part[0][q];
            }
            P[i * kPS + j] = (i == j) ? alpha : 0.f;
        }
        // the next column's norm reads only own rows; its barrier publishes
        // the diagonal entry written above
    }
    __syncthreads();
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
    if (warp == 0) {
        // column j of T from columns < j: lane p < j forms row p (the
        // columns are sequential, the rows of one column are not)
        __shared__ float Ts[kQrB][kQrB + 1];
        for (int q = 0; q < kQrB; ++q)
            if (lane < kQrB) Ts[lane][q] = 0.f;
        __syncwarp();
        for (int j = 0; j < bw; ++j) {
            if (lane < j) {
                float s = 0.f;
                for (int q = lane; q < j; ++q) s = fmaf(Ts[lane][q], G[q][j], s);
                Ts[lane][j] = -sbeta[j] * s;
            } else if (lane == j) {
                Ts[j][j] = sbeta[j];
            }
            __syncwarp();
        }
        for (int e = lane; e < kQrB * kQrB; e += 32) T[e] = Ts[e / kQrB][e % kQrB];
    }
    for (int i = tid; i < rows; i += PT)
        for (int j = 0; j < bw; ++j) X[(long long)(k + i) * l + k + j] = P[i * kPS + j];
}

// Column ownership, for panels of at most 32 RPL rows: warp q holds panel
// column q in registers (lane i: rows i, i + 32, ...).  At column step j
// the owner warp alone forms the reflector from its column (norm by a warp
// reduction), publishes it to shared memory (double-buffered) with beta, and
// finishes its column as R's; after one block barrier each warp q > j takes
// w_q = v . col_q by a warp reduction and updates its own column.  So a step
// costs one barrier and two warp reductions on its critical path, where the
// row-owning form above needs two block reductions.  Same reflectors, V and
// T layout, so k_qr_trail applies them unchanged.
template <int RPL>
__global__ void __launch_bounds__(32 * kQrB) k_qr_panel_w(float *__restrict__ X, int c, int l, int k, int bw,
                                                          float *__restrict__ V, float *__restrict__ T)
{
    constexpr int MR = 32 * RPL;
    __shared__ float vbuf[2][MR];
    __shared__ float Vs[MR][kQrB + 1];
    __shared__ float sbeta[kQrB], G[kQrB][kQrB + 1];
    const int rows = c - k, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float col[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        col[t] = (i < rows && warp < bw) ? X[(long long)(k + i) * l + k + warp] : 0.f;
    }
    for (int e = threadIdx.x; e < MR * (kQrB + 1); e += blockDim.x) (&Vs[0][0])[e] = 0.f;
    __syncthreads();
    for (int j = 0; j < bw; ++j) {
        float *vb = vbuf[j & 1];
        if (warp == j) {
            float a = 0.f;
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int i = lane + 32 * t;
                if (i >= j && i < rows) a = fmaf(col[t], col[t], a);
            }
            a = wsumf(a);
            const float x0 = __shfl_sync(0xffffffffu, col[0], j);   // row j < 16 sits in lane j, t = 0
            const float nrm = sqrtf(a);
            float beta = 0.f, v0 = 1.f, alpha = x0;
            if (rows - j > 1 && nrm > 0.f && a > x0 * x0) {
                alpha = x0 >= 0.f ? -nrm : nrm;
                v0 = x0 - alpha;
                beta = -1.f / (alpha * v0);               // 2 / (v^T v)
            }
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int i = lane + 32 * t;
                const float vi = (i < j || i >= rows) ? 0.f : (i == j ? v0 : col[t]);
                vb[i] = vi;
                Vs[i][j] = vi;
                if (i == j) col[t] = alpha;
                else if (i > j) col[t] = 0.f;
            }
            if (lane == 0) sbeta[j] = beta;
        }
        __syncthreads();
        if (warp > j && warp < bw) {
            const float beta = sbeta[j];
            if (beta != 0.f) {
                float w = 0.f;
#pragma unroll
                for (int t = 0; t < RPL; ++t) w = fmaf(vb[lane + 32 * t], col[t], w);
                w = wsumf(w);
#pragma unroll
                for (int t = 0; t < RPL; ++t) col[t] -= beta * vb[lane + 32 * t] * w;
            }
        }
    }
    __syncthreads();
    // compact WY: G = V^T V over the panel rows, then T column by column
    for (int pq = warp; pq < bw * bw; pq += kQrB) {
        const int p = pq / bw, q = pq % bw;
        if (p >= q) continue;
        float sacc = 0.f;
        for (int i = q + lane; i < rows; i += 32) sacc = fmaf(Vs[i][p], Vs[i][q], sacc);
        sacc = wsumf(sacc);
        if (lane == 0) G[p][q] = sacc;
    }
    __syncthreads();
    if (warp == 0) {
        __shared__ float Ts[kQrB][kQrB + 1];
        for (int q = 0; q < kQrB; ++q)
            if (lane < kQrB) Ts[lane][q] = 0.f;
        __syncwarp();
        for (int j = 0; j < bw; ++j) {
            if (lane < j) {
                float sacc = 0.f;
                for (int q = lane; q < j; ++q) sacc = fmaf(Ts[lane][q], G[q][j], sacc);
                Ts[lane][j] = -sbeta[j] * sacc;
            } else if (lane == j) {
                Ts[j][j] = sbeta[j];
            }
            __syncwarp();
        }
        for (int e = lane; e < kQrB * kQrB; e += 32) T[e] = Ts[e / kQrB][e % kQrB];
    }
    // R's columns back to X, the reflectors to V (rows x kQrB, zero beyond bw)
    if (warp < bw) {
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (i < rows) X[(long long)(k + i) * l + k + warp] = col[t];
        }
    }
    for (int e = threadIdx.x; e < rows * kQrB; e += blockDim.x) V[e] = Vs[e / kQrB][e % kQrB];
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
// qr32_work_bytes(c) bytes.  The panel narrows from 16 to 8 or 4 columns for
// tall matrices (c * (width + 1) floats <= 200 KB, so c up to ~17,000);
// returns DMRG_EUNSUPPORTED beyond.
dmrg_status qr_precondition32(dmrg_ctx *ctx, float *X, int c, int l, void *work)
{
    if (c <= 1 || l <= 0) return DMRG_OK;
    // panel width: 16 columns, narrower for tall panels so that a panel of c
    // rows (stride width + 1) fits the 200 KB of shared memory
    int bmax = kQrB;
    while (bmax > 2 && (size_t)c * (bmax + 1) * sizeof(float) > 200 * 1024) bmax /= 2;
    const int kPS = bmax + 1;
    const size_t smem_max = (size_t)c * kPS * sizeof(float);
    if (smem_max > 200 * 1024) return DMRG_EUNSUPPORTED;
    static bool attr = false;
    if (!attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_qr_panel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        DMRG_CUDA(cudaFuncSetAttribute(k_qr_panel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        DMRG_CUDA(cudaFuncSetAttribute(k_qr_panel<kQrPanelThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        attr = true;
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    float *V = static_cast<float *>(work);
    float *T = reinterpret_cast<float *>(static_cast<char *>(work) + al(sizeof(float) * (size_t)c * kQrB));
    const int kmax = std::min(c - 1, l);          // reflectors 0..kmax-1
    prof_mark(ctx, PROF_QR);
    for (int k = 0; k < kmax; k += bmax) {
        const int bw = std::min(bmax, kmax - k);
        const size_t smem = (size_t)(c - k) * kPS * sizeof(float);
        const int pt = qr_panel_threads(c - k);
        if (ctx->qr_wpanel && c - k <= 128)
            k_qr_panel_w<4><<<1, 32 * kQrB, 0, ctx->stream>>>(X, c, l, k, bw, V, T);
        else if (ctx->qr_wpanel && c - k <= 256)
            k_qr_panel_w<8><<<1, 32 * kQrB, 0, ctx->stream>>>(X, c, l, k, bw, V, T);
        else if (pt == 32)
            k_qr_panel<32><<<1, 32, smem, ctx->stream>>>(X, c, l, k, bw, kPS, V, T);
        else if (pt == 128)
            k_qr_panel<128><<<1, 128, smem, ctx->stream>>>(X, c, l, k, bw, kPS, V, T);
        else
            k_qr_panel<kQrPanelThreads><<<1, kQrPanelThreads, smem, ctx->stream>>>(X, c, l, k, bw, kPS, V, T);
        DMRG_COUNT_LAUNCH();
        const int ncols = l - (k + bw);
        if (ncols > 0) {
            k_qr_trail<<<(ncols + 31) / 32, kQrTrailThreads, 0, ctx->stream>>>(X, c, l, k, bw, V, T);
            DMRG_COUNT_LAUNCH();
        }
    }
    prof_mark(ctx, PROF_QR);
    prof_count(ctx, PROF_QR, 2.0 * (double)kmax * kmax * ((double)c + l - 2.0 * kmax / 3.0), 0.0);
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg
