// gemm_f64.cu -- FP64 strided batched GEMM on the CUDA cores (DFMA).
//
// Every FP64 contraction of the local update (H_eff stages 1 and 3, the
// environment update stages 1 and 3, the two-site tensor and the gauge
// moves) is one call of this kernel with the operand strides chosen so that
// no tensor is ever transposed in memory.  GB300's FP64 pipe is narrow, so
// a 64 x 64 register-tiled kernel already sits at the DFMA roof; the tiles
// are staged through shared memory with loads coalesced along whichever
// operand stride is unit.
#include "common.cuh"

#include <algorithm>

namespace dmrg {

std::atomic<long long> g_launch_count{0};

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// operand conversion: FP64 stays, FP32 narrows by integer operations
// (bit-identical to the converting instruction, which uses the narrow FP64 pipe)
template <typename T> __device__ __forceinline__ T narrow_to(double v);
template <> __device__ __forceinline__ double narrow_to<double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow_to<float>(double v) { return f64_narrow(v); }

// T = double: the FP64 path; T = float: FP32 arithmetic on FP64 operands for
// the small products of the mixed form.  In the FP32 case each BK-long
// partial sum is added into a compensated pair (hi, lo) by Knuth's TwoSum, so
// the accumulation error does not grow with K: the result carries the
// rounding of the FP32 operands and of BK-term sums only.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

// Tile BT x BT (64 or 32), 16 x 16 threads with TT = BT / 16 outputs a side.
// Split K: blockIdx.z = batch index * nsl + slice; a slice takes K range
// [slice * kps, min(K, (slice + 1) * kps)) and, when P is set, writes its
// partial sums to P[slice][b][m][n] for k_gemm_reduce (slices added in order).
template <typename T, int BT = 64>
__global__ void __launch_bounds__(NT) k_gemm_t(int M, int N, int K, double alpha, const double *__restrict__ A,
                                               long long sAm, long long sAk, long long sAb,
                                               const double *__restrict__ B, long long sBk, long long sBn,
                                               long long sBb, double beta, double *__restrict__ C, long long sCm,
                                               long long sCn, long long sCb, int nsl = 1, int kps = 0,
                                               double *__restrict__ P = nullptr)
{
    constexpr int BM = BT, BN = BT, TM = BT / 16, TN = BT / 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int bz = blockIdx.z / nsl, sl = blockIdx.z % nsl;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = nsl > 1 ? sl * kps : 0;
    const int ke = nsl > 1 ? min(K, kb + kps) : K;
    const bool plain = (alpha == 1.0) && (beta == 0.0);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    A += (long long)bz * sAb;
    B += (long long)bz * sBb;
    C += (long long)bz * sCb;
    T acc[TM][TN];
    constexpr bool kComp = sizeof(T) == 4;
    float chi[kComp ? TM : 1][kComp ? TN : 1], clo[kComp ? TM : 1][kComp ? TN : 1];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;
    if (kComp) {
#pragma unroll
        for (int i = 0; i < (kComp ? TM : 1); ++i)
#pragma unroll
            for (int j = 0; j < (kComp ? TN : 1); ++j) chi[i][j] = clo[i][j] = 0.f;
    }
    const bool a_kfast = (sAk == 1);
    const bool b_nfast = (sBn == 1);
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int it = 0; it < (BM * BK) / NT; ++it) {
            int idx = tid + it * NT;
            int mm, kk;
            if (a_kfast) { mm = idx / BK; kk = idx % BK; } else { kk = idx / BM; mm = idx % BM; }
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < ke) ? narrow_to<T>(A[(long long)gm * sAm + (long long)gk * sAk]) : (T)0;
        }
#pragma unroll
        for (int it = 0; it < (BN * BK) / NT; ++it) {
            int idx = tid + it * NT;
            int nn, kk;
            if (b_nfast) { kk = idx / BN; nn = idx % BN; } else { nn = idx / BK; kk = idx % BK; }
            int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < ke) ? narrow_to<T>(B[(long long)gk * sBk + (long long)gn * sBn]) : (T)0;
        }
        __syncthreads();
        // multiply-adds only where they can reach an output: a thread whose
        // first row or column lies beyond the matrix has none, and a short
        // last K step stops at K (the padding would be FP64 work on zeros,
        // and the FP64 pipe of this part gives ~2 a clock per SM)
        if (ty < M - m0 && tx < N - n0) {
            const int kn = ke - k0 < BK ? ke - k0 : BK;
            if (kn == BK) {
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    T a[TM], b[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                }
            } else {
                for (int kk = 0; kk < kn; ++kk) {
                    T a[TM], b[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                }
            }
        }
        if (kComp) {
#pragma unroll
            for (int i = 0; i < (kComp ? TM : 1); ++i)
#pragma unroll
                for (int j = 0; j < (kComp ? TN : 1); ++j) {
                    two_sum_acc(chi[i][j], clo[i][j], (float)acc[i][j]);
                    acc[i][j] = (T)0;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            const double sum = kComp ? f32_widen(chi[kComp ? i : 0][kComp ? j : 0]) +
                                           f32_widen(clo[kComp ? i : 0][kComp ? j : 0])
                                     : (double)acc[i][j];
            if (P) {
                P[(((long long)sl * (gridDim.z / nsl) + bz) * M + gm) * (long long)N + gn] = sum;
                continue;
            }
            double *c = C + (long long)gm * sCm + (long long)gn * sCn;
            if (plain) {
                *c = sum;
                continue;
            }
            double v = alpha * sum;
            if (beta != 0.0) v += beta * *c;
            *c = v;
        }
    }
}

// C[b][m][n] = alpha * sum_s P[s][b][m][n] + beta * C[b][m][n], slices in order
__global__ void k_gemm_reduce(const double *__restrict__ P, int nsl, int batch, int M, int N, double alpha,
                              double beta, double *__restrict__ C, long long sCm, long long sCn, long long sCb)
{
    const long long per = (long long)M * N, total = per * batch;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double a = P[e];
        for (int q = 1; q < nsl; ++q) a += P[q * total + e];
        const long long b = e / per, mn = e % per;
        const int m = (int)(mn / N), n = (int)(mn % N);
        double *c = C + b * sCb + (long long)m * sCm + (long long)n * sCn;
        double v = alpha * a;
        if (beta != 0.0) v += beta * *c;
        *c = v;
    }
}

}  // namespace

// FP64 GEMM sized to the GPU: the FP64 pipe gives each SM ~2 multiply-adds
// a clock on this part, so a product that makes a handful of 64 x 64 tiles
// runs at a few percent of the chip.  Such products take 32 x 32 tiles and,
// if that is still under one CTA per SM, split K (>= 64 terms a slice) with
// the slices added in order in FP64 (deterministic).
dmrg_status gemm_f64x(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                      long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                      double beta, double *C, long long sCm, long long sCn, long long sCb, int batch)
{
    if (M <= 0 || N <= 0 || batch <= 0) return DMRG_OK;
    if (batch > 65535) return DMRG_EINVAL;
    cudaStream_t st = ctx->stream;
    const long long t64 = (long long)((N + 63) / 64) * ((M + 63) / 64) * batch;
    if (!ctx->f64_fill || t64 >= ctx->num_sms || K < 64)
        return gemm_f64(st, M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn, sCb, batch);
    dim3 grid((N + 31) / 32, (M + 31) / 32, batch);
    if (grid.y > 65535) return DMRG_EINVAL;
    const long long t32 = (long long)grid.x * grid.y * batch;
    int nsl = (int)std::min<long long>((ctx->num_sms + t32 - 1) / t32, K / 64);
    if (nsl < 1) nsl = 1;
    if ((long long)batch * nsl > 65535) nsl = 1;
    if (nsl == 1) {
        k_gemm_t<double, 32><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm,
                                                   sCn, sCb); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        return DMRG_OK;
    }
    int kps = (K + nsl - 1) / nsl;
    kps = (kps + BK - 1) / BK * BK;
    nsl = (K + kps - 1) / kps;
    const long long total = (long long)M * N * batch;
    DMRG_TRY(ctx->f64buf.ensure(sizeof(double) * (size_t)total * nsl));
    double *P = ctx->f64buf.as<double>();
    grid.z = batch * nsl;
    k_gemm_t<double, 32><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn,
                                               sCb, nsl, kps, P); DMRG_COUNT_LAUNCH();
    long long blocks = (total + 255) / 256;
    if (blocks > 4LL * ctx->num_sms) blocks = 4LL * ctx->num_sms;
    k_gemm_reduce<<<(int)blocks, 256, 0, st>>>(P, nsl, batch, M, N, alpha, beta, C, sCm, sCn, sCb); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status gemm_f64(cudaStream_t st, int M, int N, int K, double alpha, const double *A, long long sAm,
                     long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                     double beta, double *C, long long sCm, long long sCn, long long sCb, int batch)
{
    if (M <= 0 || N <= 0 || batch <= 0) return DMRG_OK;
    if (batch > 65535) return DMRG_EINVAL;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    if (grid.y > 65535) return DMRG_EINVAL;
    if (K <= 0) {
        // C = beta * C: run the kernel with K = 0 (accumulators stay zero)
        K = 0;
    }
    k_gemm_t<double><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn, sCb); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

// FP32 small products of the mixed form, sized to the GPU like the FP64
// kernel: a product that makes fewer 64 x 64 tiles than SMs (H_eff stage 3
// at chi = 50 is 4 of them, each walking K = 250 alone) takes 32 x 32 tiles
// and, if that is still under one CTA per SM, split K (>= 32 terms a slice,
// each slice with its compensated accumulation) with the slices added in
// order in FP64 (deterministic).
dmrg_status gemm_f32c(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                      long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                      double beta, double *C, long long sCm, long long sCn, long long sCb, int batch)
{
    if (M <= 0 || N <= 0 || batch <= 0) return DMRG_OK;
    if (batch > 65535) return DMRG_EINVAL;
    cudaStream_t st = ctx->stream;
    if (K < 0) K = 0;
    const long long t64 = (long long)((N + 63) / 64) * ((M + 63) / 64) * batch;
    if (!ctx->f32_fill || t64 >= ctx->num_sms) {
        dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
        if (grid.y > 65535) return DMRG_EINVAL;
        k_gemm_t<float><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn,
                                             sCb); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        return DMRG_OK;
    }
    dim3 grid((N + 31) / 32, (M + 31) / 32, batch);
    if (grid.y > 65535) return DMRG_EINVAL;
    const long long t32 = (long long)grid.x * grid.y * batch;
    int nsl = (int)std::min<long long>((ctx->num_sms + t32 - 1) / t32, K / 32);
    if (nsl < 1) nsl = 1;
    if ((long long)batch * nsl > 65535) nsl = 1;
    if (nsl == 1) {
        k_gemm_t<float, 32><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm,
                                                  sCn, sCb); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        return DMRG_OK;
    }
    int kps = (K + nsl - 1) / nsl;
    kps = (kps + BK - 1) / BK * BK;
    nsl = (K + kps - 1) / kps;
    const long long total = (long long)M * N * batch;
    DMRG_TRY(ctx->f64buf.ensure(sizeof(double) * (size_t)total * nsl));
    double *P = ctx->f64buf.as<double>();
    grid.z = batch * nsl;
    k_gemm_t<float, 32><<<grid, NT, 0, st>>>(M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn,
                                              sCb, nsl, kps, P); DMRG_COUNT_LAUNCH();
    long long blocks = (total + 255) / 256;
    if (blocks > 4LL * ctx->num_sms) blocks = 4LL * ctx->num_sms;
    k_gemm_reduce<<<(int)blocks, 256, 0, st>>>(P, nsl, batch, M, N, alpha, beta, C, sCm, sCn, sCb); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status gemm(dmrg_ctx *ctx, int prec, int M, int N, int K, double alpha, const double *A, long long sAm,
                 long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                 double beta, double *C, long long sCm, long long sCn, long long sCb, int batch)
{
    if (prec == DMRG_PREC_FP64) {
        prof_mark(ctx, PROF_F64_GEMM);
        dmrg_status s = gemm_f64x(ctx, M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn, sCb,
                                  batch);
        prof_mark(ctx, PROF_F64_GEMM);
        prof_count(ctx, PROF_F64_GEMM, 2.0 * M * (double)N * K * batch,
                   8.0 * ((double)M * K + (double)K * N + (double)M * N) * batch);
        return s;
    }
    if (prec == DMRG_PREC_3XTF32)
        return gemm_3xtf32(ctx, M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn, sCb, batch);
    return DMRG_EUNSUPPORTED;
}

}  // namespace dmrg
