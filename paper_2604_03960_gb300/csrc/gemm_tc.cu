// gemm_tc.cu -- 3xTF32 contractions on the 5th-generation tensor cores (tcgen05).
//
// C (FP64, strided) = alpha * A B + beta * C with A, B given as FP64 strided
// operands.  Each operand value a is split into two TF32 numbers
//   hi = tf32(a),  lo = tf32(a - hi)
// and the product is taken as hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo lo
// term is below FP32 resolution).  The three products are laid end to end
// along K, so a single TF32 GEMM over K' = 3 Kp computes them:
//   A^ = [hi | hi | lo]  (M x K', K-major),   B^ = [hi | lo | hi]  (N x K', K-major)
// A prep kernel writes both operands in that K-major form (transposing
// through shared memory when the source is not K-contiguous), zero-padding K
// to a multiple of 32.  The GEMM kernel is one CTA per 128 x BN output tile:
//   * warp 0, one thread: TMA loads of 128 x 32 (A) and BN x 32 (B) FP32 tiles,
//     128-byte swizzle, into a 4-stage shared-memory ring (mbarrier
//     transaction counts);
//   * warp 1, one thread: tcgen05.mma.kind::tf32 (M = 128, N = BN, K = 8) into a
//     TMEM accumulator, tcgen05.commit releasing each stage;
//   * all four warps: tcgen05.ld of the accumulator (one TMEM lane quarter per
//     warp) and the FP64 epilogue.
// Every mbarrier wait is bounded; a wait that gives up sets the device status
// word, drains the copies it issued and frees its TMEM before returning.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace dmrg {
namespace {

constexpr int TBM = 128;           // tile rows (tcgen05 M)
constexpr int TBK = 32;            // FP32 elements per 128-byte row of a stage
constexpr int STAGES = 4;
constexpr long long kPollLimit = 1LL << 24;   // ~1-2 s with the back-off below

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < kPollLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i > 2048) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// K-major, 128-byte swizzle shared-memory matrix descriptor (tcgen05 format):
// start >> 4 in bits 0-13, leading byte offset 16 B (unused for this layout),
// stride byte offset 1024 B between 8-row groups, version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
struct TcCfg {
    static constexpr uint32_t A_BYTES = TBM * 128;
    static constexpr uint32_t B_BYTES = BN * 128;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t SMEM = STAGES * STAGE + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = BN;   // power of two >= 32
};

// Split K: blockIdx.z = batch index * nsl + slice; a slice takes K blocks
// [slice * kps, min(nk, (slice + 1) * kps)).  With P set, each slice writes its
// FP32 partial sums (as FP64) to P[slice][b][m][n] and k_tc_reduce adds the
// slices in FP64, so no FP32 accumulator sums more than kps * 32 terms.
template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int nk,
              int kps, int nsl, double *__restrict__ P, double alpha, double beta, double *__restrict__ C,
              long long sCm, long long sCn, long long sCb, int *status, float *__restrict__ C32, int kseg,
              unsigned kmap)
{
    using Cfg = TcCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;           // swizzle atoms need 1024-byte alignment
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t bar_base = base + STAGES * Cfg::STAGE;   // full[S], empty[S], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + STAGES * Cfg::STAGE + 8 * (2 * STAGES + 1));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *consumed_s = reinterpret_cast<volatile int *>(tmem_slot + 2);
    volatile int *issued_s = reinterpret_cast<volatile int *>(tmem_slot + 3);
    auto full = [&](int s) { return bar_base + 8u * s; };
    auto empty = [&](int s) { return bar_base + 8u * (STAGES + s); };
    const uint32_t done = bar_base + 8u * (2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN, bz = blockIdx.z / nsl, sl = blockIdx.z % nsl;
    const int kb0 = sl * kps;
    const int nkl = max(0, min(nk, kb0 + kps) - kb0);       // K blocks of this slice

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *consumed_s = 0;
        *issued_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int kb = 0; kb < nkl; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (*abort_flag || !mbar_wait(empty(s), ph ^ 1u)) {
                *abort_flag = 1;
                break;
            }
            mbar_expect_tx(full(s), Cfg::STAGE);
            const uint32_t a_dst = base + s * Cfg::STAGE;
            int ka = kb0 + kb, kbb = ka;
            if (kseg > 0) {
                // K' segment q (kseg blocks) of A reads stored segment nibble q of
                // kmap, that of B nibble q of kmap >> 16
                const int q = ka / kseg, w = ka - q * kseg;
                ka = (int)((kmap >> (4 * q)) & 15u) * kseg + w;
                kbb = (int)((kmap >> (16 + 4 * q)) & 15u) * kseg + w;
            }
            tma_load_3d(a_dst, &tmA, full(s), ka * TBK, m0, bz);
            tma_load_3d(a_dst + Cfg::A_BYTES, &tmB, full(s), kbb * TBK, n0, bz);
            issued = kb + 1;
        }
        *issued_s = issued;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: instruction descriptor for kind::tf32, FP32 accumulate,
        // both operands K-major, M = 128, N = BN
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TBM >> 4) << 24);
        int consumed = 0;
        for (int kb = 0; kb < nkl; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (*abort_flag || !mbar_wait(full(s), ph)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a_addr = base + s * Cfg::STAGE;
            const uint32_t b_addr = a_addr + Cfg::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TBK / 8; ++kk)
                mma_tf32(tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc,
                         (kb > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty(s));
            consumed = kb + 1;
        }
        *consumed_s = consumed;
        mma_commit(done);       // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // epilogue
    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    __syncwarp();
    if (!ok) *abort_flag = 1;
    if (!*abort_flag && nkl > 0) {
        // Each warp's 32 rows x 32 columns go through a shared-memory tile
        // (the stage buffers are idle once every MMA has completed), so that
        // a warp then stores 32 consecutive columns of one row at a time;
        // FP32 -> FP64 is widened with integer operations (the FP64 pipe,
        // which the converting instruction uses, is narrow on this part).
        float *tile = reinterpret_cast<float *>(gbase) + warp * (32 * 33);
        const long long nbatch = gridDim.z / nsl;
        const bool plain = (alpha == 1.0) && (beta == 0.0);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const int gn = n0 + c * 32 + lane;
            if (gn < N) {
#pragma unroll 4
                for (int rr = 0; rr < 32; ++rr) {
                    const int gm = m0 + warp * 32 + rr;
                    if (gm >= M) break;
                    if (C32) {
                        // FP32 result as accumulated (alpha = 1, beta = 0)
                        C32[(long long)bz * sCb + (long long)gm * sCm + (long long)gn * sCn] = tile[rr * 33 + lane];
                        continue;
                    }
                    const double x = f32_widen(tile[rr * 33 + lane]);
                    if (P) {
                        P[(((long long)sl * nbatch + bz) * M + gm) * (long long)N + gn] = x;
                    } else {
                        double *p = C + (long long)bz * sCb + (long long)gm * sCm + (long long)gn * sCn;
                        if (plain) {
                            *p = x;
                        } else {
                            double v = alpha * x;
                            if (beta != 0.0) v += beta * *p;
                            *p = v;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(status, ST_TIMEOUT);
        // drain TMA copies that were issued but never consumed (bounded)
        for (int kb = *consumed_s; kb < *issued_s; ++kb)
            (void)mbar_wait(full(kb % STAGES), (uint32_t)(kb / STAGES) & 1u);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                     : "memory");
    }
}

// C[b][m][n] = alpha * sum_s P[s][b][m][n] + beta * C[b][m][n], the slices
// added in order in FP64 (deterministic)
__global__ void k_tc_reduce(const double *__restrict__ P, int nsl, int batch, int M, int N, double alpha, double beta,
                            double *__restrict__ C, long long sCm, long long sCn, long long sCb)
{
    const long long per = (long long)M * N, total = per * batch, slice = total;
    const bool plain = (alpha == 1.0) && (beta == 0.0);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double a = P[e];
        for (int q = 1; q < nsl; ++q) a += P[q * slice + e];
        const long long b = e / per, mn = e % per;
        const int m = (int)(mn / N), n = (int)(mn % N);
        double *c = C + b * sCb + (long long)m * sCm + (long long)n * sCn;
        if (plain) {
            *c = a;
        } else {
            double v = alpha * a;
            if (beta != 0.0) v += beta * *c;
            *c = v;
        }
    }
}

__device__ __forceinline__ float to_tf32(float x) { return tf32_rna(x); }

// out[b][row][slice * Kp + col] = slice of in(b, row, col), rows R, cols Kc,
// zero for Kc <= col < Kp.  pattern 0: (hi, hi, lo); pattern 1: (hi, lo, hi).
__global__ void k_split3(const double *__restrict__ in, long long s_row, long long s_col, long long s_b, int R, int Kc,
                         int Kp, float *__restrict__ out, int pattern)
{
    __shared__ float hi_t[32][33], lo_t[32][33];
    const int b = blockIdx.z, r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const double *src = in + (long long)b * s_b;
    const bool colfast = (s_col == 1) || (s_row != 1);
    for (int i = 0; i < 4; ++i) {
        int rr, cc;
        if (colfast) { rr = threadIdx.y + 8 * i; cc = threadIdx.x; } else { rr = threadIdx.x; cc = threadIdx.y + 8 * i; }
        const int r = r0 + rr, c = c0 + cc;
        const double v = (r < R && c < Kc) ? src[(long long)r * s_row + (long long)c * s_col] : 0.0;
        float h, l;
        tf32_split(v, h, l);
        hi_t[rr][cc] = h;
        lo_t[rr][cc] = l;
    }
    __syncthreads();
    const long long K3 = 3LL * Kp;
    for (int i = 0; i < 4; ++i) {
        const int rr = threadIdx.y + 8 * i, cc = threadIdx.x;
        const int r = r0 + rr, c = c0 + cc;
        if (r >= R) continue;
        float *o = out + ((long long)b * R + r) * K3 + c;
        const float h = hi_t[rr][cc], l = lo_t[rr][cc];
        o[0] = h;
        o[Kp] = pattern == 0 ? h : l;
        o[2LL * Kp] = pattern == 0 ? l : h;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool load_encode()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

bool make_map(CUtensorMap *map, const float *base, int K3, int rows, int batch, int box_rows)
{
    cuuint64_t dims[3] = {(cuuint64_t)K3, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)K3 * 4, (cuuint64_t)K3 * 4 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// largest stored segment index in a 3-entry nibble map
inline unsigned kmap_max(unsigned m)
{
    unsigned a = m & 15u, b = (m >> 4) & 15u, c = (m >> 8) & 15u;
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

template <int BN>
dmrg_status launch_tc(dmrg_ctx *ctx, const float *Ah, const float *Bh, int M, int N, int K3, int batch, double alpha,
                      double beta, double *C, long long sCm, long long sCn, long long sCb, int nsl, double *P,
                      float *C32 = nullptr, int kseg = 0, unsigned kmap = 0u)
{
    CUtensorMap ma, mb;
    // stored K extent: the three K' segments, or the distinct stored ones
    const int Ks = kseg > 0 ? kseg * TBK * (int)(1 + max(kmap_max(kmap & 0xffffu), kmap_max(kmap >> 16))) : K3;
    if (!make_map(&ma, Ah, Ks, M, batch, TBM) || !make_map(&mb, Bh, Ks, N, batch, BN)) return DMRG_ECUDA;
    static bool attr_set = false;
    if (!attr_set) {
        DMRG_CUDA(cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN>::SMEM));
        attr_set = true;
    }
    const int nk = K3 / TBK;
    const int kps = (nk + nsl - 1) / nsl;
    dim3 grid((N + BN - 1) / BN, (M + TBM - 1) / TBM, batch * nsl);
    prof_mark(ctx, PROF_TC_GEMM);
    k_tc_gemm<BN><<<grid, 128, TcCfg<BN>::SMEM, ctx->stream>>>(ma, mb, M, N, nk, kps, nsl, nsl > 1 ? P : nullptr,
                                                               alpha, beta, C, sCm, sCn, sCb, ctx->d_status,
                                                               C32, kseg, kmap);
    DMRG_COUNT_LAUNCH();
    if (nsl > 1) {
        const long long total = (long long)M * N * batch;
        long long blocks = (total + 255) / 256;
        if (blocks > 8LL * ctx->num_sms) blocks = 8LL * ctx->num_sms;
        k_tc_reduce<<<(int)blocks, 256, 0, ctx->stream>>>(P, nsl, batch, M, N, alpha, beta, C, sCm, sCn, sCb);
        DMRG_COUNT_LAUNCH();
    }
    prof_mark(ctx, PROF_TC_GEMM);
    // work of the split product: three TF32 products of the padded shape;
    // bytes: both split operands read once and the FP64 result written once
    prof_count(ctx, PROF_TC_GEMM, 2.0 * M * N * (double)K3 * batch,
               4.0 * (double)(M + N) * K3 * batch + (C32 ? 4.0 : 8.0) * (double)M * N * batch);
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace

dmrg_status tc_gemm_split(dmrg_ctx *ctx, const float *Ah, const float *Bh, int M, int N, int K3, int batch, int bn,
                          int nsl, double *P, double *C64, float *C32, long long sCm, long long sCn, long long sCb,
                          unsigned seg_map)
{
    if (M <= 0 || N <= 0 || batch <= 0) return DMRG_OK;
    if (!tc_available(ctx)) return DMRG_EUNSUPPORTED;
    if (K3 <= 0 || K3 % (3 * TBK) || (!C64 == !C32) || (C32 && nsl != 1) || (nsl > 1 && !P) || nsl < 1 ||
        (long long)batch * nsl > 65535 || (M + TBM - 1) / TBM > 65535)
        return DMRG_EINVAL;
    // segment map: nibble q (A) and 4 + q (B) name the stored segment of K' segment q
    int kseg = 0;
    unsigned kmap = 0u;
    if (seg_map) {
        for (int q = 0; q < 6; ++q)
            if (((seg_map >> (4 * q)) & 15u) > 2u) return DMRG_EINVAL;
        kseg = K3 / (3 * TBK);
        kmap = (seg_map & 0xfffu) | ((seg_map >> 12) & 0xfffu) << 16;
    }
    {
        // no empty slice (its partial sums would never be written)
        const int nk = K3 / TBK;
        if (nsl > nk) nsl = nk;
        const int kps = (nk + nsl - 1) / nsl;
        nsl = (nk + kps - 1) / kps;
    }
    switch (bn) {
    case 64: return launch_tc<64>(ctx, Ah, Bh, M, N, K3, batch, 1.0, 0.0, C64, sCm, sCn, sCb, nsl, P, C32, kseg, kmap);
    case 128: return launch_tc<128>(ctx, Ah, Bh, M, N, K3, batch, 1.0, 0.0, C64, sCm, sCn, sCb, nsl, P, C32, kseg, kmap);
    case 256: return launch_tc<256>(ctx, Ah, Bh, M, N, K3, batch, 1.0, 0.0, C64, sCm, sCn, sCb, nsl, P, C32, kseg, kmap);
    default: return DMRG_EINVAL;
    }
}

bool tc_available(dmrg_ctx *ctx)
{
    if (ctx->tc_ok < 0) {
        cudaDeviceProp prop;
        bool ok = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess && prop.major == 10 && prop.minor == 3 &&
                  load_encode();
        ctx->tc_ok = ok ? 1 : 0;
    }
    return ctx->tc_ok == 1;
}

// Tile width choice: 256-column tiles unless that leaves most SMs idle.
int tc_pick_bn(dmrg_ctx *ctx, int M, int N, int K, int batch)
{
    if (ctx->tc_bn_override == 64 || ctx->tc_bn_override == 128 || ctx->tc_bn_override == 256)
        return ctx->tc_bn_override;
    if (batch == 1) {
        const int tuned = tune_lookup_bn(ctx, M, N, K);
        if (tuned == 64 || tuned == 128 || tuned == 256) return tuned;
    }
    long long t256 = (long long)((N + 255) / 256) * ((M + TBM - 1) / TBM) * batch;
    long long t128 = (long long)((N + 127) / 128) * ((M + TBM - 1) / TBM) * batch;
    if (N <= 64) return 64;      // half the accumulator columns and epilogue of a 128 tile
    // products that fill under one wave even with 64-column tiles are
    // latency-bound: twice the CTAs, each with half the epilogue
    const long long t64 = (long long)((N + 63) / 64) * ((M + TBM - 1) / TBM) * batch;
    if (t64 <= ctx->num_sms) return 64;
    if (N <= 128) return 128;
    // compare wave-quantised work: tiles rounded up to whole waves, weighted by tile width
    long long w256 = ((t256 + ctx->num_sms - 1) / ctx->num_sms) * 2;
    long long w128 = ((t128 + ctx->num_sms - 1) / ctx->num_sms);
    return (w128 < w256) ? 128 : 256;
}

bool tc_path(dmrg_ctx *ctx, int M, int N, int K, int batch)
{
    return M > 0 && N > 0 && batch > 0 && K > 0 && tc_available(ctx) &&
           (ctx->tc_force || (double)M * N * K * batch >= (double)ctx->tc_min_work);
}

dmrg_status split3_dev(dmrg_ctx *ctx, const double *in, long long s_row, long long s_col, long long s_b, int R,
                       int Kc, int batch, int pattern, float *out)
{
    if (R <= 0 || Kc <= 0 || batch <= 0) return DMRG_OK;
    const int Kp = split_kp(Kc);
    dim3 g(Kp / 32, (R + 31) / 32, batch);
    k_split3<<<g, dim3(32, 8), 0, ctx->stream>>>(in, s_row, s_col, s_b, R, Kc, Kp, out, pattern); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status gemm_3xtf32(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                        long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                        double beta, double *C, long long sCm, long long sCn, long long sCb, int batch)
{
    return gemm_3xtf32_pre(ctx, M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn, sCb, batch,
                           nullptr, nullptr);
}

dmrg_status gemm_3xtf32_pre(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                            long long sAk, long long sAb, const double *B, long long sBk, long long sBn,
                            long long sBb, double beta, double *C, long long sCm, long long sCn, long long sCb,
                            int batch, const float *Ah_pre, const float *Bh_pre)
{
    if (M <= 0 || N <= 0 || batch <= 0) return DMRG_OK;
    if (!tc_available(ctx)) return DMRG_EUNSUPPORTED;
    // small products: FP32 arithmetic on the CUDA cores is faster than
    // splitting into TF32 parts, at the same precision class
    if (K <= 0 || (!ctx->tc_force && (double)M * N * K * batch < (double)ctx->tc_min_work)) {
        prof_mark(ctx, PROF_F32_GEMM);
        dmrg_status e = gemm_f32c(ctx, M, N, K, alpha, A, sAm, sAk, sAb, B, sBk, sBn, sBb, beta, C, sCm, sCn,
                                  sCb, batch);
        prof_mark(ctx, PROF_F32_GEMM);
        prof_count(ctx, PROF_F32_GEMM, 2.0 * M * N * (double)(K > 0 ? K : 0) * batch, 0.0);
        return e;
    }
    if (batch > 65535 || (M + TBM - 1) / TBM > 65535) return DMRG_EINVAL;
    const int Kp = (K + 31) / 32 * 32, K3 = 3 * Kp;
    // split K so that no FP32 accumulator sums more than kSliceKb * 32 of the
    // K' = 3 Kp products (the slices meet in FP64)
    const int nk = K3 / TBK;
    int nsl = 1;
    int kb = ctx->tc_split_kb;
    if (batch == 1 && ctx->tc_bn_override == 0 && kb == 8) {
        int tkb = 0;
        if (tune_lookup_bn(ctx, M, N, K, &tkb) && (tkb == 4 || tkb == 8)) kb = tkb;   // autotuned depth
    }
    if (kb > 0 && nk > kb) {
        nsl = (nk + kb - 1) / kb;
        if (nsl > 16) nsl = 16;
        const int kps = (nk + nsl - 1) / nsl;
        nsl = (nk + kps - 1) / kps;
    }
    if ((long long)batch * nsl > 65535) nsl = 1;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t bytesA = sizeof(float) * (size_t)batch * M * K3, bytesB = sizeof(float) * (size_t)batch * N * K3;
    const size_t bytesP = nsl > 1 ? sizeof(double) * (size_t)nsl * batch * M * N : 0;
    DMRG_TRY(ctx->tcbuf.ensure(al(bytesA) + al(bytesB) + bytesP));
    float *Ah = ctx->tcbuf.as<float>();
    float *Bh = reinterpret_cast<float *>(reinterpret_cast<char *>(Ah) + al(bytesA));
    double *P = reinterpret_cast<double *>(reinterpret_cast<char *>(Bh) + al(bytesB));
    if (!Ah_pre) {
        dim3 g(Kp / 32, (M + 31) / 32, batch);
        k_split3<<<g, dim3(32, 8), 0, ctx->stream>>>(A, sAm, sAk, sAb, M, K, Kp, Ah, 0); DMRG_COUNT_LAUNCH();
    } else {
        Ah = const_cast<float *>(Ah_pre);
    }
    if (!Bh_pre) {
        dim3 g2(Kp / 32, (N + 31) / 32, batch);
        k_split3<<<g2, dim3(32, 8), 0, ctx->stream>>>(B, sBn, sBk, sBb, N, K, Kp, Bh, 1); DMRG_COUNT_LAUNCH();
    } else {
        Bh = const_cast<float *>(Bh_pre);
    }
    DMRG_CUDA(cudaGetLastError());
    const int bn = tc_pick_bn(ctx, M, N, K, batch);
    if (bn == 64) return launch_tc<64>(ctx, Ah, Bh, M, N, K3, batch, alpha, beta, C, sCm, sCn, sCb, nsl, P);
    if (bn == 128) return launch_tc<128>(ctx, Ah, Bh, M, N, K3, batch, alpha, beta, C, sCm, sCn, sCb, nsl, P);
    return launch_tc<256>(ctx, Ah, Bh, M, N, K3, batch, alpha, beta, C, sCm, sCn, sCb, nsl, P);
}

}  // namespace dmrg

using namespace dmrg;

extern "C" dmrg_status dmrg_gemm(dmrg_ctx *ctx, int prec, int force_tc, int M, int N, int K, const double *A_dev,
                                 const double *B_dev, double *C_dev)
{
    if (!ctx || !A_dev || !B_dev || !C_dev || M < 1 || N < 1 || K < 1) return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && prec != DMRG_PREC_3XTF32) return DMRG_EUNSUPPORTED;
    const int saved = ctx->tc_force;
    ctx->tc_force = force_tc;
    dmrg_status s = gemm(ctx, prec, M, N, K, 1.0, A_dev, K, 1, 0, B_dev, N, 1, 0, 0.0, C_dev, N, 1, 0, 1);
    ctx->tc_force = saved;
    if (s != DMRG_OK) return s;
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return dmrg_get_status(ctx);
}
