// common.cuh -- internal declarations of the GB300 DMRG library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/dmrg.h"

namespace dmrg {

// Number of kernels this library has launched (reported by dmrg_launch_count).
extern std::atomic<long long> g_launch_count;
#define DMRG_COUNT_LAUNCH() (::dmrg::g_launch_count.fetch_add(1, std::memory_order_relaxed))

// Device status bits, OR-ed into ctx->d_status by kernels.
enum : int {
    ST_TIMEOUT = 1,   // a bounded spin-wait gave up
    ST_NAN = 2,       // non-finite value met
    ST_NOCONV = 4,    // Jacobi did not converge
    ST_BOUNDS = 8     // an index check failed (debug builds)
};

// Upper bound on polling iterations of any device-side wait (each iteration
// sleeps ~100 ns, so the bound is of the order of a few seconds).
constexpr long long kSpinLimit = 20000000LL;

#define DMRG_CUDA(call)                                                               \
    do {                                                                              \
        cudaError_t e__ = (call);                                                     \
        if (e__ != cudaSuccess) {                                                     \
            std::fprintf(stderr, "dmrg: %s failed at %s:%d: %s\n", #call, __FILE__,   \
                         __LINE__, cudaGetErrorString(e__));                          \
            return DMRG_ECUDA;                                                        \
        }                                                                             \
    } while (0)

#define DMRG_TRY(expr)                       \
    do {                                     \
        dmrg_status s__ = (expr);            \
        if (s__ != DMRG_OK) return s__;      \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    dmrg_status ensure(size_t need) {
        if (need <= bytes) return DMRG_OK;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (cudaMalloc(&ptr, need) != cudaSuccess) return DMRG_ENOMEM;
        bytes = need;
        return DMRG_OK;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Scratch of the one-sided Jacobi SVD.
struct SvdWork {
    double *X = nullptr;    // r x l: the r vectors being orthogonalised
    double *Vm = nullptr;   // r x r: accumulated rotations
    double *nrm = nullptr;  // r    : column norms
    int *perm = nullptr;    // r    : descending order
    unsigned *sync = nullptr;  // grid barrier words (2) + rotation counters (2)
};

// FP32 Jacobi problems of at most this many floats (r vectors x length l)
// fit one CTA's shared memory: the single-CTA kernels take them.
constexpr int kSmemJacFloats = 50 * 1024;

// Bytes needed by the Jacobi scratch for r vectors of length l.
size_t svd_work_bytes(int r, int l);
SvdWork svd_work_carve(void *base, int r, int l);

}  // namespace dmrg

namespace dmrg {
// Live per-kernel timing (CUDA events on the context stream), enabled by
// dmrg_profile; used for the roofline of the dominant kernel.
enum ProfKind {
    PROF_TC_GEMM = 0, PROF_JACOBI32 = 1, PROF_JACOBI64 = 2, PROF_F64_GEMM = 3, PROF_MIX = 4, PROF_F32_GEMM = 5,
    PROF_QR = 6, PROF_LZ_VEC = 7, PROF_DECIDE = 8, PROF_KINDS = 9
};
struct ProfSlot {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    long long n = 0;
    double flops = 0.0, bytes = 0.0;
};
}  // namespace dmrg

struct dmrg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int *d_status = nullptr;     // device status word (ST_* bits)
    int *h_pinned_i = nullptr;   // pinned host readback area (64 ints)
    double *h_pinned_d = nullptr;// pinned host readback area (64 doubles)
    dmrg::DevBuf work;           // scratch for standalone calls
    dmrg::DevBuf work2;
    dmrg::DevBuf work3;
    int jacobi_max_sweeps = 60;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // tensor-core GEMM path
    dmrg::DevBuf tcbuf;          // split TF32 operands
    dmrg::DevBuf f64buf;         // split-K partial sums of the FP64 GEMM
    int tc_ok = -1;              // -1 unknown, 0 no, 1 yes
    int tc_bn_override = 0;      // force a tile width (autotuner / tests)
    int tc_force = 0;            // use the tensor cores even for tiny products
    double tc_min_work = 16777216.0;  // M*N*K below which the FP32 CUDA-core kernel takes 3xTF32 requests
                                      // (measured: chi 64 update 2.60 -> 2.41 ms against 2^22; neutral at 48, 96, 128)
    int tc_split_kb = 8;         // tensor-core GEMM: at most this many 32-wide K' blocks per FP32 accumulator
                                 // (split K with an FP64 reduction beyond; 0 = never split)
    int prof = 0;
    int prof_mask = 0x1ff;       // kinds bracketed by events while profiling (bit k = kind k)
    dmrg::ProfSlot prof_slot[dmrg::PROF_KINDS];
    int mixed_env_tc = 0;        // 1: environment updates of the mixed form on the tensor cores too
    int svd_prec = 0;            // standalone svd_truncate: 0 FP64 Jacobi, 1 mixed
    int bjac_pairs = 48;        // blocked FP32 Jacobi: target block pairs per round
    int bjac_inner = 1;          // blocked FP32 Jacobi: max inner sweeps per block pair
    double mlp_eps_target = 1e-5;// truncation-error target of the learned scheduler's label
    // autotuner decisions (autotune.cu): tensor-core tile width per GEMM
    // shape bucket, blocked-Jacobi grid target and inner sweeps per SVD
    // size bucket; buckets are ceil(log2) of each dimension
    // GEMM bucket: tile width (64, 128, 256) and split depth (K blocks per
    // FP32 accumulator, 4 or 8), with the time of each width at that depth
    struct TuneGemm { int lm, ln, lk, bn; float ms128, ms256; int kb = 0; float ms64 = 0.f; };
    // SVD bucket: the old blocked kernel's block-pair target and inner sweeps,
    // the grouped kernel's vectors per block pair (nv) and groups per CTA, and
    // the cluster kernel's size (cj: 8 or 16 CTAs, 0 = not the cluster kernel,
    // -1 = no choice recorded)
    struct TuneSvd { int lr, ll, pairs, inner; float ms; int nv, groups; int cj = -1; int tj = 0; };
    std::vector<TuneGemm> tune_gemm;
    std::vector<TuneSvd> tune_svd;
    dmrg::DevBuf work4;          // batched SVD workspace
    dmrg::DevBuf tjbuf;          // tensor-core block Jacobi workspace (tjacobi.cu)
    int tjac = 128;              // FP32 Jacobi: tensor-core block form with pairs of tjac (64, 128) vectors; 0 = off
    int tjac_min_r = 3072;       // ... from this many vectors on (ahead of the other kernels; measured faster
                                 // than the blocked grid kernel at 3072 and 4096 vectors, slower at 2048 and 2560)
    int batched_inner = 4;       // batched SVD: inner Jacobi sweeps per block pair
    int batched_ns = 1;          // FP32 batched SVD: Newton-Schulz step on each block rotation
    int jacobi_qr = 1;           // FP32 Jacobi on the R factor of the vectors (QR preconditioning)
    int jacobi_rank_drop = 1;    // ... and only on its rows above the FP32 noise (numerical row rank)
    int bjac_gram = 1;           // blocked FP32 Jacobi: inner sweep in Gram form (k_bjac32g)
    double jacobi32_floor = 1.1920928955078125e-07;   // FP32 Jacobi: vectors below this x |A|_F take no rotation
    int gbj_min_r = 0;           // FP32 Jacobi: Gram-block cooperative form from this many vectors on (0 = off)
    double jacobi32_tol = 1e-6;  // FP32 Jacobi: rotate while a pair's cosine exceeds this
    int mixed_svd64 = 0;         // 3xTF32 form with the FP64 SVD and split (contractions alone in reduced precision)
    int qr_wpanel = 1;           // QR panels of <= 256 rows: one warp per column (k_qr_panel_w)
    int f64_fill = 1;            // FP64 GEMM: 32 x 32 tiles and split K when 64 x 64 tiles leave SMs idle
    int f32_fill = 1;            // the same for the FP32 small products of the mixed form
    int tc_presplit = 1;         // matvec: L, R split once per update; x and the mix output split by their producers
    int lz_fused = 1;            // Lanczos: one cooperative launch per step for the orthogonalisation
    long long lz_cluster_n = 4096;    // ... on one thread-block cluster instead, for vectors up to this length (0 = never):
                                      // measured faster at 4096 (chi 32), slower at 16384 (chi 64)
    int cjac32 = 1;              // FP32 Jacobi: one-cluster kernel (cjacobi.cu) from cjac_min_r vectors on
    int cjac_min_r = 32;
    int cjac_force_c = 0;        // cluster Jacobi: 8 or 16 CTAs forced (autotuner, option), 0 = by size
    int gjac32 = 0;              // FP32 Jacobi: grouped block kernel (gjacobi.cu): 0 never, 1 small problems, 2 always
    int gjac_nv = 0;             // ... vectors per block pair (16, 32; 0 = by size)
    int gjac_groups = 0;         // ... max groups per CTA (0 = by shared memory)
    int jacobi64_gram = 1;       // FP64 Jacobi: grouped block kernel (0: one warp per pair)
    int jacobi64_precond = 1;    // FP64 Jacobi: FP32 preconditioning pass
    double batched_floor32 = 1.1920928955078125e-07;  // FP32 batched SVD: vectors below this x |A|_F do not rotate
    void *pinned_desc = nullptr; // batched SVD descriptors (pinned, read by the H2D copy / graph replays)
    size_t pinned_desc_bytes = 0;
};

namespace dmrg {
inline void prof_mark(dmrg_ctx *ctx, int kind)
{
    if (!ctx || !ctx->prof || !((ctx->prof_mask >> kind) & 1)) return;
    ProfSlot &p = ctx->prof_slot[kind];
    if (p.used == p.ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p.ev.push_back(e);
    }
    cudaEventRecord(p.ev[p.used++], ctx->stream);
}
inline void prof_count(dmrg_ctx *ctx, int kind, double flops, double bytes)
{
    if (!ctx || !ctx->prof || !((ctx->prof_mask >> kind) & 1)) return;
    ProfSlot &p = ctx->prof_slot[kind];
    p.n++;
    p.flops += flops;
    p.bytes += bytes;
}
}  // namespace dmrg

namespace dmrg {

// ---------------------------------------------------------------------------
// Bounded grid barrier for kernels launched cooperatively (all blocks
// co-resident).  words[0] = arrival count, words[1] = generation.
// Returns false (and sets ST_TIMEOUT) if the wait gave up.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(unsigned *words, int *status, long long spin_limit = kSpinLimit)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = words + 1;
        unsigned g = *gen;
        __threadfence();
        unsigned arrived = atomicAdd(words, 1u);
        if (arrived == gridDim.x * gridDim.y - 1) {
            atomicExch(words, 0u);
            __threadfence();
            atomicAdd(words + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (spins > 4096) __nanosleep(64);
                if (++spins > spin_limit) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Warp and block reductions (FP64).
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of blockDim.x threads (multiple of 32, <= 1024); result
// returned to every thread.  Fixed reduction order (deterministic).
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 32 */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Host-side launchers implemented in the other translation units.
// ---------------------------------------------------------------------------

// Gram-block FP32 Jacobi of one matrix on a cooperative grid (batched.cu).
size_t gbj32_padded_bytes(int r, int l);
size_t cjac32_smem_bytes(int r, int l);
bool cjac32_fits(int r, int l);
dmrg_status cjac32_run(dmrg_ctx *ctx, float *X, int r, int l, int max_sweeps, double tol, double small,
                       const double *F2, int *d_info, const int *r_eff, int force_c = 0);
bool cjac32_fits_c(int r, int l, int C);
dmrg_status gbj32_sweeps(dmrg_ctx *ctx, const double *A, int m, int n, int dir, float *X, float *Xp, void *qrw,
                         unsigned *sync, int max_sweeps, double tol, double small, int *d_info);
dmrg_status frob2_f32(dmrg_ctx *ctx, const float *A, long long n, double *F2);

// QR preconditioning of the FP32 Jacobi (qr.cu): X (c x l) <- R of X = QR.
size_t qr32_work_bytes(int c);
dmrg_status qr_precondition32(dmrg_ctx *ctx, float *X, int c, int l, void *work);

// Autotuner table lookups (autotune.cu): 0 / false when the bucket has no entry.
int tune_lookup_bn(const dmrg_ctx *ctx, int M, int N, int K, int *kb = nullptr);
int tune_lookup_cj(const dmrg_ctx *ctx, int r, int l);
// tensor-core block Jacobi chosen for this bucket: its pair width (64, 128);
// 0 another kernel; -1 no entry
int tune_lookup_tj(const dmrg_ctx *ctx, int r, int l);
bool tune_lookup_svd(const dmrg_ctx *ctx, int r, int l, int *pairs, int *inner);
bool tune_lookup_gjac(const dmrg_ctx *ctx, int r, int l, int *nv, int *groups);

// FP64 strided batched GEMM:
//   C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n)
// with A(m,k) = A[b*sAb + m*sAm + k*sAk], etc., for b < batch.
dmrg_status gemm_f64(cudaStream_t st, int M, int N, int K, double alpha, const double *A, long long sAm,
                     long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                     double beta, double *C, long long sCm, long long sCn, long long sCb, int batch);

// Same contract, with the grid sized to the GPU (32 x 32 tiles, split K)
// when 64 x 64 tiles would leave SMs idle; scratch from the context.
dmrg_status gemm_f64x(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                      long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                      double beta, double *C, long long sCm, long long sCn, long long sCb, int batch);

// Same contract with FP32 arithmetic (small products of the mixed form).
dmrg_status gemm_f32c(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                      long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                      double beta, double *C, long long sCm, long long sCn, long long sCb, int batch);

// Tensor-core GEMM (tcgen05, TF32 inputs split three ways, FP32 accumulate):
// same contract as gemm_f64 (FP64 in, FP64 out), precision ~FP32.
dmrg_status gemm_3xtf32(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                        long long sAk, long long sAb, const double *B, long long sBk, long long sBn,
                        long long sBb, double beta, double *C, long long sCm, long long sCn, long long sCb,
                        int batch);
bool tc_available(dmrg_ctx *ctx);
// Whether gemm_3xtf32 of this shape runs on the tensor cores (else on the
// FP32 CUDA-core kernel): the split operands below are only read there.
bool tc_path(dmrg_ctx *ctx, int M, int N, int K, int batch);
// Padded K of the split layout: the three TF32 parts of a row of K values
// lie at [0, Kp), [Kp, 2 Kp), [2 Kp, 3 Kp), zero beyond K, Kp = K rounded up to 32.
inline int split_kp(int K) { return (K + 31) / 32 * 32; }
// Split operand in the tensor-core layout: out[b][row][slice * Kp + col] for
// the R x Kc operand element (row, col) at in[b s_b + row s_row + col s_col].
// pattern 0 (left operand): (hi, hi, lo); pattern 1 (right operand): (hi, lo, hi).
dmrg_status split3_dev(dmrg_ctx *ctx, const double *in, long long s_row, long long s_col, long long s_b, int R,
                       int Kc, int batch, int pattern, float *out);
// gemm_3xtf32 with either operand already split (nullptr: split here).
dmrg_status gemm_3xtf32_pre(dmrg_ctx *ctx, int M, int N, int K, double alpha, const double *A, long long sAm,
                            long long sAk, long long sAb, const double *B, long long sBk, long long sBn,
                            long long sBb, double beta, double *C, long long sCm, long long sCn, long long sCb,
                            int batch, const float *Ah_pre, const float *Bh_pre);

// tcgen05 product of operands the caller has split already: Ah [batch][M][K3],
// Bh [batch][N][K3] (K-major, K3 a multiple of 32, e.g. the (hi, hi, lo) and
// (hi, lo, hi) layouts above), tile width bn (64, 128, 256).  Exactly one of
// C64 / C32 is given: C64[b sCb + m sCm + n sCn] = the product in FP64, the K'
// blocks spread over nsl slices whose FP32 sums (FP64 scratch P, nsl * batch *
// M * N doubles) are added in FP64; C32 = the FP32 accumulator itself (nsl 1).
// seg_map != 0: the operands store fewer K segments than the product reads
// (K3 = 3 segments of K3 / 3 each, e.g. (hi, lo) stored once per operand):
// nibble q (q < 3) of seg_map is the stored segment A reads as K' segment q,
// nibble 3 + q the one B reads; e.g. 0x010100 reads A as (hi, hi, lo) and B
// as (hi, lo, hi) from (hi, lo) storage of 2 K3 / 3 floats a row.
dmrg_status tc_gemm_split(dmrg_ctx *ctx, const float *Ah, const float *Bh, int M, int N, int K3, int batch, int bn,
                          int nsl, double *P, double *C64, float *C32, long long sCm, long long sCn, long long sCb,
                          unsigned seg_map = 0u);
// Tile width (64, 128, 256) the tensor-core GEMM takes for this shape.
int tc_pick_bn(dmrg_ctx *ctx, int M, int N, int K, int batch);

// FP32 -> FP64 by integer operations (exact, like the converting
// instruction, which runs on the narrow FP64 pipe of this part); zeros,
// subnormals, infinities and NaNs take the instruction.
__device__ __forceinline__ double f32_widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    if (e == 0u || e == 0xffu) return (double)f;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// FP64 -> FP32 rounded to nearest even by integer operations, bit-identical
// to the converting instruction in the normal range; zeros, subnormal or
// overflowing results, infinities and NaNs take the instruction.
__device__ __forceinline__ float f64_narrow(double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);
    if (e < 897u || e > 1150u) return (float)v;             // outside the FP32 normal exponents
    // 23 kept mantissa bits: 20 from hi, 3 from lo; 29 dropped bits in lo
    uint32_t r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t drop = lo & 0x1fffffffu;
    if (drop > 0x10000000u || (drop == 0x10000000u && (r & 1u))) ++r;   // a carry may reach the exponent
    if ((r >> 23) >= 0xffu) return (float)v;                 // rounded up to infinity
    return __uint_as_float(r | (hi & 0x80000000u));
}

// hi = tf32(float(v)), lo = tf32(float(v - hi)): the two TF32 parts of an
// FP64 value (the split of the 3xTF32 products)
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void tf32_split(double v, float &hi, float &lo)
{
    // conversions by integer operations; the one subtraction is exact
    hi = tf32_rna(f64_narrow(v));
    lo = tf32_rna(f64_narrow(v - f32_widen(hi)));
}

// Where a producer kernel also writes the right-operand split of the vector
// it produces, viewed as a K x n4 row-major matrix (element i = k n4 + c):
// h[c 3Kp + k] = hi, h[c 3Kp + Kp + k] = lo, h[c 3Kp + 2Kp + k] = hi.
struct SplitSink {
    float *h = nullptr;
    long long n4 = 0;
    int Kp = 0;
};
__device__ __forceinline__ void sink_write(const SplitSink &s, long long i, double v)
{
    float hi, lo;
    tf32_split(v, hi, lo);
    const long long k = i / s.n4, c = i - k * s.n4;
    float *o = s.h + c * 3LL * s.Kp + k;
    o[0] = hi;
    o[s.Kp] = lo;
    o[2LL * s.Kp] = hi;
}

// Dispatch on precision.
dmrg_status gemm(dmrg_ctx *ctx, int prec, int M, int N, int K, double alpha, const double *A, long long sAm,
                 long long sAk, long long sAb, const double *B, long long sBk, long long sBn, long long sBb,
                 double beta, double *C, long long sCm, long long sCn, long long sCb, int batch);

// One-sided Jacobi SVD of the row-major m x n matrix A (device).  Writes U
// (m x r), s (r, descending), Vt (r x n), r = min(m,n).  `work` must hold
// svd_work_bytes(r, max(m,n)), or svd_work_bytes_base(r, max(m,n)) with
// precond = 0.  The FP64 sweep count is written to d_info[0] (negative if
// not converged).  precond: 1 = FP32 preconditioning pass (r >= 64),
// 0 = none, -1 = the context's choice.
size_t svd_work_bytes_base(int r, int l);
dmrg_status svd_jacobi(dmrg_ctx *ctx, const double *A, int m, int n, double *U, double *s, double *Vt,
                       void *work, int max_sweeps, int *d_info, int precond = -1);

// Grouped block one-sided Jacobi (gjacobi.cu) on r extended vectors: vector
// i is X[i*ldx + e], e < l (the Gram part), then X[i*ldx + gv0 + e'], e' < rv
// (carried along).  nv = 16 or 32 vectors per block pair; max_groups > 0
// caps the groups per CTA.  sync: 4 words zeroed by the call.
template <typename T>
dmrg_status gjac_run(dmrg_ctx *ctx, T *X, int r, int l, int ldx, int gv0, int rv, int max_sweeps, double tol,
                     double small, const double *F2, unsigned *sync, int *info, const int *r_eff, int nv,
                     int max_groups);

// Blocked one-sided Jacobi with tcgen05 Gram blocks and block rotations
// (tjacobi.cu) on the r x l FP32 rows of X, in place; TB = 64 or 128 vectors
// per block pair.  DMRG_EUNSUPPORTED without tensor cores or while the
// stream is captured (it reads a convergence counter once per sweep).
dmrg_status tjac_run(dmrg_ctx *ctx, float *X, int r, int l, int max_sweeps, double tol, double small,
                     const double *F2, int *d_info, int TB);
size_t tjac_work_bytes(dmrg_ctx *ctx, int r, int l, int TB);

// FP32 one-sided Jacobi (mixed-precision form), vectors = columns (dir 0) or
// rows (dir 1) of A; see jacobi.cu.
size_t jac32_work_bytes(int r, int l);
dmrg_status svd_jacobi32(dmrg_ctx *ctx, const double *A, int m, int n, int dir, void *work, int max_sweeps,
                         int *d_info, double *s_sorted, float **X_out, double **nrm_out, int **perm_out);
dmrg_status gather_unit_vectors(dmrg_ctx *ctx, const float *X, const double *nrm, const int *perm, const int *kdev,
                                int kmax, int l, double *Q);

// Split of a truncated SVD (the retained k from res, renormalised by its
// znorm) into site tensors: A_k = U (and A_{k+1} = s Vt) when the centre moves
// right, A_k = U s and A_{k+1} = Vt otherwise; kmax bounds k for the grid.
struct BondResult;
dmrg_status launch_split(dmrg_ctx *ctx, const double *U, const double *s, const double *Vt, int m, int n, int r,
                         const BondResult *res, int go_right, double *Ak, double *Ak1, int kmax);
dmrg_status launch_init_ctrl(dmrg_ctx *ctx, dmrg_ctrl_state *st, int n, int chi0);

// Lanczos on the effective Hamiltonian (see lanczos.cu).
struct HeffOp;  // defined in dmrg_core.cu
}  // namespace dmrg
