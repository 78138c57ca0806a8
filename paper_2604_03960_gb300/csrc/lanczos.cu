// lanczos.cu -- Lanczos eigensolver for the local problem H_eff theta = E theta (Eq. 19).
//
// The paper leaves the local eigensolver unnamed; this is the K-step Lanczos
// recurrence with full reorthogonalisation by two classical Gram-Schmidt
// passes, all in FP64 and all on the device:
//   v0 = theta/|theta|;  w = H v_j;  w -= V (V^T w) (twice, against v_0..v_j);
//   alpha_j = v_j . H v_j (the first pass's coefficient on v_j; that pass also
//   removes alpha_j v_j + beta_j v_{j-1}, the three-term step);
//   beta_{j+1} = |w|;  v_{j+1} = w / beta_{j+1}
// stopping early (device flag, no host round trip) when beta < 1e-14 max|alpha|.
// The K x K tridiagonal T is solved on the device by Sturm-sequence
// bisection for its lowest eigenvalue and inverse iteration for the vector;
// the Ritz vector is V y0, normalised.  The vector kernels are HBM-bound
// streams; every reduction is deterministic (per-block partials summed in
// block order by the last block to finish).
#include "common.cuh"
#include "lanczos.cuh"

#include <cooperative_groups.h>

namespace dmrg {
namespace {

constexpr int RB = 256;        // threads per block of the vector kernels
constexpr int MAXQ = 24;       // max vectors in one multi-dot

// c[q] = sum_i V[q][i] * w[i] for q < nq, plus (if want_norm) c[nq] = |w|^2.
// Results go to out[] through `mode`:
//   mode 0: out[q] = c[q]
//   mode 1: alpha step: lz->alpha[j] = c[0], lz->amax = max
//   mode 2: beta step:  beta = sqrt(c[0]) ...
struct ReduceArgs {
    const double *V;      // vectors, stride ldv
    long long ldv;
    int nq;
    const double *w;      // second operand
    long long n;
    double *partials;     // gridDim.x * (MAXQ+1)
    unsigned *counter;    // zero on entry, reset by the last block
};

template <int MODE>
__global__ void __launch_bounds__(RB) k_multidot(ReduceArgs a, LzState *lz, int j, double *out)
{
    if (MODE != 3 && lz && !lz->active) return;
    __shared__ double sh[32];
    __shared__ bool last;
    const int nq = a.nq;
    double acc[MAXQ + 1];
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q) acc[q] = 0.0;
    const long long stride = (long long)gridDim.x * RB;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < a.n; i += stride) {
        double wi = a.w[i];
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) acc[q] = fma(a.V[(long long)q * a.ldv + i], wi, acc[q]);
        acc[MAXQ] = fma(wi, wi, acc[MAXQ]);
    }
    // block reduction of all nq + 1 sums at once: the partial sums go to
    // shared memory column by column and one warp adds up each column (FP64
    // adds are scarce on this part: 255 of them per column is the minimum,
    // where a shuffle tree per column would spend 5 x 32 per warp)
    extern __shared__ double red[];            // (MAXQ + 1) x RB
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q)
        if (q < nq || q == MAXQ) red[q * RB + threadIdx.x] = acc[q];
    __syncthreads();
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int q = warp; q <= MAXQ; q += RB / 32) {
            if (!(q < nq || q == MAXQ)) continue;
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < RB / 32; ++k) s += red[q * RB + lane + 32 * k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) a.partials[(long long)blockIdx.x * (MAXQ + 1) + q] = s;
        }
    }
    (void)sh;
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned done = atomicAdd(a.counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // final reduction, warp q' over columns q = q', q' + 8, ...: each lane sums
    // the blocks b = lane, lane + 32, ... in order, then a fixed shuffle tree
    // (all loads of a column are in flight at once; the order is fixed)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q <= MAXQ; q += RB / 32) {
        if (!(q < nq || q == MAXQ)) continue;
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            s += *(volatile double *)&a.partials[(long long)b * (MAXQ + 1) + q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane != 0) continue;
        if (MODE == 0 || MODE == 4) {
            out[q] = s;
            if (MODE == 4 && q == j) {  // first Gram-Schmidt pass on w = H v_j: alpha_j = v_j . w
                lz->alpha[j] = s;
                if (fabs(s) > lz->amax) lz->amax = fabs(s);
            }
        } else if (MODE == 1) {        // alpha_j = v_j . w
            if (q == 0) {
                lz->alpha[j] = s;
                if (fabs(s) > lz->amax) lz->amax = fabs(s);
            }
        } else if (MODE == 2) {        // beta_{j+1} = |w|, decide continuation
            if (q == MAXQ) {
                double b = sqrt(s);
                lz->beta[j + 1] = b;
                lz->m = j + 1;
                if (j + 1 >= lz->K || !(b > 1e-14 * lz->amax) || !isfinite(b)) lz->active = 0;
                if (!isfinite(b)) lz->nan = 1;
            }
        } else if (MODE == 3) {        // |theta| for the start vector / Ritz vector
            if (q == MAXQ) lz->scale = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
        }
    }
    if (threadIdx.x == 0) *a.counter = 0u;
}

// w -= sum_q c[q] V[q]   (or w = sum_q c[q] V[q] when overwrite)
__global__ void k_multiaxpy(double *__restrict__ w, const double *__restrict__ V, long long ldv, int nq,
                            const double *__restrict__ c, long long n, const LzState *lz, int check_active,
                            int overwrite)
{
    if (check_active && !lz->active) return;
    if (nq < 0) nq = lz->m;     // Ritz combination: only the vectors actually built
    __shared__ double cs[MAXQ];
    if (threadIdx.x < nq) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc = fma(cs[q], V[(long long)q * ldv + i], acc);
        w[i] = overwrite ? acc : w[i] - acc;
    }
}

// Second Gram-Schmidt pass fused with the norm: w -= sum_q c[q] V[q], then
// beta_{j+1} = |w| (per-block partial sums of squares, summed in block order
// by the last block, which also decides whether the recurrence continues).
__global__ void __launch_bounds__(RB) k_multiaxpy_norm(double *__restrict__ w, const double *__restrict__ V,
                                                       long long ldv, int nq, const double *__restrict__ c,
                                                       long long n, LzState *lz, int j, double *partials,
                                                       unsigned *counter)
{
    if (!lz->active) return;
    __shared__ double cs[MAXQ];
    __shared__ double red[RB / 32];
    __shared__ bool last;
    if (threadIdx.x < nq) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    double ss = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc = fma(cs[q], V[(long long)q * ldv + i], acc);
        const double v = w[i] - acc;
        w[i] = v;
        ss = fma(v, v, ss);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RB / 32; ++k) t += red[k];
        partials[blockIdx.x] = t;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block sums the partials in a fixed order (all loads at once)
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RB) t += *(volatile double *)&partials[b];
    __shared__ double sh[32];
    t = block_sum(t, sh);
    if (threadIdx.x != 0) return;
    const double bta = sqrt(t);
    lz->beta[j + 1] = bta;
    lz->m = j + 1;
    if (j + 1 >= lz->K || !(bta > 1e-14 * lz->amax) || !isfinite(bta)) lz->active = 0;
    if (!isfinite(bta)) lz->nan = 1;
    *counter = 0u;
}

// Column sums of acc[q] over the block (FP64, fixed order) for q < nq and,
// with `last`, q = MAXQ, written to part[q]; red: (MAXQ + 1) x OB doubles of
// shared memory (OB: block size).
template <int OB>
__device__ __forceinline__ void block_cols_to(const double *acc, int nq, bool last, double *red, double *part)
{
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q)
        if (q < nq || (last && q == MAXQ)) red[q * OB + threadIdx.x] = acc[q];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q <= MAXQ; q += OB / 32) {
        if (!(q < nq || (last && q == MAXQ))) continue;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < OB / 32; ++k) s += red[q * OB + lane + 32 * k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[q] = s;
    }
}

// Sum of the blocks' partials part[b * stride + q] (the same columns), in
// block order (every CTA gets the same bits); result to cs[q].
template <int OB>
__device__ __forceinline__ void sum_parts(const double *part, int stride, int nq, bool last, double *cs)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q <= MAXQ; q += OB / 32) {
        if (!(q < nq || (last && q == MAXQ))) continue;
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&part[(long long)b * stride + q]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cs[q] = s;
    }
    __syncthreads();
}

// grid barrier of the fused step; a one-block grid needs only the block's
__device__ __forceinline__ bool lz_barrier(unsigned *bar, int *status)
{
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    return grid_barrier(bar, status);
}

// One Lanczos step's orthogonalisation in one cooperative launch (the five
// launches above fused; two bounded grid barriers):
//   c = V^T w (v_0..v_j), alpha_j = c_j;  w1 = w - V c, and in the same pass
//   c' = V^T w1 and |w1|^2;  beta_{j+1} = |w1 - V c'| from |w1|^2 - |c'|^2,
//   continuation as in k_multiaxpy_norm;  v_{j+1} = (w1 - V c') / beta_{j+1}
//   if the recurrence goes on.
// Each thread keeps its elements' v_q in registers between the update and
// the next dot product, so V is read three times instead of four.
// part: 3 x gridDim.x x (MAXQ + 1) doubles; bar: two zeroed words.
template <int OB>
__global__ void __launch_bounds__(OB) k_lz_orth(double *__restrict__ V, double *__restrict__ w, long long n, int j,
                                                LzState *lz, double *__restrict__ part, unsigned *bar, int *status,
                                                SplitSink sink)
{
    if (!lz->active) return;                 // written by an earlier launch: the same in every CTA
    extern __shared__ double red[];          // (MAXQ + 1) x OB
    __shared__ double cs[MAXQ + 1];
    const int nq = j + 1;
    const int K = lz->K;
    const double amax0 = lz->amax;
    const int S = MAXQ + 1;
    double *p0 = part, *p1 = part + (long long)gridDim.x * S, *p2 = part + 2LL * gridDim.x * S;
    const long long stride = (long long)gridDim.x * OB;
    const long long i0 = (long long)blockIdx.x * OB + threadIdx.x;
    double acc[MAXQ + 1];
    // phase A: c = V^T w
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q) acc[q] = 0.0;
    for (long long i = i0; i < n; i += stride) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) acc[q] = fma(V[(long long)q * n + i], wi, acc[q]);
    }
    block_cols_to<OB>(acc, nq, false, red, p0 + (long long)blockIdx.x * S);
    if (!lz_barrier(bar, status)) return;
    sum_parts<OB>(p0, S, nq, false, cs);
    const double alpha = cs[j];
    const double amax = fmax(amax0, fabs(alpha));
    // phase B: w1 = w - V c; c' = V^T w1 and |w1|^2 in the same pass
    double acc2[MAXQ + 1];
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q) acc2[q] = 0.0;
    for (long long i = i0; i < n; i += stride) {
        double v[MAXQ];
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) {
                v[q] = V[(long long)q * n + i];
                a = fma(cs[q], v[q], a);
            }
        const double wi = w[i] - a;
        w[i] = wi;
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) acc2[q] = fma(v[q], wi, acc2[q]);
        acc2[MAXQ] = fma(wi, wi, acc2[MAXQ]);
    }
    __syncthreads();                         // cs is rewritten below
    block_cols_to<OB>(acc2, nq, true, red, p1 + (long long)blockIdx.x * S);   // |w1|^2 in column MAXQ
    if (!lz_barrier(bar, status)) return;
    sum_parts<OB>(p1, S, nq, true, cs);
    // phase C: beta_{j+1}^2 = |w1 - V c'|^2 = |w1|^2 - |c'|^2 (V has
    // orthonormal columns and c' = V^T w1 is tiny after the first pass, so
    // the difference loses nothing); continuation; v_{j+1} = (w1 - V c') / beta
    double cc = 0.0;
    for (int q = 0; q < nq; ++q) cc = fma(cs[q], cs[q], cc);
    const double b2 = cs[MAXQ] - cc;
    const double bta = b2 > 0.0 ? sqrt(b2) : (b2 == 0.0 ? 0.0 : b2);   // negative: not finite below
    const bool go = (j + 1 < K) && (bta > 1e-14 * amax) && isfinite(bta);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        lz->alpha[j] = alpha;
        lz->amax = amax;
        lz->beta[j + 1] = bta > 0.0 ? bta : 0.0;
        lz->m = j + 1;
        if (!go) lz->active = 0;
        if (!isfinite(bta)) lz->nan = 1;
    }
    if (go) {
        const double inv = 1.0 / bta;
        double *vn = V + (long long)(j + 1) * n;
        for (long long i = i0; i < n; i += stride) {
            double a = 0.0;
#pragma unroll
            for (int q = 0; q < MAXQ; ++q)
                if (q < nq) a = fma(cs[q], V[(long long)q * n + i], a);
            const double v = (w[i] - a) * inv;
            vn[i] = v;
            if (sink.h) sink_write(sink, i, v);   // the next matvec's split right operand
        }
    }
}

// The same step on one thread-block cluster of C CTAs (no grid barrier):
// each CTA's partial sums stay in its shared memory, and after a cluster
// barrier every CTA adds the C partials through distributed shared memory in
// rank order (lane r reads rank r, then a butterfly), so all CTAs get the
// same bits.  Three cluster barriers a step: after each pass's partials, and
// before exit (no CTA leaves while another may read its partials).
template <int OB, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(OB)
    k_lz_orth_cl(double *__restrict__ V, double *__restrict__ w, long long n, int j, LzState *lz, SplitSink sink)
{
    if (!lz->active) return;                 // the same in every CTA of the cluster
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double red[];          // (MAXQ + 1) x OB
    __shared__ double pa[MAXQ + 1], pb[MAXQ + 1], cs[MAXQ + 1];
    const int rank = (int)cluster.block_rank();
    const int nq = j + 1;
    const int K = lz->K;
    const double amax0 = lz->amax;
    const long long stride = (long long)C * OB;
    const long long i0 = (long long)rank * OB + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto cluster_sum = [&](double *part, bool last) {
        for (int q = warp; q <= MAXQ; q += OB / 32) {
            if (!(q < nq || (last && q == MAXQ))) continue;
            double s = lane < C ? cluster.map_shared_rank(part, lane)[q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) cs[q] = s;
        }
        __syncthreads();
    };
    // phase A: c = V^T w
    double acc[MAXQ + 1];
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q) acc[q] = 0.0;
    for (long long i = i0; i < n; i += stride) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) acc[q] = fma(V[(long long)q * n + i], wi, acc[q]);
    }
    block_cols_to<OB>(acc, nq, false, red, pa);
    cluster.sync();
    cluster_sum(pa, false);
    const double alpha = cs[j];
    const double amax = fmax(amax0, fabs(alpha));
    // phase B: w1 = w - V c; c' = V^T w1 and |w1|^2 in the same pass
    double acc2[MAXQ + 1];
#pragma unroll
    for (int q = 0; q <= MAXQ; ++q) acc2[q] = 0.0;
    for (long long i = i0; i < n; i += stride) {
        double v[MAXQ];
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) {
                v[q] = V[(long long)q * n + i];
                a = fma(cs[q], v[q], a);
            }
        const double wi = w[i] - a;
        w[i] = wi;
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
            if (q < nq) acc2[q] = fma(v[q], wi, acc2[q]);
        acc2[MAXQ] = fma(wi, wi, acc2[MAXQ]);
    }
    __syncthreads();                         // cs is rewritten below
    block_cols_to<OB>(acc2, nq, true, red, pb);
    cluster.sync();
    cluster_sum(pb, true);
    // phase C, as in k_lz_orth
    double cc = 0.0;
    for (int q = 0; q < nq; ++q) cc = fma(cs[q], cs[q], cc);
    const double b2 = cs[MAXQ] - cc;
    const double bta = b2 > 0.0 ? sqrt(b2) : (b2 == 0.0 ? 0.0 : b2);
    const bool go = (j + 1 < K) && (bta > 1e-14 * amax) && isfinite(bta);
    if (rank == 0 && threadIdx.x == 0) {
        lz->alpha[j] = alpha;
        lz->amax = amax;
        lz->beta[j + 1] = bta > 0.0 ? bta : 0.0;
        lz->m = j + 1;
        if (!go) lz->active = 0;
        if (!isfinite(bta)) lz->nan = 1;
    }
    if (go) {
        const double inv = 1.0 / bta;
        double *vn = V + (long long)(j + 1) * n;
        for (long long i = i0; i < n; i += stride) {
            double a = 0.0;
#pragma unroll
            for (int q = 0; q < MAXQ; ++q)
                if (q < nq) a = fma(cs[q], V[(long long)q * n + i], a);
            const double v = (w[i] - a) * inv;
            vn[i] = v;
            if (sink.h) sink_write(sink, i, v);
        }
    }
    cluster.sync();
}

// The split of a vector for the next matvec (start vector; the unfused path)
__global__ void k_sink_vec(const double *__restrict__ v, long long n, SplitSink sink, const LzState *lz)
{
    if (lz && !lz->active) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) sink_write(sink, i, v[i]);
}

// dst = src * lz->scale  (start vector / Ritz vector normalisation)
__global__ void k_scale_by(double *__restrict__ dst, const double *__restrict__ src, long long n, const LzState *lz)
{
    const double s = lz->scale;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i] * s;
}

// v_{j+1} = w / beta_{j+1}
__global__ void k_next_vec(double *__restrict__ vn, const double *__restrict__ w, long long n, const LzState *lz, int j)
{
    if (!lz->active) return;
    const double inv = 1.0 / lz->beta[j + 1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) vn[i] = w[i] * inv;
}

__global__ void k_lz_init(LzState *lz, int K)
{
    lz->K = K;
    lz->m = 0;
    lz->active = 1;
    lz->amax = 0.0;
    lz->nan = 0;
    lz->scale = 0.0;
    for (int i = 0; i < LZ_MAXK + 1; ++i) { lz->beta[i] = 0.0; }
    for (int i = 0; i < LZ_MAXK; ++i) { lz->alpha[i] = 0.0; lz->y[i] = 0.0; }
}

// Number of eigenvalues of the m x m tridiagonal (a, b[1..m-1]) below x:
// the negative pivots q_i = p_i / p_{i-1} of T - x I (Sylvester's inertia),
// read off as sign changes of the leading minors p_i = (a_i - x) p_{i-1} -
// b_i^2 p_{i-2} (b2[i] = b_i^2).  No division, and only the three FP64
// operations of the recurrence per step: signs, zero tests and the range
// test run on the integer bits (the FP64 pipe is narrow on this part).  The
// minors are rescaled by 2^-500 / 2^500 when their exponent leaves
// [-500, 500], which keeps every ratio.  A zero minor takes the sign of the
// previous one (its pivot counts as +0, as in the quotient form).
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ int sturm_count(int m, const double *a, const double *b2, double x)
{
    int cnt = 0;
    double pm = 1.0, p = a[0] - x;
    if ((dbits(p) << 1) == 0) p = 1e-300;
    cnt += dbits(p) < 0;
    for (int i = 1; i < m; ++i) {
        double pn = fma(a[i] - x, p, -b2[i] * pm);
        if ((dbits(pn) << 1) == 0) pn = dbits(p) < 0 ? -1e-300 : 1e-300;
        cnt += (dbits(pn) ^ dbits(p)) < 0;
        pm = p;
        p = pn;
        const int e = (int)((unsigned long long)dbits(p) >> 52) & 0x7ff;
        if (e > 1523) {                              // |p| >= 2^501
            p *= 3.054936363499605e-151;             // 2^-500
            pm *= 3.054936363499605e-151;
        } else if (e < 523) {                        // |p| < 2^-500
            p *= 3.273390607896142e150;              // 2^500
            pm *= 3.273390607896142e150;
        }
    }
    return cnt;
}

// The same count in FP32 on FP32 copies of T (64x the FP64 rate on this
// part): only used to narrow the bracket that the FP64 counts then refine.
__device__ int sturm_count_f(int m, const float *a, const float *b, float x)
{
    int cnt = 0;
    float pm = 1.f, p = a[0] - x;
    if (p == 0.f) p = 1e-30f;
    if (p < 0.f) cnt++;
    for (int i = 1; i < m; ++i) {
        float pn = fmaf(a[i] - x, p, -(b[i] * b[i]) * pm);
        if (pn == 0.f) pn = (p < 0.f) ? -1e-30f : 1e-30f;
        if ((pn < 0.f) != (p < 0.f)) cnt++;
        pm = p;
        p = pn;
        const float ap = fabsf(p);
        if (ap > 1.8446744e19f) {                    // 2^64
            p *= 5.421011e-20f;
            pm *= 5.421011e-20f;
        } else if (ap < 5.421011e-20f) {
            p *= 1.8446744e19f;
            pm *= 1.8446744e19f;
        }
    }
    return cnt;
}

// Lowest eigenpair of T by one warp: multisection with 32 Sturm counts per
// step (the interval shrinks 33x per step) until it is a few units in the
// last place wide, then inverse iteration on one lane.
__global__ void k_tridiag_lowest(LzState *lz, int *status)
{
    const int lane = threadIdx.x & 31;
    const int m = lz->m;
    __shared__ double a[LZ_MAXK], b[LZ_MAXK + 1], b2[LZ_MAXK + 1];  // b[i] couples i-1 and i
    __shared__ float af[LZ_MAXK], bf[LZ_MAXK + 1];
    for (int i = lane; i < m; i += 32) {
        a[i] = lz->alpha[i];
        af[i] = (float)a[i];
    }
    for (int i = lane; i <= m && i <= LZ_MAXK; i += 32) {
        b[i] = lz->beta[i];
        b2[i] = b[i] * b[i];
        bf[i] = (float)b[i];
    }
    __syncwarp();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < m ? fabs(b[i + 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    lo -= 1e-300;
    {
        // FP32 multisection down to about 1e-5 of the Gershgorin scale, then
        // a bracket widened by that much and checked with two FP64 counts
        // (none below lo, at least one below hi); if the check fails the
        // FP64 multisection starts from the Gershgorin interval instead
        const double scale = fmax(fabs(lo), fabs(hi));
        float flo = (float)lo, fhi = (float)hi;
        const float cf = (float)(lane + 1) * (1.f / 33.f);
        for (int it = 0; it < 8; ++it) {
            const float w = fhi - flo;
            if (!(w > 1e-6f * (float)scale)) break;
            const float x = fmaf(w, cf, flo);
            const unsigned below = __ballot_sync(0xffffffffu, sturm_count_f(m, af, bf, x) >= 1);
            const int f = below ? __ffs(below) - 1 : 31;
            const float xf = __shfl_sync(0xffffffffu, x, f), xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
            if (below == 0u) {
                flo = xf;                                  // every probe lies below lambda_0
            } else {
                flo = (f > 0) ? xp : flo;
                fhi = xf;
            }
        }
        const double margin = 1e-5 * scale;
        const double clo = fmax(lo, (double)flo - margin), chi = fmin(hi, (double)fhi + margin);
        int c = 0;
        if (lane < 2) c = sturm_count(m, a, b2, lane == 0 ? clo : chi);
        const int c_lo = __shfl_sync(0xffffffffu, c, 0), c_hi = __shfl_sync(0xffffffffu, c, 1);
        if (c_lo == 0 && c_hi >= 1 && clo < chi) {
            lo = clo;
            hi = chi;
        }
    }
    const double cd = (double)(lane + 1) * (1.0 / 33.0);
    for (int it = 0; it < 40; ++it) {
        const double w = hi - lo;
        if (!(w > 4.440892098500626e-16 * fmax(fabs(lo), fabs(hi)))) break;
        const double x = fmin(fma(w, cd, lo), hi);
        const unsigned below = __ballot_sync(0xffffffffu, sturm_count(m, a, b2, x) >= 1);
        const int f = below ? __ffs(below) - 1 : 31;   // first point at or above lambda_0
        const double xf = __shfl_sync(0xffffffffu, x, f), xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
        double nlo = lo, nhi = hi;
        if (below == 0u) {
            nlo = xf;
        } else {
            nhi = xf;
            nlo = (f > 0) ? xp : lo;
        }
        if (nlo == lo && nhi == hi) break;             // no representable progress
        lo = nlo;
        hi = nhi;
    }
    if (lane != 0) return;
    const double lam = 0.5 * (lo + hi);
    lz->E = lam;
    double y[LZ_MAXK], rhs[LZ_MAXK], rd[LZ_MAXK], ll[LZ_MAXK];
    const double shift = lam - 1e-13 * fmax(fabs(lam), 1e-300) - 1e-300;
    for (int i = 0; i < m; ++i) y[i] = 1.0 / sqrt((double)m) * (1.0 + 0.01 * i);
    // factor T - shift I once (LU without pivoting), keeping the reciprocal
    // pivots, so the two solves multiply instead of divide
    {
        double d = a[0] - shift;
        rd[0] = 1.0 / ((d != 0.0) ? d : 1e-300);
        for (int i = 1; i < m; ++i) {
            ll[i] = b[i] * rd[i - 1];
            d = (a[i] - shift) - ll[i] * b[i];
            rd[i] = 1.0 / ((d != 0.0) ? d : 1e-300);
        }
    }
    for (int it = 0; it < 2; ++it) {
        for (int i = 0; i < m; ++i) rhs[i] = y[i];
        for (int i = 1; i < m; ++i) rhs[i] -= ll[i] * rhs[i - 1];
        y[m - 1] = rhs[m - 1] * rd[m - 1];
        for (int i = m - 2; i >= 0; --i) y[i] = (rhs[i] - b[i + 1] * y[i + 1]) * rd[i];
        double nn = 0.0;
        for (int i = 0; i < m; ++i) nn += y[i] * y[i];
        nn = 1.0 / sqrt(nn);
        for (int i = 0; i < m; ++i) y[i] *= nn;
    }
    double sgn = 1.0;
    for (int i = 0; i < m; ++i) if (y[i] != 0.0) { sgn = (y[i] < 0.0) ? -1.0 : 1.0; break; }
    for (int i = 0; i < m; ++i) lz->y[i] = sgn * y[i];
    if (!isfinite(lam) || lz->nan) atomicOr(status, ST_NAN);
}

// multi-dot grid: one block per SM, so each thread accumulates several
// elements before the (FP64-add bound) block reduction
int grid_dot(long long n, int num_sms)
{
    long long b = (n + RB - 1) / RB;
    if (b > num_sms) b = num_sms;
    if (b < 1) b = 1;
    return (int)b;
}

// fused orthogonalisation: 128-thread blocks, one element a thread up to one
// block per SM (all co-resident: the launch is cooperative).  The FP64
// multiply-adds of the passes and of the block sums (2 a clock per SM on
// this part) grow with elements + threads per SM, and the grid barrier and
// the sum over blocks' partials with the block count; measured at 16,384
// elements: 28.4 us a step with 256 threads, 25.8 with 128, 40.9 with 64.
constexpr int kOB = 128;
int grid_orth(long long n, int num_sms)
{
    long long b = (n + kOB - 1) / kOB;
    if (b > num_sms) b = num_sms;
    if (b < 1) b = 1;
    return (int)b;
}

constexpr int kOBC = 256;     // threads per CTA of the cluster form (199 registers a thread)

// Whether a cluster of C CTAs of the cluster form can be resident (queried
// once per size; a launch that cannot is not attempted).
template <int C>
bool lz_cluster_fits()
{
    static int ok = -1;
    if (ok >= 0) return ok == 1;
    ok = 0;
    const int smem = (int)(sizeof(double) * (MAXQ + 1) * kOBC);
    if (cudaFuncSetAttribute(k_lz_orth_cl<kOBC, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (C > 8 && cudaFuncSetAttribute(k_lz_orth_cl<kOBC, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kOBC);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int nc = 0;
    ok = (cudaOccupancyMaxActiveClusters(&nc, (const void *)k_lz_orth_cl<kOBC, C>, &cfg) == cudaSuccess && nc >= 1)
             ? 1
             : 0;
    cudaGetLastError();
    return ok == 1;
}

int grid_for(long long n, int num_sms)
{
    long long b = (n + RB - 1) / RB;
    long long cap = (long long)num_sms * 4;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

size_t lanczos_work_bytes(long long n, int K, int num_sms)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t vecs = al(sizeof(double) * (size_t)n * (K + 1));   // V (K vectors) + w
    size_t parts = al(sizeof(double) * (size_t)num_sms * 4 * (MAXQ + 1));
    return vecs + parts + al(sizeof(LzState)) + al(sizeof(double) * (MAXQ + 1)) + al(64);
}

LanczosWork lanczos_work_carve(void *base, long long n, int K, int num_sms)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(base);
    LanczosWork w;
    w.V = reinterpret_cast<double *>(p);
    w.w = w.V + (size_t)n * K;
    p += al(sizeof(double) * (size_t)n * (K + 1));
    w.partials = reinterpret_cast<double *>(p); p += al(sizeof(double) * (size_t)num_sms * 4 * (MAXQ + 1));
    w.lz = reinterpret_cast<LzState *>(p); p += al(sizeof(LzState));
    w.c = reinterpret_cast<double *>(p); p += al(sizeof(double) * (MAXQ + 1));
    w.counter = reinterpret_cast<unsigned *>(p);
    return w;
}

dmrg_status lanczos_run(dmrg_ctx *ctx, const LanczosWork &w, long long n, int K, double *theta,
                        const MatvecFn &matvec, const SplitSink *sink_p)
{
    SplitSink sink;
    if (sink_p) sink = *sink_p;
    if (K < 1) K = 1;
    if (K > LZ_MAXK) K = LZ_MAXK;
    if ((long long)K > n) K = (int)n;
    cudaStream_t st = ctx->stream;
    const int g = grid_for(n, ctx->num_sms), gd = grid_dot(n, ctx->num_sms);
    const size_t dsm = sizeof(double) * (MAXQ + 1) * RB;
    static bool dsm_attr = false;
    if (!dsm_attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_multidot<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
        DMRG_CUDA(cudaFuncSetAttribute(k_multidot<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
        DMRG_CUDA(cudaFuncSetAttribute(k_multidot<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
        dsm_attr = true;
    }
    DMRG_CUDA(cudaMemsetAsync(w.counter, 0, 64, st));    // last-block counter and grid-barrier words
    k_lz_init<<<1, 1, 0, st>>>(w.lz, K); DMRG_COUNT_LAUNCH();
    ReduceArgs ra{nullptr, n, 0, theta, n, w.partials, w.counter};
    k_multidot<3><<<gd, RB, dsm, st>>>(ra, w.lz, 0, nullptr); DMRG_COUNT_LAUNCH();          // |theta|
    k_scale_by<<<g, RB, 0, st>>>(w.V, theta, n, w.lz); DMRG_COUNT_LAUNCH();                // v0
    if (sink.h) { k_sink_vec<<<g, RB, 0, st>>>(w.V, n, sink, nullptr); DMRG_COUNT_LAUNCH(); }
    DMRG_CUDA(cudaGetLastError());
    const int gc = grid_orth(n, ctx->num_sms);
    static bool orth_attr = false;
    if (!orth_attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_lz_orth<kOB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * (MAXQ + 1) * kOB)));
        orth_attr = true;
    }
    // cluster size of the cluster form (0: not available)
    const int lz_c = ctx->lz_cluster_n > 0 ? (lz_cluster_fits<16>() ? 16 : (lz_cluster_fits<8>() ? 8 : 0)) : 0;
    for (int j = 0; j < K; ++j) {
        double *vj = w.V + (size_t)n * j;
        DMRG_TRY(matvec(vj, w.w));
        prof_mark(ctx, PROF_LZ_VEC);
        if (ctx->lz_fused && n <= ctx->lz_cluster_n && (lz_c == 16 || lz_c == 8)) {
            // the same step on one thread-block cluster: hardware cluster
            // barriers instead of grid barriers
            const size_t sm = sizeof(double) * (MAXQ + 1) * kOBC;
            if (lz_c == 16)
                k_lz_orth_cl<kOBC, 16><<<16, kOBC, sm, st>>>(w.V, w.w, n, j, w.lz, sink);
            else
                k_lz_orth_cl<kOBC, 8><<<8, kOBC, sm, st>>>(w.V, w.w, n, j, w.lz, sink);
            DMRG_COUNT_LAUNCH();
            prof_mark(ctx, PROF_LZ_VEC);
            prof_count(ctx, PROF_LZ_VEC, 0.0, 8.0 * (double)n * (3.0 * (j + 1) + 7.0));
            DMRG_CUDA(cudaGetLastError());
            continue;
        }
        if (ctx->lz_fused) {
            // both Gram-Schmidt passes, the norm and v_{j+1} in one cooperative launch
            double *Vp = w.V, *wp = w.w, *pp = w.partials;
            long long nn = n;
            int jj = j;
            LzState *lzp = w.lz;
            unsigned *bar = w.counter + 4;
            int *stp = ctx->d_status;
            void *args[] = {&Vp, &wp, &nn, &jj, &lzp, &pp, &bar, &stp, &sink};
            DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_lz_orth<kOB>, dim3(gc), dim3(kOB), args,
                                                  sizeof(double) * (MAXQ + 1) * kOB, st));
            DMRG_COUNT_LAUNCH();
            prof_mark(ctx, PROF_LZ_VEC);
            prof_count(ctx, PROF_LZ_VEC, 0.0, 8.0 * (double)n * (3.0 * (j + 1) + 7.0));
            DMRG_CUDA(cudaGetLastError());
            continue;
        }
        // Full reorthogonalisation by two classical Gram-Schmidt passes on
        // w = H v_j against v_0..v_j.  The first pass subtracts alpha_j v_j and
        // beta_j v_{j-1} with the rest (the three-term step is contained in
        // it), and its coefficient on v_j is alpha_j = v_j . H v_j; the second
        // pass also yields beta_{j+1} = |w|.
        ReduceArgs a2{w.V, n, j + 1, w.w, n, w.partials, w.counter};
        k_multidot<4><<<gd, RB, dsm, st>>>(a2, w.lz, j, w.c); DMRG_COUNT_LAUNCH();
        k_multiaxpy<<<g, RB, 0, st>>>(w.w, w.V, n, j + 1, w.c, n, w.lz, 1, 0); DMRG_COUNT_LAUNCH();
        k_multidot<0><<<gd, RB, dsm, st>>>(a2, w.lz, j, w.c); DMRG_COUNT_LAUNCH();
        k_multiaxpy_norm<<<gd, RB, 0, st>>>(w.w, w.V, n, j + 1, w.c, n, w.lz, j, w.partials, w.counter);
        DMRG_COUNT_LAUNCH();
        if (j + 1 < K) {
            k_next_vec<<<g, RB, 0, st>>>(w.V + (size_t)n * (j + 1), w.w, n, w.lz, j); DMRG_COUNT_LAUNCH();
            if (sink.h) {
                k_sink_vec<<<g, RB, 0, st>>>(w.V + (size_t)n * (j + 1), n, sink, w.lz); DMRG_COUNT_LAUNCH();
            }
        }
        prof_mark(ctx, PROF_LZ_VEC);
        // two Gram-Schmidt passes: (j + 1) basis vectors read twice in each,
        // the work vector about six times, 8 B each
        prof_count(ctx, PROF_LZ_VEC, 0.0, 8.0 * (double)n * (4.0 * (j + 1) + 6.0));
        DMRG_CUDA(cudaGetLastError());
    }
    k_tridiag_lowest<<<1, 32, 0, st>>>(w.lz, ctx->d_status); DMRG_COUNT_LAUNCH();
    // theta = V y0 (only the first m vectors carry weight: y is zero beyond m)
    {
        // copy y to the coefficient buffer (device to device)
        DMRG_CUDA(cudaMemcpyAsync(w.c, w.lz->y, sizeof(double) * K, cudaMemcpyDeviceToDevice, st));
        k_multiaxpy<<<g, RB, 0, st>>>(theta, w.V, n, -1, w.c, n, w.lz, 0, 1); DMRG_COUNT_LAUNCH();
        ReduceArgs a4{nullptr, n, 0, theta, n, w.partials, w.counter};
        k_multidot<3><<<gd, RB, dsm, st>>>(a4, w.lz, 0, nullptr); DMRG_COUNT_LAUNCH();
        k_scale_by<<<g, RB, 0, st>>>(theta, theta, n, w.lz); DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg
