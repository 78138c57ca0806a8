// jacobi.cu -- one-sided (Hestenes) Jacobi SVD of the two-site tensor.
//
// The SVD of Eq. (20) is computed by orthogonalising r = min(m, n) vectors of
// length l = max(m, n) (the columns of theta when n <= m, its rows when
// m < n) with plane rotations: for a pair (x_i, x_j) with Gram entries
// alpha = |x_i|^2, beta = |x_j|^2, gamma = x_i.x_j the rotation
//   zeta = (beta - alpha) / (2 gamma),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2),  s = c t,   x_i <- c x_i - s x_j,  x_j <- s x_i + c x_j
// makes them orthogonal (Hestenes 1958; the 2x2 symmetric Schur step of
// Golub & Van Loan 8.5.2).  A sweep visits every pair once in round-robin
// ("circle method") order: each round is a perfect matching of the vectors,
// so all r/2 rotations of a round are independent and run one per warp.
// The sweep loop runs inside one persistent cooperative kernel with a
// bounded grid barrier between rounds; the iteration stops after a sweep
// without rotations.  On exit s_i = |x_i|, u_i = x_i / s_i and the
// accumulated rotations give V.
#include "common.cuh"
#include "mma_tf32.cuh"

#include <cooperative_groups.h>
#include <algorithm>

namespace dmrg {

size_t svd_work_bytes_base(int r, int l)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(sizeof(double) * (size_t)r * l) + al(sizeof(double) * (size_t)r * r) + al(sizeof(double) * r) +
           al(sizeof(int) * r) + al(sizeof(unsigned) * 8);
}

// + the FP32 copy of the extended vectors and two r x r FP64 matrices of the
// preconditioned FP64 Jacobi
size_t svd_work_bytes(int r, int l)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return svd_work_bytes_base(r, l) + al(sizeof(float) * (size_t)r * (l + r)) + 2 * al(sizeof(double) * (size_t)r * r);
}

SvdWork svd_work_carve(void *base, int r, int l)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(base);
    SvdWork w;
    w.X = reinterpret_cast<double *>(p); p += al(sizeof(double) * (size_t)r * l);
    w.Vm = reinterpret_cast<double *>(p); p += al(sizeof(double) * (size_t)r * r);
    w.nrm = reinterpret_cast<double *>(p); p += al(sizeof(double) * r);
    w.perm = reinterpret_cast<int *>(p); p += al(sizeof(int) * r);
    w.sync = reinterpret_cast<unsigned *>(p);
    return w;
}

namespace {

// X[i][j] = theta column i (tr = 0) or row i (tr = 1); Vm = identity.
__global__ void k_jac_load(const double *__restrict__ A, int m, int n, int tr, int r, int l, double *__restrict__ X,
                           double *__restrict__ Vm, unsigned *sync)
{
    __shared__ double tile[32][33];
    // transposed copy through a shared tile when tr == 0
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    if (!tr) {
        // X (r x l) = A^T: X[i][j] = A[j][i], i < n = r, j < m = l
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int row = by + yy, col = bx + threadIdx.x;          // read A[row][col]
            tile[yy][threadIdx.x] = (row < m && col < n) ? A[(long long)row * n + col] : 0.0;
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = bx + yy, j = by + threadIdx.x;              // write X[i][j] = A[j][i]
            if (i < r && j < l) X[(long long)i * l + j] = tile[threadIdx.x][yy];
        }
    } else {
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = by + yy, j = bx + threadIdx.x;
            if (i < r && j < l) X[(long long)i * l + j] = A[(long long)i * n + j];
        }
    }
    // identity (grid covers at least r x r when launched for max(l, r))
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        int i = by + yy, j = bx + threadIdx.x;
        if (i < r && j < r) Vm[(long long)i * r + j] = (i == j) ? 1.0 : 0.0;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.y == 0 && threadIdx.x < 8) sync[threadIdx.x] = 0u;
}

__device__ __forceinline__ void rr_pair(int rp, int t, int p, int &i, int &j)
{
    // circle method on rp (even) players: player rp-1 fixed, the others rotate
    const int q = rp - 1;
    if (p == 0) {
        i = q;
        j = t;
    } else {
        i = (t + p) % q;
        j = (t - p + q) % q;
    }
}

__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rotation for the pair with Gram entries (a, b, g), all FP32 (the FP32 path
// rotates FP32 data, and GB300's FP64 pipe is far too narrow to evaluate
// square roots and divisions on every lane).  Returns false if none needed.
__device__ __forceinline__ bool rot32(float a, float b, float g, float floor2, float tol, float &c, float &sn)
{
    if (!(a > floor2 && b > floor2)) return false;
    if (!(fabsf(g) > tol * sqrtf(a) * sqrtf(b))) return false;
    const float zeta = (b - a) / (2.0f * g);
    const float tt = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
    c = rsqrtf(fmaf(tt, tt, 1.0f));
    sn = c * tt;
    return true;
}

__device__ __forceinline__ bool block_barrier(unsigned *words, int *status)
{
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    return grid_barrier(words, status);
}

// F2[0] = sum of squares of all entries (|A|_F^2), for the negligible-vector test
// (it only scales the floor below which vectors count as zero, so each
// thread's share is accumulated in FP32; the block sum is FP64)
__global__ void k_frob2(const double *__restrict__ A, long long n, double *F2)
{
    __shared__ double sh[32];
    float a = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const float x = (float)A[i];
        a = fmaf(x, x, a);
    }
    const double t = block_sum((double)a, sh);
    if (threadIdx.x == 0) F2[0] = t;
}

__global__ void __launch_bounds__(256) k_jac_sweeps(double *__restrict__ X, double *__restrict__ Vm, int r, int l,
                                                    int max_sweeps, double tol, unsigned *sync, int *status,
                                                    int *info, const double *F2, double small)
{
    // vectors with |x|^2 below small^2 |A|_F^2 are numerically zero: their
    // mutual angles are rounding noise and they are never retained
    const double floor2 = small * small * F2[0];
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int gwarp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * warps_per_block;
    const int rp = r + (r & 1);
    const int npairs = rp / 2;
    unsigned *barrier = sync;       // [0], [1]
    unsigned *rotc = sync + 2;      // [2], [3] alternating per sweep
    __shared__ unsigned block_rot;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) block_rot = 0;
        __syncthreads();
        unsigned my_rot = 0;
        for (int t = 0; t < rp - 1; ++t) {
            for (int p = gwarp; p < npairs; p += nwarps) {
                int i, j;
                rr_pair(rp, t, p, i, j);
                if (i >= r || j >= r) continue;
                double *xi = X + (long long)i * l, *xj = X + (long long)j * l;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int k = lane; k < l; k += 32) {
                    double u = xi[k], v = xj[k];
                    a = fma(u, u, a);
                    b = fma(v, v, b);
                    g = fma(u, v, g);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (!(a > floor2 && b > floor2)) continue;
                if (!(fabs(g) > tol * sqrt(a) * sqrt(b))) continue;
                // rotation parameters on one lane, broadcast (FP64 square roots
                // and divisions are expensive on GB300)
                double c = 0.0, s = 0.0;
                if (lane == 0) {
                    double zeta = (b - a) / (2.0 * g);
                    double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = c * tt;
                }
                c = __shfl_sync(0xffffffffu, c, 0);
                s = __shfl_sync(0xffffffffu, s, 0);
                for (int k = lane; k < l; k += 32) {
                    double u = xi[k], v = xj[k];
                    xi[k] = c * u - s * v;
                    xj[k] = s * u + c * v;
                }
                double *vi = Vm + (long long)i * r, *vj = Vm + (long long)j * r;
                for (int k = lane; k < r; k += 32) {
                    double u = vi[k], v = vj[k];
                    vi[k] = c * u - s * v;
                    vj[k] = s * u + c * v;
                }
                if (lane == 0) my_rot++;
            }
            if (!block_barrier(barrier, status)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
                return;
            }
        }
        if (lane == 0 && my_rot) atomicAdd(&block_rot, my_rot);
        __syncthreads();
        if (threadIdx.x == 0 && block_rot) atomicAdd(&rotc[sweep & 1], block_rot);
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
        unsigned total = *(volatile unsigned *)&rotc[sweep & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) rotc[(sweep + 1) & 1] = 0u;
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
        // make the reset of the next counter visible before anyone adds to it
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

// nrm[i] = |x_i|, one warp per vector
__global__ void k_jac_norms(const double *__restrict__ X, int r, int l, long long ldx, double *__restrict__ nrm)
{
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= r) return;
    const double *x = X + (long long)w * ldx;
    double a = 0.0;
    for (int k = lane; k < l; k += 32) a = fma(x[k], x[k], a);
    a = warp_sum(a);
    if (lane == 0) nrm[w] = sqrt(a);
}

// perm[rank] = i, descending by norm, ties by index
// Order-preserving integer key of a norm: for v >= 0 (also -0.0) the bits
// of |v| plus one, monotone in v; NaN and negatives map to 0 and sort last.
// Ranking on the keys uses integer compares only (FP64 compares run on the
// narrow FP64 pipe of this part, r of them per element).
__device__ __forceinline__ unsigned long long norm_key(double v)
{
    return (v >= 0.0) ? ((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL) + 1ULL : 0ULL;
}

constexpr int kRankSmemKeys = 6144;
__global__ void k_jac_rank(const double *__restrict__ nrm, int r, int *__restrict__ perm)
{
    __shared__ unsigned long long keys[kRankSmemKeys];
    const bool staged = r <= kRankSmemKeys;
    if (staged) {
        for (int j = threadIdx.x; j < r; j += blockDim.x) keys[j] = norm_key(nrm[j]);
        __syncthreads();
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    const unsigned long long v = staged ? keys[i] : norm_key(nrm[i]);
    int rank = 0;
    for (int j = 0; j < r; ++j) {
        const unsigned long long w = staged ? keys[j] : norm_key(nrm[j]);
        rank += (w > v) || (w == v && j < i);
    }
    perm[rank] = i;
}

// One block per output index c: writes s[c], U[:, c], Vt[c, :] with the sign
// convention "largest |entry| of U[:, c] positive".
__global__ void k_jac_out(const double *__restrict__ X, const double *__restrict__ Vm, const double *__restrict__ nrm,
                          const int *__restrict__ perm, int m, int n, int tr, int r, int l, long long ldx,
                          long long ldv, double *__restrict__ U, double *__restrict__ s, double *__restrict__ Vt)
{
    __shared__ double sh_v[32];
    __shared__ int sh_i[32];
    const int c = blockIdx.x;
    int i = perm[c];
    if (i < 0 || i >= r) i = c;
    const double sig = nrm[i];
    const double inv = (sig > 0.0) ? 1.0 / sig : 0.0;
    // U column source: X row i scaled (tr = 0, length m = l) or Vm row i (tr = 1, length m = r)
    const double *usrc = tr ? (Vm + (long long)i * ldv) : (X + (long long)i * ldx);
    const double uscale = tr ? 1.0 : inv;
    // argmax |u|
    double best = -1.0;
    int bidx = 0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double a = fabs(usrc[k]);
        if (a > best) { best = a; bidx = k; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sh_v[threadIdx.x >> 5] = best; sh_i[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sh_v[0];
        int bi = sh_i[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sh_v[w] > bv || (sh_v[w] == bv && sh_i[w] < bi)) { bv = sh_v[w]; bi = sh_i[w]; }
        sh_i[0] = bi;
        s[c] = sig;
    }
    __syncthreads();
    const double sign = (usrc[sh_i[0]] < 0.0) ? -1.0 : 1.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) U[(long long)k * r + c] = sign * uscale * usrc[k];
    const double *vsrc = tr ? (X + (long long)i * ldx) : (Vm + (long long)i * ldv);
    const double vscale = tr ? inv : 1.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) Vt[(long long)c * n + k] = sign * vscale * vsrc[k];
}

// ---------------------------------------------------------------------------
// FP32 variant for the mixed-precision form: vectors only (no V), dot
// products accumulated per lane in FP32 (two chains) and across lanes in FP64.
// ---------------------------------------------------------------------------
__global__ void k_jac32_load(const double *__restrict__ A, int m, int n, int dir, int r, int l, float *__restrict__ X,
                             unsigned *sync)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    if (dir == 0) {
        // vectors are the columns of A: X[i][t] = A[t][i], i < n = r, t < m = l
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int row = by + yy, col = bx + threadIdx.x;
            tile[yy][threadIdx.x] = (row < m && col < n) ? (float)A[(long long)row * n + col] : 0.0f;
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = bx + yy, t = by + threadIdx.x;
            if (i < r && t < l) X[(long long)i * l + t] = tile[threadIdx.x][yy];
        }
    } else {
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = by + yy, t = bx + threadIdx.x;
            if (i < r && t < l) X[(long long)i * l + t] = (float)A[(long long)i * n + t];
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.y == 0 && threadIdx.x < 8) sync[threadIdx.x] = 0u;
}

// Single-CTA FP32 Jacobi with the vectors resident in shared memory (r*l
// floats <= kSmemJacFloats): the rounds synchronise with __syncthreads only.

__global__ void __launch_bounds__(1024) k_jac32_smem(float *__restrict__ Xg, int r_all, int l, int max_sweeps,
                                                     double tol, int *status, int *info, const double *F2, double small,
                                                     const int *r_eff)
{
    extern __shared__ float xs[];
    __shared__ unsigned rot_count;
    const long long n = (long long)r_all * l;
    // rows beyond r_eff (negligible after QR preconditioning) are carried, not rotated
    const int r = r_eff ? min(r_all, max(1, *r_eff)) : r_all;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) xs[e] = Xg[e];
    const float floor2f = (float)(small * small * F2[0]), tolf = (float)tol;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rp = r + (r & 1), npairs = rp / 2;
    int sweep = 0;
    bool converged = false;
    __syncthreads();
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rot_count = 0;
        __syncthreads();
        unsigned my_rot = 0;
        for (int t = 0; t < rp - 1; ++t) {
            for (int p = warp; p < npairs; p += nw) {
                int i, j;
                rr_pair(rp, t, p, i, j);
                if (i >= r || j >= r) continue;
                float *xi = xs + (long long)i * l, *xj = xs + (long long)j * l;
                float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, g0 = 0.f, g1 = 0.f;
                int k = lane;
                for (; k + 32 < l; k += 64) {
                    float u = xi[k], v = xj[k], u2 = xi[k + 32], v2 = xj[k + 32];
                    a0 = fmaf(u, u, a0); b0 = fmaf(v, v, b0); g0 = fmaf(u, v, g0);
                    a1 = fmaf(u2, u2, a1); b1 = fmaf(v2, v2, b1); g1 = fmaf(u2, v2, g1);
                }
                if (k < l) {
                    float u = xi[k], v = xj[k];
                    a0 = fmaf(u, u, a0); b0 = fmaf(v, v, b0); g0 = fmaf(u, v, g0);
                }
                const float a = warp_sum_f(a0 + a1), b = warp_sum_f(b0 + b1), g = warp_sum_f(g0 + g1);
                float c, sn;
                if (!rot32(a, b, g, floor2f, tolf, c, sn)) continue;
                for (int q = lane; q < l; q += 32) {
                    float u = xi[q], v = xj[q];
                    xi[q] = fmaf(c, u, -sn * v);
                    xj[q] = fmaf(sn, u, c * v);
                }
                if (lane == 0) my_rot++;
            }
            __syncthreads();
        }
        if (lane == 0 && my_rot) atomicAdd(&rot_count, my_rot);
        __syncthreads();
        const unsigned total = rot_count;
        __syncthreads();
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
    }
    for (long long e = threadIdx.x; e < n; e += blockDim.x) Xg[e] = xs[e];
    if (threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

// Blocked FP32 Jacobi: the vectors are grouped in blocks of BW; a sweep
// pairs the blocks in round-robin order, and the CTA that owns a block pair
// loads its 2 BW vectors into shared memory and applies inner sweeps of plane
// rotations over every pair among them before writing them back.  The grid
// barrier is paid once per block round, and each vector crosses L2 once per
// block round.  Each vector pair is handled by WPP = 16 / BW warps, every
// warp owning a slice of the vector length; the slice dot products meet in
// shared memory and are summed in a fixed order, so all warps of a pair
// derive the same rotation.
constexpr int kBjacThreads = 512;

template <int BW>
__global__ void __launch_bounds__(kBjacThreads) k_bjac32(float *__restrict__ X, int r_all, int l, int max_sweeps,
                                                         double tol, unsigned *sync, int *status, int *info,
                                                         const double *F2, double small, int max_inner,
                                                         const int *r_eff)
{
    // rows beyond r_eff (negligible after QR preconditioning) are carried, not rotated
    const int r = r_eff ? min(r_all, max(1, *r_eff)) : r_all;
    constexpr int NW = kBjacThreads / 32;
    constexpr int WPP = (NW / BW) > 0 ? (NW / BW) : 1;    // warps per pair
    constexpr int PPR = NW / WPP;                         // pairs in flight per inner round
    extern __shared__ float xs[];            // [2 BW][l]
    __shared__ int vid[2 * BW];
    __shared__ float part[NW][3];
    __shared__ unsigned block_rot, inner_rot;
    const float floor2f = (float)(small * small * F2[0]), tolf = (float)tol;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = warp / WPP, sub = warp % WPP;        // pair slot and slice of this warp
    const int chunk = (l + WPP - 1) / WPP;
    const int e0 = sub * chunk, e1 = min(l, e0 + chunk);
    const int nb = (r + BW - 1) / BW;
    const int nbp = nb + (nb & 1);
    const int npairs = nbp / 2;
    unsigned *barrier = sync;
    unsigned *rotc = sync + 2;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) block_rot = 0;
        __syncthreads();
        unsigned my_rot = 0;
        for (int t = 0; t < nbp - 1; ++t) {
            for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
                int I, J;
                rr_pair(nbp, t, p, I, J);
                if (threadIdx.x < 2 * BW) {
                    const int blk = threadIdx.x < BW ? I : J;
                    const int v = blk * BW + (threadIdx.x % BW);
                    vid[threadIdx.x] = (blk < nb && v < r) ? v : -1;
                }
                __syncthreads();
                for (int q = warp; q < 2 * BW; q += NW) {
                    const int v = vid[q];
                    if (v >= 0) {
                        const float *src = X + (long long)v * l;
                        float *dst = xs + (long long)q * l;
                        for (int e = lane; e < l; e += 32) dst[e] = src[e];
                    }
                }
                __syncthreads();
                constexpr int nv = 2 * BW;
                for (int inner = 0; inner < max_inner; ++inner) {
                    if (threadIdx.x == 0) inner_rot = 0;
                    __syncthreads();
                    for (int u = 0; u < nv - 1; ++u) {
                        for (int pp0 = 0; pp0 < BW; pp0 += PPR) {
                            const int pp = pp0 + slot;
                            int a_ = 0, b_ = 0;
                            bool act = pp < BW;
                            if (act) {
                                rr_pair(nv, u, pp, a_, b_);
                                act = vid[a_] >= 0 && vid[b_] >= 0;
                            }
                            float *xi = xs + (long long)a_ * l, *xj = xs + (long long)b_ * l;
                            float a0 = 0.f, b0 = 0.f, g0 = 0.f, a1 = 0.f, b1 = 0.f, g1 = 0.f;
                            if (act) {
                                int k = e0 + lane;
                                for (; k + 32 < e1; k += 64) {
                                    float x0 = xi[k], y0 = xj[k], x1 = xi[k + 32], y1 = xj[k + 32];
                                    a0 = fmaf(x0, x0, a0); b0 = fmaf(y0, y0, b0); g0 = fmaf(x0, y0, g0);
                                    a1 = fmaf(x1, x1, a1); b1 = fmaf(y1, y1, b1); g1 = fmaf(x1, y1, g1);
                                }
                                if (k < e1) {
                                    float x0 = xi[k], y0 = xj[k];
                                    a0 = fmaf(x0, x0, a0); b0 = fmaf(y0, y0, b0); g0 = fmaf(x0, y0, g0);
                                }
                                const float pa = warp_sum_f(a0 + a1), pb = warp_sum_f(b0 + b1), pg = warp_sum_f(g0 + g1);
                                if (lane == 0) { part[warp][0] = pa; part[warp][1] = pb; part[warp][2] = pg; }
                            }
                            __syncthreads();
                            float c = 1.f, sn = 0.f;
                            bool rot = false;
                            if (act) {
                                float a = 0.f, b = 0.f, g = 0.f;
                                const int w0 = slot * WPP;
                                for (int w = 0; w < WPP; ++w) { a += part[w0 + w][0]; b += part[w0 + w][1]; g += part[w0 + w][2]; }
                                rot = rot32(a, b, g, floor2f, tolf, c, sn);
                            }
                            if (rot) {
                                for (int q = e0 + lane; q < e1; q += 32) {
                                    const float x0 = xi[q], y0 = xj[q];
                                    xi[q] = fmaf(c, x0, -sn * y0);
                                    xj[q] = fmaf(sn, x0, c * y0);
                                }
                                if (sub == 0 && lane == 0) { my_rot++; atomicAdd(&inner_rot, 1u); }
                            }
                            __syncthreads();
                        }
                    }
                    const unsigned ir = inner_rot;
                    __syncthreads();
                    if (ir == 0u || BW == 1) break;
                }
                for (int q = warp; q < 2 * BW; q += NW) {
                    const int v = vid[q];
                    if (v >= 0) {
                        const float *src = xs + (long long)q * l;
                        float *dst = X + (long long)v * l;
                        for (int e = lane; e < l; e += 32) dst[e] = src[e];
                    }
                }
                __syncthreads();
            }
            if (!block_barrier(barrier, status)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
                return;
            }
        }
        if (lane == 0 && my_rot) atomicAdd(&block_rot, my_rot);
        __syncthreads();
        if (threadIdx.x == 0 && block_rot) atomicAdd(&rotc[sweep & 1], block_rot);
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
        const unsigned total = *(volatile unsigned *)&rotc[sweep & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) rotc[(sweep + 1) & 1] = 0u;
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

// Blocked FP32 Jacobi with the inner sweep in Gram form.  The CTA that owns a
// block pair stages its NV = 2 BW vectors in shared memory and
//   1. forms their Gram matrix G = X X^T on the tensor cores (3xTF32);
//   2. runs one cyclic Jacobi sweep on G -- the rotations an inner sweep over
//      the vector pairs would apply, in exact arithmetic -- accumulating the
//      product Q of the rotations, then one FP32 Newton-Schulz step on Q;
//   3. writes x_j <- sum_i Q[i][j] x_i with FP32 FMAs (3xTF32 products carry
//      ~2^-22 relative error, which would accumulate in the vectors over the
//      rounds; in G it only perturbs the rotations, which stay orthogonal).
// A round is a few dozen dependent steps on a small matrix, where the vector
// form takes 2 BW - 1 steps of reductions over length-l vectors.  Outer
// rounds, grid barrier and convergence test as k_bjac32.
//
// Rotation of pair (p, q): x_p <- c x_p - s x_q, x_q <- s x_p + c x_q, i.e.
// X <- X J with J[x][x] = c, J[partner][x] = -s for x = p and +s for x = q.
// Then G <- J^T G J and Q <- Q J entrywise from the previous step's buffer
// (double-buffered: one barrier per step).  The rotation of step u + 1 is
// taken in step u by the thread that owns its pair, from the same
// expressions that produce the new entries.  Entry (i, j) is evaluated in
// the order of (min, max), so G stays bitwise symmetric.
template <int BW>
__global__ void __launch_bounds__(kBjacThreads) k_bjac32g(float *__restrict__ X, int r_all, int l, int ls,
                                                          int max_sweeps, double tol, unsigned *sync, int *status,
                                                          int *info, const double *F2, double small,
                                                          const int *r_eff)
{
    constexpr int NW = kBjacThreads / 32;
    constexpr int NV = 2 * BW;
    constexpr int MT = (NV + 15) / 16, NT = NV / 8;     // Gram tiles of 16 x 8
    constexpr int WPT = NW / (MT * NT);                  // warps per Gram tile (k split)
    static_assert(NV >= 8 && WPT >= 1, "block width");
    extern __shared__ __align__(16) float xs[];          // [NV][ls]: vector q at xs + q ls
    __shared__ int vid[NV];
    __shared__ float Gb[2][NV][NV + 1], Qb[2][NV][NV + 1];
    __shared__ float part[NW][16][8];
    __shared__ float pc[2][NV], psn[2][NV];              // step parameters per index: c, J[partner][x]
    __shared__ int ppt[2][NV];                           // partner (the index itself when not rotated)
    __shared__ unsigned block_rot, pair_rot;
    const int r = r_eff ? min(r_all, max(1, *r_eff)) : r_all;
    const float floor2f = (float)(small * small * F2[0]), tolf = (float)tol;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, c4 = lane & 3;
    const int nb = (r + BW - 1) / BW;
    const int nbp = nb + (nb & 1);
    const int npairs = nbp / 2;
    const int nchunk = (l + 7) / 8;                      // positions in chunks of 8 (zero tail up to ls)
    const bool vec4 = (l & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;   // rows 16-byte aligned
    unsigned *barrier = sync;
    unsigned *rotc = sync + 2;
    int sweep = 0;
    bool converged = false;

    // new G entry (i <= j) of step parameters `pb` from buffer `gb`
    auto gnew = [&](int pb, int gb, int i, int j) {
        const float ci = pc[pb][i], si = psn[pb][i], cj = pc[pb][j], sj = psn[pb][j];
        const int pi = ppt[pb][i], pj = ppt[pb][j];
        float v = ci * cj * Gb[gb][i][j];
        v = fmaf(ci * sj, Gb[gb][i][pj], v);
        v = fmaf(si * cj, Gb[gb][pi][j], v);
        return fmaf(si * sj, Gb[gb][pi][pj], v);
    };
    // parameters of pair (a, b) from its three Gram entries; true if it rotates
    auto setpar = [&](int pb, int a, int b, float gaa, float gbb, float gab) {
        float c = 1.f, sn = 0.f;
        const bool rot = vid[a] >= 0 && vid[b] >= 0 && rot32(gaa, gbb, gab, floor2f, tolf, c, sn);
        pc[pb][a] = c; psn[pb][a] = rot ? -sn : 0.f; ppt[pb][a] = rot ? b : a;
        pc[pb][b] = c; psn[pb][b] = rot ? sn : 0.f; ppt[pb][b] = rot ? a : b;
        return rot;
    };

    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) block_rot = 0;
        __syncthreads();
        for (int t = 0; t < nbp - 1; ++t) {
            for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
                int I, J;
                rr_pair(nbp, t, p, I, J);
                if (threadIdx.x < NV) {
                    const int blk = threadIdx.x < BW ? I : J;
                    const int v = blk * BW + (threadIdx.x % BW);
                    vid[threadIdx.x] = (blk < nb && v < r) ? v : -1;
                }
                if (threadIdx.x == 0) pair_rot = 0;
                __syncthreads();
                if (vec4) {
                    // every load of a thread issued before its stores: one L2
                    // round trip per round instead of one per few elements
                    const int l4 = l >> 2, ls4 = ls >> 2;
                    float4 *xs4 = reinterpret_cast<float4 *>(xs);
#pragma unroll 4
                    for (int idx = threadIdx.x; idx < NV * l4; idx += kBjacThreads) {
                        const int q = idx / l4, e4 = idx - q * l4;
                        const int v = vid[q];
                        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (v >= 0) val = reinterpret_cast<const float4 *>(X + (long long)v * l)[e4];
                        xs4[q * ls4 + e4] = val;
                    }
                    const int tail = ls - l;
                    for (int idx = threadIdx.x; idx < NV * tail; idx += kBjacThreads)
                        xs[(idx / tail) * ls + l + idx % tail] = 0.f;
                } else {
                    for (int q = warp; q < NV; q += NW) {
                        const int v = vid[q];
                        float *dst = xs + (long long)q * ls;
                        const float *src = X + (long long)(v < 0 ? 0 : v) * l;
                        for (int e = lane; e < ls; e += 32) dst[e] = (v >= 0 && e < l) ? src[e] : 0.f;
                    }
                }
                __syncthreads();
                // 1. Gram matrix: warp w adds chunks w % WPT, + WPT, ... of tile w / WPT
                {
                    const int tile = warp / WPT, kp = warp % WPT;
                    const int mi = tile / NT, ni = tile % NT;
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    auto fa = [&](int m, int k) { return m < NV ? xs[m * ls + k] : 0.f; };
                    auto fb = [&](int k, int n) { return xs[n * ls + k]; };
                    for (int ck = kp; ck < nchunk; ck += WPT) mma3(acc, g, c4, fa, fb, 16 * mi, 8 * ni, 8 * ck);
                    part[warp][g][2 * c4] = acc[0];
                    part[warp][g][2 * c4 + 1] = acc[1];
                    part[warp][g + 8][2 * c4] = acc[2];
                    part[warp][g + 8][2 * c4 + 1] = acc[3];
                }
                __syncthreads();
                for (int e = threadIdx.x; e < NV * NV; e += kBjacThreads) {
                    const int i = e / NV, j = e % NV;
                    Qb[0][i][j] = (i == j) ? 1.f : 0.f;
                    if (i > j) continue;
                    const int tile = (i / 16) * NT + j / 8;
                    float a = 0.f;
                    for (int kp = 0; kp < WPT; ++kp) a += part[tile * WPT + kp][i % 16][j % 8];
                    Gb[0][i][j] = a;
                    Gb[0][j][i] = a;
                }
                __syncthreads();
                unsigned myrot = 0;
                if (threadIdx.x < BW) {
                    int a_, b_;
                    rr_pair(NV, 0, threadIdx.x, a_, b_);
                    myrot += setpar(0, a_, b_, Gb[0][a_][a_], Gb[0][b_][b_], Gb[0][min(a_, b_)][max(a_, b_)]);
                }
                __syncthreads();
                // 2. the sweep on G; step u reads buffer u & 1 and its parameters u & 1
                for (int u = 0; u < NV - 1; ++u) {
                    const int cb = u & 1, nbf = cb ^ 1;
                    for (int e = threadIdx.x; e < 2 * NV * NV; e += kBjacThreads) {
                        if (e < NV * NV) {
                            const int i = e / NV, j = e % NV;
                            if (i > j) continue;
                            const float v = gnew(cb, cb, i, j);
                            Gb[nbf][i][j] = v;
                            Gb[nbf][j][i] = v;
                        } else {
                            const int e2 = e - NV * NV, i = e2 / NV, j = e2 % NV;
                            Qb[nbf][i][j] = fmaf(psn[cb][j], Qb[cb][i][ppt[cb][j]], pc[cb][j] * Qb[cb][i][j]);
                        }
                    }
                    if (u + 1 < NV - 1 && threadIdx.x < BW) {
                        int a_, b_;
                        rr_pair(NV, u + 1, threadIdx.x, a_, b_);
                        const float gaa = gnew(cb, cb, a_, a_), gbb = gnew(cb, cb, b_, b_);
                        const float gab = gnew(cb, cb, min(a_, b_), max(a_, b_));
                        myrot += setpar(nbf, a_, b_, gaa, gbb, gab);
                    }
                    __syncthreads();
                }
                if (myrot) atomicAdd(&pair_rot, myrot);
                __syncthreads();
                constexpr int qf = (NV - 1) & 1;                 // buffer holding the final Q
                const float(*Qf)[NV + 1] = Qb[qf];
                const unsigned prot = pair_rot;
                if (prot) {
                    // Q <- Q (3 I - Q^T Q) / 2: orthogonal again at FP32 rounding
                    for (int e = threadIdx.x; e < NV * NV; e += kBjacThreads) {
                        const int i = e / NV, j = e % NV;
                        float a = 0.f;
                        for (int k2 = 0; k2 < NV; ++k2) a = fmaf(Qb[qf][k2][i], Qb[qf][k2][j], a);
                        Gb[qf ^ 1][i][j] = (i == j ? 1.5f : 0.f) - 0.5f * a;
                    }
                    __syncthreads();
                    for (int e = threadIdx.x; e < NV * NV; e += kBjacThreads) {
                        const int i = e / NV, j = e % NV;
                        float a = 0.f;
                        for (int k2 = 0; k2 < NV; ++k2) a = fmaf(Qb[qf][i][k2], Gb[qf ^ 1][k2][j], a);
                        Qb[qf ^ 1][i][j] = a;
                    }
                    __syncthreads();
                    Qf = Qb[qf ^ 1];
                    if (threadIdx.x == 0) block_rot += prot;
                    // 3. x_j <- sum_i Q[i][j] x_i in FP32 (the vectors carry FP32
                    // rounding only), straight to X: a thread keeps OPT columns
                    // of Q in registers and walks positions with its group
                    constexpr int OPT = NV >= 32 ? 2 : 4, NG = NV / OPT, TPG = kBjacThreads / NG;
                    const int gi = threadIdx.x / TPG, t0 = threadIdx.x % TPG;
                    float qr[OPT][NV];
                    int vo[OPT];
#pragma unroll
                    for (int o = 0; o < OPT; ++o) {
                        vo[o] = vid[gi * OPT + o];
#pragma unroll
                        for (int i = 0; i < NV; ++i) qr[o][i] = Qf[i][gi * OPT + o];
                    }
                    for (int e = t0; e < l; e += TPG) {
                        float acc[OPT];
#pragma unroll
                        for (int o = 0; o < OPT; ++o) acc[o] = 0.f;
#pragma unroll
                        for (int i = 0; i < NV; ++i) {
                            const float x = xs[i * ls + e];
#pragma unroll
                            for (int o = 0; o < OPT; ++o) acc[o] = fmaf(qr[o][i], x, acc[o]);
                        }
#pragma unroll
                        for (int o = 0; o < OPT; ++o)
                            if (vo[o] >= 0) X[(long long)vo[o] * l + e] = acc[o];
                    }
                }
                __syncthreads();
            }
            if (!block_barrier(barrier, status)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
                return;
            }
        }
        if (threadIdx.x == 0 && block_rot) atomicAdd(&rotc[sweep & 1], block_rot);
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
        const unsigned total = *(volatile unsigned *)&rotc[sweep & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) rotc[(sweep + 1) & 1] = 0u;
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
        if (!block_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

// shared-memory row stride of the Gram form: l rounded up to whole 8-position
// chunks, + 4 (odd multiple of 4 floats: the mma fragment reads of 8 rows x 4
// columns fall in 32 distinct banks)
inline int bjac32g_stride(int l) { return ((l + 7) / 8) * 8 + 4; }

template <int BW>
dmrg_status launch_bjac32g(dmrg_ctx *ctx, float *X, int r, int l, int max_sweeps, double tol, unsigned *sync,
                           int *d_info, const double *F2, double small, const int *r_eff)
{
    int ls = bjac32g_stride(l);
    const size_t smem = sizeof(float) * 2 * BW * (size_t)ls;
    static size_t attr = 0;
    if (attr < smem) {
        DMRG_CUDA(cudaFuncSetAttribute(k_bjac32g<BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    int per_sm = 0;
    DMRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bjac32g<BW>, kBjacThreads, smem));
    if (per_sm < 1) return DMRG_EUNSUPPORTED;
    const int nb = (r + BW - 1) / BW;
    const int npairs = (nb + (nb & 1)) / 2;
    int blocks = std::min(npairs, per_sm * ctx->num_sms);
    if (blocks < 1) blocks = 1;
    int *status = ctx->d_status;
    void *args[] = {&X, (void *)&r, (void *)&l, &ls, &max_sweeps, (void *)&tol, &sync, &status, &d_info,
                    (void *)&F2, (void *)&small, (void *)&r_eff};
    DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_bjac32g<BW>, dim3(blocks), dim3(kBjacThreads), args, smem,
                                          ctx->stream)); DMRG_COUNT_LAUNCH();
    return DMRG_OK;
}

template <int BW>
dmrg_status launch_bjac32(dmrg_ctx *ctx, float *X, int r, int l, int max_sweeps, double tol, unsigned *sync,
                          int *d_info, const double *F2, double small, int max_inner, const int *r_eff)
{
    const size_t smem = sizeof(float) * 2 * BW * (size_t)l;
    static size_t attr = 0;
    if (attr < smem) {
        DMRG_CUDA(cudaFuncSetAttribute(k_bjac32<BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = smem;
    }
    int per_sm = 0;
    DMRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bjac32<BW>, kBjacThreads, smem));
    if (per_sm < 1) return DMRG_EUNSUPPORTED;
    const int nb = (r + BW - 1) / BW;
    const int npairs = (nb + (nb & 1)) / 2;
    int blocks = std::min(npairs, per_sm * ctx->num_sms);
    if (blocks < 1) blocks = 1;
    int *status = ctx->d_status;
    void *args[] = {&X, (void *)&r, (void *)&l, &max_sweeps, (void *)&tol, &sync, &status, &d_info, (void *)&F2,
                    (void *)&small, &max_inner, (void *)&r_eff};
    DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_bjac32<BW>, dim3(blocks), dim3(kBjacThreads), args, smem,
                                          ctx->stream)); DMRG_COUNT_LAUNCH();
    return DMRG_OK;
}

__global__ void k_frob2_f(const float *__restrict__ A, long long n, double *F2)
{
    __shared__ double sh[32];
    float a = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) a = fmaf(A[i], A[i], a);
    const double t = block_sum((double)a, sh);
    if (threadIdx.x == 0) F2[0] = t;
}

// vectors shorter than 2^-22 |A|_F are unresolved after the FP32 rounding of
// A (Weyl) and were not orthogonalised (pairs below 2^-23 |A|_F are skipped):
// their norm is reported as zero so they sort last and are never retained
__global__ void k_jac32_norms(const float *__restrict__ X, int r, int l, double *__restrict__ nrm, const double *F2)
{
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= r) return;
    const float *x = X + (long long)w * l;
    double a = 0.0;
    for (int k = lane; k < l; k += 32) a = fma((double)x[k], (double)x[k], a);
    a = warp_sum(a);
    const double cut = 2.384185791015625e-07 * sqrt(F2[0]);
    if (lane == 0) nrm[w] = sqrt(a) > cut ? sqrt(a) : 0.0;
}

__global__ void k_sorted_values(const double *__restrict__ nrm, const int *__restrict__ perm, int r_out,
                                double *__restrict__ s)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < r_out) s[c] = nrm[perm[c]];
}

// Q[j][t] = X[perm[j]][t] / nrm[perm[j]]  (FP64), j < k
__global__ void k_gather_unit(const float *__restrict__ X, const double *__restrict__ nrm, const int *__restrict__ perm,
                              const int *__restrict__ kdev, int l, double *__restrict__ Q, double rel_floor)
{
    const int k = *kdev;
    const double cut = rel_floor * nrm[perm[0]];   // unresolved vectors are returned as zero
    const long long total = (long long)k * l;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int j = (int)(e / l), t = (int)(e % l);
        const int i = perm[j];
        const double nv = nrm[i];
        Q[e] = nv > cut ? (double)X[(long long)i * l + t] / nv : 0.0;
    }
}

}  // namespace

static dmrg_status svd_jacobi_scalar(dmrg_ctx *ctx, const double *A, int m, int n, double *U, double *s, double *Vt,
                                     void *work, int max_sweeps, int *d_info)
{
    if (m <= 0 || n <= 0) return DMRG_EINVAL;
    const int tr = (m < n);
    const int r = tr ? m : n, l = tr ? n : m;
    SvdWork w = svd_work_carve(work, r, l);
    cudaStream_t st = ctx->stream;
    {
        int big = l > r ? l : r;
        dim3 grid((big + 31) / 32, (big + 31) / 32);
        if (!tr) grid = dim3((n + 31) / 32 > (r + 31) / 32 ? (n + 31) / 32 : (r + 31) / 32,
                             (m + 31) / 32 > (r + 31) / 32 ? (m + 31) / 32 : (r + 31) / 32);
        k_jac_load<<<grid, dim3(32, 8), 0, st>>>(A, m, n, tr, r, l, w.X, w.Vm, w.sync); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
    }
    // rotate only while |x_i.x_j| > l eps |x_i||x_j|: the rounding noise of the
    // computed dot product is ~ sqrt(l) eps, so this margin of sqrt(l) lets the
    // sweep loop terminate instead of rotating on noise
    const double tol = (double)(l > 16 ? l : 16) * 2.220446049250313e-16;
    const int rp = r + (r & 1);
    const int npairs = rp / 2;
    // GB300's per-SM FP64 rate is low, so even small problems are spread over
    // several CTAs (one warp per pair) as soon as there are enough pairs
    int threads = 256;
    int blocks = 1;
    if (r > 48) {
        int per_sm = 0;
        DMRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jac_sweeps, threads, 0));
        int maxb = per_sm * ctx->num_sms;
        blocks = (npairs + 3) / 4;      // two pairs per warp per round at most
        if (blocks > maxb) blocks = maxb;
        if (blocks < 1) blocks = 1;
    }
    double *X = w.X, *Vm = w.Vm;
    unsigned *sync = w.sync;
    int *status = ctx->d_status;
    const double *F2 = reinterpret_cast<const double *>(w.sync + 4);
    const double small = (double)(l > 16 ? l : 16) * 2.220446049250313e-16;
    k_frob2<<<1, 1024, 0, st>>>(X, (long long)r * l, reinterpret_cast<double *>(w.sync + 4)); DMRG_COUNT_LAUNCH();
    void *args[] = {&X, &Vm, (void *)&r, (void *)&l, &max_sweeps, (void *)&tol, &sync, &status, &d_info, &F2,
                    (void *)&small};
    prof_mark(ctx, PROF_JACOBI64);
    if (blocks == 1) {
        k_jac_sweeps<<<1, threads, 0, st>>>(X, Vm, r, l, max_sweeps, tol, sync, status, d_info, F2, small); DMRG_COUNT_LAUNCH();
    } else {
        DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_jac_sweeps, dim3(blocks), dim3(threads), args, 0, st)); DMRG_COUNT_LAUNCH();
    }
    prof_mark(ctx, PROF_JACOBI64);
    // nominal full-SVD flop count (4 m^2 n + 8 m n^2 + 9 n^3, m >= n) and the
    // minimum bytes of one pass over the vectors and V
    prof_count(ctx, PROF_JACOBI64, 4.0 * l * (double)l * r + 8.0 * l * (double)r * r + 9.0 * (double)r * r * r,
               8.0 * ((double)r * l + (double)r * r) * 2.0);
    DMRG_CUDA(cudaGetLastError());
    k_jac_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(X, r, l, l, w.nrm); DMRG_COUNT_LAUNCH();
    k_jac_rank<<<(r + 255) / 256, 256, 0, st>>>(w.nrm, r, w.perm); DMRG_COUNT_LAUNCH();
    k_jac_out<<<r, 256, 0, st>>>(X, Vm, w.nrm, w.perm, m, n, tr, r, l, l, r, U, s, Vt); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}


namespace {

int grid_ln(long long n, int num_sms)
{
    long long b = (n + 255) / 256;
    if (b > 4LL * num_sms) b = 4LL * num_sms;
    return (int)(b < 1 ? 1 : b);
}

// Extended vectors for the grouped Jacobi: row i of Xe (row stride ldx) is
// [theta column i (tr = 0) or row i (tr = 1), length l | row i of the r x r
// identity at offset l], in T.
template <typename T>
__global__ void k_gj_load(const double *__restrict__ A, int m, int n, int tr, int r, int l, int ldx,
                          T *__restrict__ Xe, int with_v)
{
    __shared__ double tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    if (!tr) {
        // vectors are the columns of A: Xe[i][j] = A[j][i], i < n = r, j < m = l
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int row = by + yy, col = bx + threadIdx.x;
            tile[yy][threadIdx.x] = (row < m && col < n) ? A[(long long)row * n + col] : 0.0;
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = bx + yy, j = by + threadIdx.x;
            if (i < r && j < l) Xe[(long long)i * ldx + j] = (T)tile[threadIdx.x][yy];
        }
    } else {
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = by + yy, j = bx + threadIdx.x;
            if (i < r && j < l) Xe[(long long)i * ldx + j] = (T)A[(long long)i * n + j];
        }
    }
    if (with_v) {
        // the grid covers at least r x r
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            int i = by + yy, j = bx + threadIdx.x;
            if (i < r && j < r) Xe[(long long)i * ldx + l + j] = (i == j) ? (T)1 : (T)0;
        }
    }
}

// Q[i][j] = (double) second part of FP32 extended row i (the rows of V^T)
__global__ void k_gj_take_q(const float *__restrict__ X32, int r, int l, int ldx, double *__restrict__ Q)
{
    const long long total = (long long)r * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), j = (int)(e % r);
        Q[e] = (double)X32[(long long)i * ldx + l + j];
    }
}

// second part of FP64 extended row i = row i of Q
__global__ void k_gj_put_q(const double *__restrict__ Q, int r, int l, int ldx, double *__restrict__ Xe)
{
    const long long total = (long long)r * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), j = (int)(e % r);
        Xe[(long long)i * ldx + l + j] = Q[e];
    }
}

}  // namespace

// FP64 one-sided Jacobi SVD on the grouped block kernel.
//  - The vectors are extended by the rows of V^T (the identity at the start),
//    so the rotations that orthogonalise them also accumulate V.
//  - With precond (r >= 64): a first pass runs the same iteration in FP32 on
//    an FP32 copy (rotate while a cosine exceeds 1e-5).  Its accumulated
//    V32^T is made orthogonal to FP64 precision by two Newton-Schulz steps
//    Q <- (3 I - Q Q^T) Q / 2, and the FP64 iteration starts from the
//    vectors Q X and V^T = Q: nearly orthogonal already, they converge in two
//    or three FP64 sweeps.  The FP64 result does not depend on the FP32 pass
//    beyond its starting point: the stopping rule is the FP64 one.
dmrg_status svd_jacobi(dmrg_ctx *ctx, const double *A, int m, int n, double *U, double *s, double *Vt, void *work,
                       int max_sweeps, int *d_info, int precond)
{
    if (m <= 0 || n <= 0) return DMRG_EINVAL;
    if (!ctx->jacobi64_gram) return svd_jacobi_scalar(ctx, A, m, n, U, s, Vt, work, max_sweeps, d_info);
    const int tr = (m < n);
    const int r = tr ? m : n, l = tr ? n : m;
    const int ldx = l + r;
    SvdWork w = svd_work_carve(work, r, l);
    double *Xe = w.X;                      // r x (l + r): spans the X and Vm slots of the base layout
    cudaStream_t st = ctx->stream;
    unsigned *sync = w.sync;
    double *F2 = reinterpret_cast<double *>(w.sync + 4);
    int *info32 = reinterpret_cast<int *>(w.sync + 6);
    k_frob2<<<1, 1024, 0, st>>>(A, (long long)m * n, F2); DMRG_COUNT_LAUNCH();
    const int big = l > r ? l : r;
    const dim3 lgrid((big + 31) / 32, (big + 31) / 32);
    const double tol = (double)(l > 16 ? l : 16) * 2.220446049250313e-16;
    const double small = tol;
    const int nv = r <= 128 ? 32 : 16;
    if (precond < 0) precond = ctx->jacobi64_precond;
    prof_mark(ctx, PROF_JACOBI64);
    if (precond && r >= 64) {
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        char *p = static_cast<char *>(work) + svd_work_bytes_base(r, l);
        float *X32 = reinterpret_cast<float *>(p); p += al(sizeof(float) * (size_t)r * ldx);
        double *Q = reinterpret_cast<double *>(p); p += al(sizeof(double) * (size_t)r * r);
        double *T = reinterpret_cast<double *>(p);
        k_gj_load<float><<<lgrid, dim3(32, 8), 0, st>>>(A, m, n, tr, r, l, ldx, X32, 1); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        DMRG_TRY(gjac_run<float>(ctx, X32, r, l, ldx, l, r, max_sweeps, 1.0e-5, ctx->jacobi32_floor, F2, sync, info32,
                                 nullptr, nv, 0));
        k_gj_take_q<<<grid_ln((long long)r * r, ctx->num_sms), 256, 0, st>>>(X32, r, l, ldx, Q); DMRG_COUNT_LAUNCH();
        for (int it = 0; it < 2; ++it) {
            // T = Q Q^T, then Q <- 1.5 Q - 0.5 T Q (into X32's FP64-sized slot would alias; use Xe as scratch)
            DMRG_TRY(gemm_f64(st, r, r, r, 1.0, Q, r, 1, 0, Q, 1, r, 0, 0.0, T, r, 1, 0, 1));
            DMRG_CUDA(cudaMemcpyAsync(Xe, Q, sizeof(double) * (size_t)r * r, cudaMemcpyDeviceToDevice, st));
            DMRG_TRY(gemm_f64(st, r, r, r, -0.5, T, r, 1, 0, Q, r, 1, 0, 1.5, Xe, r, 1, 0, 1));
            DMRG_CUDA(cudaMemcpyAsync(Q, Xe, sizeof(double) * (size_t)r * r, cudaMemcpyDeviceToDevice, st));
        }
        // first part of the FP64 vectors: Q op(A), op(A) the r x l matrix of vectors
        const long long sBk = tr ? n : 1, sBn = tr ? 1 : n;
        DMRG_TRY(gemm_f64(st, r, l, r, 1.0, Q, r, 1, 0, A, sBk, sBn, 0, 0.0, Xe, ldx, 1, 0, 1));
        k_gj_put_q<<<grid_ln((long long)r * r, ctx->num_sms), 256, 0, st>>>(Q, r, l, ldx, Xe); DMRG_COUNT_LAUNCH();
    } else {
        k_gj_load<double><<<lgrid, dim3(32, 8), 0, st>>>(A, m, n, tr, r, l, ldx, Xe, 1); DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    DMRG_TRY(gjac_run<double>(ctx, Xe, r, l, ldx, l, r, max_sweeps, tol, small, F2, sync, d_info, nullptr, nv, 0));
    prof_mark(ctx, PROF_JACOBI64);
    prof_count(ctx, PROF_JACOBI64, 4.0 * l * (double)l * r + 8.0 * l * (double)r * r + 9.0 * (double)r * r * r,
               8.0 * ((double)r * l + (double)r * r) * 2.0);
    k_jac_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(Xe, r, l, ldx, w.nrm); DMRG_COUNT_LAUNCH();
    k_jac_rank<<<(r + 255) / 256, 256, 0, st>>>(w.nrm, r, w.perm); DMRG_COUNT_LAUNCH();
    k_jac_out<<<r, 256, 0, st>>>(Xe, Xe + l, w.nrm, w.perm, m, n, tr, r, l, ldx, ldx, U, s, Vt); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg

namespace dmrg {

size_t jac32_work_bytes(int r, int l)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(sizeof(float) * (size_t)r * l) + al(sizeof(double) * r) + al(sizeof(int) * r) + al(sizeof(unsigned) * 8) +
           al(qr32_work_bytes(r)) + gbj32_padded_bytes(r, l);
}

dmrg_status frob2_f32(dmrg_ctx *ctx, const float *A, long long n, double *F2)
{
    k_frob2_f<<<1, 256, 0, ctx->stream>>>(A, n, F2); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

// Numerical row rank of R after the QR preconditioning: the smallest r_eff
// such that the rows r_eff.. together have Frobenius norm <= 2^-23 |X|_F.
// Dropping them moves no singular value by more than that (Weyl), the size of
// the FP32 rounding X already carries; the Jacobi then rotates r_eff rows.
constexpr int kRowRankSmem = 4096;
__global__ void k_row_rank32(const float *__restrict__ X, int r, int l, double *__restrict__ rn, int *r_eff)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < r; i += nw) {
        float a = 0.f;
        for (int k = lane; k < l; k += 32) a = fmaf(X[(long long)i * l + k], X[(long long)i * l + k], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) rn[i] = (double)a;
    }
    __syncthreads();
    // the scans below run on one thread: stage the row norms in shared memory
    __shared__ double rs[kRowRankSmem];
    const double *q = rn;
    if (r <= kRowRankSmem) {
        for (int i = threadIdx.x; i < r; i += blockDim.x) rs[i] = rn[i];
        __syncthreads();
        q = rs;
    }
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < r; ++i) tot += q[i];
        const double thr = tot * 1.4210854715202004e-14;   // (2^-23)^2 |X|_F^2
        double suffix = 0.0;
        int j = r;
        while (j > 1 && suffix + q[j - 1] <= thr) suffix += q[--j];
        *r_eff = j;
    }
}

// FP32 one-sided Jacobi on the columns (dir 0) or rows (dir 1) of theta; on
// return s_sorted[0..min(m,n)) holds the vector norms in descending order and
// perm the vector of each.  Scratch layout: X32 | nrm | perm | sync.
dmrg_status svd_jacobi32(dmrg_ctx *ctx, const double *A, int m, int n, int dir, void *work, int max_sweeps,
                         int *d_info, double *s_sorted, float **X_out, double **nrm_out, int **perm_out)
{
    if (m <= 0 || n <= 0) return DMRG_EINVAL;
    const int r = dir == 0 ? n : m, l = dir == 0 ? m : n;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(work);
    float *X = reinterpret_cast<float *>(p); p += al(sizeof(float) * (size_t)r * l);
    double *nrm = reinterpret_cast<double *>(p); p += al(sizeof(double) * r);
    int *perm = reinterpret_cast<int *>(p); p += al(sizeof(int) * r);
    unsigned *sync = reinterpret_cast<unsigned *>(p); p += al(sizeof(unsigned) * 8);
    void *qrw = p; p += al(qr32_work_bytes(r));
    float *Xp = reinterpret_cast<float *>(p);
    cudaStream_t st = ctx->stream;
    // rotate while the cosine exceeds 1e-5 (see below)
    if (ctx->gbj_min_r > 0 && r >= ctx->gbj_min_r) {
        // Gram-block Jacobi on a cooperative grid (tensor-core Gram and
        // rotation tiles), QR-preconditioned
        prof_mark(ctx, PROF_JACOBI32);
        DMRG_TRY(gbj32_sweeps(ctx, A, m, n, dir, X, Xp, qrw, sync, max_sweeps, 1.0e-5, ctx->jacobi32_floor, d_info));
        prof_mark(ctx, PROF_JACOBI32);
        {
            const double M_ = l > r ? l : r, N_ = l > r ? r : l;
            prof_count(ctx, PROF_JACOBI32, 4.0 * M_ * M_ * N_ + 8.0 * M_ * N_ * N_ + 9.0 * N_ * N_ * N_,
                       4.0 * (double)r * l * 2.0);
        }
        const double *F2g = reinterpret_cast<const double *>(sync + 4);
        k_jac32_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(X, r, l, nrm, F2g); DMRG_COUNT_LAUNCH();
        k_jac_rank<<<(r + 255) / 256, 256, 0, st>>>(nrm, r, perm); DMRG_COUNT_LAUNCH();
        const int r_out = m < n ? m : n;
        k_sorted_values<<<(r_out + 255) / 256, 256, 0, st>>>(nrm, perm, r_out, s_sorted); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
        *X_out = X;
        *nrm_out = nrm;
        *perm_out = perm;
        return DMRG_OK;
    }
    {
        dim3 grid = dir == 0 ? dim3((n + 31) / 32, (m + 31) / 32) : dim3((n + 31) / 32, (m + 31) / 32);
        k_jac32_load<<<grid, dim3(32, 8), 0, st>>>(A, m, n, dir, r, l, X, sync); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
    }
    // QR preconditioning: rotate the rows of R (X = Q R) instead of the rows
    // of X -- same singular values and directions, a third of the sweeps
    const int *reff = nullptr;
    if (ctx->jacobi_qr && r >= 32) {
        dmrg_status e = qr_precondition32(ctx, X, r, l, qrw);
        if (e != DMRG_OK && e != DMRG_EUNSUPPORTED) return e;
        if (e == DMRG_OK && ctx->jacobi_rank_drop) {
            // row norms go to the norm slot (rewritten after the sweeps); r_eff to sync[6]
            k_row_rank32<<<1, 512, 0, st>>>(X, r, l, nrm, reinterpret_cast<int *>(sync + 6)); DMRG_COUNT_LAUNCH();
            reff = reinterpret_cast<const int *>(sync + 6);
        }
    }
    // rotate while the cosine exceeds jacobi32_tol (1e-6): the Gram entries
    // of the blocked kernels (3xTF32) resolve a few 1e-7, and vectors left at
    // cosines of 1e-5 span a retained subspace rotated by ~1e-5 s_i s_j /
    // (s_i^2 - s_j^2) towards the discarded one -- measured, that raised the
    // mixed form's energy by 1.4e-8 per site against FP64 on the same
    // retained dimensions (1.3e-10 at 1e-6); the FP64 Newton-Schulz step that
    // follows makes the retained vectors orthonormal to ~k tol^2
    const double tol = ctx->jacobi32_tol;
    int *status = ctx->d_status;
    // F2 = |A|_F^2 from the FP32 copy; vectors below 2^-23 |A|_F are dropped anyway
    const double *F2 = reinterpret_cast<const double *>(sync + 4);
    const double small = ctx->jacobi32_floor;
    k_frob2_f<<<1, 1024, 0, st>>>(X, (long long)r * l, reinterpret_cast<double *>(sync + 4)); DMRG_COUNT_LAUNCH();
    prof_mark(ctx, PROF_JACOBI32);
    // grouped block Jacobi (Gram form, one 128-thread group per block pair):
    // option gjac32 = 1 for the problems that fit one CTA, 2 for every size.
    // Off by default: measured, the single-CTA kernel below takes 2.45 ms on
    // a 128 x 128 two-site tensor where the grouped one takes 3.85 ms, and
    // the blocked kernel is 1.2-2x faster at the bulk sizes
    bool done = false;
    // blocked form with tcgen05 Gram blocks and block rotations (tjacobi.cu):
    // an autotuned bucket's choice, else by size
    const int tj = tune_lookup_tj(ctx, r, l);
    const int tb = tj > 0 ? tj : (tj < 0 && ctx->tjac && r >= ctx->tjac_min_r ? ctx->tjac : 0);
    if (tb) {
        dmrg_status e = tjac_run(ctx, X, r, l, max_sweeps, tol, small, F2, d_info, tb);
        if (e == DMRG_OK) done = true;
        else if (e != DMRG_EUNSUPPORTED) return e;
    }
    // an autotuned bucket may pick the cluster size (8, 16) or another kernel (0)
    const int cj = (ctx->cjac32 && ctx->cjac_force_c == 0) ? tune_lookup_cj(ctx, r, l) : -1;
    const int force_c = ctx->cjac_force_c ? ctx->cjac_force_c : (cj > 0 ? cj : 0);
    if (!done && ctx->cjac32 && cj != 0 && r >= ctx->cjac_min_r &&
        (force_c ? cjac32_fits_c(r, l, force_c) : cjac32_fits(r, l))) {
        // one thread-block cluster: blocks of vectors in the CTAs' shared
        // memory, moved between them through distributed shared memory
        DMRG_TRY(cjac32_run(ctx, X, r, l, max_sweeps, tol, small, F2, d_info, reff, force_c));
        done = true;
    }
    if (done) {
    } else if (ctx->gjac32 == 2 || (ctx->gjac32 == 1 && (long long)r * l <= kSmemJacFloats)) {
        int nv = ctx->gjac_nv ? ctx->gjac_nv : (r <= 128 ? 32 : 16), groups = ctx->gjac_groups;
        if (!ctx->gjac_nv && !ctx->gjac_groups) tune_lookup_gjac(ctx, r, l, &nv, &groups);   // autotuned bucket
        DMRG_TRY(gjac_run<float>(ctx, X, r, l, l, l, 0, max_sweeps, tol, small, F2, sync, d_info, reff, nv, groups));
    } else if ((long long)r * l <= kSmemJacFloats) {
        const int smem = (int)(sizeof(float) * (size_t)r * l);
        static bool attr = false;
        if (!attr) {
            DMRG_CUDA(cudaFuncSetAttribute(k_jac32_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(float) * kSmemJacFloats)));
            attr = true;
        }
        int thr = r >= 64 ? 1024 : (r >= 16 ? 256 : 64);
        k_jac32_smem<<<1, thr, smem, st>>>(X, r, l, max_sweeps, tol, status, d_info, F2, small, reff);
        DMRG_COUNT_LAUNCH();
    } else {
        // blocked form: block width so that about one block pair per SM is
        // available each round and 2 BW vectors fit in shared memory
        // each grid barrier costs a few microseconds with ~100 CTAs arriving,
        // so aim for ~48 block pairs per round: fewer, heavier rounds
        const long long cap = (200LL * 1024) / (8LL * l);      // max BW for shared memory
        int pairs = ctx->bjac_pairs, inner = ctx->bjac_inner;
        tune_lookup_svd(ctx, r, l, &pairs, &inner);            // autotuned bucket, if any
        int bw = 1;
        while (bw < 16 && 2LL * bw <= cap && (r / (2 * bw)) > pairs) bw *= 2;
        while (bw > 1 && (long long)bw > cap) bw /= 2;
        dmrg_status e = DMRG_EUNSUPPORTED;
        // Gram-form inner sweep (one inner sweep per block pair, BW >= 4)
        const bool gram = ctx->bjac_gram && inner == 1 && bw >= 4 &&
                          8LL * bw * bjac32g_stride(l) <= 192LL * 1024;
        if (gram) {
            switch (bw) {
            case 16: e = launch_bjac32g<16>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, reff); break;
            case 8: e = launch_bjac32g<8>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, reff); break;
            default: e = launch_bjac32g<4>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, reff); break;
            }
        } else switch (bw) {
        case 16: e = launch_bjac32<16>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, inner, reff); break;
        case 8: e = launch_bjac32<8>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, inner, reff); break;
        case 4: e = launch_bjac32<4>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, inner, reff); break;
        case 2: e = launch_bjac32<2>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, inner, reff); break;
        default: e = launch_bjac32<1>(ctx, X, r, l, max_sweeps, tol, sync, d_info, F2, small, inner, reff); break;
        }
        if (e != DMRG_OK) return e;
    }
    prof_mark(ctx, PROF_JACOBI32);
    {
        const double M_ = l > r ? l : r, N_ = l > r ? r : l;
        prof_count(ctx, PROF_JACOBI32, 4.0 * M_ * M_ * N_ + 8.0 * M_ * N_ * N_ + 9.0 * N_ * N_ * N_,
                   4.0 * (double)r * l * 2.0);
    }
    DMRG_CUDA(cudaGetLastError());
    k_jac32_norms<<<(r * 32 + 255) / 256, 256, 0, st>>>(X, r, l, nrm, F2); DMRG_COUNT_LAUNCH();
    k_jac_rank<<<(r + 255) / 256, 256, 0, st>>>(nrm, r, perm); DMRG_COUNT_LAUNCH();
    const int r_out = m < n ? m : n;
    k_sorted_values<<<(r_out + 255) / 256, 256, 0, st>>>(nrm, perm, r_out, s_sorted); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    *X_out = X;
    *nrm_out = nrm;
    *perm_out = perm;
    return DMRG_OK;
}

dmrg_status gather_unit_vectors(dmrg_ctx *ctx, const float *X, const double *nrm, const int *perm, const int *kdev,
                                int kmax, int l, double *Q)
{
    long long total = (long long)kmax * l;
    long long b = (total + 255) / 256;
    if (b > ctx->num_sms * 8LL) b = ctx->num_sms * 8LL;
    if (b < 1) b = 1;
    k_gather_unit<<<(int)b, 256, 0, ctx->stream>>>(X, nrm, perm, kdev, l, Q, 2.384185791015625e-07); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg
