// gjacobi.cu -- grouped block one-sided Jacobi in Gram form, FP32 and FP64.
//
// The one-sided (Hestenes) Jacobi SVD of Eq. (20) orthogonalises r vectors
// of length l by plane rotations.  Here the vectors are grouped in blocks of
// BW = NV / 2; a sweep visits every pair of blocks once in circle-method
// order, and one round of that order is a perfect matching of the blocks, so
// all block pairs of a round are independent.  A block pair is the work of a
// *group* of 128 threads (four warps) that synchronise with a named barrier
// of their own; a CTA holds several groups, so small problems run in one CTA
// with __syncthreads between rounds and larger ones on a few co-resident
// CTAs with a bounded grid barrier.  For its block pair a group
//   1. stages the NV vectors in shared memory (zero-padded to whole chunks
//      of 8 positions);
//   2. forms their Gram matrix G = X X^T over the first l positions: FP32 as
//      3xTF32 tensor-core products (mma.sync m16n8k8), FP64 with DFMA;
//   3. runs one cyclic Jacobi sweep on G -- in exact arithmetic the rotations
//      an inner sweep over the vector pairs would apply -- accumulating their
//      product Q (double-buffered, one group barrier per step), then one
//      Newton-Schulz step Q <- Q (3 I - Q^T Q) / 2;
//   4. writes x_j <- sum_i Q[i][j] x_i over the whole extended vector with
//      FMAs of the vectors' own precision.
// The iteration stops after a sweep without rotations.
//
// Extended vectors: a vector may carry a second part of rv positions (the
// row of V^T it accumulates: the same rotations applied to the identity).
// The Gram matrix is taken over the first part only.  In global memory
// vector i is X[i * ldx + e] for e < l and X[i * ldx + gv0 + e'] for the
// second part, e' < rv.
#include "common.cuh"
#include "mma_tf32.cuh"

#include <algorithm>

namespace dmrg {
namespace {

constexpr int GT = 128;               // threads of a group
constexpr int GW = GT / 32;           // warps of a group
constexpr int kMaxGroups = 4;          // 512 threads: up to 128 registers a thread

__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

// circle method on np (even) players: player np-1 fixed, the others rotate
__device__ __forceinline__ void circle(int np, int t, int p, int &i, int &j)
{
    const int q = np - 1;
    if (p == 0) {
        i = q;
        j = t;
    } else {
        i = (t + p) % q;
        j = (t - p + q) % q;
    }
}

// Rotation of a pair with Gram entries a = |x_p|^2, b = |x_q|^2, g = x_p.x_q:
// zeta = (b - a) / (2 g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t (the 2 x 2 symmetric Schur step, Golub &
// Van Loan 8.5.2).  None when a vector is below the floor or the pair is
// orthogonal to the tolerance.
__device__ __forceinline__ bool rot_params(float a, float b, float g, float floor2, float tol, float &c, float &s)
{
    if (!(a > floor2 && b > floor2)) return false;
    if (!(fabsf(g) > tol * sqrtf(a) * sqrtf(b))) return false;
    const float zeta = (b - a) / (2.0f * g);
    const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = c * t;
    return true;
}
__device__ __forceinline__ bool rot_params(double a, double b, double g, double floor2, double tol, double &c,
                                           double &s)
{
    if (!(a > floor2 && b > floor2)) return false;
    if (!(fabs(g) > tol * sqrt(a) * sqrt(b))) return false;
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
    return true;
}

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// one element from global to shared memory without a register round trip;
// zero-filled when !valid (no global read then)
__device__ __forceinline__ void cp_async_elem(float *dst, const float *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_elem(double *dst, const double *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}

// per-group shared memory (after the vectors): Gram and rotation buffers,
// Gram partial sums, step parameters, vector ids, a rotation counter
template <typename T, int NV>
struct GroupSmem {
    T Gb[2][NV][NV + 1];
    T Qb[2][NV][NV + 1];
    float part[GW][16][8];
    T pc[2][NV], psn[2][NV];
    int ppt[2][NV];
    int vid[NV];
    unsigned rot;
};

template <typename T, int NV>
__host__ __device__ constexpr size_t group_bytes(int ls)
{
    return (size_t)round_up((int)(sizeof(T) * (size_t)NV * ls), 16) + round_up((int)sizeof(GroupSmem<T, NV>), 16);
}

// Gram matrix G = X X^T of the group's NV vectors over positions [0, lpad).
template <int NV>
__device__ __forceinline__ void gram(const float *xs, int ls, int lpad, GroupSmem<float, NV> &S, int tg)
{
    constexpr int MT = NV / 16, NT = NV / 8, TILES = MT * NT;
    constexpr int WPT = TILES >= GW ? 1 : GW / TILES;     // warps per tile (k split)
    const int lane = tg & 31, warp = tg >> 5, g = lane >> 2, c4 = lane & 3;
    const int nchunk = lpad / 8;
    auto fa = [&](int m, int k) { return xs[m * ls + k]; };
    auto fb = [&](int k, int n) { return xs[n * ls + k]; };
    if (TILES >= GW) {
        for (int tile = warp; tile < TILES; tile += GW) {
            const int mi = tile / NT, ni = tile % NT;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ck = 0; ck < nchunk; ++ck) mma3(acc, g, c4, fa, fb, 16 * mi, 8 * ni, 8 * ck);
            S.Gb[0][16 * mi + g][8 * ni + 2 * c4] = acc[0];
            S.Gb[0][16 * mi + g][8 * ni + 2 * c4 + 1] = acc[1];
            S.Gb[0][16 * mi + g + 8][8 * ni + 2 * c4] = acc[2];
            S.Gb[0][16 * mi + g + 8][8 * ni + 2 * c4 + 1] = acc[3];
        }
    } else {
        const int tile = warp / WPT, kp = warp % WPT;
        const int mi = tile / NT, ni = tile % NT;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int ck = kp; ck < nchunk; ck += WPT) mma3(acc, g, c4, fa, fb, 16 * mi, 8 * ni, 8 * ck);
        S.part[warp][g][2 * c4] = acc[0];
        S.part[warp][g][2 * c4 + 1] = acc[1];
        S.part[warp][g + 8][2 * c4] = acc[2];
        S.part[warp][g + 8][2 * c4 + 1] = acc[3];
    }
    if (TILES < GW) {
        // sum the k parts of each tile in a fixed order
        asm volatile("bar.sync %0, %1;" ::"r"((int)(threadIdx.x / GT) + 1), "r"(GT) : "memory");
        for (int e = tg; e < NV * NV; e += GT) {
            const int i = e / NV, j = e % NV;
            const int tile = (i / 16) * NT + j / 8;
            float a = 0.f;
            for (int kp = 0; kp < WPT; ++kp) a += S.part[tile * WPT + kp][i % 16][j % 8];
            S.Gb[0][i][j] = a;
        }
    }
}

template <int NV>
__device__ __forceinline__ void gram(const double *xs, int ls, int lpad, GroupSmem<double, NV> &S, int tg)
{
    // upper triangle, each entry's dot product split over 4 consecutive lanes
    constexpr int NE = NV * (NV + 1) / 2;
    const int items = NE * 4;
    for (int w0 = 0; w0 < items; w0 += GT) {
        const int w = w0 + tg;
        double a = 0.0;
        int i = 0, j = 0;
        const bool ok = w < items;
        if (ok) {
            int e = w >> 2;
            // entry e of the row-major upper triangle -> (i, j)
            while (e >= NV - i) { e -= NV - i; ++i; }
            j = i + e;
            const double *xi = xs + i * ls, *xj = xs + j * ls;
            for (int k = w & 3; k < lpad; k += 4) a = fma(xi[k], xj[k], a);
        }
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (ok && (w & 3) == 0) {
            S.Gb[0][i][j] = a;
            S.Gb[0][j][i] = a;
        }
    }
}

template <typename T, int NV>
__global__ void __launch_bounds__(GT *kMaxGroups)
    k_gjac(T *__restrict__ X, int r_all, int l, int lpad, int ldx, int gv0, int rv, int ls, int max_sweeps,
           double tol, double small, const double *F2, unsigned *sync, int *status, int *info, const int *r_eff)
{
    constexpr int BW = NV / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned block_rot;
    const int ngroups = blockDim.x / GT;
    const int grp = threadIdx.x / GT, tg = threadIdx.x % GT;
    const size_t gb = group_bytes<T, NV>(ls);
    T *xs = reinterpret_cast<T *>(smem_raw + gb * grp);
    GroupSmem<T, NV> &S =
        *reinterpret_cast<GroupSmem<T, NV> *>(smem_raw + gb * grp + round_up((int)(sizeof(T) * (size_t)NV * ls), 16));
    const int r = r_eff ? min(r_all, max(1, *r_eff)) : r_all;
    const T floor2 = (T)(small * small * F2[0]), tolT = (T)tol;
    const int nb = (r + BW - 1) / BW;
    const int nbp = nb + (nb & 1);
    const int npairs = nbp / 2;
    const int gid = blockIdx.x * ngroups + grp, total_groups = gridDim.x * ngroups;
    const int lv = lpad + rv;                    // extended length in shared memory
    unsigned *barrier = sync;
    unsigned *rotc = sync + 2;
    int sweep = 0;
    bool converged = false;

    auto gnew = [&](int pb, int gbuf, int i, int j) {
        const T ci = S.pc[pb][i], si = S.psn[pb][i], cj = S.pc[pb][j], sj = S.psn[pb][j];
        const int pi = S.ppt[pb][i], pj = S.ppt[pb][j];
        T v = ci * cj * S.Gb[gbuf][i][j];
        v = fma(ci * sj, S.Gb[gbuf][i][pj], v);
        v = fma(si * cj, S.Gb[gbuf][pi][j], v);
        return fma(si * sj, S.Gb[gbuf][pi][pj], v);
    };
    auto setpar = [&](int pb, int a, int b, T gaa, T gbb, T gab) {
        T c = (T)1, sn = (T)0;
        const bool rot = S.vid[a] >= 0 && S.vid[b] >= 0 && rot_params(gaa, gbb, gab, floor2, tolT, c, sn);
        S.pc[pb][a] = c; S.psn[pb][a] = rot ? -sn : (T)0; S.ppt[pb][a] = rot ? b : a;
        S.pc[pb][b] = c; S.psn[pb][b] = rot ? sn : (T)0; S.ppt[pb][b] = rot ? a : b;
        return rot;
    };

    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) block_rot = 0;
        __syncthreads();
        for (int t = 0; t < nbp - 1; ++t) {
            for (int p = gid; p < npairs; p += total_groups) {
                int I, J;
                circle(nbp, t, p, I, J);
                if (tg < NV) {
                    const int blk = tg < BW ? I : J;
                    const int v = blk * BW + (tg % BW);
                    S.vid[tg] = (blk < nb && v < r) ? v : -1;
                }
                if (tg == 0) S.rot = 0;
                group_sync(grp);
                // 1. stage the vectors (positions l..lpad zero) with asynchronous
                //    copies: every copy of a thread is in flight at once, one
                //    L2 round trip per round instead of one per element
                for (int q = 0; q < NV; ++q) {
                    const int v = S.vid[q];
                    const T *src = X + (long long)(v < 0 ? 0 : v) * ldx;
                    T *dst = xs + q * ls;
                    for (int e = tg; e < lv; e += GT) {
                        const bool valid = v >= 0 && (e < l || e >= lpad);
                        const T *g = valid ? (e < l ? src + e : src + gv0 + (e - lpad)) : X;
                        cp_async_elem(dst + e, g, valid);
                    }
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                group_sync(grp);
                // 2. Gram matrix, made bitwise symmetric (upper triangle mirrored)
                gram<NV>(xs, ls, lpad, S, tg);
                group_sync(grp);
                for (int e = tg; e < NV * NV; e += GT) {
                    const int i = e / NV, j = e % NV;
                    S.Qb[0][i][j] = (i == j) ? (T)1 : (T)0;
                    if (i > j) S.Gb[0][i][j] = S.Gb[0][j][i];
                }
                group_sync(grp);
                // 3. one cyclic sweep on G, accumulating Q
                unsigned myrot = 0;
                if (tg < BW) {
                    int a_, b_;
                    circle(NV, 0, tg, a_, b_);
                    myrot += setpar(0, a_, b_, S.Gb[0][a_][a_], S.Gb[0][b_][b_], S.Gb[0][min(a_, b_)][max(a_, b_)]);
                }
                group_sync(grp);
                for (int u = 0; u < NV - 1; ++u) {
                    const int cb = u & 1, nbf = cb ^ 1;
                    for (int e = tg; e < 2 * NV * NV; e += GT) {
                        if (e < NV * NV) {
                            const int i = e / NV, j = e % NV;
                            if (i > j) continue;
                            const T v = gnew(cb, cb, i, j);
                            S.Gb[nbf][i][j] = v;
                            S.Gb[nbf][j][i] = v;
                        } else {
                            const int e2 = e - NV * NV, i = e2 / NV, j = e2 % NV;
                            S.Qb[nbf][i][j] =
                                fma(S.psn[cb][j], S.Qb[cb][i][S.ppt[cb][j]], S.pc[cb][j] * S.Qb[cb][i][j]);
                        }
                    }
                    if (u + 1 < NV - 1 && tg < BW) {
                        int a_, b_;
                        circle(NV, u + 1, tg, a_, b_);
                        const T gaa = gnew(cb, cb, a_, a_), gbb = gnew(cb, cb, b_, b_);
                        const T gab = gnew(cb, cb, min(a_, b_), max(a_, b_));
                        myrot += setpar(nbf, a_, b_, gaa, gbb, gab);
                    }
                    group_sync(grp);
                }
                if (myrot) atomicAdd(&S.rot, myrot);
                group_sync(grp);
                const unsigned prot = S.rot;
                if (prot) {
                    constexpr int qf = (NV - 1) & 1;             // buffer holding the final Q
                    // Q <- Q (3 I - Q^T Q) / 2: orthogonal again at the working precision
                    for (int e = tg; e < NV * NV; e += GT) {
                        const int i = e / NV, j = e % NV;
                        T a = (T)0;
                        for (int k2 = 0; k2 < NV; ++k2) a = fma(S.Qb[qf][k2][i], S.Qb[qf][k2][j], a);
                        S.Gb[qf ^ 1][i][j] = (i == j ? (T)1.5 : (T)0) - (T)0.5 * a;
                    }
                    group_sync(grp);
                    for (int e = tg; e < NV * NV; e += GT) {
                        const int i = e / NV, j = e % NV;
                        T a = (T)0;
                        for (int k2 = 0; k2 < NV; ++k2) a = fma(S.Qb[qf][i][k2], S.Gb[qf ^ 1][k2][j], a);
                        S.Qb[qf ^ 1][i][j] = a;
                    }
                    group_sync(grp);
                    if (tg == 0) atomicAdd(&block_rot, prot);
                    // 4. x_j <- sum_i Q[i][j] x_i over the extended vector, straight to X:
                    //    a thread keeps OPT columns of Q in registers and walks positions
                    constexpr int OPT = sizeof(T) == 4 ? (NV >= 32 ? 2 : 4) : (NV >= 32 ? 1 : 2);
                    constexpr int NG = NV / OPT, TPG = GT / NG;
                    static_assert(GT % NG == 0, "output groups");
                    const T(*Qf)[NV + 1] = S.Qb[qf ^ 1];
                    const int gi = tg / TPG, t0 = tg % TPG;
                    T qr[OPT][NV];
                    int vo[OPT];
#pragma unroll
                    for (int o = 0; o < OPT; ++o) {
                        vo[o] = S.vid[gi * OPT + o];
#pragma unroll
                        for (int i = 0; i < NV; ++i) qr[o][i] = Qf[i][gi * OPT + o];
                    }
                    for (int e = t0; e < lv; e += TPG) {
                        if (e >= l && e < lpad) continue;        // zero padding stays zero
                        T acc[OPT];
#pragma unroll
                        for (int o = 0; o < OPT; ++o) acc[o] = (T)0;
#pragma unroll
                        for (int i = 0; i < NV; ++i) {
                            const T x = xs[i * ls + e];
#pragma unroll
                            for (int o = 0; o < OPT; ++o) acc[o] = fma(qr[o][i], x, acc[o]);
                        }
                        const long long ge = e < l ? e : (long long)gv0 + (e - lpad);
#pragma unroll
                        for (int o = 0; o < OPT; ++o)
                            if (vo[o] >= 0) X[(long long)vo[o] * ldx + ge] = acc[o];
                    }
                }
                group_sync(grp);
            }
            // every block pair of this round is written before the next round reads
            if (gridDim.x == 1) {
                __syncthreads();
            } else if (!grid_barrier(barrier, status)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
                return;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && block_rot) atomicAdd(&rotc[sweep & 1], block_rot);
        if (gridDim.x == 1) {
            __syncthreads();
        } else if (!grid_barrier(barrier, status)) {
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
        // the reset of the next counter is visible before anyone adds to it
        if (gridDim.x == 1) {
            __syncthreads();
        } else if (!grid_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

template <typename T, int NV>
dmrg_status launch_gjac(dmrg_ctx *ctx, T *X, int r, int l, int ldx, int gv0, int rv, int max_sweeps, double tol,
                        double small, const double *F2, unsigned *sync, int *info, const int *r_eff, int max_groups)
{
    const int lpad = round_up(l, 8);
    // shared-memory row stride: whole chunks of 8, + 4 floats (FP32: the mma
    // fragment reads of 8 rows x 4 positions fall in 32 distinct banks) or + 1
    // double (FP64)
    const int ls = sizeof(T) == 4 ? round_up(lpad + rv, 8) + 4 : round_up(lpad + rv, 2) + 1;
    const size_t gb = group_bytes<T, NV>(ls);
    const size_t smem_cap = 220 * 1024;
    const int Gfit = (int)std::min<size_t>(kMaxGroups, smem_cap / gb);
    if (Gfit < 1) return DMRG_EUNSUPPORTED;
    const int BW = NV / 2;
    const int nb = (r + BW - 1) / BW;
    const int npairs = (nb + (nb & 1)) / 2;
    // groups per CTA: all block pairs in one CTA when they fit (no grid
    // barrier), else one pair per SM as long as there are SMs for them
    int G;
    if (max_groups > 0) G = std::min(Gfit, max_groups);
    else if (npairs <= Gfit) G = npairs;
    else G = std::min(Gfit, (npairs + ctx->num_sms - 1) / ctx->num_sms);
    if (G > npairs) G = npairs;
    if (G < 1) G = 1;
    const int threads = G * GT;
    const size_t smem = gb * G;
    static size_t attr[2] = {0, 0};
    size_t &a = attr[NV == 32 ? 1 : 0];
    if (a < smem) {
        DMRG_CUDA(cudaFuncSetAttribute(k_gjac<T, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        a = smem;
    }
    int blocks = (npairs + G - 1) / G;
    int *status = ctx->d_status;
    DMRG_CUDA(cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned), ctx->stream));
    if (blocks == 1) {
        k_gjac<T, NV><<<1, threads, smem, ctx->stream>>>(X, r, l, lpad, ldx, gv0, rv, ls, max_sweeps, tol, small, F2,
                                                         sync, status, info, r_eff);
        DMRG_COUNT_LAUNCH();
    } else {
        int per_sm = 0;
        DMRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gjac<T, NV>, threads, smem));
        if (per_sm < 1) return DMRG_EUNSUPPORTED;
        blocks = std::min(blocks, per_sm * ctx->num_sms);
        int lpad_ = lpad, ls_ = ls;
        void *args[] = {&X, (void *)&r, (void *)&l, &lpad_, (void *)&ldx, (void *)&gv0, (void *)&rv, &ls_,
                        (void *)&max_sweeps, (void *)&tol, (void *)&small, (void *)&F2, (void *)&sync, &status,
                        (void *)&info, (void *)&r_eff};
        DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_gjac<T, NV>, dim3(blocks), dim3(threads), args, smem,
                                              ctx->stream));
        DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace

template <typename T>
dmrg_status gjac_run(dmrg_ctx *ctx, T *X, int r, int l, int ldx, int gv0, int rv, int max_sweeps, double tol,
                     double small, const double *F2, unsigned *sync, int *info, const int *r_eff, int nv,
                     int max_groups)
{
    if (r < 1 || l < 1 || ldx < l || (rv > 0 && gv0 < l)) return DMRG_EINVAL;
    if (nv == 32) return launch_gjac<T, 32>(ctx, X, r, l, ldx, gv0, rv, max_sweeps, tol, small, F2, sync, info, r_eff,
                                            max_groups);
    return launch_gjac<T, 16>(ctx, X, r, l, ldx, gv0, rv, max_sweeps, tol, small, F2, sync, info, r_eff, max_groups);
}

template dmrg_status gjac_run<float>(dmrg_ctx *, float *, int, int, int, int, int, int, double, double,
                                     const double *, unsigned *, int *, const int *, int, int);
template dmrg_status gjac_run<double>(dmrg_ctx *, double *, int, int, int, int, int, int, double, double,
                                      const double *, unsigned *, int *, const int *, int, int);

}  // namespace dmrg
