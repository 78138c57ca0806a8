// cjacobi.cu -- FP32 one-sided Jacobi (Eq. 20) on one thread-block cluster.
//
// The mixed form's SVD of the two-site tensor orthogonalises r vectors (the
// rows of X, length l) by plane rotations.  On one CTA every round of a sweep
// moves all r x l values through one SM's shared-memory pipe; on a grid the
// rounds pay a global barrier.  Here the work is spread over the C CTAs of
// one cluster (8; 16, the opt-in size, when 8 CTAs' shared memory cannot
// hold the blocks) and only block moves cross SMs:
//   * the vectors form 2C blocks of b = ceil(r / 2C); CTA c holds two of them
//     (its "top" and "bottom" block) in shared memory;
//   * a sweep first rotates the pairs inside every block (circle method on
//     the b vectors of a block, both blocks of all CTAs at once), then runs
//     2C - 1 block rounds: the b^2 pairs between the CTA's two blocks in b
//     inner rounds of b disjoint pairs (top i with bottom (i + s) mod b),
//     after which the blocks advance one place along the circle-method cycle
//         bottom_0 -> top_1 -> ... -> top_{C-1} -> bottom_{C-1} -> ... -> bottom_0
//     (top_0 stays), pushed into the receiving CTA's shared memory through
//     distributed shared memory, and one cluster barrier;
//   * so every pair of vectors meets exactly once a sweep (a cyclic
//     ordering), and a sweep costs 2C cluster barriers;
//   * one warp handles a pair: x_i . x_j from registers (two FP32 chains and
//     a butterfly, so every lane holds the same sum), the 2 x 2 symmetric
//     Schur rotation, and the squared norms carried along as
//     |x_i'|^2 = |x_i|^2 - t g, |x_j'|^2 = |x_j|^2 + t g (recomputed at the
//     start of every sweep).
// The iteration stops after a sweep without rotations (cosine above the
// tolerance), counted across the cluster in CTA 0's shared memory.  Vectors
// keep their identity (an index travels with each), so the result is written
// back to the rows it came from.
#include "common.cuh"

#include <algorithm>
#include <cooperative_groups.h>
#include <unordered_map>

namespace dmrg {
namespace {

namespace cg = cooperative_groups;

constexpr int kCjMaxB = 32;         // vectors per block: one warp per pair, <= 1024 threads

__device__ __forceinline__ void cj_circle(int np, int t, int p, int &i, int &j)
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

// One pair on one warp.  xi, xj: the two vectors (shared memory, rows of
// ldl floats, zero beyond l); na, nb: their squared norms.  Lane i holds the
// float4 chunks i, i + 32, ... of each (one 512-byte span per load or store
// instruction, no bank conflicts; 32 TM >= ldl).  Returns true if a
// rotation was applied.
template <int TM>
__device__ __forceinline__ bool cj_pair(float *__restrict__ xi, float *__restrict__ xj, float *na, float *nb, int ldl,
                                        float floor2, float tol, int lane)
{
    const float a = *na, b = *nb;
    if (!(a > floor2 && b > floor2)) return false;
    constexpr int V4 = TM / 4;
    float4 u[V4], v[V4];
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int q = 0; q < V4; ++q) {
        const int k = 4 * (lane + 32 * q);
        if (k < ldl) {
            u[q] = *reinterpret_cast<const float4 *>(xi + k);
            v[q] = *reinterpret_cast<const float4 *>(xj + k);
        } else {
            u[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            v[q] = u[q];
        }
        g0 = fmaf(u[q].x, v[q].x, g0);
        g1 = fmaf(u[q].y, v[q].y, g1);
        g0 = fmaf(u[q].z, v[q].z, g0);
        g1 = fmaf(u[q].w, v[q].w, g1);
    }
    float g = g0 + g1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    // the rotation from the special-function unit (reciprocal and reciprocal
    // square root, a few ulp): any angle this close to the Jacobi angle
    // orthogonalises the pair to well below the tolerance, and c, s come
    // from one rsqrt so c^2 + s^2 = 1 to its accuracy
    if (!(fabsf(g) * rsqrtf(a) * rsqrtf(b) > tol)) return false;
    const float zeta = __fdividef(b - a, 2.0f * g);
    const float az = fabsf(zeta);
    float t;
    if (az > 1e15f) {
        t = __fdividef(0.5f, az);
    } else {
        const float q = fmaf(zeta, zeta, 1.0f);
        t = __fdividef(1.0f, az + q * rsqrtf(q));
    }
    t = copysignf(t, zeta);
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = c * t;
#pragma unroll
    for (int q = 0; q < V4; ++q) {
        const int k = 4 * (lane + 32 * q);
        if (k < ldl) {
            float4 x, y;
            x.x = fmaf(c, u[q].x, -s * v[q].x);
            x.y = fmaf(c, u[q].y, -s * v[q].y);
            x.z = fmaf(c, u[q].z, -s * v[q].z);
            x.w = fmaf(c, u[q].w, -s * v[q].w);
            y.x = fmaf(s, u[q].x, c * v[q].x);
            y.y = fmaf(s, u[q].y, c * v[q].y);
            y.z = fmaf(s, u[q].z, c * v[q].z);
            y.w = fmaf(s, u[q].w, c * v[q].w);
            *reinterpret_cast<float4 *>(xi + k) = x;
            *reinterpret_cast<float4 *>(xj + k) = y;
        }
    }
    if (lane == 0) {
        *na = a - t * g;
        *nb = b + t * g;
    }
    return true;
}

// Shared memory (dynamic, 16-byte aligned):
//   blocks  [2 parities][2: top, bottom][b][ldl] floats
//   norms   [2][2][b] floats
//   ids     [2][2][b] ints
//   counts  [3] unsigned: [0], [1] the cluster's rotations of even / odd
//           sweeps (used on rank 0), [2] this CTA's rotations of the sweep
template <int TM, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(1024)
    k_cjac32(float *__restrict__ X, int r_all, int l, int ldl, int b, int max_sweeps, float tol,
             const double *__restrict__ F2, double small, const int *__restrict__ r_eff_p, int *status, int *info)
{
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float cj_sm[];
    const int crank = (int)cluster.block_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long blk = (long long)b * ldl;
    float *const nrm = cj_sm + 4 * blk;
    int *const ids = reinterpret_cast<int *>(nrm + 4 * b);
    unsigned *const cnt = reinterpret_cast<unsigned *>(ids + 4 * b);
    auto slot = [&](int par, int tb) { return cj_sm + (long long)(par * 2 + tb) * blk; };
    auto nslot = [&](int par, int tb) { return nrm + (par * 2 + tb) * b; };
    auto islot = [&](int par, int tb) { return ids + (par * 2 + tb) * b; };

    const int r_eff = r_eff_p ? min(r_all, max(1, *r_eff_p)) : r_all;
    // initial placement: CTA c holds blocks c (top) and C + c (bottom)
    for (int v = warp; v < 2 * b; v += nw) {
        const int tb = v / b, i = v - tb * b;
        const int beta = tb ? C + crank : crank;
        const int id = beta * b + i;
        float *x = slot(0, tb) + (long long)i * ldl;
        for (int k = lane; k < ldl; k += 32) x[k] = (id < r_eff && k < l) ? X[(long long)id * l + k] : 0.f;
        if (lane == 0) islot(0, tb)[i] = id;
    }
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0u;
    const float floor2 = (float)(small * small * F2[0]);
    // every CTA of the cluster is running and initialised before any remote access
    cluster.sync();

    // destinations of the two blocks along the cycle (rank, slot)
    const int dt_rank = crank == 0 ? 0 : (crank < C - 1 ? crank + 1 : crank);
    const int dt_tb = crank == C - 1 ? 1 : 0;
    const int db_rank = crank == 0 ? 1 : crank - 1;
    const int db_tb = crank == 0 ? 0 : 1;
    unsigned *const cnt_r0 = cluster.map_shared_rank(cnt, 0);

    const int rp = b + (b & 1), half = rp / 2;
    int par = 0, sweep = 0;
    bool converged = false;
    unsigned my_rot = 0u;                    // this warp's rotations in the sweep
    for (; sweep < max_sweeps; ++sweep) {
        // squared norms of the CTA's two blocks
        for (int v = warp; v < 2 * b; v += nw) {
            const int tb = v / b, i = v - tb * b;
            const float *x = slot(par, tb) + (long long)i * ldl;
            float a0 = 0.f, a1 = 0.f;
            int k = lane;
            for (; k + 32 < l; k += 64) {
                a0 = fmaf(x[k], x[k], a0);
                a1 = fmaf(x[k + 32], x[k + 32], a1);
            }
            if (k < l) a0 = fmaf(x[k], x[k], a0);
            float a = a0 + a1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) nslot(par, tb)[i] = a;
        }
        __syncthreads();
        // 1. the pairs inside each block
        for (int t = 0; t < rp - 1; ++t) {
            if (warp < 2 * half) {
                const int tb = warp / half, p = warp - tb * half;
                int i, j;
                cj_circle(rp, t, p, i, j);
                if (i < b && j < b) {
                    float *x = slot(par, tb);
                    float *n = nslot(par, tb);
                    my_rot += cj_pair<TM>(x + (long long)i * ldl, x + (long long)j * ldl, n + i, n + j, ldl, floor2,
                                          tol, lane);
                }
            }
            __syncthreads();
        }
        // 2. block rounds
        for (int br = 0; br < 2 * C - 1; ++br) {
            for (int s = 0; s < b; ++s) {
                if (warp < b) {
                    const int i = warp, j = (warp + s) % b;
                    my_rot += cj_pair<TM>(slot(par, 0) + (long long)i * ldl, slot(par, 1) + (long long)j * ldl,
                                          nslot(par, 0) + i, nslot(par, 1) + j, ldl, floor2, tol, lane);
                }
                __syncthreads();
            }
            // advance the blocks: push into the receivers' other parity
            const int np = par ^ 1;
            {
                const float4 *st = reinterpret_cast<const float4 *>(slot(par, 0));
                const float4 *sb = reinterpret_cast<const float4 *>(slot(par, 1));
                float4 *dt = reinterpret_cast<float4 *>(cluster.map_shared_rank(slot(np, dt_tb), dt_rank));
                float4 *db = reinterpret_cast<float4 *>(cluster.map_shared_rank(slot(np, db_tb), db_rank));
                const int n4 = (int)(blk >> 2);
                for (int e = threadIdx.x; e < n4; e += blockDim.x) {
                    dt[e] = st[e];
                    db[e] = sb[e];
                }
                if (threadIdx.x < b) {
                    cluster.map_shared_rank(nslot(np, dt_tb), dt_rank)[threadIdx.x] = nslot(par, 0)[threadIdx.x];
                    cluster.map_shared_rank(islot(np, dt_tb), dt_rank)[threadIdx.x] = islot(par, 0)[threadIdx.x];
                } else if (threadIdx.x >= 32 && threadIdx.x < 32 + b) {
                    const int i = threadIdx.x - 32;
                    cluster.map_shared_rank(nslot(np, db_tb), db_rank)[i] = nslot(par, 1)[i];
                    cluster.map_shared_rank(islot(np, db_tb), db_rank)[i] = islot(par, 1)[i];
                }
            }
            cluster.sync();
            par = np;
        }
        // convergence: rotations of this sweep over the cluster
        if (lane == 0 && my_rot) atomicAdd(&cnt[2], my_rot);
        my_rot = 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&cnt_r0[sweep & 1], cnt[2]);
            cnt[2] = 0u;
        }
        cluster.sync();
        const unsigned total = *reinterpret_cast<volatile unsigned *>(&cnt_r0[sweep & 1]);
        if (crank == 0 && threadIdx.x == 0) cnt[(sweep + 1) & 1] = 0u;
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
    }
    // write back to the rows the vectors came from
    for (int v = warp; v < 2 * b; v += nw) {
        const int tb = v / b, i = v - tb * b;
        const int id = islot(par, tb)[i];
        if (id >= r_eff) continue;
        const float *x = slot(par, tb) + (long long)i * ldl;
        for (int k = lane; k < l; k += 32) X[(long long)id * l + k] = x[k];
    }
    if (crank == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

template <int TM, int C>
dmrg_status launch_cjac32(dmrg_ctx *ctx, float *X, int r, int l, int ldl, int b, int threads, size_t smem,
                          int max_sweeps, float tol, const double *F2, double small, int *d_info, const int *r_eff)
{
    static bool attr = false;
    if (!attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_cjac32<TM, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        if (C > 8) DMRG_CUDA(cudaFuncSetAttribute(k_cjac32<TM, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr = true;
    }
    k_cjac32<TM, C><<<C, threads, smem, ctx->stream>>>(X, r, l, ldl, b, max_sweeps, tol, F2, small, r_eff,
                                                       ctx->d_status, d_info);
    DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

// Whether a cluster of C CTAs of `threads` threads and `smem` bytes can be
// resident (occupancy query, cached per size class); a launch that cannot is
// not attempted.
template <int TM, int C>
bool cjac_cluster_fits(int threads, size_t smem)
{
    static std::unordered_map<unsigned long long, bool> seen;
    const unsigned long long key = ((unsigned long long)threads << 32) | (unsigned long long)smem;
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    if (cudaFuncSetAttribute(k_cjac32<TM, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
        return false;
    if (C > 8 && cudaFuncSetAttribute(k_cjac32<TM, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, (const void *)k_cjac32<TM, C>, &cfg) == cudaSuccess && n >= 1;
    cudaGetLastError();
    seen[key] = ok;
    return ok;
}

struct CjPlan {
    int C = 0, b = 0, ldl = 0, threads = 0, tm = 0;
    size_t smem = 0;
};

CjPlan cj_plan(int r, int l, int C)
{
    CjPlan p;
    p.C = C;
    p.b = (r + 2 * C - 1) / (2 * C);
    p.ldl = (l + 3) & ~3;
    const int rp = p.b + (p.b & 1);
    p.threads = 32 * std::max(4, std::max(rp, p.b));
    p.smem = sizeof(float) * (4ull * p.b * p.ldl + 4ull * p.b) + sizeof(int) * 4ull * p.b + 4 * sizeof(unsigned);
    const int tm = (l + 31) / 32;
    p.tm = tm <= 4 ? 4 : tm <= 8 ? 8 : tm <= 12 ? 12 : 16;
    return p;
}

bool cj_plan_ok(const CjPlan &p, int r, int l)
{
    return r >= 1 && l >= 1 && l <= 512 && p.b <= kCjMaxB && p.smem <= 227 * 1024;
}

template <int C>
bool cj_fits_dispatch(const CjPlan &p)
{
    switch (p.tm) {
    case 4: return cjac_cluster_fits<4, C>(p.threads, p.smem);
    case 8: return cjac_cluster_fits<8, C>(p.threads, p.smem);
    case 12: return cjac_cluster_fits<12, C>(p.threads, p.smem);
    default: return cjac_cluster_fits<16, C>(p.threads, p.smem);
    }
}

// 8 CTAs where the blocks fit them, else 16 (opt-in cluster size) if the GPU
// can hold such a cluster; 0 if neither.  force_c = 8 or 16 takes that size
// if it fits (the autotuner's choice), else 0.
int cj_choose(int r, int l, CjPlan *out, int force_c = 0)
{
    if (force_c == 8 || force_c == 16) {
        CjPlan p = cj_plan(r, l, force_c);
        if (!cj_plan_ok(p, r, l)) return 0;
        if (force_c == 16 && !cj_fits_dispatch<16>(p)) return 0;
        *out = p;
        return force_c;
    }
    CjPlan p8 = cj_plan(r, l, 8);
    if (cj_plan_ok(p8, r, l)) {
        *out = p8;
        return 8;
    }
    CjPlan p16 = cj_plan(r, l, 16);
    if (cj_plan_ok(p16, r, l) && cj_fits_dispatch<16>(p16)) {
        *out = p16;
        return 16;
    }
    return 0;
}

}  // namespace

size_t cjac32_smem_bytes(int r, int l)
{
    CjPlan p;
    return cj_choose(r, l, &p) ? p.smem : 0;
}

bool cjac32_fits(int r, int l)
{
    CjPlan p;
    return cj_choose(r, l, &p) != 0;
}

bool cjac32_fits_c(int r, int l, int C)
{
    CjPlan p;
    return cj_choose(r, l, &p, C) == C;
}

// X: r x l row-major FP32 (device), rotated in place; r_eff (device, may be
// null): only the first *r_eff rows take part, the rest are left untouched.
dmrg_status cjac32_run(dmrg_ctx *ctx, float *X, int r, int l, int max_sweeps, double tol, double small,
                       const double *F2, int *d_info, const int *r_eff, int force_c)
{
    CjPlan p;
    const int C = cj_choose(r, l, &p, force_c);
    if (!C) return DMRG_EUNSUPPORTED;
    const float tf = (float)tol;
#define CJ_LAUNCH(TMV, CV)                                                                                           \
    return launch_cjac32<TMV, CV>(ctx, X, r, l, p.ldl, p.b, p.threads, p.smem, max_sweeps, tf, F2, small, d_info, r_eff)
    if (C == 8) {
        switch (p.tm) {
        case 4: CJ_LAUNCH(4, 8);
        case 8: CJ_LAUNCH(8, 8);
        case 12: CJ_LAUNCH(12, 8);
        default: CJ_LAUNCH(16, 8);
        }
    }
    switch (p.tm) {
    case 4: CJ_LAUNCH(4, 16);
    case 8: CJ_LAUNCH(8, 16);
    case 12: CJ_LAUNCH(12, 16);
    default: CJ_LAUNCH(16, 16);
    }
#undef CJ_LAUNCH
}

}  // namespace dmrg
