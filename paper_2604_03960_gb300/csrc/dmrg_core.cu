// dmrg_core.cu -- contraction plans, the per-bond local update, the sweep
// driver and the C ABI (include/dmrg.h).
//
// Layouts in device memory (row-major, last index fastest):
//   site i      A[a][s][b]            chi_i x 2 x chi_{i+1}
//   env slot i  L_i[w][a'][a]          when the orthogonality centre is right of i
//               Rt_i[w][b][b']         when it is left of i (R stored transposed:
//                                      ket index first), so that every contraction
//                                      below is one strided GEMM without copies.
// One slot per position serves L_i or R_i (never both live), which halves the
// environment memory: at N = 400, chi = 2048, D = 8 the slots take ~100 GB.
//
// H_eff theta (Eq. 19) = three steps per Lanczos matvec:
//   X[(w,a')][(s1,s2,b)] = L[(w,a')][a] theta[a][(s1,s2,b)]                GEMM  M=D cl, N=4 cr, K=cl
//   Y[a'][q'][u][b]      = sum_{w,q} C[(u,q')][(w,q)] X[w][a'][q][b]        mix   C = W_k W_{k+1} over the shared MPO index
//   y[(a',q')][b']       = Y[(a',q')][(u,b)] Rt[(u,b)][b']                  GEMM  M=4 cl, N=cr, K=D cr
// Environment updates follow the same GEMM / mix / GEMM pattern.
#include "common.cuh"
#include "ctrl.cuh"
#include "lanczos.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>

namespace dmrg {
namespace {

constexpr int kMaxCh = 32;   // max channels of a mix (4 D for D <= 8)
// singular values below 2^-22 s_0 are not resolved by the FP32 Jacobi of the
// mixed form (rounding theta to FP32 moves every singular value by up to
// 2^-24 |theta|, Weyl) and count as zero there
constexpr double kMixedRankFloor = 2.384185791015625e-07;   // 2^-22

// ---------------------------------------------------------------------------
// MPO (Eq. 18 generalised; lower-triangular, left boundary row D-1, right
// boundary column 0).  One thread per site.
// ---------------------------------------------------------------------------
__device__ void put(double *Wi, int D, int wl, int wr, double o00, double o01, double o10, double o11, double c)
{
    double *p = Wi + ((size_t)wl * D + wr) * 4;
    p[0] += c * o00; p[1] += c * o01; p[2] += c * o10; p[3] += c * o11;
}

__global__ void k_build_mpo(int model, int N, double J, double Delta, double J2, double *W)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int D = (model == DMRG_XXZ) ? 5 : (model == DMRG_J1J2 ? 8 : 3);
    double *Wi = W + (size_t)i * D * D * 4;
    for (int x = 0; x < D * D * 4; ++x) Wi[x] = 0.0;
    // basis 0 = up, 1 = down; operators as (00, 01, 10, 11)
    const double Id[4] = {1, 0, 0, 1}, Sz[4] = {0.5, 0, 0, -0.5}, Sp[4] = {0, 1, 0, 0}, Sm[4] = {0, 0, 1, 0};
    const double Pz[4] = {1, 0, 0, -1}, Px[4] = {0, 1, 1, 0};
#define PUT(wl, wr, O, c) put(Wi, D, wl, wr, O[0], O[1], O[2], O[3], c)
    if (model == DMRG_XXZ) {
        PUT(0, 0, Id, 1.0); PUT(1, 0, Sp, 1.0); PUT(2, 0, Sm, 1.0); PUT(3, 0, Sz, 1.0);
        PUT(4, 1, Sm, 0.5 * J); PUT(4, 2, Sp, 0.5 * J); PUT(4, 3, Sz, J * Delta); PUT(4, 4, Id, 1.0);
    } else if (model == DMRG_J1J2) {
        PUT(0, 0, Id, 1.0); PUT(7, 7, Id, 1.0);
        PUT(7, 1, Sp, 1.0); PUT(7, 2, Sm, 1.0); PUT(7, 3, Sz, 1.0);
        PUT(1, 0, Sm, 0.5 * J); PUT(2, 0, Sp, 0.5 * J); PUT(3, 0, Sz, J * Delta);
        PUT(1, 4, Id, 1.0); PUT(2, 5, Id, 1.0); PUT(3, 6, Id, 1.0);
        PUT(4, 0, Sm, 0.5 * J2); PUT(5, 0, Sp, 0.5 * J2); PUT(6, 0, Sz, J2);
    } else {
        PUT(0, 0, Id, 1.0); PUT(2, 2, Id, 1.0); PUT(2, 1, Pz, -J); PUT(1, 0, Pz, 1.0); PUT(2, 0, Px, -Delta);
    }
#undef PUT
}

// ---------------------------------------------------------------------------
// Mixing coefficients.
//   kind 0 (H_eff):   C[(u*4+q')][(w*4+q)] = sum_v W1[w][v][s1'][s1] W2[v][u][s2'][s2], q = 2 s1 + s2
//   kind 1 (L env):   C[(v*2+s')][(w*2+s)] = W[w][v][s'][s]
//   kind 2 (R env):   C[(w*2+s')][(v*2+s)] = W[w][v][s'][s]
// ---------------------------------------------------------------------------
__global__ void k_build_coef(int kind, int D, const double *W1, const double *W2, double *C)
{
    const int nch = (kind == 0) ? 4 * D : 2 * D;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nch * nch) return;
    const int o = idx / nch, i = idx % nch;
    double v = 0.0;
    if (kind == 0) {
        int u = o / 4, qp = o % 4, w = i / 4, q = i % 4;
        int s1p = qp / 2, s2p = qp % 2, s1 = q / 2, s2 = q % 2;
        for (int m = 0; m < D; ++m)
            v += W1[(((size_t)w * D + m) * 2 + s1p) * 2 + s1] * W2[(((size_t)m * D + u) * 2 + s2p) * 2 + s2];
    } else if (kind == 1) {
        int vv = o / 2, sp = o % 2, w = i / 2, s = i % 2;
        v = W1[(((size_t)w * D + vv) * 2 + sp) * 2 + s];
    } else {
        int w = o / 2, sp = o % 2, vv = i / 2, s = i % 2;
        v = W1[(((size_t)w * D + vv) * 2 + sp) * 2 + s];
    }
    C[idx] = v;
}

struct MixDesc {
    int nin, nout, in_ny, out_ny;
    long long in_sx, in_sy, in_sa, out_sx, out_sy, out_sa;
    int An, Bn;
    int f32;        // 1: multiply-adds in FP32 (the mixed form's H_eff, whose GEMMs are FP32-accurate)
    float *yh = nullptr;   // also write the left-operand split of the output, viewed as rows of y_rs
    long long y_rs = 0;
    int ykp = 0;
};

// out[channel o][a][b] = sum_i C[o][i] in[channel i][a][b]; b is unit stride.
// A block takes 32 consecutive elements (one per lane) and stages their
// inputs in shared memory; warp w then forms the output channels w, w + 8,
// ...  The coefficient table (an MPO product, mostly zeros) is the same for
// every lane, so a zero coefficient is skipped by a warp-uniform branch and
// each output costs one multiply-add per nonzero coefficient, in channel
// order.  The mixed form (f32) mixes in FP32, with its inputs narrowed and
// its outputs widened by integer operations (bit-identical to the
// converting instructions, which would use the narrow FP64 pipe).
constexpr int kMixThreads = 256;
constexpr int kMixW = kMixThreads / 32;
template <typename T>
__global__ void __launch_bounds__(kMixThreads) k_mix(const double *__restrict__ in, double *__restrict__ out,
                                                     const double *__restrict__ C, MixDesc d)
{
    __shared__ T cs[kMaxCh * kMaxCh];
    __shared__ T xs[kMaxCh][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long total = (long long)d.An * d.Bn;
    const long long e = (long long)blockIdx.x * 32 + lane;
    const bool ok = e < total;
    const int a = ok ? (int)(e / d.Bn) : 0, b = ok ? (int)(e % d.Bn) : 0;
    for (int q = threadIdx.x; q < d.nout * d.nin; q += kMixThreads) {
        const double v = C[q];
        if constexpr (sizeof(T) == 4) cs[q] = f64_narrow(v); else cs[q] = v;
    }
    for (int c = warp; c < d.nin; c += kMixW) {
        const int x = c / d.in_ny, y = c % d.in_ny;
        const double v = ok ? in[x * d.in_sx + y * d.in_sy + a * d.in_sa + b] : 0.0;
        if constexpr (sizeof(T) == 4) xs[c][lane] = f64_narrow(v); else xs[c][lane] = v;
    }
    __syncthreads();
    if (!ok) return;
    for (int o = warp; o < d.nout; o += kMixW) {
        T acc = (T)0;
        const T *crow = cs + o * d.nin;
        for (int c = 0; c < d.nin; ++c) {
            const T cv = crow[c];
            if (cv != (T)0) {
                if constexpr (sizeof(T) == 4) acc = fmaf(cv, xs[c][lane], acc); else acc = fma(cv, xs[c][lane], acc);
            }
        }
        const int x = o / d.out_ny, y = o % d.out_ny;
        const long long f = x * d.out_sx + y * d.out_sy + a * d.out_sa + b;
        if constexpr (sizeof(T) == 4) {
            if (d.yh) {
                // only the next GEMM's left-operand parts (hi, hi, lo), the
                // bits its split of (double)acc would give: acc - hi is exact in FP32
                const float hi = tf32_rna(acc), lo = tf32_rna(acc - hi);
                const long long mrow = f / d.y_rs, kk = f - mrow * d.y_rs;
                float *q = d.yh + mrow * 3LL * d.ykp + kk;
                q[0] = hi;
                q[d.ykp] = hi;
                q[2LL * d.ykp] = lo;
            } else {
                out[f] = f32_widen(acc);
            }
        } else {
            out[f] = acc;
        }
    }
}

// batched transpose: out[b][j][i] = in[b][i][j] (n x n blocks)
__global__ void k_transpose_sq(const double *__restrict__ in, double *__restrict__ out, int n, int batch)
{
    __shared__ double t[32][33];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const double *src = in + (size_t)b * n * n;
    double *dst = out + (size_t)b * n * n;
    for (int y = threadIdx.y; y < 32; y += 8) {
        int i = i0 + y, j = j0 + threadIdx.x;
        t[y][threadIdx.x] = (i < n && j < n) ? src[(size_t)i * n + j] : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        int j = j0 + y, i = i0 + threadIdx.x;
        if (i < n && j < n) dst[(size_t)j * n + i] = t[threadIdx.x][y];
    }
}

// After truncation to k: A_k = U[:, :k] (x s/z if the centre stays left),
// A_{k+1} = (s/z x) Vt[:k, :] (if the centre moves right).
__global__ void k_split(const double *__restrict__ U, const double *__restrict__ s, const double *__restrict__ Vt,
                        int m, int n, int r, const BondResult *res, int go_right, double *__restrict__ Ak,
                        double *__restrict__ Ak1)
{
    const int k = res->k;
    const double z = res->znorm;
    const long long nA = (long long)m * k, nB = (long long)k * n;
    const long long total = nA > nB ? nA : nB;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        if (e < nA) {
            int i = (int)(e / k), j = (int)(e % k);
            double v = U[(long long)i * r + j];
            Ak[e] = go_right ? v : v * (s[j] / z);
        }
        if (e < nB) {
            int j = (int)(e / n), c = (int)(e % n);
            double v = Vt[(long long)j * n + c];
            Ak1[e] = go_right ? v * (s[j] / z) : v;
        }
    }
}

// dst[i][j] = src[i][j] * (scale_cols ? s[j] : 1) for an m x k block
__global__ void k_copy_scale(const double *__restrict__ src, double *__restrict__ dst, long long m, int k,
                             const double *__restrict__ s)
{
    const long long total = m * k;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        int j = (int)(e % k);
        dst[e] = s ? src[e] * s[j] : src[e];
    }
}

// normalise a small vector in place (single block)
__global__ void k_normalise(double *x, int n)
{
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += x[i] * x[i];
    a = block_sum(a, sh);
    double inv = (a > 0.0) ? 1.0 / sqrt(a) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
}

__global__ void k_init_ctrl(dmrg_ctrl_state *st, int n, int chi0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dmrg_ctrl_state z;
    z.Sbar = z.Sbar_prev = z.Sbar_prev2 = z.e_prev = z.I = 0.0;
    for (int j = 0; j < 8; ++j) z.hist[j] = 0.0;
    z.chi = chi0;
    z.initialized = 0;
    z.nhist = 0;
    z.pad = 0;
    st[i] = z;
}

__global__ void k_boundary_env(double *E, int D, int w)
{
    int i = threadIdx.x;
    if (i < D) E[i] = (i == w) ? 1.0 : 0.0;
}

// out (C x R) = in (R x C)^T
__global__ void k_transpose_rect(const double *__restrict__ in, double *__restrict__ out, int R, int C)
{
    __shared__ double t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        int r = r0 + y, c = c0 + threadIdx.x;
        t[y][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = t[threadIdx.x][y];
    }
}

// E = x.y / x.x into a Lanczos state (FP64 Rayleigh quotient), single block
__global__ void k_rayleigh(const double *__restrict__ x, const double *__restrict__ y, long long n, LzState *lz)
{
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        a = fma(x[i], y[i], a);
        b = fma(x[i], x[i], b);
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0 && b > 0.0) lz->E = a / b;
}

// two-pass deterministic normalisation of a vector to unit 2-norm
constexpr int kNormBlocks = 256;
__global__ void k_sumsq_partial(const double *__restrict__ x, long long n, double *__restrict__ part)
{
    __shared__ double sh[32];
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a = fma(x[i], x[i], a);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_scale_partials(double *__restrict__ x, long long n, const double *__restrict__ part, int nparts)
{
    // every block sums the partials in the same fixed order (all threads load
    // at once, then the block reduction), so all blocks get the same scale
    __shared__ double sh[32];
    __shared__ double inv;
    double a = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) a += part[b];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) inv = (a > 0.0) ? 1.0 / sqrt(a) : 0.0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= inv;
}

__global__ void k_fill_int(int *p, int v) { *p = v; }

// Norms of the rows of P (r x n) or of its columns (m x r), in FP64.
__global__ void k_row_norms(const double *__restrict__ P, int r, int n, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= r) return;
    double a = 0.0;
    for (int j = lane; j < n; j += 32) a = fma(P[(long long)row * n + j], P[(long long)row * n + j], a);
    a = warp_sum(a);
    if (lane == 0) out[row] = sqrt(a);
}
__global__ void k_col_norms(const double *__restrict__ P, int m, int r, double *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= r) return;
    double a = 0.0;
    for (int i = 0; i < m; ++i) a = fma(P[(long long)i * r + c], P[(long long)i * r + c], a);
    out[c] = sqrt(a);
}
// perm[rank] = i with ranks by descending value, ties by index; s[c] = v[perm[c]]
__global__ void k_rank_sorted(const double *__restrict__ v, int r, int *__restrict__ perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    const double x = v[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) rank += (v[j] > x) || (v[j] == x && j < i);
    perm[rank] = i;
}
__global__ void k_take_sorted(const double *__restrict__ v, const int *__restrict__ perm, int r, double *__restrict__ s)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < r) s[c] = v[perm[c]];
}
// out[c][j] = in[perm[c]][j] * (scale ? 1 / s[c] : 1)   (r x n rows)
__global__ void k_gather_rows(const double *__restrict__ in, const int *__restrict__ perm, const double *__restrict__ s,
                              int r, int n, double *__restrict__ out)
{
    const long long total = (long long)r * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n), j = (int)(e % n);
        const double f = s ? (s[c] > 0.0 ? 1.0 / s[c] : 0.0) : 1.0;
        out[e] = in[(long long)perm[c] * n + j] * f;
    }
}
// out[i][c] = in[perm[c]][i]  (in r x m, out m x r)
__global__ void k_gather_rows_t(const double *__restrict__ in, const int *__restrict__ perm, int r, int m,
                                double *__restrict__ out)
{
    const long long total = (long long)m * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), c = (int)(e % r);
        out[e] = in[(long long)perm[c] * m + i];
    }
}
// out[i][c] = in[i][perm[c]] / s[c]  (m x r)
__global__ void k_gather_cols_scaled(const double *__restrict__ in, const int *__restrict__ perm,
                                     const double *__restrict__ s, int m, int r, double *__restrict__ out)
{
    const long long total = (long long)m * r;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / r), c = (int)(e % r);
        out[e] = s[c] > 0.0 ? in[(long long)i * r + perm[c]] / s[c] : 0.0;
    }
}

int grid1d(long long n, int threads, int num_sms)
{
    long long b = (n + threads - 1) / threads;
    long long cap = (long long)num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

// ---------------------------------------------------------------------------
// Contraction plans
// ---------------------------------------------------------------------------
// Split of a truncated SVD into two site tensors (used by the circuit path too)
dmrg_status launch_split(dmrg_ctx *ctx, const double *U, const double *s, const double *Vt, int m, int n, int r,
                         const BondResult *res, int go_right, double *Ak, double *Ak1, int kmax)
{
    const long long tot = std::max((long long)m * kmax, (long long)kmax * n);
    k_split<<<grid1d(tot, 256, ctx->num_sms), 256, 0, ctx->stream>>>(U, s, Vt, m, n, r, res, go_right, Ak, Ak1);
    DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status launch_init_ctrl(dmrg_ctx *ctx, dmrg_ctrl_state *st, int n, int chi0)
{
    k_init_ctrl<<<(n + 127) / 128, 128, 0, ctx->stream>>>(st, n, chi0); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

static dmrg_status mix(dmrg_ctx *ctx, const double *in, double *out, const double *C, const MixDesc &d)
{
    long long total = (long long)d.An * d.Bn;
    prof_mark(ctx, PROF_MIX);
    if (total <= 0) return DMRG_OK;
    const long long blocks = (total + 31) / 32;
    if (blocks > 0x7fffffffLL) return DMRG_EINVAL;
    if (d.f32)
        k_mix<float><<<(unsigned)blocks, kMixThreads, 0, ctx->stream>>>(in, out, C, d);
    else
        k_mix<double><<<(unsigned)blocks, kMixThreads, 0, ctx->stream>>>(in, out, C, d);
    DMRG_COUNT_LAUNCH();
    prof_mark(ctx, PROF_MIX);
    prof_count(ctx, PROF_MIX, 0.0, 8.0 * (double)total * (d.nin + d.nout));   // each input and output channel once
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

// y = H_eff x. L: [w][a'][a] (D cl cl); Rt: [u][b][b'] (D cr cr); C: (4D)^2;
// X, Y: D*cl*4*cr doubles each.
// Pre-split tensor-core operands of the matvec's two GEMMs (any may be null).
struct HeffPre {
    const float *Lh = nullptr, *Rh = nullptr, *xh = nullptr;
    float *Yh = nullptr;
};

dmrg_status heff_apply_dev(dmrg_ctx *ctx, int prec, int D, int cl, int cr, const double *L, const double *Rt,
                           const double *C, double *X, double *Y, const double *x, double *y,
                           const HeffPre *pre = nullptr)
{
    const long long n4 = 4LL * cr;
    const bool p1 = pre && prec == DMRG_PREC_3XTF32 && pre->Lh && pre->xh;
    const bool p2 = pre && prec == DMRG_PREC_3XTF32 && pre->Yh && pre->Rh;
    if (p1)
        DMRG_TRY(gemm_3xtf32_pre(ctx, D * cl, (int)n4, cl, 1.0, L, cl, 1, 0, x, n4, 1, 0, 0.0, X, n4, 1, 0, 1, pre->Lh,
                                 pre->xh));
    else
        DMRG_TRY(gemm(ctx, prec, D * cl, (int)n4, cl, 1.0, L, cl, 1, 0, x, n4, 1, 0, 0.0, X, n4, 1, 0, 1));
    MixDesc md;
    md.f32 = prec != DMRG_PREC_FP64;
    md.nin = 4 * D; md.nout = 4 * D; md.in_ny = 4; md.out_ny = 4;
    md.in_sx = (long long)cl * n4; md.in_sy = cr; md.in_sa = n4;
    md.out_sx = cr; md.out_sy = (long long)D * cr; md.out_sa = 4LL * D * cr;
    md.An = cl; md.Bn = cr;
    if (p2) {
        md.yh = pre->Yh;
        md.y_rs = (long long)D * cr;
        md.ykp = split_kp(D * cr);
    }
    DMRG_TRY(mix(ctx, X, Y, C, md));
    if (p2)
        DMRG_TRY(gemm_3xtf32_pre(ctx, 4 * cl, cr, D * cr, 1.0, Y, (long long)D * cr, 1, 0, Rt, cr, 1, 0, 0.0, y, cr,
                                 1, 0, 1, pre->Yh, pre->Rh));
    else
        DMRG_TRY(gemm(ctx, prec, 4 * cl, cr, D * cr, 1.0, Y, (long long)D * cr, 1, 0, Rt, cr, 1, 0, 0.0, y, cr, 1, 0,
                      1));
    return DMRG_OK;
}

// Lnew[v][b'][b] from L (D cl cl), coefficient C (kind 1), A (cl x 2 x ck)
dmrg_status env_left_dev(dmrg_ctx *ctx, int prec, int D, int cl, int ck, const double *L, const double *C,
                         const double *A, double *Lnew, double *T1, double *T2)
{
    const long long n2 = 2LL * ck;
    DMRG_TRY(gemm(ctx, prec, D * cl, (int)n2, cl, 1.0, L, cl, 1, 0, A, n2, 1, 0, 0.0, T1, n2, 1, 0, 1));
    MixDesc md;
    md.f32 = prec != DMRG_PREC_FP64;
    md.nin = 2 * D; md.nout = 2 * D; md.in_ny = 2; md.out_ny = 2;
    md.in_sx = (long long)cl * n2; md.in_sy = ck; md.in_sa = n2;
    md.out_sx = (long long)cl * n2; md.out_sy = ck; md.out_sa = n2;
    md.An = cl; md.Bn = ck;
    DMRG_TRY(mix(ctx, T1, T2, C, md));
    DMRG_TRY(gemm(ctx, prec, ck, ck, 2 * cl, 1.0, A, 1, ck, 0, T2, ck, 1, (long long)2 * cl * ck, 0.0, Lnew, ck, 1,
                  (long long)ck * ck, D));
    return DMRG_OK;
}

// Rtnew[w][a][a'] from Rt (D cr cr, [v][b][b']), coefficient C (kind 2), B (ck x 2 x cr)
dmrg_status env_right_dev(dmrg_ctx *ctx, int prec, int D, int ck, int cr, const double *Rt, const double *C,
                          const double *B, double *Rtnew, double *T1, double *T2)
{
    DMRG_TRY(gemm(ctx, prec, 2 * ck, cr, cr, 1.0, B, cr, 1, 0, Rt, cr, 1, (long long)cr * cr, 0.0, T1, cr, 1,
                  (long long)2 * ck * cr, D));
    MixDesc md;
    md.f32 = prec != DMRG_PREC_FP64;
    md.nin = 2 * D; md.nout = 2 * D; md.in_ny = 2; md.out_ny = 2;
    md.in_sx = (long long)2 * ck * cr; md.in_sy = cr; md.in_sa = 2LL * cr;
    md.out_sx = (long long)2 * ck * cr; md.out_sy = cr; md.out_sa = 2LL * cr;
    md.An = ck; md.Bn = cr;
    DMRG_TRY(mix(ctx, T1, T2, C, md));
    DMRG_TRY(gemm(ctx, prec, ck, ck, 2 * cr, 1.0, T2, 2LL * cr, 1, (long long)ck * 2 * cr, B, 1, 2LL * cr, 0, 0.0,
                  Rtnew, ck, 1, (long long)ck * ck, D));
    return DMRG_OK;
}

static dmrg_status normalise(dmrg_ctx *ctx, double *x, long long n, double *part)
{
    k_sumsq_partial<<<kNormBlocks, 256, 0, ctx->stream>>>(x, n, part); DMRG_COUNT_LAUNCH();
    k_scale_partials<<<grid1d(n, 256, ctx->num_sms), 256, 0, ctx->stream>>>(x, n, part, kNormBlocks); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

static dmrg_status build_coef(dmrg_ctx *ctx, int kind, int D, const double *W1, const double *W2, double *C)
{
    int nch = (kind == 0) ? 4 * D : 2 * D;
    k_build_coef<<<(nch * nch + 255) / 256, 256, 0, ctx->stream>>>(kind, D, W1, W2, C); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

static dmrg_status transpose_sq(dmrg_ctx *ctx, const double *in, double *out, int n, int batch)
{
    dim3 g((n + 31) / 32, (n + 31) / 32, batch);
    k_transpose_sq<<<g, dim3(32, 8), 0, ctx->stream>>>(in, out, n, batch); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

double matvec_flops(int D, int cl, int cr)
{
    return 2.0 * D * cl * 4.0 * cr * cl + 2.0 * (4.0 * D) * (4.0 * D) * cl * cr + 2.0 * 4.0 * cl * cr * D * cr;
}

double svd_nominal_flops(int m, int n)
{
    double M = std::max(m, n), Nn = std::min(m, n);
    return 4.0 * M * M * Nn + 8.0 * M * Nn * Nn + 9.0 * Nn * Nn * Nn;
}

double env_flops(int D, int cl, int ck)
{
    return 2.0 * D * cl * 2.0 * ck * cl + 2.0 * (2.0 * D) * (2.0 * D) * cl * ck + 2.0 * D * ck * ck * 2.0 * cl;
}

}  // namespace dmrg

using namespace dmrg;

// ===========================================================================
// State
// ===========================================================================
struct dmrg_state {
    dmrg_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;   // copy of ctx->stream (destroy does not touch ctx)
    int N = 0, D = 0;
    dmrg_params p{};
    dmrg_model_params mp{};
    std::vector<int> chi, cap;
    DevBuf arena;
    double *W = nullptr, *coef_mv = nullptr, *coef_l = nullptr, *coef_r = nullptr;
    std::vector<double *> A, env;
    dmrg_ctrl_state *ctrl = nullptr;
    double *theta = nullptr, *X = nullptr, *Y = nullptr;
    // tensor-core split operands of the matvec, made once per local update
    // (L, R) or by their producers (the Lanczos vector, the mix output)
    float *Lh = nullptr, *Rh = nullptr, *xh = nullptr, *Yh = nullptr;
    double *U = nullptr, *s = nullptr, *Vt = nullptr;
    void *svdw = nullptr;
    LanczosWork lw;
    BondResult *d_res = nullptr;
    BondResult *h_res = nullptr;   // pinned
    int *d_info = nullptr;
    dmrg_visit_record *d_visits = nullptr;
    float *mlp = nullptr;
    int has_mlp = 0;
    int sweep_index = 0;
    long long nmax = 0;
    int K = 20;
    cudaEvent_t ev_res = nullptr;    // recorded after the bond result is copied to h_res
    dmrg_ctrl_state *gctrl = nullptr;  // global adaptive chi: the one controller (device)
    int global_chi = 0;                // ... and its current chi (host copy, set at sweep ends)
    std::vector<int> sched;            // DMRG_CTRL_REPLAY: chi of each visit of the next sweeps
    int cur_visit = -1;                // visit index within the running sweep (-1 outside dmrg_sweep)
    // a bond step between its two phases (bond_step_a / bond_step_b)
    struct Pending {
        int k = 0, go_right = 0, direction = 1, m = 0, n = 0, r = 0, cl = 0, cm = 0, cr = 0, K = 0;
        float *X32 = nullptr;
        double *nrm = nullptr;
        int *perm = nullptr;
    } pend;
};

extern "C" {

const char *dmrg_status_string(dmrg_status s)
{
    switch (s) {
    case DMRG_OK: return "ok";
    case DMRG_EINVAL: return "invalid argument";
    case DMRG_ENOMEM: return "out of device memory";
    case DMRG_ENOCONV: return "Jacobi SVD did not converge";
    case DMRG_ENAN: return "non-finite value";
    case DMRG_ETIMEOUT: return "device-side wait timed out";
    case DMRG_ECUDA: return "CUDA runtime error";
    case DMRG_EUNSUPPORTED: return "unsupported option";
    }
    return "unknown";
}

dmrg_status dmrg_set_option(dmrg_ctx *ctx, const char *name, double value)
{
    if (!ctx || !name) return DMRG_EINVAL;
    if (!std::strcmp(name, "tc_force")) { ctx->tc_force = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "tc_min_work")) {
        if (!(value >= 0.0)) return DMRG_EINVAL;
        ctx->tc_min_work = value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "tc_bn")) {
        int v = (int)value;
        if (v != 0 && v != 64 && v != 128 && v != 256) return DMRG_EINVAL;
        ctx->tc_bn_override = v;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "cjac_force_c")) {
        if (value != 0.0 && value != 8.0 && value != 16.0) return DMRG_EINVAL;
        ctx->cjac_force_c = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "mixed_env_tc")) { ctx->mixed_env_tc = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "mlp_eps_target")) {
        if (!(value > 0.0 && value < 1.0)) return DMRG_EINVAL;
        ctx->mlp_eps_target = value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "bjac_pairs")) {
        if (!(value >= 1.0 && value <= 100000.0)) return DMRG_EINVAL;
        ctx->bjac_pairs = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "batched_inner")) {
        if (!(value >= 1.0 && value <= 16.0)) return DMRG_EINVAL;
        ctx->batched_inner = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "batched_ns")) { ctx->batched_ns = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "jacobi_qr")) { ctx->jacobi_qr = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "jacobi_rank_drop")) { ctx->jacobi_rank_drop = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "bjac_gram")) { ctx->bjac_gram = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "gbj_min_r")) {
        if (!(value >= 0.0 && value <= 1e6)) return DMRG_EINVAL;
        ctx->gbj_min_r = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "jacobi32_floor")) {
        if (!(value >= 0.0 && value < 1e-2)) return DMRG_EINVAL;
        ctx->jacobi32_floor = value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "batched_floor32")) {
        if (!(value >= 0.0 && value < 1e-2)) return DMRG_EINVAL;
        ctx->batched_floor32 = value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "bjac_inner")) {
        if (!(value >= 1.0 && value <= 8.0)) return DMRG_EINVAL;
        ctx->bjac_inner = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "svd_prec")) {
        if (value != 0.0 && value != 1.0) return DMRG_EINVAL;
        ctx->svd_prec = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "mixed_svd64")) { ctx->mixed_svd64 = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "jacobi32_tol")) {
        if (!(value >= 1e-8 && value <= 1e-2)) return DMRG_EINVAL;
        ctx->jacobi32_tol = value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "qr_wpanel")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->qr_wpanel = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "f64_fill")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->f64_fill = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "f32_fill")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->f32_fill = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "tc_presplit")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->tc_presplit = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "lz_cluster_n")) {
        if (!(value >= 0.0 && value <= 1e9)) return DMRG_EINVAL;
        ctx->lz_cluster_n = (long long)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "lz_fused")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->lz_fused = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "cjac32")) {
        if (!(value == 0.0 || value == 1.0)) return DMRG_EINVAL;
        ctx->cjac32 = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "cjac_min_r")) {
        if (!(value >= 2.0 && value <= 1e6)) return DMRG_EINVAL;
        ctx->cjac_min_r = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "tjac")) {
        if (value != 0.0 && value != 64.0 && value != 128.0) return DMRG_EINVAL;
        ctx->tjac = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "tjac_min_r")) {
        if (!(value >= 2.0 && value <= 1e6)) return DMRG_EINVAL;
        ctx->tjac_min_r = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "gjac32")) {
        if (value != 0.0 && value != 1.0 && value != 2.0) return DMRG_EINVAL;
        ctx->gjac32 = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "tc_split_kb")) {
        if (!(value >= 0.0 && value <= 1e6) || value != (double)(int)value) return DMRG_EINVAL;
        ctx->tc_split_kb = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "gjac_nv")) {
        if (value != 0.0 && value != 16.0 && value != 32.0) return DMRG_EINVAL;
        ctx->gjac_nv = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "gjac_groups")) {
        if (!(value >= 0.0 && value <= 4.0)) return DMRG_EINVAL;
        ctx->gjac_groups = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "jacobi64_gram")) { ctx->jacobi64_gram = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "jacobi64_precond")) { ctx->jacobi64_precond = value != 0.0; return DMRG_OK; }
    if (!std::strcmp(name, "prof_mask")) {
        if (!(value >= 1.0 && value <= (double)((1 << PROF_KINDS) - 1)) || value != (double)(int)value)
            return DMRG_EINVAL;
        ctx->prof_mask = (int)value;
        return DMRG_OK;
    }
    if (!std::strcmp(name, "jacobi_max_sweeps")) {
        if (!(value >= 1.0 && value <= 1000.0)) return DMRG_EINVAL;
        ctx->jacobi_max_sweeps = (int)value;
        return DMRG_OK;
    }
    return DMRG_EINVAL;
}

int dmrg_mpo_dim(int model)
{
    switch (model) {
    case DMRG_XXZ: return 5;
    case DMRG_J1J2: return 8;
    case DMRG_TFIM: return 3;
    }
    return -1;
}

dmrg_status dmrg_create(dmrg_ctx **out, int device, void *cuda_stream)
{
    if (!out) return DMRG_EINVAL;
    *out = nullptr;
    DMRG_CUDA(cudaSetDevice(device));
    dmrg_ctx *c = new (std::nothrow) dmrg_ctx();
    if (!c) return DMRG_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return DMRG_ECUDA; }
    c->num_sms = prop.multiProcessorCount;
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) { delete c; return DMRG_ENOMEM; }
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) { cudaFree(c->d_status); delete c; return DMRG_ECUDA; }
    if (cudaMallocHost(&c->h_pinned_i, 64 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned_d, 64 * sizeof(double)) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return DMRG_ENOMEM;
    }
    std::memset(c->h_pinned_i, 0, 64 * sizeof(int));
    std::memset(c->h_pinned_d, 0, 64 * sizeof(double));
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    *out = c;
    return DMRG_OK;
}

void dmrg_destroy(dmrg_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    ctx->work.release();
    ctx->work2.release();
    ctx->work3.release();
    ctx->tcbuf.release();
    ctx->f64buf.release();
    ctx->work4.release();
    ctx->tjbuf.release();
    if (ctx->pinned_desc) cudaFreeHost(ctx->pinned_desc);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_pinned_i) cudaFreeHost(ctx->h_pinned_i);
    if (ctx->h_pinned_d) cudaFreeHost(ctx->h_pinned_d);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (auto &p : ctx->prof_slot)
        for (auto e : p.ev) cudaEventDestroy(e);
    delete ctx;
}

static dmrg_status status_from_bits(int bits)
{
    if (bits & ST_TIMEOUT) return DMRG_ETIMEOUT;
    if (bits & ST_NAN) return DMRG_ENAN;
    if (bits & ST_NOCONV) return DMRG_ENOCONV;
    if (bits) return DMRG_EINVAL;
    return DMRG_OK;
}

dmrg_status dmrg_get_status(dmrg_ctx *ctx)
{
    if (!ctx) return DMRG_EINVAL;
    DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_i, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return status_from_bits(ctx->h_pinned_i[0]);
}

dmrg_status dmrg_build_mpo(dmrg_ctx *ctx, dmrg_model model, const dmrg_model_params *mp, double *W_dev)
{
    if (!ctx || !mp || !W_dev || mp->N < 2 || dmrg_mpo_dim(model) < 0) return DMRG_EINVAL;
    k_build_mpo<<<(mp->N + 63) / 64, 64, 0, ctx->stream>>>((int)model, mp->N, mp->J, mp->Delta, mp->J2, W_dev); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

// ---------------------------------------------------------------------------
// one local update (Section 10): theta, Lanczos, SVD, entropy + controller +
// truncation, split, environment update
// ---------------------------------------------------------------------------
// A bond step runs in two phases.  Phase A enqueues the two-site tensor, the
// Lanczos solve, the SVD and the entropy/controller/truncation decision, and
// starts the copy of the decision to pinned host memory (event ev_res).
// Phase B waits for that copy (the one host synchronisation of a bond step:
// the retained k sizes every later launch) and enqueues the split and the
// environment update.  Several chains interleave their phases (A for all,
// then B for all) so that their kernels overlap on the device.
static dmrg_status bond_step_a(dmrg_state *st, int k, int go_right, int do_ctrl, dmrg_visit_record *visit,
                               int direction)
{
    dmrg_ctx *ctx = st->ctx;
    const int D = st->D, prec = st->p.prec;
    const int cl = st->chi[k], cm = st->chi[k + 1], cr = st->chi[k + 2];
    const int m = 2 * cl, n = 2 * cr, r = std::min(m, n);
    const long long nn = (long long)m * n;
    auto &P = st->pend;
    P.k = k; P.go_right = go_right; P.direction = direction;
    P.m = m; P.n = n; P.r = r; P.cl = cl; P.cm = cm; P.cr = cr;
    // two-site tensor (Eq. 20's left-hand side)
    DMRG_TRY(gemm(ctx, prec, m, n, cm, 1.0, st->A[k], cm, 1, 0, st->A[k + 1], n, 1, 0, 0.0, st->theta, n, 1, 0, 1));
    // Lanczos on H_eff (Eq. 19)
    const double *L = st->env[k], *Rt = st->env[k + 2];
    const double *C = st->coef_mv + (size_t)k * (4 * D) * (4 * D);
    // tensor-core matvecs: L and R split once for the whole Lanczos run, the
    // Lanczos vector and the mix output split by the kernels that make them
    HeffPre pre;
    SplitSink sink;
    if (prec == DMRG_PREC_3XTF32 && ctx->tc_presplit) {
        if (tc_path(ctx, D * cl, 4 * cr, cl, 1)) {
            DMRG_TRY(split3_dev(ctx, L, cl, 1, 0, D * cl, cl, 1, 0, st->Lh));
            pre.Lh = st->Lh;
            pre.xh = st->xh;
            sink.h = st->xh;
            sink.n4 = 4LL * cr;
            sink.Kp = split_kp(cl);
            // the producers write columns k < K only: the padding must read as zero
            DMRG_CUDA(cudaMemsetAsync(st->xh, 0, sizeof(float) * (size_t)4 * cr * 3 * split_kp(cl), ctx->stream));
        }
        if (tc_path(ctx, 4 * cl, cr, D * cr, 1)) {
            DMRG_TRY(split3_dev(ctx, Rt, 1, cr, 0, cr, D * cr, 1, 1, st->Rh));
            pre.Rh = st->Rh;
            pre.Yh = st->Yh;
            DMRG_CUDA(cudaMemsetAsync(st->Yh, 0, sizeof(float) * (size_t)4 * cl * 3 * split_kp(D * cr), ctx->stream));
        }
    }
    MatvecFn mv = [&](const double *x, double *y) {
        return heff_apply_dev(ctx, prec, D, cl, cr, L, Rt, C, st->X, st->Y, x, y, &pre);
    };
    const int K = (int)std::min<long long>(st->K, nn);
    P.K = K;
    DMRG_TRY(lanczos_run(ctx, st->lw, nn, K, st->theta, mv, sink.h ? &sink : nullptr));
    if (prec != DMRG_PREC_FP64 && k == 0 && direction == -1) {
        // last visit of a sweep: the sweep energy is the FP64 Rayleigh
        // quotient of the Ritz vector (second order in its error), so the
        // FP32 accumulation of the tensor-core matvecs does not reach it
        DMRG_TRY(heff_apply_dev(ctx, DMRG_PREC_FP64, D, cl, cr, L, Rt, C, st->X, st->Y, st->theta, st->lw.w));
        k_rayleigh<<<1, 256, 0, ctx->stream>>>(st->theta, st->lw.w, nn, st->lw.lz); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
    }
    const float *mlp = st->has_mlp ? st->mlp : nullptr;
    int chi_global = st->p.ctrl == DMRG_CTRL_GLOBAL ? st->global_chi : 0;
    if (st->p.ctrl == DMRG_CTRL_REPLAY) {
        // the recorded schedule decides (the controllers do not step)
        const int V = 2 * st->N - 3;
        const int v = st->cur_visit;
        if (v < 0 || (int)st->sched.size() < V) return DMRG_EINVAL;
        chi_global = st->sched[v];
    }
    if (prec == DMRG_PREC_FP64 || ctx->mixed_svd64) {
        // SVD (Eq. 20) in FP64, then entropy, controller and truncation
        DMRG_TRY(svd_jacobi(ctx, st->theta, m, n, st->U, st->s, st->Vt, st->svdw, st->p.jacobi_max_sweeps,
                            st->d_info));
        DMRG_TRY(launch_decide(ctx, st->s, r, st->ctrl + k, st->p, do_ctrl, chi_global, mlp, k, st->N,
                               st->sweep_index, st->lw.lz, st->d_res, visit, direction,
                               (double)r * 2.220446049250313e-16, st->d_info));
    } else {
        // Mixed form: FP32 Jacobi on the vectors that become the isometry
        // (columns of theta if the centre moves right, rows if it moves left)
        const int dir = go_right ? 0 : 1;
        DMRG_TRY(svd_jacobi32(ctx, st->theta, m, n, dir, st->svdw, st->p.jacobi_max_sweeps, st->d_info, st->s,
                              &P.X32, &P.nrm, &P.perm));
        DMRG_TRY(launch_decide(ctx, st->s, r, st->ctrl + k, st->p, do_ctrl, chi_global, mlp, k, st->N,
                               st->sweep_index, st->lw.lz, st->d_res, visit, direction, kMixedRankFloor, st->d_info));
    }
    DMRG_CUDA(cudaMemcpyAsync(st->h_res, st->d_res, sizeof(BondResult), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaEventRecord(st->ev_res, ctx->stream));
    return DMRG_OK;
}

static dmrg_status bond_step_b(dmrg_state *st, double *flops, int *k_out, double *E_out)
{
    dmrg_ctx *ctx = st->ctx;
    const int D = st->D, prec = st->p.prec;
    const auto &P = st->pend;
    const int k = P.k, go_right = P.go_right, m = P.m, n = P.n, r = P.r, cl = P.cl, cm = P.cm, cr = P.cr;
    DMRG_CUDA(cudaEventSynchronize(st->ev_res));
    const int kk = st->h_res->k;
    if (kk < 1 || kk > r || kk > st->cap[k + 1]) {
        std::fprintf(stderr, "dmrg: bond %d: retained k = %d outside [1, min(r = %d, cap = %d)] (S = %g)\n", k, kk, r,
                     st->cap[k + 1], st->h_res->S);
        return DMRG_ENAN;
    }
    if (prec == DMRG_PREC_FP64 || ctx->mixed_svd64) {
        long long tot = std::max((long long)m * kk, (long long)kk * n);
        k_split<<<grid1d(tot, 256, ctx->num_sms), 256, 0, ctx->stream>>>(st->U, st->s, st->Vt, m, n, r, st->d_res,
                                                                         go_right, st->A[k], st->A[k + 1]); DMRG_COUNT_LAUNCH();
        DMRG_CUDA(cudaGetLastError());
    } else {
        // one FP64 Newton-Schulz step Q <- Q - (Q Q^T - I) Q / 2 on the k
        // retained unit vectors, and the centre tensor as the projection of
        // theta on them (3xTF32), renormalised
        const int dir = go_right ? 0 : 1;
        const int len = dir == 0 ? m : n;
        double *Q = st->X, *T = st->Y, *E = st->Vt;
        DMRG_TRY(gather_unit_vectors(ctx, P.X32, P.nrm, P.perm, &st->d_res->k, kk, len, Q));
        DMRG_TRY(gemm_f64x(ctx, kk, kk, len, 1.0, Q, len, 1, 0, Q, 1, len, 0, 0.0, E, kk, 1, 0, 1));
        DMRG_CUDA(cudaMemcpyAsync(T, Q, sizeof(double) * (size_t)kk * len, cudaMemcpyDeviceToDevice, ctx->stream));
        DMRG_TRY(gemm_f64x(ctx, kk, len, kk, -0.5, E, kk, 1, 0, Q, len, 1, 0, 1.5, T, len, 1, 0, 1));
        if (dir == 0) {
            // A_k = T^T (m x kk): k_transpose_rect(in = T (kk x m), out = A_k (m x kk))
            k_transpose_rect<<<dim3((m + 31) / 32, (kk + 31) / 32), dim3(32, 8), 0, ctx->stream>>>(T, st->A[k], kk, m); DMRG_COUNT_LAUNCH();
            DMRG_CUDA(cudaGetLastError());
            DMRG_TRY(gemm(ctx, prec, kk, n, m, 1.0, T, m, 1, 0, st->theta, n, 1, 0, 0.0, st->A[k + 1], n, 1, 0, 1));
            DMRG_TRY(normalise(ctx, st->A[k + 1], (long long)kk * n, st->s + r));
        } else {
            DMRG_CUDA(cudaMemcpyAsync(st->A[k + 1], T, sizeof(double) * (size_t)kk * n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
            DMRG_TRY(gemm(ctx, prec, m, kk, n, 1.0, st->theta, n, 1, 0, T, 1, n, 0, 0.0, st->A[k], kk, 1, 0, 1));
            DMRG_TRY(normalise(ctx, st->A[k], (long long)m * kk, st->s + r));
        }
    }
    st->chi[k + 1] = kk;
    double f = 2.0 * m * n * cm + P.K * matvec_flops(D, cl, cr) + svd_nominal_flops(m, n);
    // Environments carry the energy of whole blocks and each is built from the
    // previous one, so FP32-accumulated errors would add up along the chain:
    // the mixed form keeps them in FP64 unless the context asks otherwise.
    const int eprec = (prec == DMRG_PREC_3XTF32 && !ctx->mixed_env_tc) ? DMRG_PREC_FP64 : prec;
    if (go_right) {
        DMRG_TRY(env_left_dev(ctx, eprec, D, cl, kk, st->env[k], st->coef_l + (size_t)k * 4 * D * D, st->A[k],
                              st->env[k + 1], st->X, st->Y));
        f += env_flops(D, cl, kk);
    } else if (k + 1 >= 2) {
        DMRG_TRY(env_right_dev(ctx, eprec, D, kk, cr, st->env[k + 2], st->coef_r + (size_t)(k + 1) * 4 * D * D,
                               st->A[k + 1], st->env[k + 1], st->X, st->Y));
        f += env_flops(D, cr, kk);
    }
    if (flops) *flops += f;
    if (k_out) *k_out = kk;
    if (E_out) *E_out = st->h_res->E;
    return DMRG_OK;
}

static dmrg_status bond_step(dmrg_state *st, int k, int go_right, int do_ctrl, dmrg_visit_record *visit,
                             int direction, double *flops, int *k_out, double *E_out)
{
    DMRG_TRY(bond_step_a(st, k, go_right, do_ctrl, visit, direction));
    return bond_step_b(st, flops, k_out, E_out);
}

dmrg_status dmrg_state_create(dmrg_ctx *ctx, int D, const dmrg_model_params *mp, const double *W_dev,
                              const dmrg_params *p, const double *mps_init_dev, dmrg_state **out)
{
    if (!ctx || !mp || !W_dev || !p || !mps_init_dev || !out) return DMRG_EINVAL;
    const int N = mp->N;
    if (N < 3 || D < 1 || 4 * D > kMaxCh || p->chi_min < 1 || p->chi_max < p->chi_min || p->chi_init < 1 ||
        p->chi_init > p->chi_max || p->lanczos_steps < 1 || p->lanczos_steps > LZ_MAXK)
        return DMRG_EINVAL;
    if (p->prec != DMRG_PREC_FP64 && p->prec != DMRG_PREC_3XTF32) return DMRG_EUNSUPPORTED;
    if (p->prec == DMRG_PREC_3XTF32 && !tc_available(ctx)) return DMRG_EUNSUPPORTED;
    dmrg_state *st = new (std::nothrow) dmrg_state();
    if (!st) return DMRG_ENOMEM;
    st->ctx = ctx;
    st->stream = ctx->stream;
    st->N = N;
    st->D = D;
    st->p = *p;
    if (st->p.jacobi_max_sweeps <= 0) st->p.jacobi_max_sweeps = 60;
    st->mp = *mp;
    st->K = p->lanczos_steps;
    st->chi.resize(N + 1);
    st->cap.resize(N + 1);
    auto powcap = [](int e, long long c) { long long v = 1; for (int i = 0; i < e && v < c; ++i) v *= 2; return v; };
    for (int i = 0; i <= N; ++i) {
        long long c = p->chi_max;
        c = std::min(c, powcap(i, c));
        c = std::min(c, powcap(N - i, c));
        st->cap[i] = (int)c;
        long long c0 = std::min<long long>(p->chi_init, c);
        st->chi[i] = (int)c0;
    }
    // sizes
    long long nmax = 1, svd_bytes = 0, umax = 1, vtmax = 1, smax = 1;
    for (int k = 0; k + 2 <= N; ++k) {
        long long m = 2LL * st->cap[k], n = 2LL * st->cap[k + 2];
        nmax = std::max(nmax, m * n);
        long long r = std::min(m, n), l = std::max(m, n);
        svd_bytes = std::max<long long>(svd_bytes, (long long)svd_work_bytes((int)r, (int)l));
        umax = std::max(umax, m * r);
        vtmax = std::max(vtmax, r * n);
        smax = std::max(smax, r);
    }
    for (int i = 0; i < N; ++i) {  // initial gauge move: chi_i x 2 chi_{i+1}
        long long m = st->chi[i], n = 2LL * st->chi[i + 1];
        long long r = std::min(m, n), l = std::max(m, n);
        svd_bytes = std::max<long long>(svd_bytes, (long long)svd_work_bytes((int)r, (int)l));
        umax = std::max(umax, m * r);
        vtmax = std::max(vtmax, r * n);
        smax = std::max(smax, r);
    }
    for (int i = 0; i < N; ++i) {  // gauge-move temporaries and initial environments
        nmax = std::max(nmax, 4LL * st->cap[i] * st->cap[i + 1]);
        nmax = std::max(nmax, (long long)st->cap[i] * st->cap[i]);
    }
    st->nmax = nmax;
    size_t total = 0;
    std::vector<size_t> site_off(N), env_off(N + 1);
    total += al256(sizeof(double) * (size_t)N * D * D * 4);                  // W
    total += al256(sizeof(double) * (size_t)(N - 1) * 16 * D * D);           // coef_mv
    total += al256(sizeof(double) * (size_t)N * 4 * D * D) * 2;              // coef_l, coef_r
    for (int i = 0; i < N; ++i) { site_off[i] = total; total += al256(sizeof(double) * (size_t)st->cap[i] * 2 * st->cap[i + 1]); }
    for (int i = 0; i <= N; ++i) { env_off[i] = total; total += al256(sizeof(double) * (size_t)D * st->cap[i] * st->cap[i]); }
    size_t off_ctrl = total; total += al256(sizeof(dmrg_ctrl_state) * (N - 1));
    size_t off_gctrl = total; total += al256(sizeof(dmrg_ctrl_state));
    size_t off_theta = total; total += al256(sizeof(double) * nmax);
    size_t off_X = total; total += al256(sizeof(double) * nmax * D);
    size_t off_Y = total; total += al256(sizeof(double) * nmax * D);
    size_t off_U = total; total += al256(sizeof(double) * umax);
    size_t off_s = total; total += al256(sizeof(double) * (smax + 2 * kNormBlocks));
    size_t off_Vt = total; total += al256(sizeof(double) * vtmax);
    size_t off_svd = total; total += al256(svd_bytes);
    size_t off_lz = total; total += al256(lanczos_work_bytes(nmax, st->K, ctx->num_sms));
    size_t off_res = total; total += al256(sizeof(BondResult));
    size_t off_info = total; total += al256(sizeof(int) * 4);
    size_t off_vis = total; total += al256(sizeof(dmrg_visit_record) * (2 * N));
    size_t off_mlp = total; total += al256(sizeof(float) * MLP_NPARAM);
    long long cmax = 1;
    for (int i = 0; i <= N; ++i) cmax = std::max<long long>(cmax, st->cap[i]);
    const long long kp_c = split_kp((int)cmax), kp_dc = split_kp((int)(D * cmax));
    size_t off_Lh = total; total += al256(sizeof(float) * (size_t)(D * cmax) * 3 * kp_c);
    size_t off_Rh = total; total += al256(sizeof(float) * (size_t)cmax * 3 * kp_dc);
    size_t off_xh = total; total += al256(sizeof(float) * (size_t)(4 * cmax) * 3 * kp_c);
    size_t off_Yh = total; total += al256(sizeof(float) * (size_t)(4 * cmax) * 3 * kp_dc);
    if (st->arena.ensure(total) != DMRG_OK) { delete st; return DMRG_ENOMEM; }
    char *base = st->arena.as<char>();
    size_t o = 0;
    st->W = reinterpret_cast<double *>(base + o); o += al256(sizeof(double) * (size_t)N * D * D * 4);
    st->coef_mv = reinterpret_cast<double *>(base + o); o += al256(sizeof(double) * (size_t)(N - 1) * 16 * D * D);
    st->coef_l = reinterpret_cast<double *>(base + o); o += al256(sizeof(double) * (size_t)N * 4 * D * D);
    st->coef_r = reinterpret_cast<double *>(base + o); o += al256(sizeof(double) * (size_t)N * 4 * D * D);
    st->A.resize(N);
    st->env.resize(N + 1);
    for (int i = 0; i < N; ++i) st->A[i] = reinterpret_cast<double *>(base + site_off[i]);
    for (int i = 0; i <= N; ++i) st->env[i] = reinterpret_cast<double *>(base + env_off[i]);
    st->ctrl = reinterpret_cast<dmrg_ctrl_state *>(base + off_ctrl);
    st->gctrl = reinterpret_cast<dmrg_ctrl_state *>(base + off_gctrl);
    st->global_chi = p->chi_min;
    st->theta = reinterpret_cast<double *>(base + off_theta);
    st->X = reinterpret_cast<double *>(base + off_X);
    st->Y = reinterpret_cast<double *>(base + off_Y);
    st->U = reinterpret_cast<double *>(base + off_U);
    st->s = reinterpret_cast<double *>(base + off_s);
    st->Vt = reinterpret_cast<double *>(base + off_Vt);
    st->svdw = base + off_svd;
    st->lw = lanczos_work_carve(base + off_lz, nmax, st->K, ctx->num_sms);
    st->d_res = reinterpret_cast<BondResult *>(base + off_res);
    st->d_info = reinterpret_cast<int *>(base + off_info);
    st->d_visits = reinterpret_cast<dmrg_visit_record *>(base + off_vis);
    st->mlp = reinterpret_cast<float *>(base + off_mlp);
    st->Lh = reinterpret_cast<float *>(base + off_Lh);
    st->Rh = reinterpret_cast<float *>(base + off_Rh);
    st->xh = reinterpret_cast<float *>(base + off_xh);
    st->Yh = reinterpret_cast<float *>(base + off_Yh);
    if (cudaMallocHost(&st->h_res, sizeof(BondResult)) != cudaSuccess) { st->arena.release(); delete st; return DMRG_ENOMEM; }
    if (cudaEventCreateWithFlags(&st->ev_res, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(st->h_res); st->arena.release(); delete st; return DMRG_ECUDA;
    }
    cudaStream_t cs = ctx->stream;
    auto fail = [&](dmrg_status s) {
        cudaStreamSynchronize(cs); cudaEventDestroy(st->ev_res); cudaFreeHost(st->h_res); st->arena.release();
        delete st; return s;
    };
    if (cudaMemcpyAsync(st->W, W_dev, sizeof(double) * (size_t)N * D * D * 4, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
        return fail(DMRG_ECUDA);
    // coefficient tables
    for (int k = 0; k + 1 < N; ++k) {
        dmrg_status s0 = build_coef(ctx, 0, D, st->W + (size_t)k * D * D * 4, st->W + (size_t)(k + 1) * D * D * 4,
                                    st->coef_mv + (size_t)k * 16 * D * D);
        if (s0 != DMRG_OK) return fail(s0);
    }
    for (int i = 0; i < N; ++i) {
        dmrg_status s1 = build_coef(ctx, 1, D, st->W + (size_t)i * D * D * 4, nullptr, st->coef_l + (size_t)i * 4 * D * D);
        dmrg_status s2 = build_coef(ctx, 2, D, st->W + (size_t)i * D * D * 4, nullptr, st->coef_r + (size_t)i * 4 * D * D);
        if (s1 != DMRG_OK || s2 != DMRG_OK) return fail(DMRG_ECUDA);
    }
    // initial MPS entries
    {
        size_t off = 0;
        for (int i = 0; i < N; ++i) {
            size_t sz = (size_t)st->chi[i] * 2 * st->chi[i + 1];
            if (cudaMemcpyAsync(st->A[i], mps_init_dev + off, sizeof(double) * sz, cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
                return fail(DMRG_ECUDA);
            off += sz;
        }
    }
    // right-canonical form: M_i = U S Vt, A_i <- Vt, A_{i-1} <- A_{i-1} U S
    for (int i = N - 1; i >= 1; --i) {
        int rows = st->chi[i], cols = 2 * st->chi[i + 1];
        int r = std::min(rows, cols);
        dmrg_status s0 = svd_jacobi(ctx, st->A[i], rows, cols, st->U, st->s, st->Vt, st->svdw, 60, st->d_info);
        if (s0 != DMRG_OK) return fail(s0);
        if (r != rows) return fail(DMRG_EINVAL);
        k_copy_scale<<<grid1d((long long)r * cols, 256, ctx->num_sms), 256, 0, cs>>>(st->Vt, st->A[i], r, cols, nullptr); DMRG_COUNT_LAUNCH();
        // the state is normalised at the end; renormalising S at every step
        // keeps the carried norm (a product over the sites, about 2^N for a
        // random MPS) from overflowing on long chains
        k_normalise<<<1, 256, 0, cs>>>(st->s, r); DMRG_COUNT_LAUNCH();
        k_copy_scale<<<grid1d((long long)rows * r, 256, ctx->num_sms), 256, 0, cs>>>(st->U, st->theta, rows, r, st->s); DMRG_COUNT_LAUNCH();
        int pr = 2 * st->chi[i - 1];
        s0 = gemm_f64(cs, pr, r, rows, 1.0, st->A[i - 1], rows, 1, 0, st->theta, r, 1, 0, 0.0, st->X, r, 1, 0, 1);
        if (s0 != DMRG_OK) return fail(s0);
        k_copy_scale<<<grid1d((long long)pr * r, 256, ctx->num_sms), 256, 0, cs>>>(st->X, st->A[i - 1], pr, r, nullptr); DMRG_COUNT_LAUNCH();
        if (cudaGetLastError() != cudaSuccess) return fail(DMRG_ECUDA);
    }
    k_normalise<<<1, 256, 0, cs>>>(st->A[0], 2 * st->chi[1]); DMRG_COUNT_LAUNCH();
    k_boundary_env<<<1, 32, 0, cs>>>(st->env[0], D, D - 1); DMRG_COUNT_LAUNCH();
    k_boundary_env<<<1, 32, 0, cs>>>(st->env[N], D, 0); DMRG_COUNT_LAUNCH();
    for (int i = N - 1; i >= 2; --i) {
        dmrg_status s0 = env_right_dev(ctx, st->p.prec, D, st->chi[i], st->chi[i + 1], st->env[i + 1],
                                       st->coef_r + (size_t)i * 4 * D * D, st->A[i], st->env[i], st->X, st->Y);
        if (s0 != DMRG_OK) return fail(s0);
    }
    k_init_ctrl<<<(N - 1 + 127) / 128, 128, 0, cs>>>(st->ctrl, N - 1, p->chi_min); DMRG_COUNT_LAUNCH();
    k_init_ctrl<<<1, 128, 0, cs>>>(st->gctrl, 1, p->chi_min); DMRG_COUNT_LAUNCH();
    if (cudaGetLastError() != cudaSuccess) return fail(DMRG_ECUDA);
    if (cudaStreamSynchronize(cs) != cudaSuccess) return fail(DMRG_ECUDA);
    *out = st;
    return DMRG_OK;
}

void dmrg_state_destroy(dmrg_state *st)
{
    if (!st) return;
    cudaStreamSynchronize(st->stream);
    if (st->ev_res) cudaEventDestroy(st->ev_res);
    if (st->h_res) cudaFreeHost(st->h_res);
    st->arena.release();
    delete st;
}

// Visit v of a sweep of N sites: bond k, whether the centre moves right, the
// direction and whether the controller steps (Section 10's sweep order).
static void visit_of(const dmrg_state *st, int v, int &k, int &go_right, int &direction, int &do_ctrl)
{
    const int N = st->N;
    const int half = v < N - 1 ? 0 : 1;
    const int q = half == 0 ? v : v - (N - 1);
    k = (half == 0) ? q : N - 3 - q;
    go_right = (half == 0 && k < N - 2);
    direction = half == 0 ? 1 : -1;
    do_ctrl = ((st->p.pid_steps_per_sweep >= 2) || (half == 0)) && st->p.ctrl != DMRG_CTRL_HOLD &&
              st->p.ctrl != DMRG_CTRL_REPLAY;
}

// End of a sweep: copy the visit records, fill the sweep record, advance the
// sweep index and read the status word.
static dmrg_status sweep_close(dmrg_state *st, double E_last, double flops, double seconds,
                               dmrg_sweep_record *rec, dmrg_visit_record *visits_host)
{
    const int V = 2 * st->N - 3;
    std::vector<dmrg_visit_record> vis(V);
    DMRG_CUDA(cudaMemcpyAsync(vis.data(), st->d_visits, sizeof(dmrg_visit_record) * V, cudaMemcpyDeviceToHost,
                              st->ctx->stream));
    DMRG_CUDA(cudaStreamSynchronize(st->ctx->stream));
    if (visits_host) std::memcpy(visits_host, vis.data(), sizeof(dmrg_visit_record) * V);
    if (rec) {
        dmrg_sweep_record r{};
        r.E = E_last;
        double mx = 0.0, sum = 0.0;
        int mk = 0;
        for (auto &x : vis) { mx = std::max(mx, x.trunc_err); sum += x.k; mk = std::max(mk, x.k); }
        r.max_trunc_err = mx;
        r.mean_chi = sum / V;
        r.max_chi = mk;
        r.n_visits = V;
        r.seconds = seconds;
        r.flops = flops;
        *rec = r;
    }
    if (st->p.ctrl == DMRG_CTRL_GLOBAL) {
        // global adaptive chi: one controller step per sweep, on the mean of
        // the bonds' filtered entropies; its chi truncates every bond next sweep
        DMRG_TRY(launch_global_step(st->ctx, st->ctrl, st->N - 1, st->gctrl, st->p));
        DMRG_CUDA(cudaMemcpyAsync(st->ctx->h_pinned_i + 48, &st->gctrl->chi, sizeof(int), cudaMemcpyDeviceToHost,
                                  st->ctx->stream));
        DMRG_CUDA(cudaStreamSynchronize(st->ctx->stream));
        st->global_chi = st->ctx->h_pinned_i[48];
    }
    st->sweep_index++;
    dmrg_status ds = dmrg_get_status(st->ctx);
    if (ds != DMRG_OK && ds != DMRG_ENOCONV) return ds;
    return DMRG_OK;
}

dmrg_status dmrg_sweep(dmrg_ctx *ctx, dmrg_state *st, int n_sweeps, int stop_on_conv, dmrg_sweep_record *rec_host,
                       dmrg_visit_record *visits_host, int *sweeps_done)
{
    if (!ctx || !st || st->ctx != ctx || n_sweeps < 0) return DMRG_EINVAL;
    const int V = 2 * st->N - 3;
    double E_prev = 0.0;
    int done = 0;
    for (int t = 0; t < n_sweeps; ++t) {
        double flops = 0.0, E_last = 0.0;
        DMRG_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
        for (int v = 0; v < V; ++v) {
            int k, go_right, direction, do_ctrl, kk;
            visit_of(st, v, k, go_right, direction, do_ctrl);
            st->cur_visit = v;
            dmrg_status bs = bond_step(st, k, go_right, do_ctrl, st->d_visits + v, direction, &flops, &kk, &E_last);
            st->cur_visit = -1;
            if (bs != DMRG_OK) return bs;
        }
        DMRG_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
        DMRG_CUDA(cudaEventSynchronize(ctx->ev1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        DMRG_TRY(sweep_close(st, E_last, flops, ms * 1e-3, rec_host ? rec_host + t : nullptr,
                             visits_host ? visits_host + (size_t)t * V : nullptr));
        done = t + 1;
        if (stop_on_conv && t > 0 && std::fabs((E_last - E_prev) / E_last) < st->p.eps_conv) break;
        E_prev = E_last;
    }
    if (sweeps_done) *sweeps_done = done;
    return DMRG_OK;
}

dmrg_status dmrg_sweep_chains(int n_chains, dmrg_ctx *const *ctxs, dmrg_state *const *states, int n_sweeps,
                              dmrg_sweep_record *rec_host, double *seconds_out)
{
    if (n_chains < 1 || !ctxs || !states || n_sweeps < 0) return DMRG_EINVAL;
    for (int c = 0; c < n_chains; ++c) {
        if (!ctxs[c] || !states[c] || states[c]->ctx != ctxs[c]) return DMRG_EINVAL;
        for (int d = 0; d < c; ++d)
            if (ctxs[d] == ctxs[c] || states[d] == states[c]) return DMRG_EINVAL;   // one context per chain
    }
    struct Run {
        int v = 0, sweep = 0;
        double flops = 0.0, E_last = 0.0;
    };
    std::vector<Run> run(n_chains);
    auto t0 = std::chrono::steady_clock::now();
    int live = n_sweeps > 0 ? n_chains : 0;
    std::vector<int> active;
    while (live > 0) {
        active.clear();
        for (int c = 0; c < n_chains; ++c)
            if (run[c].sweep < n_sweeps) active.push_back(c);
        // phase A of every live chain, then phase B of every live chain
        for (int c : active) {
            dmrg_state *st = states[c];
            int k, go_right, direction, do_ctrl;
            visit_of(st, run[c].v, k, go_right, direction, do_ctrl);
            st->cur_visit = run[c].v;
            DMRG_TRY(bond_step_a(st, k, go_right, do_ctrl, st->d_visits + run[c].v, direction));
        }
        for (int c : active) {
            dmrg_state *st = states[c];
            int kk;
            DMRG_TRY(bond_step_b(st, &run[c].flops, &kk, &run[c].E_last));
            if (++run[c].v == 2 * st->N - 3) {
                dmrg_sweep_record *rec = rec_host ? rec_host + (size_t)c * n_sweeps + run[c].sweep : nullptr;
                DMRG_TRY(sweep_close(st, run[c].E_last, run[c].flops, 0.0, rec, nullptr));
                run[c].v = 0;
                run[c].flops = 0.0;
                if (++run[c].sweep == n_sweeps) --live;
            }
        }
    }
    for (int c = 0; c < n_chains; ++c) DMRG_CUDA(cudaStreamSynchronize(ctxs[c]->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (seconds_out) *seconds_out = secs;
    return DMRG_OK;
}

dmrg_status bond_update(dmrg_ctx *ctx, dmrg_state *st, int bond, int direction, double *E_out, int *k_out)
{
    if (!ctx || !st || st->ctx != ctx || bond < 0 || bond > st->N - 2 || (direction != 1 && direction != -1))
        return DMRG_EINVAL;
    if (st->p.ctrl == DMRG_CTRL_REPLAY) return DMRG_EINVAL;   // a schedule is per sweep visit
    int go_right = (direction == 1) && (bond < st->N - 2);
    const int do_ctrl = st->p.ctrl != DMRG_CTRL_HOLD;
    DMRG_TRY(bond_step(st, bond, go_right, do_ctrl, st->d_visits, direction, nullptr, k_out, E_out));
    return DMRG_OK;
}

dmrg_status dmrg_state_chi(dmrg_state *st, int *chi_host)
{
    if (!st || !chi_host) return DMRG_EINVAL;
    std::memcpy(chi_host, st->chi.data(), sizeof(int) * (st->N + 1));
    return DMRG_OK;
}

dmrg_status dmrg_state_site(dmrg_state *st, int i, const double **A_dev)
{
    if (!st || !A_dev || i < 0 || i >= st->N) return DMRG_EINVAL;
    *A_dev = st->A[i];
    return DMRG_OK;
}

dmrg_status dmrg_state_env(dmrg_state *st, int left, int k, double *E_out_dev)
{
    if (!st || !E_out_dev || k < 0 || k > st->N) return DMRG_EINVAL;
    const int c = st->chi[k], D = st->D;
    if (left) {
        DMRG_CUDA(cudaMemcpyAsync(E_out_dev, st->env[k], sizeof(double) * D * c * c, cudaMemcpyDeviceToDevice,
                                  st->ctx->stream));
    } else {
        DMRG_TRY(transpose_sq(st->ctx, st->env[k], E_out_dev, c, D));
    }
    DMRG_CUDA(cudaStreamSynchronize(st->ctx->stream));
    return DMRG_OK;
}

dmrg_status dmrg_state_ctrl(dmrg_state *st, dmrg_ctrl_state **ctrl_dev)
{
    if (!st || !ctrl_dev) return DMRG_EINVAL;
    *ctrl_dev = st->ctrl;
    return DMRG_OK;
}

long long dmrg_state_mps_size(dmrg_state *st)
{
    if (!st) return -1;
    long long n = 0;
    for (int i = 0; i < st->N; ++i) n += (long long)st->chi[i] * 2 * st->chi[i + 1];
    return n;
}

dmrg_status dmrg_state_get_mps(dmrg_state *st, double *out)
{
    if (!st || !out) return DMRG_EINVAL;
    long long off = 0;
    for (int i = 0; i < st->N; ++i) {
        size_t n = (size_t)st->chi[i] * 2 * st->chi[i + 1];
        DMRG_CUDA(cudaMemcpyAsync(out + off, st->A[i], sizeof(double) * n, cudaMemcpyDefault, st->ctx->stream));
        off += (long long)n;
    }
    DMRG_CUDA(cudaStreamSynchronize(st->ctx->stream));
    return DMRG_OK;
}

dmrg_status dmrg_state_put_mps(dmrg_state *st, const double *in)
{
    if (!st || !in) return DMRG_EINVAL;
    long long off = 0;
    for (int i = 0; i < st->N; ++i) {
        size_t n = (size_t)st->chi[i] * 2 * st->chi[i + 1];
        DMRG_CUDA(cudaMemcpyAsync(st->A[i], in + off, sizeof(double) * n, cudaMemcpyDefault, st->ctx->stream));
        off += (long long)n;
    }
    DMRG_CUDA(cudaStreamSynchronize(st->ctx->stream));
    return DMRG_OK;
}

long long dmrg_launch_count(void) { return g_launch_count.load(); }

int dmrg_svd_last_sweeps(const dmrg_ctx *ctx) { return ctx ? ctx->h_pinned_i[32] : 0; }

}  // extern "C"

namespace dmrg {
namespace {
// Two co-resident blocks meet at the bounded grid barrier; with `absent` set,
// block 0 never arrives, so block 1 polls until spin_limit, records
// ST_TIMEOUT in the status word and returns.  Nothing traps or faults.
__global__ void k_wait_selftest(unsigned *words, int *status, long long spin_limit, int absent, int *result)
{
    if (absent && blockIdx.x == 0) return;
    const bool ok = grid_barrier(words, status, spin_limit);
    if (threadIdx.x == 0) result[blockIdx.x] = ok ? 1 : -1;
}
}  // namespace
}  // namespace dmrg

extern "C" {

dmrg_status dmrg_wait_selftest(dmrg_ctx *ctx, long long spin_limit, int absent)
{
    if (!ctx || spin_limit < 1) return DMRG_EINVAL;
    void *buf = nullptr;
    DMRG_CUDA(cudaMalloc(&buf, 64));
    DMRG_CUDA(cudaMemsetAsync(buf, 0, 64, ctx->stream));
    unsigned *words = static_cast<unsigned *>(buf);
    int *result = reinterpret_cast<int *>(static_cast<char *>(buf) + 32);
    int *status = ctx->d_status;
    void *args[] = {&words, &status, &spin_limit, &absent, &result};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_wait_selftest, dim3(2), dim3(32), args, 0, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return DMRG_ECUDA;
    return dmrg_get_status(ctx);
}

dmrg_status dmrg_profile(dmrg_ctx *ctx, int on)
{
    if (!ctx) return DMRG_EINVAL;
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto &p : ctx->prof_slot) { p.used = 0; p.n = 0; p.flops = 0.0; p.bytes = 0.0; }
    ctx->prof = on ? 1 : 0;
    return DMRG_OK;
}

dmrg_status dmrg_profile_read(dmrg_ctx *ctx, int kind, double *ms, long long *launches, double *flops, double *bytes)
{
    if (!ctx || kind < 0 || kind >= PROF_KINDS) return DMRG_EINVAL;
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    ProfSlot &p = ctx->prof_slot[kind];
    double t = 0.0;
    for (size_t i = 0; i + 1 < p.used; i += 2) {
        float x = 0.f;
        if (cudaEventElapsedTime(&x, p.ev[i], p.ev[i + 1]) == cudaSuccess) t += x;
    }
    if (ms) *ms = t;
    if (launches) *launches = p.n;
    if (flops) *flops = p.flops;
    if (bytes) *bytes = p.bytes;
    return DMRG_OK;
}

dmrg_status dmrg_state_set_params(dmrg_state *st, const dmrg_params *p)
{
    if (!st || !p) return DMRG_EINVAL;
    const dmrg_params &o = st->p;
    // the state's memory and precision were sized for these: they stay
    if (p->chi_max != o.chi_max || p->prec != o.prec || p->lanczos_steps != o.lanczos_steps ||
        p->chi_min < 1 || p->chi_min > p->chi_max || p->ctrl < DMRG_CTRL_PID || p->ctrl > DMRG_CTRL_REPLAY)
        return DMRG_EINVAL;
    const int jms = o.jacobi_max_sweeps;
    st->p = *p;
    if (st->p.jacobi_max_sweeps <= 0) st->p.jacobi_max_sweeps = jms;
    return DMRG_OK;
}

dmrg_status dmrg_state_set_schedule(dmrg_state *st, const int *chi_host, int n)
{
    if (!st || !chi_host || n != 2 * st->N - 3) return DMRG_EINVAL;
    for (int v = 0; v < n; ++v)
        if (chi_host[v] < 1 || chi_host[v] > st->p.chi_max) return DMRG_EINVAL;
    st->sched.assign(chi_host, chi_host + n);
    return DMRG_OK;
}

dmrg_status dmrg_state_set_mlp(dmrg_state *st, const float *params_dev)
{
    if (!st) return DMRG_EINVAL;
    if (!params_dev) { st->has_mlp = 0; return DMRG_OK; }
    DMRG_CUDA(cudaMemcpyAsync(st->mlp, params_dev, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, st->ctx->stream));
    st->has_mlp = 1;
    return DMRG_OK;
}

// ---------------------------------------------------------------------------
// standalone building blocks
// ---------------------------------------------------------------------------
// Mixed-precision SVD (context option svd_prec = 1): FP32 Jacobi on the
// min(m,n) vectors of the longer side, one FP64 Newton-Schulz step on the
// unit vectors, and the FP64 projection of theta on them.  The singular
// values are the norms of the projection: they depend on the isometry's
// direction errors only to second order, while the FP32 Jacobi norms carry
// the rounding of every rotation (about 1e-4 relative at n ~ 1000) and a
// 3xTF32 projection its own (about 1e-5).  The other factor is the
// projection scaled by 1/s.  Singular values below 2^-22 s_0 are not resolved.
static dmrg_status svd_mixed_full(dmrg_ctx *ctx, const double *A, int m, int n, double *U, double *s, double *Vt,
                                  BondResult *res, int *info)
{
    const int dir = (n <= m) ? 0 : 1;          // vectors = columns (length m) or rows (length n)
    const int r = std::min(m, n), len = dir == 0 ? m : n;
    const size_t w1 = al256(jac32_work_bytes(dir == 0 ? n : m, len));
    const size_t need = w1 + 3 * al256(sizeof(double) * (size_t)r * len) + al256(sizeof(double) * (size_t)r * r) +
                        al256(sizeof(double) * 512) + al256(sizeof(int) * 4) + al256(sizeof(double) * r) +
                        al256(sizeof(int) * r);
    DMRG_TRY(ctx->work3.ensure(need));
    char *b = ctx->work3.as<char>();
    void *jw = b; b += w1;
    double *Q = reinterpret_cast<double *>(b); b += al256(sizeof(double) * (size_t)r * len);
    double *T = reinterpret_cast<double *>(b); b += al256(sizeof(double) * (size_t)r * len);
    double *P = reinterpret_cast<double *>(b); b += al256(sizeof(double) * (size_t)r * len);
    double *E = reinterpret_cast<double *>(b); b += al256(sizeof(double) * (size_t)r * r);
    int *rdev = reinterpret_cast<int *>(b); b += al256(sizeof(int) * 4);
    double *pn = reinterpret_cast<double *>(b); b += al256(sizeof(double) * r);
    int *pperm = reinterpret_cast<int *>(b);
    float *X32;
    double *nrm;
    int *perm;
    DMRG_TRY(svd_jacobi32(ctx, A, m, n, dir, jw, ctx->jacobi_max_sweeps, info, s, &X32, &nrm, &perm));
    // all r vectors
    (void)res;
    k_fill_int<<<1, 1, 0, ctx->stream>>>(rdev, r); DMRG_COUNT_LAUNCH();
    DMRG_TRY(gather_unit_vectors(ctx, X32, nrm, perm, rdev, r, len, Q));
    DMRG_TRY(gemm_f64(ctx->stream, r, r, len, 1.0, Q, len, 1, 0, Q, 1, len, 0, 0.0, E, r, 1, 0, 1));
    DMRG_CUDA(cudaMemcpyAsync(T, Q, sizeof(double) * (size_t)r * len, cudaMemcpyDeviceToDevice, ctx->stream));
    DMRG_TRY(gemm_f64(ctx->stream, r, len, r, -0.5, E, r, 1, 0, Q, len, 1, 0, 1.5, T, len, 1, 0, 1));
    const int rb = (r + 255) / 256;
    if (dir == 0) {
        // P = T A (r x n); s = |rows of P|, re-ranked; U = T^T, Vt = diag(1/s) P in that order
        DMRG_TRY(gemm(ctx, DMRG_PREC_FP64, r, n, m, 1.0, T, m, 1, 0, A, n, 1, 0, 0.0, P, n, 1, 0, 1));
        k_row_norms<<<(r * 32 + 255) / 256, 256, 0, ctx->stream>>>(P, r, n, pn); DMRG_COUNT_LAUNCH();
        k_rank_sorted<<<rb, 256, 0, ctx->stream>>>(pn, r, pperm); DMRG_COUNT_LAUNCH();
        k_take_sorted<<<rb, 256, 0, ctx->stream>>>(pn, pperm, r, s); DMRG_COUNT_LAUNCH();
        k_gather_rows_t<<<grid1d((long long)m * r, 256, ctx->num_sms), 256, 0, ctx->stream>>>(T, pperm, r, m, U); DMRG_COUNT_LAUNCH();
        k_gather_rows<<<grid1d((long long)r * n, 256, ctx->num_sms), 256, 0, ctx->stream>>>(P, pperm, s, r, n, Vt); DMRG_COUNT_LAUNCH();
    } else {
        // P = A T^T (m x r); s = |columns of P|, re-ranked; Vt = T, U = P diag(1/s) in that order
        DMRG_TRY(gemm(ctx, DMRG_PREC_FP64, m, r, n, 1.0, A, n, 1, 0, T, 1, n, 0, 0.0, P, r, 1, 0, 1));
        k_col_norms<<<rb, 256, 0, ctx->stream>>>(P, m, r, pn); DMRG_COUNT_LAUNCH();
        k_rank_sorted<<<rb, 256, 0, ctx->stream>>>(pn, r, pperm); DMRG_COUNT_LAUNCH();
        k_take_sorted<<<rb, 256, 0, ctx->stream>>>(pn, pperm, r, s); DMRG_COUNT_LAUNCH();
        k_gather_rows<<<grid1d((long long)r * n, 256, ctx->num_sms), 256, 0, ctx->stream>>>(T, pperm, nullptr, r, n, Vt); DMRG_COUNT_LAUNCH();
        k_gather_cols_scaled<<<grid1d((long long)m * r, 256, ctx->num_sms), 256, 0, ctx->stream>>>(P, pperm, s, m, r, U); DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status svd_truncate(dmrg_ctx *ctx, const double *theta_dev, int m, int n, int chi_max, double eps, double *U_dev,
                         double *s_dev, double *Vt_dev, int *k_out, double *S_out, double *trunc_err_out)
{
    if (!ctx || !theta_dev || !U_dev || !s_dev || !Vt_dev || m < 1 || n < 1 || chi_max < 1 || !(eps >= 0.0))
        return DMRG_EINVAL;
    const int r = std::min(m, n), l = std::max(m, n);
    if (ctx->svd_prec == 1) {
        if (!tc_available(ctx)) return DMRG_EUNSUPPORTED;
        DMRG_TRY(ctx->work.ensure(al256(sizeof(BondResult)) + al256(sizeof(int) * 4)));
        BondResult *res = reinterpret_cast<BondResult *>(ctx->work.as<char>());
        int *info = reinterpret_cast<int *>(ctx->work.as<char>() + al256(sizeof(BondResult)));
        DMRG_TRY(svd_mixed_full(ctx, theta_dev, m, n, U_dev, s_dev, Vt_dev, res, info));
        dmrg_params p{};
        p.eps_trunc = eps;
        p.chi_min = 1;
        p.chi_max = chi_max;
        p.ctrl = DMRG_CTRL_FIXED;
        DMRG_TRY(launch_decide(ctx, s_dev, r, nullptr, p, 0, chi_max, nullptr, 0, 1, 0, nullptr, res, nullptr, 0,
                               kMixedRankFloor));
        DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_d, res, sizeof(BondResult), cudaMemcpyDeviceToHost, ctx->stream));
        DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_i + 32, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
        BondResult br;
        std::memcpy(&br, ctx->h_pinned_d, sizeof(BondResult));
        if (k_out) *k_out = br.k;
        if (S_out) *S_out = br.S;
        if (trunc_err_out) *trunc_err_out = br.eps;
        dmrg_status ds = dmrg_get_status(ctx);
        if (ctx->h_pinned_i[32] < 0) return DMRG_ENOCONV;
        return ds == DMRG_ENOCONV ? DMRG_OK : ds;
    }
    size_t need = al256(svd_work_bytes(r, l)) + al256(sizeof(BondResult)) + al256(sizeof(int) * 4);
    DMRG_TRY(ctx->work.ensure(need));
    char *base = ctx->work.as<char>();
    BondResult *res = reinterpret_cast<BondResult *>(base + al256(svd_work_bytes(r, l)));
    int *info = reinterpret_cast<int *>(base + al256(svd_work_bytes(r, l)) + al256(sizeof(BondResult)));
    DMRG_TRY(svd_jacobi(ctx, theta_dev, m, n, U_dev, s_dev, Vt_dev, base, ctx->jacobi_max_sweeps, info));
    dmrg_params p{};
    p.eps_trunc = eps;
    p.chi_min = 1;
    p.chi_max = chi_max;
    p.multiplet_guard = 0;
    p.ctrl = DMRG_CTRL_FIXED;
    DMRG_TRY(launch_decide(ctx, s_dev, r, nullptr, p, 0, chi_max, nullptr, 0, 1, 0, nullptr, res, nullptr, 0,
                           (double)r * 2.220446049250313e-16));
    DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_d, res, sizeof(BondResult), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaMemcpyAsync(ctx->h_pinned_i + 32, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    BondResult br;
    std::memcpy(&br, ctx->h_pinned_d, sizeof(BondResult));
    if (k_out) *k_out = br.k;
    if (S_out) *S_out = br.S;
    if (trunc_err_out) *trunc_err_out = br.eps;
    dmrg_status ds = dmrg_get_status(ctx);
    if (ctx->h_pinned_i[32] < 0) return DMRG_ENOCONV;
    return ds == DMRG_ENOCONV ? DMRG_OK : ds;
}

dmrg_status entropy_pid_step(dmrg_ctx *ctx, int n_bonds, const double *S_raw_dev, dmrg_ctrl_state *st_dev,
                             const dmrg_params *p_host, int *chi_out_dev)
{
    if (!ctx || !S_raw_dev || !st_dev || !p_host || !chi_out_dev || n_bonds < 0) return DMRG_EINVAL;
    return launch_ctrl_steps(ctx, n_bonds, S_raw_dev, st_dev, *p_host, chi_out_dev);
}

dmrg_status dmrg_entropy(dmrg_ctx *ctx, int n, const double *s_dev, double *S_dev, double *eps_dev)
{
    if (!ctx || !s_dev || !S_dev || n < 1) return DMRG_EINVAL;
    return launch_entropy(ctx, n, s_dev, S_dev, eps_dev);
}

// scratch for the standalone contraction calls: coefficient table, Rt, X, Y
static dmrg_status standalone_scratch(dmrg_ctx *ctx, int D, int cl, int cr, double **C, double **Rt, double **X,
                                      double **Y, size_t extra, void **extra_ptr)
{
    size_t nX = (size_t)D * 4 * cl * cr + (size_t)D * 4 * cl * cl + 64;
    size_t need = al256(sizeof(double) * 1024) + al256(sizeof(double) * (size_t)D * std::max(cr, cl) * std::max(cr, cl)) +
                  2 * al256(sizeof(double) * nX) + al256(extra);
    DMRG_TRY(ctx->work2.ensure(need));
    char *b = ctx->work2.as<char>();
    *C = reinterpret_cast<double *>(b); b += al256(sizeof(double) * 1024);
    *Rt = reinterpret_cast<double *>(b); b += al256(sizeof(double) * (size_t)D * std::max(cr, cl) * std::max(cr, cl));
    *X = reinterpret_cast<double *>(b); b += al256(sizeof(double) * nX);
    *Y = reinterpret_cast<double *>(b); b += al256(sizeof(double) * nX);
    if (extra_ptr) *extra_ptr = b;
    return DMRG_OK;
}

dmrg_status dmrg_heff_apply(dmrg_ctx *ctx, int prec, int D, int cl, int cr, const double *L_dev, const double *W1_dev,
                            const double *W2_dev, const double *R_dev, const double *theta_dev, double *y_dev)
{
    if (!ctx || !L_dev || !W1_dev || !W2_dev || !R_dev || !theta_dev || !y_dev || D < 1 || 4 * D > kMaxCh || cl < 1 ||
        cr < 1)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && !(prec == DMRG_PREC_3XTF32 && tc_available(ctx))) return DMRG_EUNSUPPORTED;
    double *C, *Rt, *X, *Y;
    DMRG_TRY(standalone_scratch(ctx, D, cl, cr, &C, &Rt, &X, &Y, 0, nullptr));
    DMRG_TRY(build_coef(ctx, 0, D, W1_dev, W2_dev, C));
    DMRG_TRY(transpose_sq(ctx, R_dev, Rt, cr, D));
    DMRG_TRY(heff_apply_dev(ctx, prec, D, cl, cr, L_dev, Rt, C, X, Y, theta_dev, y_dev));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return dmrg_get_status(ctx);
}

dmrg_status dmrg_env_left(dmrg_ctx *ctx, int prec, int D, int cl, int ck, const double *L_dev, const double *W_dev,
                          const double *A_dev, double *Lnew_dev)
{
    if (!ctx || !L_dev || !W_dev || !A_dev || !Lnew_dev || D < 1 || 2 * D > kMaxCh || cl < 1 || ck < 1)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && !(prec == DMRG_PREC_3XTF32 && tc_available(ctx))) return DMRG_EUNSUPPORTED;
    double *C, *Rt, *X, *Y;
    DMRG_TRY(standalone_scratch(ctx, D, cl, ck, &C, &Rt, &X, &Y, 0, nullptr));
    DMRG_TRY(build_coef(ctx, 1, D, W_dev, nullptr, C));
    DMRG_TRY(env_left_dev(ctx, prec, D, cl, ck, L_dev, C, A_dev, Lnew_dev, X, Y));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return dmrg_get_status(ctx);
}

dmrg_status dmrg_env_right(dmrg_ctx *ctx, int prec, int D, int ck, int cr, const double *R_dev, const double *W_dev,
                           const double *B_dev, double *Rnew_dev)
{
    if (!ctx || !R_dev || !W_dev || !B_dev || !Rnew_dev || D < 1 || 2 * D > kMaxCh || cr < 1 || ck < 1)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && !(prec == DMRG_PREC_3XTF32 && tc_available(ctx))) return DMRG_EUNSUPPORTED;
    double *C, *Rt, *X, *Y;
    void *extra;
    DMRG_TRY(standalone_scratch(ctx, D, ck, cr, &C, &Rt, &X, &Y, sizeof(double) * (size_t)D * ck * ck, &extra));
    double *Rtn = static_cast<double *>(extra);
    DMRG_TRY(build_coef(ctx, 2, D, W_dev, nullptr, C));
    DMRG_TRY(transpose_sq(ctx, R_dev, Rt, cr, D));
    DMRG_TRY(env_right_dev(ctx, prec, D, ck, cr, Rt, C, B_dev, Rtn, X, Y));
    DMRG_TRY(transpose_sq(ctx, Rtn, Rnew_dev, ck, D));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return dmrg_get_status(ctx);
}

dmrg_status dmrg_lanczos(dmrg_ctx *ctx, int prec, int D, int cl, int cr, const double *L_dev, const double *W1_dev,
                         const double *W2_dev, const double *R_dev, double *theta_dev, int K, double *E_out,
                         int *steps_out)
{
    if (!ctx || !L_dev || !W1_dev || !W2_dev || !R_dev || !theta_dev || D < 1 || 4 * D > kMaxCh || cl < 1 || cr < 1 ||
        K < 1 || K > LZ_MAXK)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && !(prec == DMRG_PREC_3XTF32 && tc_available(ctx))) return DMRG_EUNSUPPORTED;
    const long long n = 4LL * cl * cr;
    double *C, *Rt, *X, *Y;
    void *extra;
    DMRG_TRY(standalone_scratch(ctx, D, cl, cr, &C, &Rt, &X, &Y, lanczos_work_bytes(n, K, ctx->num_sms), &extra));
    LanczosWork lw = lanczos_work_carve(extra, n, K, ctx->num_sms);
    DMRG_TRY(build_coef(ctx, 0, D, W1_dev, W2_dev, C));
    DMRG_TRY(transpose_sq(ctx, R_dev, Rt, cr, D));
    MatvecFn mv = [&](const double *x, double *y) { return heff_apply_dev(ctx, prec, D, cl, cr, L_dev, Rt, C, X, Y, x, y); };
    int Ke = (int)std::min<long long>(K, n);
    DMRG_TRY(lanczos_run(ctx, lw, n, Ke, theta_dev, mv));
    LzState h;
    DMRG_CUDA(cudaMemcpyAsync(&h, lw.lz, sizeof(LzState), cudaMemcpyDeviceToHost, ctx->stream));
    DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (E_out) *E_out = h.E;
    if (steps_out) *steps_out = h.m;
    return dmrg_get_status(ctx);
}

}  // extern "C"
