// batched.cu -- many independent SVD + entropy + truncation problems in one
// launch (the uneven isolated-SVD batch).  One CTA per matrix runs a one-sided
// block Jacobi (Hestenes) iteration in Gram form:
//
//   the r vectors (columns or rows of A, whichever are fewer) are split into
//   blocks of 16; in each round of a round-robin schedule over the blocks, a
//   team of 4 warps takes a pair of blocks W = [X_I X_J] (32 vectors), forms
//   the 32 x 32 Gram matrix G = W^T W over tiles of 32 positions staged in
//   shared memory, diagonalises G with cyclic two-sided Jacobi (one warp,
//   accumulating the rotation Q), and applies W <- W Q, V <- V Q as small
//   matrix products.  A block pair whose G already has every cosine below the
//   tolerance is left untouched; a sweep with no rotation anywhere ends the
//   iteration.
//
// Compared with rotating one vector pair at a time this needs 2r/16 dependent
// rounds per sweep instead of 2r, and the vector traffic of a round is three
// passes over the 32 vectors (Gram, update of X, update of V) whatever the
// number of rotations inside the pair.  FP64, or FP32 for the mixed form.
// The call performs no host synchronisation, so once a first call has sized
// the workspace the launch sequence can be captured in a CUDA graph
// (dmrg_graph_*).
#include "common.cuh"
#include "mma_tf32.cuh"

#include <algorithm>
#include <numeric>

namespace dmrg {
namespace {

struct BDesc {
    int m, n, r, l, tr, nb;            // nb: number of 16-vector blocks (even)
    int ldx, ldv;                      // padded vector lengths (multiples of 32)
    int idx, pad;                      // position of the matrix in the caller's arrays
    long long off_in, off_U, off_s, off_Vt;
    long long off_X, off_V, off_P;     // workspace: vectors, rotations, permutation + sorted values
    long long off_R;                   // workspace: Householder reflectors of the QR preconditioning
};

constexpr int kBT = 512;                       // threads per matrix
constexpr int kWarps = kBT / 32;
constexpr int kTeamWarps = 4;                  // warps sharing one block pair
constexpr int kTeams = kWarps / kTeamWarps;
constexpr int kBlk = 16;                       // vectors per block; a pair is one warp wide

template <typename T> struct TileStride;       // row stride of a [position][vector] tile
template <> struct TileStride<float> { static constexpr int v = 44; };   // 176 B rows: conflict-free MMA fragments
template <> struct TileStride<double> { static constexpr int v = 34; };  // 272 B rows

template <typename T> struct GbjSmem {
    T tile[kWarps][32][TileStride<T>::v];      // per-warp staging tile; also the Gram partials
    T G[kTeams][32][33];
    T Q[kTeams][32][33];
    T Qa[kTeams][32][sizeof(T) == 4 ? 44 : 1];   // FP32: the block rotation in the MMA-friendly stride
    T rc[kTeams][2][16], rs[kTeams][2][16];   // rotations of a Jacobi step, double-buffered by step parity
    int rp[kTeams][2][16], rq[kTeams][2][16];
    unsigned rmask[kTeams][2];
    int team_rot[kTeams];
    unsigned rot_count;
    double red[32];
    BDesc d;
};

template <typename T> __device__ __forceinline__ T wsum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 32 consecutive elements (16-byte aligned) of one vector into column `lane`
// of a [position][vector] tile
__device__ __forceinline__ void stage32(const float *__restrict__ p, float (*tile)[44], int lane)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 x = q[i];
        tile[4 * i][lane] = x.x; tile[4 * i + 1][lane] = x.y;
        tile[4 * i + 2][lane] = x.z; tile[4 * i + 3][lane] = x.w;
    }
}
__device__ __forceinline__ void stage32(const double *__restrict__ p, double (*tile)[34], int lane)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const double2 x = q[i];
        tile[2 * i][lane] = x.x; tile[2 * i + 1][lane] = x.y;
    }
}

// ---------------------------------------------------------------------------
// FP32 form: the per-tile products on the tensor cores, 3xTF32 (x = hi + lo,
// hi = tf32(x), lo = tf32(x - hi); a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b),
// mma.m16n8k8 with FP32 accumulation.  Fragment layout of m16n8k8 (g = lane/4,
// c = lane%4): A a0..a3 = (g, c), (g+8, c), (g, c+4), (g+8, c+4); B b0, b1 =
// (k=c, n=g), (k=c+4, n=g); D d0..d3 = (g, 2c), (g, 2c+1), (g+8, 2c), (g+8, 2c+1).
// ---------------------------------------------------------------------------
// Gram partial of a tile: acc[mi][ni][.] += sum_t tile[t][m] tile[t][n],
// m = 16 mi + ..., n = 8 ni + ... (mma D layout)
__device__ __forceinline__ void tile_gram_tc(const float (*tile)[44], int lane, float (&acc)[2][4][4])
{
    const int g = lane >> 2, c = lane & 3;
    auto a = [&](int m, int k) { return tile[k][m]; };
    auto b = [&](int k, int n) { return tile[k][n]; };
#pragma unroll
    for (int ks = 0; ks < 32; ks += 8)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma3(acc[mi][ni], g, c, a, b, 16 * mi, 8 * ni, ks);
}

// p[j][t] = sum_q tile[t][q] Q[q][j] for the warp's 32 vectors j (lane = j writes
// its own vector's 32 positions); the tile is overwritten by the result
__device__ __forceinline__ void tile_apply_tc(float (*tile)[44], const float (*Qa)[44], int lane,
                                              float *__restrict__ p)
{
    const int g = lane >> 2, c = lane & 3;
    float d[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[mi][ni][e] = 0.f;
    auto a = [&](int m, int k) { return tile[m][k]; };   // A[position][old vector]
    auto b = [&](int k, int n) { return Qa[k][n]; };     // B[old vector][new vector]
#pragma unroll
    for (int ks = 0; ks < 32; ks += 8)
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma3(d[mi][ni], g, c, a, b, 16 * mi, 8 * ni, ks);
    __syncwarp();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int r0 = 16 * mi + g, c0 = 8 * ni + 2 * c;
            tile[r0][c0] = d[mi][ni][0];
            tile[r0][c0 + 1] = d[mi][ni][1];
            tile[r0 + 8][c0] = d[mi][ni][2];
            tile[r0 + 8][c0 + 1] = d[mi][ni][3];
        }
    __syncwarp();
    float4 *o4 = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < 8; ++i)
        o4[i] = make_float4(tile[4 * i][lane], tile[4 * i + 1][lane], tile[4 * i + 2][lane], tile[4 * i + 3][lane]);
}

// FP64: acc[q] += sum_t tile[t][lane] * tile[t][q]   (row t broadcast to the warp)
__device__ __forceinline__ void tile_gram(const double (*tile)[34], int lane, double (&acc)[32])
{
#pragma unroll 4
    for (int t = 0; t < 32; ++t) {
        const double o = tile[t][lane];
#pragma unroll
        for (int q = 0; q < 32; q += 2) {
            const double2 x = *reinterpret_cast<const double2 *>(&tile[t][q]);
            acc[q] = fma(o, x.x, acc[q]); acc[q + 1] = fma(o, x.y, acc[q + 1]);
        }
    }
}
// FP64: p[t] = sum_q qc[q] * tile[t][q] for the 32 positions, written in pieces of 8
__device__ __forceinline__ void tile_apply(const double (*tile)[34], const double (&qc)[32], double *__restrict__ p)
{
#pragma unroll 1
    for (int h = 0; h < 32; h += 8) {
        double out[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int q = 0; q < 32; q += 2) {
                const double2 x = *reinterpret_cast<const double2 *>(&tile[h + t][q]);
                a0 = fma(qc[q], x.x, a0); a1 = fma(qc[q + 1], x.y, a1);
            }
            out[t] = a0 + a1;
        }
        double2 *o2 = reinterpret_cast<double2 *>(p + h);
#pragma unroll
        for (int i = 0; i < 4; ++i) o2[i] = make_double2(out[2 * i], out[2 * i + 1]);
    }
}

__device__ __forceinline__ void team_bar(int team)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(kTeamWarps * 32) : "memory");
}

// vector index of local vector j (0..31) of block pair (bi, bj)
__device__ __forceinline__ int pair_vec(int bi, int bj, int j) { return j < kBlk ? bi * kBlk + j : bj * kBlk + j - kBlk; }

// round-robin (circle) pairing of n (even) items: pair k of round t
__device__ __forceinline__ void circle_pair(int n, int t, int k, int &p, int &q)
{
    if (k == 0) { p = n - 1; q = t; }
    else { p = (t + k) % (n - 1); q = (t - k + n - 1) % (n - 1); }
}

// ---------------------------------------------------------------------------
// QR preconditioning inside the CTA: [X | V] <- Q^T [X | V] with X = Q R
// (Householder reflectors on the vector index, panels of 16 columns of X).
// The Jacobi then rotates the rows of R, which converges in a third of the
// sweeps on graded spectra, and V starts from Q^T instead of the identity so
// that it still ends as the left factor.  The panel lives in the staging
// tiles; the reflectors go to Vr (rows x 16, workspace); T and the panel's
// small arrays go to the G/Q areas of team 0.
// ---------------------------------------------------------------------------
constexpr int kQB = 16;

template <typename T>
__device__ void cta_qr(GbjSmem<T> &S, T *__restrict__ X, T *__restrict__ V, T *__restrict__ Vr, int c, int l, int ldx,
                       int ldv)
{
    T *P = &S.tile[0][0][0];                 // panel: rows x bw
    T(*Tm)[33] = S.G[0];                     // compact-WY factor (16 x 16)
    T(*Gv)[33] = S.Q[0];                     // V^T V of the panel
    T *beta = &S.rc[0][0][0], *misc = &S.rs[0][0][0];
    T *wv = &S.rc[0][1][0];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kmax = c - 1 < l ? c - 1 : l;
    for (int k = 0; k < kmax; k += kQB) {
        const int bw = kmax - k < kQB ? kmax - k : kQB;
        const int rows = c - k;
        for (int e = tid; e < rows * bw; e += kBT) P[e] = X[(long long)(k + e / bw) * ldx + k + e % bw];
        for (int e = tid; e < rows * kQB; e += kBT) Vr[e] = (T)0;
        __syncthreads();
        for (int j = 0; j < bw; ++j) {
            // column norm in the working precision (FP64 is scarce on this part)
            T a = (T)0;
            for (int i = j + tid; i < rows; i += kBT) {
                const T x = P[i * bw + j];
                a = fma(x, x, a);
            }
            a = wsum(a);
            if (lane == 0) S.red[warp] = (double)a;
            __syncthreads();
            if (tid == 0) {
                T sacc = (T)0;
                for (int w = 0; w < kWarps; ++w) sacc += (T)S.red[w];
                a = sacc;
                const T x0 = P[j * bw + j];
                const T nrm = sqrt(a);
                T b = (T)0, v0 = (T)1, alpha = x0;
                if (rows - j > 1 && nrm > (T)0 && a > x0 * x0) {
                    alpha = x0 >= (T)0 ? -nrm : nrm;
                    v0 = x0 - alpha;
                    b = (T)-1 / (alpha * v0);          // 2 / (v^T v)
                }
                beta[j] = b;
                misc[0] = v0;
                misc[1] = alpha;
            }
            __syncthreads();
            const T b = beta[j], v0 = misc[0];
            for (int i = j + tid; i < rows; i += kBT) Vr[(long long)i * kQB + j] = i == j ? v0 : P[i * bw + j];
            if (b != (T)0) {
                for (int q = j + 1 + warp; q < bw; q += kWarps) {
                    T sacc = (T)0;
                    for (int i = j + lane; i < rows; i += 32) sacc = fma(i == j ? v0 : P[i * bw + j], P[i * bw + q], sacc);
                    sacc = wsum(sacc);
                    if (lane == 0) wv[q] = sacc;
                }
                __syncthreads();
                const int nq = bw - j - 1;
                for (int e = tid; e < (rows - j) * nq; e += kBT) {
                    const int i = j + e / nq, q = j + 1 + e % nq;
                    const T vi = i == j ? v0 : P[i * bw + j];
                    P[i * bw + q] -= b * vi * wv[q];
                }
            }
            __syncthreads();
            const T alpha = misc[1];
            for (int i = j + tid; i < rows; i += kBT) P[i * bw + j] = (i == j) ? alpha : (T)0;
            __syncthreads();
        }
        for (int e = tid; e < rows * bw; e += kBT) X[(long long)(k + e / bw) * ldx + k + e % bw] = P[e];
        // Gram of the reflectors, then T (H_0 ... H_{bw-1} = I - V T V^T)
        for (int pq = warp; pq < bw * bw; pq += kWarps) {
            const int pp = pq / bw, qq = pq % bw;
            if (pp >= qq) continue;
            T sacc = (T)0;
            for (int i = qq + lane; i < rows; i += 32) sacc = fma(Vr[(long long)i * kQB + pp], Vr[(long long)i * kQB + qq], sacc);
            sacc = wsum(sacc);
            if (lane == 0) Gv[pp][qq] = sacc;
        }
        __syncthreads();
        if (tid == 0) {
            for (int pp = 0; pp < kQB; ++pp)
                for (int qq = 0; qq < kQB; ++qq) Tm[pp][qq] = (T)0;
            for (int j = 0; j < bw; ++j) {
                Tm[j][j] = beta[j];
                for (int pp = 0; pp < j; ++pp) {
                    T sacc = (T)0;
                    for (int qq = pp; qq < j; ++qq) sacc = fma(Tm[pp][qq], Gv[qq][j], sacc);
                    Tm[pp][j] = -beta[j] * sacc;
                }
            }
        }
        __syncthreads();
        // trailing columns: X[k:, k+bw:ldx) and all of V[k:, 0:ldv), 32 per warp-group
        const int nx = ldx - (k + bw), ntot = nx + ldv;
        for (int g0 = warp * 32; g0 < ntot; g0 += kWarps * 32) {
            const int u = g0 + lane;
            T *col = nullptr;
            long long ld = 0;
            if (u < nx) { col = X + k + bw + u; ld = ldx; }
            else if (u < ntot) { col = V + (u - nx); ld = ldv; }
            T w[kQB];
#pragma unroll
            for (int j = 0; j < kQB; ++j) w[j] = (T)0;
            if (col)
                for (int i = 0; i < rows; ++i) {
                    const T x = col[(long long)(k + i) * ld];
                    const T *vi = Vr + (long long)i * kQB;
#pragma unroll
                    for (int j = 0; j < kQB; ++j) w[j] = fma(vi[j], x, w[j]);
                }
            T z[kQB];
#pragma unroll
            for (int j = 0; j < kQB; ++j) {
                T sacc = (T)0;
#pragma unroll
                for (int t2 = 0; t2 <= j; ++t2) sacc = fma(Tm[t2][j], w[t2], sacc);
                z[j] = sacc;
            }
            if (col)
                for (int i = 0; i < rows; ++i) {
                    const T *vi = Vr + (long long)i * kQB;
                    T sacc = (T)0;
#pragma unroll
                    for (int j = 0; j < kQB; ++j) sacc = fma(vi[j], z[j], sacc);
                    col[(long long)(k + i) * ld] -= sacc;
                }
        }
        __syncthreads();
    }
}

// One block pair (bi, bj) of a round, processed by the calling team of four
// warps: Gram partials over the team's tiles, team-parallel cyclic Jacobi on
// the 32 x 32 Gram matrix, the rotation applied to the 32 vectors (and to V
// when ntv > 0).  The number of first-inner-sweep rotations goes to
// *rot_counter (shared or global memory).
template <typename T>
__device__ __forceinline__ void gbj_pair(GbjSmem<T> &S, T *__restrict__ X, T *__restrict__ V, int ldx, int ldv,
                                         int ntx, int ntv, int bi, int bj, T floor2T, T tolT, int max_inner,
                                         int do_ns, unsigned *rot_counter)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int team = warp / kTeamWarps, tw = warp % kTeamWarps;
                const int vj = pair_vec(bi, bj, lane);
                // 1. Gram partial over this warp's tiles of positions
                if constexpr (sizeof(T) == 4) {
                    float acc[2][4][4];
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
                    for (int tt = tw; tt < ntx; tt += kTeamWarps) {
                        stage32(X + (long long)vj * ldx + tt * 32, S.tile[warp], lane);
                        __syncwarp();
                        tile_gram_tc(S.tile[warp], lane, acc);
                        __syncwarp();
                    }
                    const int g = lane >> 2, c = lane & 3;
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 4; ++ni) {
                            const int r0 = 16 * mi + g, c0 = 8 * ni + 2 * c;
                            S.tile[warp][r0][c0] = acc[mi][ni][0];
                            S.tile[warp][r0][c0 + 1] = acc[mi][ni][1];
                            S.tile[warp][r0 + 8][c0] = acc[mi][ni][2];
                            S.tile[warp][r0 + 8][c0 + 1] = acc[mi][ni][3];
                        }
                } else {
                    T acc[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc[q] = (T)0;
                    for (int tt = tw; tt < ntx; tt += kTeamWarps) {
                        stage32(X + (long long)vj * ldx + tt * 32, S.tile[warp], lane);
                        __syncwarp();
                        tile_gram(S.tile[warp], lane, acc);
                        __syncwarp();
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q) S.tile[warp][q][lane] = acc[q];
                }
                team_bar(team);
                // 2. the team: reduce the partials, diagonalise G with cyclic
                // Jacobi (16 disjoint rotations per step, rows then columns),
                // accumulate Q
                {
                    T(*G)[33] = S.G[team];
                    T(*Qm)[33] = S.Q[team];
                    const int tt = tw * 32 + lane;            // 0..127 within the team
                    const int w0 = team * kTeamWarps;
                    for (int e = tt; e < 32 * 32; e += kTeamWarps * 32) {
                        const int q = e >> 5, j = e & 31;
                        T g = S.tile[w0][q][j];
#pragma unroll
                        for (int w = 1; w < kTeamWarps; ++w) g += S.tile[w0 + w][q][j];
                        G[q][j] = g;
                        Qm[q][j] = (q == j) ? (T)1 : (T)0;
                    }
                    team_bar(team);
                    int first = 0, any = 0;
                    int gstep = 0;   // running step count: consecutive steps use alternate buffers,
                                     // including across inner sweeps (31 steps per sweep is odd)
                    for (int isw = 0; isw < max_inner; ++isw) {
                        int nrot = 0;
                        for (int st = 0; st < 31; ++st, ++gstep) {
                            const int buf = gstep & 1;
                            if (tw == 0) {
                                bool rot = false;
                                if (lane < 16) {
                                    int p, q;
                                    circle_pair(32, st, lane, p, q);
                                    const T a = G[p][p], b = G[q][q], g = G[p][q];
                                    // |g| > tol sqrt(a b), both norms above the floor (in T:
                                    // FP64 arithmetic is scarce on this part)
                                    rot = a > floor2T && b > floor2T && fabs(g) > tolT * sqrt(a) * sqrt(b);
                                    T c = (T)1, sn = (T)0;
                                    if (rot) {
                                        const T zeta = (b - a) / (T(2) * g);
                                        const T t = (zeta >= T(0) ? T(1) : T(-1)) /
                                                    (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                                        c = T(1) / sqrt(T(1) + t * t);
                                        sn = c * t;
                                    }
                                    S.rc[team][buf][lane] = c; S.rs[team][buf][lane] = sn;
                                    S.rp[team][buf][lane] = p; S.rq[team][buf][lane] = q;
                                }
                                const unsigned msk = __ballot_sync(0xffffffffu, rot);
                                if (lane == 0) S.rmask[team][buf] = msk;
                            }
                            team_bar(team);
                            const unsigned msk = S.rmask[team][buf];
                            if (msk == 0u) continue;                 // uniform over the team
                            nrot += __popc(msk);
                            // rows p, q of G: element (pair kk, column j)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int e = tt + 128 * i, kk = e >> 5, j = e & 31;
                                if ((msk >> kk) & 1u) {
                                    const int p = S.rp[team][buf][kk], q = S.rq[team][buf][kk];
                                    const T c = S.rc[team][buf][kk], sn = S.rs[team][buf][kk];
                                    const T x = G[p][j], y = G[q][j];
                                    G[p][j] = c * x - sn * y;
                                    G[q][j] = sn * x + c * y;
                                }
                            }
                            team_bar(team);
                            // columns p, q of G and Q: element (pair kk, row j)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int e = tt + 128 * i, kk = e >> 5, j = e & 31;
                                if ((msk >> kk) & 1u) {
                                    const int p = S.rp[team][buf][kk], q = S.rq[team][buf][kk];
                                    const T c = S.rc[team][buf][kk], sn = S.rs[team][buf][kk];
                                    const T x = G[j][p], y = G[j][q];
                                    G[j][p] = c * x - sn * y;
                                    G[j][q] = sn * x + c * y;
                                    const T u = Qm[j][p], w = Qm[j][q];
                                    Qm[j][p] = c * u - sn * w;
                                    Qm[j][q] = sn * u + c * w;
                                }
                            }
                            team_bar(team);
                        }
                        if (isw == 0) first = nrot;
                        any += nrot;
                        if (nrot == 0) break;
                    }
                    if (sizeof(T) == 4 && any && do_ns) {
                        // Q holds up to max_inner x 31 FP32 rotations per column:
                        // one Newton-Schulz step Q <- Q (3 I - Q^T Q) / 2 brings it
                        // back to orthogonal at FP32 rounding before it is applied.
                        // N = (3 I - Q^T Q) / 2 goes to G (no longer needed).
                        T nv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int e = tt + 128 * i, r0 = e >> 5, c0 = e & 31;
                            T a = (T)0;
#pragma unroll 8
                            for (int k2 = 0; k2 < 32; ++k2) a = fma(Qm[k2][r0], Qm[k2][c0], a);
                            nv[i] = (r0 == c0 ? T(1.5) : T(0)) - T(0.5) * a;
                        }
                        team_bar(team);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int e = tt + 128 * i;
                            G[e >> 5][e & 31] = nv[i];
                        }
                        team_bar(team);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int e = tt + 128 * i, r0 = e >> 5, c0 = e & 31;
                            T a = (T)0;
#pragma unroll 8
                            for (int k2 = 0; k2 < 32; ++k2) a = fma(Qm[r0][k2], G[k2][c0], a);
                            nv[i] = a;
                        }
                        team_bar(team);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int e = tt + 128 * i;
                            Qm[e >> 5][e & 31] = nv[i];
                        }
                    }
                    if constexpr (sizeof(T) == 4) {
                        if (any) {
                            team_bar(team);
                            for (int e = tt; e < 32 * 32; e += kTeamWarps * 32) S.Qa[team][e >> 5][e & 31] = Qm[e >> 5][e & 31];
                        }
                    }
                    if (tt == 0) {
                        S.team_rot[team] = any;
                        if (first) atomicAdd(rot_counter, (unsigned)first);
                    }
                }
                team_bar(team);
                // 3. W <- W Q and V <- V Q (skipped when nothing rotated)
                if (S.team_rot[team]) {
                    if constexpr (sizeof(T) == 4) {
                        for (int tt = tw; tt < ntx + ntv; tt += kTeamWarps) {
                            T *base = tt < ntx ? X + (long long)vj * ldx + tt * 32
                                               : V + (long long)vj * ldv + (tt - ntx) * 32;
                            stage32(base, S.tile[warp], lane);
                            __syncwarp();
                            tile_apply_tc(S.tile[warp], S.Qa[team], lane, base);
                            __syncwarp();
                        }
                    } else {
                        T qc[32];
#pragma unroll
                        for (int q = 0; q < 32; ++q) qc[q] = S.Q[team][q][lane];
                        for (int tt = tw; tt < ntx + ntv; tt += kTeamWarps) {
                            T *base = tt < ntx ? X + (long long)vj * ldx + tt * 32
                                               : V + (long long)vj * ldv + (tt - ntx) * 32;
                            stage32(base, S.tile[warp], lane);
                            __syncwarp();
                            tile_apply(S.tile[warp], qc, base);
                            __syncwarp();
                        }
                    }
                }
}

template <typename T>
__global__ void __launch_bounds__(kBT) k_svd_batched(const BDesc *__restrict__ desc, const double *__restrict__ theta,
                                                    T *__restrict__ work, double *__restrict__ U,
                                                    double *__restrict__ s, double *__restrict__ Vt, int max_sweeps,
                                                    int max_inner, int do_ns, int do_qr, double tol_unit,
                                                    int tol_by_l, double small, int *info, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GbjSmem<T> &S = *reinterpret_cast<GbjSmem<T> *>(smem_raw);
    if (threadIdx.x == 0) S.d = desc[blockIdx.x];
    __syncthreads();
    const BDesc &d = S.d;
    const int m = d.m, n = d.n, r = d.r, l = d.l, tr = d.tr, nb = d.nb, ldx = d.ldx, ldv = d.ldv;
    T *X = work + d.off_X, *V = work + d.off_V;
    const double *A = theta + d.off_in;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int team = warp / kTeamWarps;
    const int rpad = nb * kBlk;
    // rotate while a cosine exceeds l eps (FP64) or 1e-5 (FP32)
    const double tol = tol_by_l ? tol_unit * (double)(l > 16 ? l : 16) : tol_unit;

    // load: X[i][t] = vector i (column i of A when tr = 0, row i when tr = 1),
    // zero padded to rpad x ldx; V = identity on the first r vectors
    double f2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)rpad * ldx; e += kBT) {
        const int i = (int)(e / ldx), t = (int)(e % ldx);
        double v = 0.0;
        if (i < r && t < l) v = tr ? A[(long long)i * n + t] : A[(long long)t * n + i];
        X[e] = (T)v;
        f2 += v * v;
    }
    for (long long e = threadIdx.x; e < (long long)rpad * ldv; e += kBT) {
        const int i = (int)(e / ldv), k = (int)(e % ldv);
        V[e] = (i == k && i < r) ? (T)1 : (T)0;
    }
    f2 = block_sum(f2, S.red);
    const double floor2 = small * small * f2;
    const T floor2T = (T)floor2, tolT = (T)tol;
    __syncthreads();
    if (do_qr && r >= 32 && (long long)r * kQB <= (long long)kWarps * 32 * TileStride<T>::v)
        cta_qr(S, X, V, work + d.off_R, r, l, ldx, ldv);

    int sweep = 0;
    bool converged = false;
    const int npairs = nb / 2, ntx = ldx / 32, ntv = ldv / 32;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) S.rot_count = 0u;
        __syncthreads();
        for (int rnd = 0; rnd < nb - 1; ++rnd) {
            for (int k = team; k < npairs; k += kTeams) {
                int bi, bj;
                circle_pair(nb, rnd, k, bi, bj);
                gbj_pair(S, X, V, ldx, ldv, ntx, ntv, bi, bj, floor2T, tolT, max_inner, do_ns, &S.rot_count);
            }
            __syncthreads();
        }
        const unsigned tot = S.rot_count;
        __syncthreads();
        if (tot == 0u) {
            converged = true;
            ++sweep;
            break;
        }
    }
    if (threadIdx.x == 0) {
        info[d.idx] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
    // norms into the s slot (unsorted), then rank and write the factors
    double *sb = s + d.off_s;
    for (int i = warp; i < r; i += kWarps) {
        const T *x = X + (long long)i * ldx;
        double a = 0.0;
        for (int k = lane; k < l; k += 32) a = fma((double)x[k], (double)x[k], a);
        a = wsum(a);
        if (lane == 0) sb[i] = sqrt(a);
    }
    __syncthreads();
    // rank by counting (descending, ties by index), one thread per vector
    int *perm = reinterpret_cast<int *>(work + d.off_P);
    double *tmp = reinterpret_cast<double *>(perm + ((r + 1) & ~1));
    for (int i = threadIdx.x; i < r; i += kBT) {
        const double v = sb[i];
        int rank = 0;
        for (int j = 0; j < r; ++j) {
            const double w = sb[j];
            rank += (w > v) || (w == v && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    double *Ub = U + d.off_U, *Vb = Vt + d.off_Vt;
    // one warp per output index: sign convention "largest |U[:, c]| positive"
    for (int c = warp; c < r; c += kWarps) {
        const int i = perm[c];
        const double sig = sb[i];
        const double inv = sig > 0.0 ? 1.0 / sig : 0.0;
        const T *usrc = tr ? (V + (long long)i * ldv) : (X + (long long)i * ldx);
        const double usc = tr ? 1.0 : inv;
        double best = -1.0;
        int bi = 0;
        for (int k = lane; k < m; k += 32) {
            const double a = fabs((double)usrc[k]);
            if (a > best) { best = a; bi = k; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const double sign = ((double)usrc[bi] < 0.0) ? -1.0 : 1.0;
        for (int k = lane; k < m; k += 32) Ub[(long long)k * r + c] = sign * usc * (double)usrc[k];
        const T *vsrc = tr ? (X + (long long)i * ldx) : (V + (long long)i * ldv);
        const double vsc = tr ? inv : 1.0;
        for (int k = lane; k < n; k += 32) Vb[(long long)c * n + k] = sign * vsc * (double)vsrc[k];
    }
    __syncthreads();
    // sorted singular values back into the s slot
    for (int c = threadIdx.x; c < r; c += kBT) tmp[c] = sb[perm[c]];
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += kBT) sb[c] = tmp[c];
}

// One matrix on many CTAs (cooperative launch): the block pairs of each
// round are spread over all teams of the grid, with a grid barrier between
// rounds.  FP32 vectors only (the mixed form's isometry; the other factor is
// a projection, so no V).  X: rpad x ldx (zero padded), rotated in place.
// sync: [0..1] barrier words, [2..3] rotation counters by sweep parity.
__global__ void __launch_bounds__(kBT) k_gbj32_coop(float *__restrict__ X, int nb, int ldx, int l, int max_sweeps,
                                                   double tol, const double *__restrict__ F2, double small,
                                                   unsigned *sync, int *status, int *info, int max_inner)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GbjSmem<float> &S = *reinterpret_cast<GbjSmem<float> *>(smem_raw);
    const int warp = threadIdx.x >> 5, team = warp / kTeamWarps;
    unsigned *barrier = sync, *rotc = sync + 2;
    const float floor2T = (float)(small * small * F2[0]);
    const float tolT = (float)tol;
    const int npairs = nb / 2, ntx = ldx / 32;
    const int gteam = blockIdx.x * kTeams + team, nteams = gridDim.x * kTeams;
    (void)l;
    int sweep = 0;
    bool converged = false;
    for (; sweep < max_sweeps; ++sweep) {
        for (int rnd = 0; rnd < nb - 1; ++rnd) {
            for (int k = gteam; k < npairs; k += nteams) {
                int bi, bj;
                circle_pair(nb, rnd, k, bi, bj);
                gbj_pair<float>(S, X, nullptr, ldx, 0, ntx, 0, bi, bj, floor2T, tolT, max_inner, 1,
                                &rotc[sweep & 1]);
            }
            if (!grid_barrier(barrier, status)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
                return;
            }
        }
        const unsigned total = *(volatile unsigned *)&rotc[sweep & 1];
        if (blockIdx.x == 0 && threadIdx.x == 0) rotc[(sweep + 1) & 1] = 0u;
        if (total == 0u) {
            converged = true;
            ++sweep;
            break;
        }
        if (!grid_barrier(barrier, status)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) info[0] = -(sweep + 1);
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = converged ? sweep : -sweep;
        if (!converged) atomicOr(status, ST_NOCONV);
    }
}

// A: m x n row-major FP64; vectors = columns (dir 0, r = n, l = m) or rows
// (dir 1, r = m, l = n) -> Xp (rpad x ldx FP32, zero padded); clears sync[0..3]
__global__ void k_load_padded32(const double *__restrict__ A, int m, int n, int dir, int r, int l, int rpad, int ldx,
                                float *__restrict__ Xp, unsigned *sync)
{
    const long long total = (long long)rpad * ldx;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldx), t = (int)(e % ldx);
        float v = 0.f;
        if (i < r && t < l) v = (float)(dir == 0 ? A[(long long)t * n + i] : A[(long long)i * n + t]);
        Xp[e] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) sync[threadIdx.x] = 0u;
}

// Xp (rpad x ldx) -> X (r x l), dropping the padding
__global__ void k_unpad32(const float *__restrict__ Xp, int r, int l, int ldx, float *__restrict__ X)
{
    const long long total = (long long)r * l;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        X[e] = Xp[(long long)(e / l) * ldx + e % l];
}

// entropy, truncation error and k for every matrix (one CTA each)
// (rank floor: floor_unit * r * s_0 when floor_by_r, else floor_unit * s_0)
__global__ void k_decide_batched(const BDesc *__restrict__ desc, const double *__restrict__ s, int chi_max, double eps,
                                 double floor_unit, int floor_by_r, int *k_out, double *S_out, double *err_out)
{
    __shared__ double sh[32];
    const BDesc d = desc[blockIdx.x];
    const double *sb = s + d.off_s;
    const int r = d.r;
    double z = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x) z += sb[j] * sb[j];
    const double Z = block_sum(z, sh);
    double en = 0.0, cr = 0.0, ca = 0.0;
    const double rank_floor = floor_by_r ? floor_unit * (double)r : floor_unit;
    const double nz = sqrt(Z), rtol = rank_floor * (r > 0 ? sb[0] : 0.0);
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double pj = Z > 0.0 ? sb[j] * sb[j] / Z : 0.0;
        if (pj > 0.0) en -= pj * log(pj);
        if (sb[j] > rtol) cr += 1.0;
        if (nz > 0.0 && sb[j] / nz > eps) ca += 1.0;
    }
    const double S = block_sum(en, sh);
    const int rank = (int)block_sum(cr, sh), above = (int)block_sum(ca, sh);
    int k = chi_max;
    if (rank < k) k = rank;
    if (above < k) k = above;
    if (k < 1) k = 1;
    double t = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x)
        if (j >= k) t += Z > 0.0 ? sb[j] * sb[j] / Z : 0.0;
    const double T = block_sum(t, sh);
    if (threadIdx.x == 0) {
        k_out[d.idx] = k;
        S_out[d.idx] = S;
        err_out[d.idx] = sqrt(fmax(T, 0.0));
    }
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

int grid1d_batched(long long n, int num_sms)
{
    long long b = (n + 255) / 256;
    if (b > (long long)num_sms * 8) b = (long long)num_sms * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace dmrg

using namespace dmrg;

namespace dmrg {

size_t gbj32_padded_bytes(int r, int l)
{
    int nb = (r + kBlk - 1) / kBlk;
    nb += nb & 1;
    const size_t ldx = (size_t)((l + 31) & ~31);
    return (((size_t)nb * kBlk * ldx * sizeof(float)) + 255) & ~size_t(255);
}

// FP32 one-sided Jacobi of the r vectors of A (columns for dir 0, rows for
// dir 1) in Gram-block form on a cooperative grid, QR-preconditioned when the
// context asks; the rotated vectors end in X (r x l).  Xp is the padded
// scratch (gbj32_padded_bytes), qrw the QR scratch, sync the barrier/counter
// words with F2 = |A|_F^2 written at sync + 4.
dmrg_status gbj32_sweeps(dmrg_ctx *ctx, const double *A, int m, int n, int dir, float *X, float *Xp, void *qrw,
                         unsigned *sync, int max_sweeps, double tol, double small, int *d_info)
{
    const int r = dir == 0 ? n : m, l = dir == 0 ? m : n;
    int nb = (r + kBlk - 1) / kBlk;
    nb += nb & 1;
    const int rpad = nb * kBlk, ldx = (l + 31) & ~31;
    cudaStream_t st = ctx->stream;
    k_load_padded32<<<grid1d_batched((long long)rpad * ldx, ctx->num_sms), 256, 0, st>>>(A, m, n, dir, r, l, rpad, ldx,
                                                                                         Xp, sync); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    if (ctx->jacobi_qr && r >= 32) {
        dmrg_status e = qr_precondition32(ctx, Xp, r, ldx, qrw);
        if (e != DMRG_OK && e != DMRG_EUNSUPPORTED) return e;
    }
    double *F2 = reinterpret_cast<double *>(sync + 4);
    DMRG_TRY(frob2_f32(ctx, Xp, (long long)rpad * ldx, F2));
    static bool attr = false;
    if (!attr) {
        DMRG_CUDA(cudaFuncSetAttribute(k_gbj32_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(GbjSmem<float>)));
        attr = true;
    }
    int per_sm = 0;
    DMRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gbj32_coop, kBT, sizeof(GbjSmem<float>)));
    if (per_sm < 1) return DMRG_EUNSUPPORTED;
    const int npairs = nb / 2;
    int blocks = (npairs + kTeams - 1) / kTeams;
    blocks = std::max(1, std::min(blocks, per_sm * ctx->num_sms));
    int *status = ctx->d_status;
    int max_inner = ctx->batched_inner;
    const double *F2c = F2;
    void *args[] = {&Xp, (void *)&nb, (void *)&ldx, (void *)&l, &max_sweeps, (void *)&tol, (void *)&F2c,
                    (void *)&small, &sync, &status, &d_info, &max_inner};
    DMRG_CUDA(cudaLaunchCooperativeKernel((const void *)k_gbj32_coop, dim3(blocks), dim3(kBT), args,
                                          sizeof(GbjSmem<float>), st)); DMRG_COUNT_LAUNCH();
    k_unpad32<<<grid1d_batched((long long)r * l, ctx->num_sms), 256, 0, st>>>(Xp, r, l, ldx, X); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // namespace dmrg

extern "C" dmrg_status svd_truncate_batched(dmrg_ctx *ctx, int prec, int batch, const int *m, const int *n,
                                            const double *theta_dev, const long long *off_in, double *U_dev,
                                            const long long *off_U, double *s_dev, const long long *off_s,
                                            double *Vt_dev, const long long *off_Vt, int chi_max, double eps,
                                            int *k_dev, double *S_dev, double *err_dev, int *sweeps_dev)
{
    if (!ctx || batch < 1 || !m || !n || !theta_dev || !off_in || !U_dev || !off_U || !s_dev || !off_s || !Vt_dev ||
        !off_Vt || chi_max < 1 || !(eps >= 0.0) || !k_dev || !S_dev || !err_dev)
        return DMRG_EINVAL;
    if (prec != DMRG_PREC_FP64 && prec != DMRG_PREC_3XTF32) return DMRG_EUNSUPPORTED;
    const size_t esz = prec == DMRG_PREC_FP64 ? sizeof(double) : sizeof(float);
    std::vector<BDesc> h(batch);
    std::vector<double> cost(batch);
    long long wo = 0;
    auto take = [&](size_t bytes) {   // element offset of a 256-byte aligned region
        const long long o = wo;
        wo += (long long)(al256(bytes) / esz);
        return o;
    };
    for (int b = 0; b < batch; ++b) {
        if (m[b] < 1 || n[b] < 1) return DMRG_EINVAL;
        BDesc &d = h[b];
        d.m = m[b];
        d.n = n[b];
        d.tr = m[b] < n[b];
        d.r = std::min(m[b], n[b]);
        d.l = std::max(m[b], n[b]);
        d.nb = (d.r + kBlk - 1) / kBlk;
        d.nb += d.nb & 1;
        d.ldx = (d.l + 31) & ~31;
        d.ldv = (d.r + 31) & ~31;
        d.idx = b;
        d.pad = 0;
        d.off_in = off_in[b];
        d.off_U = off_U[b];
        d.off_s = off_s[b];
        d.off_Vt = off_Vt[b];
        const long long rpad = (long long)d.nb * kBlk;
        d.off_X = take(esz * rpad * d.ldx);
        d.off_V = take(esz * rpad * d.ldv);
        d.off_P = take(sizeof(int) * (d.r + 2) + sizeof(double) * d.r + 16);
        d.off_R = take(esz * (size_t)d.r * kQB);
        cost[b] = (double)rpad * rpad * (double)(d.ldx + d.ldv);
    }
    // largest problems first, so that the CTAs that run longest start first
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    {
        std::vector<BDesc> sorted(batch);
        for (int b = 0; b < batch; ++b) sorted[b] = h[order[b]];
        h.swap(sorted);
    }
    const size_t need_desc = al256(sizeof(BDesc) * batch), need_info = al256(sizeof(int) * batch);
    const size_t need = need_desc + need_info + esz * (size_t)wo;
    DMRG_TRY(ctx->work4.ensure(need));
    if ((size_t)batch * sizeof(BDesc) > ctx->pinned_desc_bytes) {
        if (ctx->pinned_desc) cudaFreeHost(ctx->pinned_desc);
        ctx->pinned_desc = nullptr;
        ctx->pinned_desc_bytes = 0;
        DMRG_CUDA(cudaMallocHost(&ctx->pinned_desc, sizeof(BDesc) * batch));
        ctx->pinned_desc_bytes = sizeof(BDesc) * batch;
    }
    std::memcpy(ctx->pinned_desc, h.data(), sizeof(BDesc) * batch);
    char *base = ctx->work4.as<char>();
    BDesc *ddesc = reinterpret_cast<BDesc *>(base);
    int *info = sweeps_dev ? sweeps_dev : reinterpret_cast<int *>(base + need_desc);
    void *work = base + need_desc + need_info;
    DMRG_CUDA(cudaMemcpyAsync(ddesc, ctx->pinned_desc, sizeof(BDesc) * batch, cudaMemcpyHostToDevice, ctx->stream));
    const int sweeps = ctx->jacobi_max_sweeps;
    const int inner = ctx->batched_inner;
    // descriptors are in cost order; results go to each matrix's own index (BDesc::idx)
    if (prec == DMRG_PREC_FP64) {
        static bool attr = false;
        if (!attr) {
            DMRG_CUDA(cudaFuncSetAttribute(k_svd_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(GbjSmem<double>)));
            attr = true;
        }
        k_svd_batched<double><<<batch, kBT, sizeof(GbjSmem<double>), ctx->stream>>>(
            ddesc, theta_dev, static_cast<double *>(work), U_dev, s_dev, Vt_dev, sweeps, inner, 0, ctx->jacobi_qr,
            2.220446049250313e-16, 1, 16.0 * 2.220446049250313e-16, info, ctx->d_status); DMRG_COUNT_LAUNCH();
        k_decide_batched<<<batch, 256, 0, ctx->stream>>>(ddesc, s_dev, chi_max, eps, 2.220446049250313e-16, 1,
                                                         k_dev, S_dev, err_dev); DMRG_COUNT_LAUNCH();
    } else {
        static bool attr = false;
        if (!attr) {
            DMRG_CUDA(cudaFuncSetAttribute(k_svd_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(GbjSmem<float>)));
            attr = true;
        }
        k_svd_batched<float><<<batch, kBT, sizeof(GbjSmem<float>), ctx->stream>>>(
            ddesc, theta_dev, static_cast<float *>(work), U_dev, s_dev, Vt_dev, sweeps, inner, ctx->batched_ns, ctx->jacobi_qr, 1e-5, 0,
            ctx->batched_floor32, info, ctx->d_status); DMRG_COUNT_LAUNCH();
        k_decide_batched<<<batch, 256, 0, ctx->stream>>>(ddesc, s_dev, chi_max, eps, 2.384185791015625e-07, 0,
                                                         k_dev, S_dev, err_dev); DMRG_COUNT_LAUNCH();
    }
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_begin(dmrg_ctx *ctx)
{
    if (!ctx || !ctx->stream) return DMRG_EINVAL;   // the legacy default stream cannot be captured
    DMRG_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_end(dmrg_ctx *ctx, void **graph_exec)
{
    if (!ctx || !graph_exec) return DMRG_EINVAL;
    cudaGraph_t g = nullptr;
    DMRG_CUDA(cudaStreamEndCapture(ctx->stream, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return DMRG_ECUDA;
    *graph_exec = ex;
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_launch(dmrg_ctx *ctx, void *graph_exec)
{
    if (!ctx || !graph_exec) return DMRG_EINVAL;
    DMRG_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), ctx->stream));
    return DMRG_OK;
}

extern "C" dmrg_status dmrg_graph_destroy(void *graph_exec)
{
    if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
    return DMRG_OK;
}
