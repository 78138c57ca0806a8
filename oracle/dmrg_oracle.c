/*
 * dmrg_oracle.c -- plain, slow, FP64 CPU oracle for the adaptive two-site
 * DMRG local update of arXiv 2604.03960 ("Adaptive Tensor Network Simulation
 * via Entropy-Feedback PID Control and GPU-Accelerated SVD").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header or constant table with the
 * CUDA library.
 *
 * Every routine is written from the mathematical definition in the paper (or,
 * where the paper is silent, from a textbook definition named in place) with
 * plain loops and no blocking or fusion.  Compile with -ffp-contract=off so
 * that a*b+c is never fused: the controller's integer output must be
 * reproducible bit for bit.
 *
 * Conventions (0-based):
 *   W[i][wl][wr][s][sp]   MPO of site i, s = bra (row) index, sp = ket index.
 *   A[i][a][s][b]         MPS site tensor, chi[i] x d x chi[i+1].
 *   L[k][w][a'][a]        left environment of sites 0..k-1 (a' bra, a ket).
 *   R[k][w][b'][b]        right environment of sites k..N-1.
 *   theta[a][s1][s2][b]   two-site tensor of bond k (sites k, k+1).
 *   Boundary vectors: L[0][w] = delta(w, D-1), R[N][w] = delta(w, 0).
 *
 * Functions that no independent pin covers say "parity unpinned" here:
 *   none at present (see the tests for the pin of each routine).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <fenv.h>

#define REF_OK 0
#define REF_EINVAL 1
#define REF_ENOMEM 2
#define REF_ENOCONV 3

/* ------------------------------------------------------------------------ */
/* Parameters (mirrors the meaning of the library's parameter block; this is
 * the oracle's own declaration).                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alpha_ema;   /* EMA smoothing, Eq. (8)                            */
    double gamma;       /* margin factor of the direct map, Eq. (7)          */
    double S_target;    /* target entropy, Eq. (9)                           */
    double Kp, Ki, Kd;  /* PID gains, Eq. (10) / Algorithm 2                 */
    double beta;        /* predictor aggressiveness, Eq. (16)                */
    double eps_trunc;   /* singular-value threshold on the normalised spectrum */
    double eps_conv;    /* sweep convergence |dE/E|                          */
    int chi_min, chi_max;
    int lanczos_steps;
    int max_sweeps;
    int jacobi_max_sweeps;
    int prec;           /* ignored by the oracle (always FP64)               */
    int ctrl;           /* 0 PID, 1 DIRECT, 2 FIXED, 3 THRESHOLD, 4 MLP       */
    int ema_init_zero;  /* 1: first EMA value is alpha*S instead of S        */
    int multiplet_guard;/* 1: never cut inside a group of equal s            */
    int pid_steps_per_sweep; /* 2: one controller step per bond visit; 1: only L->R visits */
    int chi_init;       /* initial bond dimension of the random MPS          */
    int chi_fixed;      /* bond dimension for ctrl == FIXED                  */
    int second_order;   /* 1: add the curvature term of the second-order predictor */
} ref_params;

enum { CTRL_PID = 0, CTRL_DIRECT = 1, CTRL_FIXED = 2, CTRL_THRESHOLD = 3, CTRL_MLP = 4, CTRL_GLOBAL = 5 };

/* Per-bond controller state (Algorithm 2 requirements plus the predictor's
 * previous EMA value and the MLP's window of EMA values).                   */
typedef struct {
    double Sbar;        /* EMA-smoothed entropy  S-bar_i(t)                   */
    double Sbar_prev;   /* S-bar_i(t-1)                                       */
    double Sbar_prev2;  /* S-bar_i(t-2) (second-order predictor)              */
    double e_prev;      /* e_i(t-1)                                           */
    double I;           /* integral accumulator I_i                           */
    double hist[8];     /* last 8 EMA values, oldest first (MLP features)     */
    int chi;            /* chi_i(t)                                           */
    int initialized;
    int nhist;
    int pad;
} ref_ctrl_state;

/* ------------------------------------------------------------------------ */
/* Spin-1/2 operators, basis index 0 = up (+1/2), 1 = down (-1/2).           */
/* ------------------------------------------------------------------------ */
static void op_identity(double o[4]) { o[0] = 1; o[1] = 0; o[2] = 0; o[3] = 1; }
static void op_sz(double o[4])       { o[0] = 0.5; o[1] = 0; o[2] = 0; o[3] = -0.5; }
static void op_splus(double o[4])    { o[0] = 0; o[1] = 1; o[2] = 0; o[3] = 0; }  /* |up><down| */
static void op_sminus(double o[4])   { o[0] = 0; o[1] = 0; o[2] = 1; o[3] = 0; }  /* |down><up| */
static void op_pauli_z(double o[4])  { o[0] = 1; o[1] = 0; o[2] = 0; o[3] = -1; }
static void op_pauli_x(double o[4])  { o[0] = 0; o[1] = 1; o[2] = 1; o[3] = 0; }

static void mpo_set(double *Wsite, int D, int wl, int wr, const double op[4], double c)
{
    for (int s = 0; s < 2; ++s)
        for (int sp = 0; sp < 2; ++sp)
            Wsite[(((size_t)wl * D + wr) * 2 + s) * 2 + sp] += c * op[s * 2 + sp];
}

/*
 * MPO of the Hamiltonians used by the paper's benchmarks.
 *   model 0: XXZ  H = J sum_i [ (S+_i S-_{i+1} + S-_i S+_{i+1})/2 + Delta Sz_i Sz_{i+1} ]
 *            (Delta = 1 is the Heisenberg chain of Eq. (18)); D = 5.
 *   model 1: J1-J2 Heisenberg  H = J sum S_i.S_{i+1} + J2 sum S_i.S_{i+2}; D = 8.
 *   model 2: transverse-field Ising with Pauli matrices
 *            H = -J sum sz_i sz_{i+1} - h sum sx_i  (h passed in `Delta`); D = 3
 *            (the "Ising critical/ordered" rows of Table 5).
 * Lower-triangular convention: the left boundary selects row D-1 ("nothing
 * placed yet"), the right boundary selects column 0 ("all terms completed").
 * Returns D, or -1 for an unknown model.  W must hold N*D*D*4 doubles.
 */
int ref_mpo_dim(int model)
{
    switch (model) { case 0: return 5; case 1: return 8; case 2: return 3; default: return -1; }
}

int ref_build_mpo(int model, int N, double J, double Delta, double J2, double *W)
{
    int D = ref_mpo_dim(model);
    if (D < 0 || N < 2) return -1;
    double I2[4], Sz[4], Sp[4], Sm[4], Z[4], X[4];
    op_identity(I2); op_sz(Sz); op_splus(Sp); op_sminus(Sm); op_pauli_z(Z); op_pauli_x(X);
    size_t site = (size_t)D * D * 4;
    memset(W, 0, sizeof(double) * site * N);
    for (int i = 0; i < N; ++i) {
        double *Wi = W + site * i;
        if (model == 0) {
            mpo_set(Wi, D, 0, 0, I2, 1.0);
            mpo_set(Wi, D, 1, 0, Sp, 1.0);
            mpo_set(Wi, D, 2, 0, Sm, 1.0);
            mpo_set(Wi, D, 3, 0, Sz, 1.0);
            mpo_set(Wi, D, 4, 1, Sm, 0.5 * J);
            mpo_set(Wi, D, 4, 2, Sp, 0.5 * J);
            mpo_set(Wi, D, 4, 3, Sz, J * Delta);
            mpo_set(Wi, D, 4, 4, I2, 1.0);
        } else if (model == 1) {
            /* states: 7 start, 1..3 "S+,S-,Sz placed one site back",
             * 4..6 "placed two sites back", 0 done */
            mpo_set(Wi, D, 7, 7, I2, 1.0);
            mpo_set(Wi, D, 7, 1, Sp, 1.0);
            mpo_set(Wi, D, 7, 2, Sm, 1.0);
            mpo_set(Wi, D, 7, 3, Sz, 1.0);
            mpo_set(Wi, D, 1, 0, Sm, 0.5 * J);
            mpo_set(Wi, D, 2, 0, Sp, 0.5 * J);
            mpo_set(Wi, D, 3, 0, Sz, J * Delta);
            mpo_set(Wi, D, 1, 4, I2, 1.0);
            mpo_set(Wi, D, 2, 5, I2, 1.0);
            mpo_set(Wi, D, 3, 6, I2, 1.0);
            mpo_set(Wi, D, 4, 0, Sm, 0.5 * J2);
            mpo_set(Wi, D, 5, 0, Sp, 0.5 * J2);
            mpo_set(Wi, D, 6, 0, Sz, J2);
            mpo_set(Wi, D, 0, 0, I2, 1.0);
        } else {
            mpo_set(Wi, D, 2, 2, I2, 1.0);
            mpo_set(Wi, D, 2, 1, Z, -J);
            mpo_set(Wi, D, 1, 0, Z, 1.0);
            mpo_set(Wi, D, 2, 0, X, -Delta);
            mpo_set(Wi, D, 0, 0, I2, 1.0);
        }
    }
    return D;
}

/* Contract the MPO of N sites into the dense 2^N x 2^N Hamiltonian
 * (site 0 is the most significant index).  Only for tiny N.               */
int ref_mpo_to_dense(int N, int D, const double *W, double *H)
{
    int d = 2;
    size_t dim = (size_t)1 << N;
    /* M[w][row][col] for the block of sites 0..i-1 */
    size_t cur = 1;
    double *M = calloc((size_t)D, sizeof(double));
    if (!M) return REF_ENOMEM;
    M[D - 1] = 1.0;
    for (int i = 0; i < N; ++i) {
        size_t nxt = cur * d;
        double *M2 = calloc((size_t)D * nxt * nxt, sizeof(double));
        if (!M2) { free(M); return REF_ENOMEM; }
        const double *Wi = W + (size_t)D * D * 4 * i;
        for (int w = 0; w < D; ++w)
            for (int v = 0; v < D; ++v)
                for (size_t r = 0; r < cur; ++r)
                    for (size_t c = 0; c < cur; ++c) {
                        double m = M[((size_t)w * cur + r) * cur + c];
                        if (m == 0.0) continue;
                        for (int s = 0; s < d; ++s)
                            for (int sp = 0; sp < d; ++sp) {
                                double o = Wi[(((size_t)w * D + v) * d + s) * d + sp];
                                if (o == 0.0) continue;
                                M2[((size_t)v * nxt + r * d + s) * nxt + c * d + sp] += m * o;
                            }
                    }
        free(M);
        M = M2;
        cur = nxt;
    }
    for (size_t r = 0; r < dim; ++r)
        for (size_t c = 0; c < dim; ++c)
            H[r * dim + c] = M[r * dim + c]; /* w = 0 block */
    free(M);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers                                                            */
/* ------------------------------------------------------------------------ */
/* C[m][n] = sum_k A[m][k] B[k][n]   (row-major, plain triple loop)          */
static void mm(int m, int n, int k, const double *A, const double *B, double *C)
{
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = 0.0;
        for (int p = 0; p < k; ++p) {
            double a = A[(size_t)i * k + p];
            if (a == 0.0) continue;
            const double *b = B + (size_t)p * n;
            double *c = C + (size_t)i * n;
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/*
 * Householder QR of a row-major m x n matrix A (m >= n), textbook form
 * (Golub & Van Loan, Algorithm 5.2.1).  On return Q (m x n, orthonormal
 * columns) and R (n x n upper triangular) with A = Q R.
 */
int ref_qr(int m, int n, const double *A, double *Q, double *R)
{
    if (m < n) return REF_EINVAL;
    double *Wk = malloc(sizeof(double) * (size_t)m * n);
    double *V = malloc(sizeof(double) * (size_t)m * n);
    double *beta = malloc(sizeof(double) * (size_t)n);
    if (!Wk || !V || !beta) { free(Wk); free(V); free(beta); return REF_ENOMEM; }
    memcpy(Wk, A, sizeof(double) * (size_t)m * n);
    memset(V, 0, sizeof(double) * (size_t)m * n);
    for (int j = 0; j < n; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += Wk[(size_t)i * n + j] * Wk[(size_t)i * n + j];
        nrm = sqrt(nrm);
        double x0 = Wk[(size_t)j * n + j];
        double alpha = (x0 >= 0.0) ? -nrm : nrm;   /* reflect x onto alpha e1 */
        /* v = x - alpha e1 */
        double vnorm2 = 0.0;
        for (int i = j; i < m; ++i) {
            double vi = Wk[(size_t)i * n + j] - (i == j ? alpha : 0.0);
            V[(size_t)i * n + j] = vi;
            vnorm2 += vi * vi;
        }
        beta[j] = (vnorm2 > 0.0) ? 2.0 / vnorm2 : 0.0;
        /* apply H = I - beta v v^T to columns j..n-1 */
        for (int c = j; c < n; ++c) {
            double dot = 0.0;
            for (int i = j; i < m; ++i) dot += V[(size_t)i * n + j] * Wk[(size_t)i * n + c];
            dot *= beta[j];
            for (int i = j; i < m; ++i) Wk[(size_t)i * n + c] -= dot * V[(size_t)i * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < n; ++c) R[(size_t)i * n + c] = (c >= i) ? Wk[(size_t)i * n + c] : 0.0;
    /* Q = H_0 H_1 ... H_{n-1} [I_n; 0] accumulated backwards */
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < n; ++c) Q[(size_t)i * n + c] = (i == c) ? 1.0 : 0.0;
    for (int j = n - 1; j >= 0; --j) {
        for (int c = 0; c < n; ++c) {
            double dot = 0.0;
            for (int i = j; i < m; ++i) dot += V[(size_t)i * n + j] * Q[(size_t)i * n + c];
            dot *= beta[j];
            for (int i = j; i < m; ++i) Q[(size_t)i * n + c] -= dot * V[(size_t)i * n + j];
        }
    }
    free(Wk); free(V); free(beta);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Symmetric eigenproblem by the cyclic Jacobi method (Golub & Van Loan      */
/* Section 8.5): used for the small Lanczos tridiagonal matrix and for the  */
/* dense checks.  A (n x n, row-major) is overwritten; on return w holds the */
/* eigenvalues ascending and Z (row-major) the eigenvectors as columns.     */
/* ------------------------------------------------------------------------ */
int ref_sym_eig(int n, double *A, double *w, double *Z)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Z[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a = A[(size_t)i * n + j];
                tot += a * a;
                if (i != j) off += a * a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                /* rotation angle from the symmetric Schur decomposition of the 2x2 block */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J = rotation in the (p,q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * zkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
    /* selection sort ascending, permuting eigenvector columns */
    for (int i = 0; i < n - 1; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j) if (w[j] < w[best]) best = j;
        if (best != i) {
            double t = w[i]; w[i] = w[best]; w[best] = t;
            for (int k = 0; k < n; ++k) {
                double z = Z[(size_t)k * n + i];
                Z[(size_t)k * n + i] = Z[(size_t)k * n + best];
                Z[(size_t)k * n + best] = z;
            }
        }
    }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Two-sided Jacobi SVD (Golub & Van Loan Section 8.6.4, Kogbetliantz form). */
/* For a square n x n matrix: repeatedly pick (p,q), make the 2x2 block      */
/* symmetric by one rotation, diagonalise it by a second, and apply both to  */
/* rows/columns p,q while accumulating U and V.                              */
/* ------------------------------------------------------------------------ */
static int svd_square_two_sided(int n, double *A, double *U, double *V, double *s, int max_sweeps)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            U[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
            V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
        }
    double frob = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) frob += A[i] * A[i];
    double tol_abs = 1e-18 * sqrt(frob);     /* entries below this cannot move any s_k */
    int converged = 0;
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        converged = 1;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double w = A[(size_t)p * n + p], x = A[(size_t)p * n + q];
                double y = A[(size_t)q * n + p], z = A[(size_t)q * n + q];
                double scale = sqrt(fabs(w * z)) + 1e-300;
                if (fabs(x) <= 1e-15 * scale && fabs(y) <= 1e-15 * scale) continue;
                if (fabs(x) <= tol_abs && fabs(y) <= tol_abs) continue;
                if (x == 0.0 && y == 0.0) continue;
                converged = 0;
                /* (1) left rotation G1 = [[c1, s1], [-s1, c1]] making G1*B symmetric:
                 *     c1*x + s1*z = -s1*w + c1*y  ->  tan(psi) = (y - x)/(w + z)       */
                double psi = atan2(y - x, w + z);
                double c1 = cos(psi), s1 = sin(psi);
                double b00 = c1 * w + s1 * y, b01 = c1 * x + s1 * z;
                double b11 = -s1 * x + c1 * z;
                /* (2) symmetric Schur rotation J = [[c2, s2], [-s2, c2]] so J^T S J is diagonal */
                double c2 = 1.0, s2 = 0.0;
                if (b01 != 0.0) {
                    double tau = (b11 - b00) / (2.0 * b01);
                    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c2 = 1.0 / sqrt(1.0 + t * t);
                    s2 = t * c2;
                }
                /* rows p,q are transformed by Lrot = J^T G1 with J^T = [[c2, -s2], [s2, c2]] */
                double l00 = c2 * c1 + s2 * s1, l01 = c2 * s1 - s2 * c1;
                double l10 = s2 * c1 - c2 * s1, l11 = s2 * s1 + c2 * c1;
                for (int k = 0; k < n; ++k) {
                    double ap = A[(size_t)p * n + k], aq = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = l00 * ap + l01 * aq;
                    A[(size_t)q * n + k] = l10 * ap + l11 * aq;
                }
                /* A <- A J, J = [[c2, s2], [-s2, c2]] acting on columns p,q */
                for (int k = 0; k < n; ++k) {
                    double ap = A[(size_t)k * n + p], aq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c2 * ap - s2 * aq;
                    A[(size_t)k * n + q] = s2 * ap + c2 * aq;
                }
                /* U <- U Lrot^T, V <- V J  so that A_orig = U A V^T stays true */
                for (int k = 0; k < n; ++k) {
                    double up = U[(size_t)k * n + p], uq = U[(size_t)k * n + q];
                    U[(size_t)k * n + p] = l00 * up + l01 * uq;
                    U[(size_t)k * n + q] = l10 * up + l11 * uq;
                    double vp = V[(size_t)k * n + p], vq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c2 * vp - s2 * vq;
                    V[(size_t)k * n + q] = s2 * vp + c2 * vq;
                }
                A[(size_t)p * n + q] = 0.0;
                A[(size_t)q * n + p] = 0.0;
            }
    }
    for (int i = 0; i < n; ++i) {
        double d = A[(size_t)i * n + i];
        if (d < 0.0) {   /* flip the sign into U */
            d = -d;
            for (int k = 0; k < n; ++k) U[(size_t)k * n + i] = -U[(size_t)k * n + i];
        }
        s[i] = d;
    }
    return converged ? REF_OK : REF_ENOCONV;
}

/*
 * Full SVD of a row-major m x n matrix: A = U diag(s) Vt, U m x r, Vt r x n,
 * r = min(m,n), s descending.  Rectangular inputs are first reduced to a
 * square triangular factor by Householder QR (of A if m > n, of A^T if
 * m < n).  Sign convention: the entry of largest magnitude in every column
 * of U is made positive (the matching row of Vt flips with it).
 */
int ref_svd(int m, int n, const double *A, double *U, double *s, double *Vt, int max_sweeps)
{
    if (m <= 0 || n <= 0) return REF_EINVAL;
    int tr = (m < n);
    int M = tr ? n : m, Nn = tr ? m : n;    /* work on B = A or A^T, M >= Nn */
    double *B = malloc(sizeof(double) * (size_t)M * Nn);
    double *Q = malloc(sizeof(double) * (size_t)M * Nn);
    double *Rm = malloc(sizeof(double) * (size_t)Nn * Nn);
    double *Ur = malloc(sizeof(double) * (size_t)Nn * Nn);
    double *Vr = malloc(sizeof(double) * (size_t)Nn * Nn);
    double *sv = malloc(sizeof(double) * (size_t)Nn);
    double *UB = malloc(sizeof(double) * (size_t)M * Nn);
    int *ord = malloc(sizeof(int) * (size_t)Nn);
    if (!B || !Q || !Rm || !Ur || !Vr || !sv || !UB || !ord) {
        free(B); free(Q); free(Rm); free(Ur); free(Vr); free(sv); free(UB); free(ord);
        return REF_ENOMEM;
    }
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < Nn; ++j)
            B[(size_t)i * Nn + j] = tr ? A[(size_t)j * n + i] : A[(size_t)i * n + j];
    int st = ref_qr(M, Nn, B, Q, Rm);
    if (st == REF_OK) st = svd_square_two_sided(Nn, Rm, Ur, Vr, sv, max_sweeps);
    if (st == REF_OK || st == REF_ENOCONV) {
        mm(M, Nn, Nn, Q, Ur, UB);           /* B = (Q Ur) diag(sv) Vr^T */
        for (int i = 0; i < Nn; ++i) ord[i] = i;
        for (int i = 0; i < Nn - 1; ++i) {  /* sort descending (selection) */
            int best = i;
            for (int j = i + 1; j < Nn; ++j) if (sv[ord[j]] > sv[ord[best]]) best = j;
            int t = ord[i]; ord[i] = ord[best]; ord[best] = t;
        }
        int r = Nn;
        for (int c = 0; c < r; ++c) {
            int o = ord[c];
            s[c] = sv[o];
            /* left vectors of A: UB (if !tr) or Vr (if tr); right: the other */
            double maxabs = -1.0, sign = 1.0;
            for (int i = 0; i < m; ++i) {
                double u = tr ? Vr[(size_t)i * Nn + o] : UB[(size_t)i * Nn + o];
                if (fabs(u) > maxabs) { maxabs = fabs(u); sign = (u < 0.0) ? -1.0 : 1.0; }
            }
            for (int i = 0; i < m; ++i)
                U[(size_t)i * r + c] = sign * (tr ? Vr[(size_t)i * Nn + o] : UB[(size_t)i * Nn + o]);
            for (int j = 0; j < n; ++j)
                Vt[(size_t)c * n + j] = sign * (tr ? UB[(size_t)j * Nn + o] : Vr[(size_t)j * Nn + o]);
        }
    }
    free(B); free(Q); free(Rm); free(Ur); free(Vr); free(sv); free(UB); free(ord);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Entropy and truncation error, Eqs. (4)-(5).                               */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } neum;
static void neum_add(neum *a, double x)
{   /* Neumaier compensated summation */
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

/* S = -sum_k p_k ln p_k, p_k = s_k^2 / sum_j s_j^2 over the full spectrum;
 * terms with p_k == 0 contribute 0.  eps_out[k] (optional, length n+1):
 * truncation error sqrt(sum_{j>=k} p_j) when the first k values are kept.  */
double ref_entropy(int n, const double *s, double *eps_out)
{
    neum tot = {0, 0};
    for (int k = 0; k < n; ++k) neum_add(&tot, s[k] * s[k]);
    double Z = tot.s + tot.c;
    neum S = {0, 0};
    if (Z > 0.0) {
        for (int k = 0; k < n; ++k) {
            double p = s[k] * s[k] / Z;
            if (p > 0.0) neum_add(&S, -p * log(p));
        }
    }
    if (eps_out) {
        neum tail = {0, 0};
        eps_out[n] = 0.0;
        for (int k = n - 1; k >= 0; --k) {
            neum_add(&tail, (Z > 0.0) ? s[k] * s[k] / Z : 0.0);
            eps_out[k] = sqrt(fmax(tail.s + tail.c, 0.0));
        }
    }
    return S.s + S.c;
}

/* ------------------------------------------------------------------------ */
/* Controller: EMA (Eq. 8) -> predictor (Eq. 16) -> PID (Algorithm 2,        */
/* Eqs. 9-11) with rounding, clamping and anti-windup; DIRECT (Algorithm 1). */
/* Readings where the paper is ambiguous:                                   */
/*  - error sign e = S_hat - S_target (Eq. 9 / Algorithm 2; Eq. 17's sign   */
/*    would invert the loop),                                               */
/*  - the first step initialises S-bar = S (Section 4) unless ema_init_zero */
/*    (Section 10 initialisation), and sets S-bar_prev = S-bar and          */
/*    e_prev = e so the predictor and derivative terms start at 0,          */
/*  - rounding is half-to-even,                                             */
/*  - anti-windup fires on either clamp bound (Algorithm 2).               */
/* Plain mul/add only, in a fixed order, so the result is reproducible.    */
/* `chi_out` receives the controller's bond dimension for this visit.      */
/* ------------------------------------------------------------------------ */
static int clamp_int(double x, int lo, int hi)
{
    if (x < (double)lo) return lo;
    if (x > (double)hi) return hi;
    return (int)x;
}

/* EMA (Eq. 8) and predictor (Eq. 16) of one visit; returns S-hat. */
static double ctrl_filter(ref_ctrl_state *st, double S, const ref_params *p)
{
    double a = p->alpha_ema;
    if (!st->initialized) {
        st->Sbar = p->ema_init_zero ? a * S : S;
        st->Sbar_prev = st->Sbar;
        st->Sbar_prev2 = st->Sbar;
    } else {
        double nb = a * S + (1.0 - a) * st->Sbar;
        st->Sbar_prev2 = st->Sbar_prev;
        st->Sbar_prev = st->Sbar;
        st->Sbar = nb;
    }
    /* window of EMA values for the learned scheduler */
    if (st->nhist < 8) {
        st->hist[st->nhist++] = st->Sbar;
    } else {
        for (int i = 0; i < 7; ++i) st->hist[i] = st->hist[i + 1];
        st->hist[7] = st->Sbar;
    }
    double Shat = st->Sbar + p->beta * (st->Sbar - st->Sbar_prev);
    if (p->second_order)
        Shat = Shat + p->beta * ((st->Sbar - 2.0 * st->Sbar_prev) + st->Sbar_prev2);
    return Shat;
}

/* PID control signal before rounding (Algorithm 2, Eq. 10): error e (Eq. 9),
 * integral update, derivative on e - e_prev.  Returns u; e in *e_out. */
static double ctrl_pid_u(ref_ctrl_state *st, double Shat, const ref_params *p, double *e_out)
{
    double e = Shat - p->S_target;
    if (!st->initialized) st->e_prev = e;
    double P = p->Kp * e;
    st->I = st->I + p->Ki * e;
    double Dt = p->Kd * (e - st->e_prev);
    *e_out = e;
    return (P + st->I) + Dt;
}

int ref_ctrl_step(ref_ctrl_state *st, double S, const ref_params *p, int *chi_out)
{
    double Shat = ctrl_filter(st, S, p);
    int chi_new;
    if (p->ctrl == CTRL_DIRECT) {
        double tgt = ceil(p->gamma * exp(st->Sbar));
        chi_new = clamp_int(tgt, p->chi_min, p->chi_max);
    } else if (p->ctrl == CTRL_FIXED) {
        chi_new = p->chi_fixed;
    } else if (p->ctrl == CTRL_THRESHOLD) {
        chi_new = p->chi_max;
    } else {
        double e;
        double u = ctrl_pid_u(st, Shat, p, &e);
        double delta = nearbyint(u);               /* FE_TONEAREST: half to even */
        double raw = (double)st->chi + delta;
        chi_new = clamp_int(raw, p->chi_min, p->chi_max);
        if ((double)chi_new != raw) st->I = st->I - p->Ki * e;   /* anti-windup */
        st->e_prev = e;
    }
    st->chi = chi_new;
    st->initialized = 1;
    *chi_out = chi_new;
    return REF_OK;
}

/* The same EMA -> predictor -> PID step with rounding and clamping switched
 * off (so anti-windup never fires) and chi carried as a real number in
 * *chi_real: chi <- chi + u.  This is the linear loop that the stability
 * analysis of Section 5 reasons about; it exists only to pin the filter and
 * PID arithmetic above against the closed-form solution of that loop. */
int ref_ctrl_step_real(ref_ctrl_state *st, double S, const ref_params *p, double *chi_real)
{
    double Shat = ctrl_filter(st, S, p);
    double e;
    double u = ctrl_pid_u(st, Shat, p, &e);
    *chi_real = *chi_real + u;
    st->e_prev = e;
    st->initialized = 1;
    return REF_OK;
}

/* Replay a recorded sequence of raw entropies through n_bonds controllers:
 * S_seq[t*n_bonds + i] is the entropy of bond i at step t; chi_seq receives
 * the controller output in the same layout.                                */
int ref_ctrl_replay(int n_steps, int n_bonds, const double *S_seq, const ref_params *p,
                    ref_ctrl_state *states, int *chi_seq)
{
    for (int t = 0; t < n_steps; ++t)
        for (int i = 0; i < n_bonds; ++i)
            ref_ctrl_step(&states[i], S_seq[(size_t)t * n_bonds + i], p, &chi_seq[(size_t)t * n_bonds + i]);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Learned scheduler: 10 -> 64 -> 64 -> 1 MLP with exact-erf GELU, MSE loss, */
/* Adam.  Parameter vector layout: W1[64][10], b1[64], W2[64][64], b2[64],   */
/* W3[1][64], b3[1]  (4929 values).                                          */
/* ------------------------------------------------------------------------ */
#define MLP_IN 10
#define MLP_H 64
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

int ref_mlp_nparam(void) { return MLP_NPARAM; }

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_grad(double x)
{
    double Phi = 0.5 * (1.0 + erf(x / sqrt(2.0)));
    double phi = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
    return Phi + x * phi;
}

/* forward for a batch; y[b] = network output.  Optional caches z1,h1,z2,h2 (B x 64). */
static void mlp_forward_cache(const double *P, int B, const double *X, double *y,
                              double *z1, double *h1, double *z2, double *h2)
{
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    double a1[MLP_H], g1[MLP_H], a2[MLP_H], g2[MLP_H];
    for (int b = 0; b < B; ++b) {
        const double *x = X + (size_t)b * MLP_IN;
        for (int j = 0; j < MLP_H; ++j) {
            double acc = b1[j];
            for (int i = 0; i < MLP_IN; ++i) acc += W1[j * MLP_IN + i] * x[i];
            a1[j] = acc; g1[j] = gelu(acc);
        }
        for (int j = 0; j < MLP_H; ++j) {
            double acc = b2[j];
            for (int i = 0; i < MLP_H; ++i) acc += W2[j * MLP_H + i] * g1[i];
            a2[j] = acc; g2[j] = gelu(acc);
        }
        double out = b3[0];
        for (int i = 0; i < MLP_H; ++i) out += W3[i] * g2[i];
        y[b] = out;
        if (z1) for (int j = 0; j < MLP_H; ++j) {
            z1[(size_t)b * MLP_H + j] = a1[j]; h1[(size_t)b * MLP_H + j] = g1[j];
            z2[(size_t)b * MLP_H + j] = a2[j]; h2[(size_t)b * MLP_H + j] = g2[j];
        }
    }
}

int ref_mlp_forward(const double *P, int B, const double *X, double *y)
{
    mlp_forward_cache(P, B, X, y, NULL, NULL, NULL, NULL);
    return REF_OK;
}

/* loss = mean_b (y_b - t_b)^2; grad (length nparam) = d loss / d P.        */
int ref_mlp_loss_grad(const double *P, int B, const double *X, const double *t, double *loss, double *grad)
{
    const double *W2 = P + MLP_H * MLP_IN + MLP_H, *W3 = W2 + MLP_H * MLP_H + MLP_H;
    double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    double *z1 = malloc(sizeof(double) * (size_t)B * MLP_H * 4), *y = malloc(sizeof(double) * (size_t)B);
    if (!z1 || !y) { free(z1); free(y); return REF_ENOMEM; }
    double *h1 = z1 + (size_t)B * MLP_H, *z2 = h1 + (size_t)B * MLP_H, *h2 = z2 + (size_t)B * MLP_H;
    mlp_forward_cache(P, B, X, y, z1, h1, z2, h2);
    memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double L = 0.0;
    for (int b = 0; b < B; ++b) {
        double r = y[b] - t[b];
        L += r * r;
        double dy = 2.0 * r / B;
        double dz2[MLP_H], dz1[MLP_H];
        gb3[0] += dy;
        for (int i = 0; i < MLP_H; ++i) {
            gW3[i] += dy * h2[(size_t)b * MLP_H + i];
            dz2[i] = dy * W3[i] * gelu_grad(z2[(size_t)b * MLP_H + i]);
        }
        for (int j = 0; j < MLP_H; ++j) {
            gb2[j] += dz2[j];
            for (int i = 0; i < MLP_H; ++i) gW2[j * MLP_H + i] += dz2[j] * h1[(size_t)b * MLP_H + i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double acc = 0.0;
            for (int j = 0; j < MLP_H; ++j) acc += W2[j * MLP_H + i] * dz2[j];
            dz1[i] = acc * gelu_grad(z1[(size_t)b * MLP_H + i]);
        }
        const double *x = X + (size_t)b * MLP_IN;
        for (int j = 0; j < MLP_H; ++j) {
            gb1[j] += dz1[j];
            for (int i = 0; i < MLP_IN; ++i) gW1[j * MLP_IN + i] += dz1[j] * x[i];
        }
    }
    *loss = L / B;
    free(z1); free(y);
    return REF_OK;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1); step is the 1-based t.    */
int ref_adam_step(int n, double *P, const double *g, double *m, double *v, int step,
                  double lr, double b1, double b2, double eps)
{
    double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
    for (int i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        P[i] -= lr * mh / (sqrt(vh) + eps);
    }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Environments and the effective Hamiltonian (Eq. 19).                      */
/* ------------------------------------------------------------------------ */
/* y = H_eff theta at a bond with environments L (D x cl x cl), R (D x cr x cr)
 * and MPO tensors W1, W2 (D x D x d x d):
 *   y[a'][s1'][s2'][b'] = sum L[w][a'][a] W1[w][v][s1'][s1] W2[v][u][s2'][s2] R[u][b'][b] theta[a][s1][s2][b]
 * evaluated in four stages (over a, then (w,s1), then (v,s2), then (u,b)). */
int ref_heff_apply(int cl, int cr, int d, int D, const double *L, const double *W1, const double *W2,
                   const double *R, const double *theta, double *y)
{
    size_t n4 = (size_t)d * d * cr;               /* (s1,s2,b) */
    double *T1 = calloc((size_t)D * cl * n4, sizeof(double));   /* [w][a'][s1][s2][b] */
    double *T2 = calloc((size_t)D * cl * n4, sizeof(double));   /* [v][a'][s1'][s2][b] */
    double *T3 = calloc((size_t)D * cl * n4, sizeof(double));   /* [u][a'][s1'][s2'][b] */
    if (!T1 || !T2 || !T3) { free(T1); free(T2); free(T3); return REF_ENOMEM; }
    for (int w = 0; w < D; ++w)
        mm(cl, (int)n4, cl, L + (size_t)w * cl * cl, theta, T1 + (size_t)w * cl * n4);
    for (int w = 0; w < D; ++w)
        for (int v = 0; v < D; ++v)
            for (int s1p = 0; s1p < d; ++s1p)
                for (int s1 = 0; s1 < d; ++s1) {
                    double c = W1[(((size_t)w * D + v) * d + s1p) * d + s1];
                    if (c == 0.0) continue;
                    for (int ap = 0; ap < cl; ++ap) {
                        const double *src = T1 + (((size_t)w * cl + ap) * d + s1) * d * cr;
                        double *dst = T2 + (((size_t)v * cl + ap) * d + s1p) * d * cr;
                        for (size_t x = 0; x < (size_t)d * cr; ++x) dst[x] += c * src[x];
                    }
                }
    for (int v = 0; v < D; ++v)
        for (int u = 0; u < D; ++u)
            for (int s2p = 0; s2p < d; ++s2p)
                for (int s2 = 0; s2 < d; ++s2) {
                    double c = W2[(((size_t)v * D + u) * d + s2p) * d + s2];
                    if (c == 0.0) continue;
                    for (int ap = 0; ap < cl; ++ap)
                        for (int s1p = 0; s1p < d; ++s1p) {
                            const double *src = T2 + ((((size_t)v * cl + ap) * d + s1p) * d + s2) * cr;
                            double *dst = T3 + ((((size_t)u * cl + ap) * d + s1p) * d + s2p) * cr;
                            for (int b = 0; b < cr; ++b) dst[b] += c * src[b];
                        }
                }
    /* y[a',s1',s2'][b'] = sum_u sum_b T3[u][a',s1',s2'][b] R[u][b'][b] */
    size_t rows = (size_t)cl * d * d;
    memset(y, 0, sizeof(double) * rows * cr);
    for (int u = 0; u < D; ++u) {
        const double *Ru = R + (size_t)u * cr * cr;
        const double *T = T3 + (size_t)u * rows * cr;
        for (size_t r = 0; r < rows; ++r)
            for (int bp = 0; bp < cr; ++bp) {
                double acc = 0.0;
                for (int b = 0; b < cr; ++b) acc += T[r * cr + b] * Ru[(size_t)bp * cr + b];
                y[r * cr + bp] += acc;
            }
    }
    free(T1); free(T2); free(T3);
    return REF_OK;
}

/* L_new[v][b'][b] = sum A[a'][s'][b'] W[w][v][s'][s] L[w][a'][a] A[a][s][b]
 * (A: cl x d x ck, left-canonical site).                                    */
int ref_env_left(int cl, int ck, int d, int D, const double *L, const double *W, const double *A, double *Lnew)
{
    size_t n2 = (size_t)d * ck;
    double *T1 = calloc((size_t)D * cl * n2, sizeof(double));  /* [w][a'][s][b] */
    double *T2 = calloc((size_t)D * cl * n2, sizeof(double));  /* [v][a'][s'][b] */
    if (!T1 || !T2) { free(T1); free(T2); return REF_ENOMEM; }
    for (int w = 0; w < D; ++w) mm(cl, (int)n2, cl, L + (size_t)w * cl * cl, A, T1 + (size_t)w * cl * n2);
    for (int w = 0; w < D; ++w)
        for (int v = 0; v < D; ++v)
            for (int sp = 0; sp < d; ++sp)
                for (int s = 0; s < d; ++s) {
                    double c = W[(((size_t)w * D + v) * d + sp) * d + s];
                    if (c == 0.0) continue;
                    for (int ap = 0; ap < cl; ++ap) {
                        const double *src = T1 + (((size_t)w * cl + ap) * d + s) * ck;
                        double *dst = T2 + (((size_t)v * cl + ap) * d + sp) * ck;
                        for (int b = 0; b < ck; ++b) dst[b] += c * src[b];
                    }
                }
    for (int v = 0; v < D; ++v)
        for (int bp = 0; bp < ck; ++bp)
            for (int b = 0; b < ck; ++b) {
                double acc = 0.0;
                for (int ap = 0; ap < cl; ++ap)
                    for (int sp = 0; sp < d; ++sp)
                        acc += A[((size_t)ap * d + sp) * ck + bp] * T2[(((size_t)v * cl + ap) * d + sp) * ck + b];
                Lnew[((size_t)v * ck + bp) * ck + b] = acc;
            }
    free(T1); free(T2);
    return REF_OK;
}

/* R_new[w][a'][a] = sum B[a'][s'][b'] W[w][v][s'][s] R[v][b'][b] B[a][s][b]
 * (B: ck x d x cr, right-canonical site).                                   */
int ref_env_right(int ck, int cr, int d, int D, const double *R, const double *W, const double *B, double *Rnew)
{
    /* T1[v][a][s][b'] = sum_b B[a][s][b] R[v][b'][b] */
    size_t n2 = (size_t)d * cr;
    double *T1 = calloc((size_t)D * ck * n2, sizeof(double));
    double *T2 = calloc((size_t)D * ck * n2, sizeof(double));  /* [w][a][s'][b'] */
    if (!T1 || !T2) { free(T1); free(T2); return REF_ENOMEM; }
    for (int v = 0; v < D; ++v)
        for (int a = 0; a < ck; ++a)
            for (int s = 0; s < d; ++s)
                for (int bp = 0; bp < cr; ++bp) {
                    double acc = 0.0;
                    for (int b = 0; b < cr; ++b)
                        acc += B[((size_t)a * d + s) * cr + b] * R[((size_t)v * cr + bp) * cr + b];
                    T1[(((size_t)v * ck + a) * d + s) * cr + bp] = acc;
                }
    for (int w = 0; w < D; ++w)
        for (int v = 0; v < D; ++v)
            for (int sp = 0; sp < d; ++sp)
                for (int s = 0; s < d; ++s) {
                    double c = W[(((size_t)w * D + v) * d + sp) * d + s];
                    if (c == 0.0) continue;
                    for (int a = 0; a < ck; ++a) {
                        const double *src = T1 + (((size_t)v * ck + a) * d + s) * cr;
                        double *dst = T2 + (((size_t)w * ck + a) * d + sp) * cr;
                        for (int bp = 0; bp < cr; ++bp) dst[bp] += c * src[bp];
                    }
                }
    for (int w = 0; w < D; ++w)
        for (int ap = 0; ap < ck; ++ap)
            for (int a = 0; a < ck; ++a) {
                double acc = 0.0;
                for (int sp = 0; sp < d; ++sp)
                    for (int bp = 0; bp < cr; ++bp)
                        acc += B[((size_t)ap * d + sp) * cr + bp] * T2[(((size_t)w * ck + a) * d + sp) * cr + bp];
                Rnew[((size_t)w * ck + ap) * ck + a] = acc;
            }
    free(T1); free(T2);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Lanczos for the lowest eigenpair of H_eff (the paper leaves the local     */
/* eigensolver unnamed; this is the textbook Lanczos recurrence with full    */
/* reorthogonalisation by two classical Gram-Schmidt passes).               */
/*   v0 = theta/|theta|;  w = H v_j;  alpha_j = v_j.w;                       */
/*   w -= alpha_j v_j + beta_j v_{j-1};  w -= V (V^T w) twice;               */
/*   beta_{j+1} = |w|;  stop after K steps or when beta < 1e-14 max|alpha|.  */
/* T is solved by cyclic Jacobi; the Ritz vector is V y0, normalised.       */
/* ------------------------------------------------------------------------ */
int ref_lanczos(int cl, int cr, int d, int D, const double *L, const double *W1, const double *W2,
                const double *R, double *theta, int K, double *E_out, int *k_used,
                double *alpha_out, double *beta_out)
{
    size_t n = (size_t)cl * d * d * cr;
    if (K > (int)n) K = (int)n;
    if (K < 1) K = 1;
    double *V = malloc(sizeof(double) * n * (size_t)(K + 1));
    double *w = malloc(sizeof(double) * n);
    double *al = calloc((size_t)K, sizeof(double)), *be = calloc((size_t)K + 1, sizeof(double));
    double *c = malloc(sizeof(double) * (size_t)(K + 1));
    if (!V || !w || !al || !be || !c) { free(V); free(w); free(al); free(be); free(c); return REF_ENOMEM; }
    double nrm = 0.0;
    for (size_t i = 0; i < n; ++i) nrm += theta[i] * theta[i];
    nrm = sqrt(nrm);
    for (size_t i = 0; i < n; ++i) V[i] = theta[i] / nrm;
    int m = 0;
    double amax = 0.0;
    for (int j = 0; j < K; ++j) {
        double *vj = V + n * j;
        ref_heff_apply(cl, cr, d, D, L, W1, W2, R, vj, w);
        double a = 0.0;
        for (size_t i = 0; i < n; ++i) a += vj[i] * w[i];
        al[j] = a;
        if (fabs(a) > amax) amax = fabs(a);
        for (size_t i = 0; i < n; ++i) w[i] -= a * vj[i];
        if (j > 0) { double *vm = V + n * (j - 1); for (size_t i = 0; i < n; ++i) w[i] -= be[j] * vm[i]; }
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = 0; q <= j; ++q) {
                double acc = 0.0;
                const double *vq = V + n * q;
                for (size_t i = 0; i < n; ++i) acc += vq[i] * w[i];
                c[q] = acc;
            }
            for (int q = 0; q <= j; ++q) {
                const double *vq = V + n * q;
                for (size_t i = 0; i < n; ++i) w[i] -= c[q] * vq[i];
            }
        }
        double b = 0.0;
        for (size_t i = 0; i < n; ++i) b += w[i] * w[i];
        b = sqrt(b);
        m = j + 1;
        be[j + 1] = b;
        if (j == K - 1 || b < 1e-14 * amax) break;
        double *vn = V + n * (j + 1);
        for (size_t i = 0; i < n; ++i) vn[i] = w[i] / b;
    }
    double *T = calloc((size_t)m * m, sizeof(double)), *ev = malloc(sizeof(double) * m), *Z = malloc(sizeof(double) * (size_t)m * m);
    for (int i = 0; i < m; ++i) {
        T[(size_t)i * m + i] = al[i];
        if (i + 1 < m) { T[(size_t)i * m + i + 1] = be[i + 1]; T[(size_t)(i + 1) * m + i] = be[i + 1]; }
    }
    ref_sym_eig(m, T, ev, Z);
    memset(theta, 0, sizeof(double) * n);
    for (int j = 0; j < m; ++j) {
        double y = Z[(size_t)j * m + 0];
        const double *vj = V + n * j;
        for (size_t i = 0; i < n; ++i) theta[i] += y * vj[i];
    }
    nrm = 0.0;
    for (size_t i = 0; i < n; ++i) nrm += theta[i] * theta[i];
    nrm = sqrt(nrm);
    for (size_t i = 0; i < n; ++i) theta[i] /= nrm;
    *E_out = ev[0];
    *k_used = m;
    if (alpha_out) for (int i = 0; i < m; ++i) alpha_out[i] = al[i];
    if (beta_out) for (int i = 0; i < m; ++i) beta_out[i] = be[i + 1];
    free(T); free(ev); free(Z);
    free(V); free(w); free(al); free(be); free(c);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Truncation decision (Section 10):                                         */
/*   k = min(chi_ctrl, rank, #{s_j > eps_trunc}) on the normalised spectrum, */
/*   at least 1; with multiplet_guard k never ends inside a group of         */
/*   singular values equal to relative 1e-10.                                */
/* ------------------------------------------------------------------------ */
int ref_trunc_k(int r, const double *s, int chi_ctrl, double eps_trunc, int multiplet_guard)
{
    double Z = 0.0;
    for (int j = 0; j < r; ++j) Z += s[j] * s[j];
    double nz = sqrt(Z);
    int rank = 0, above = 0;
    double rank_tol = (double)r * 2.220446049250313e-16 * (r > 0 ? s[0] : 0.0);
    for (int j = 0; j < r; ++j) {
        if (s[j] > rank_tol) rank++;
        if (nz > 0.0 && s[j] / nz > eps_trunc) above++;
    }
    int k = chi_ctrl;
    if (rank < k) k = rank;
    if (above < k) k = above;
    if (k < 1) k = 1;
    if (multiplet_guard && k < r) {
        while (k > 1 && fabs(s[k - 1] - s[k]) <= 1e-10 * s[k - 1]) k--;
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* DMRG sweeps (Section 10).                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N, d, D;
    int *chi;            /* N+1 bond dimensions */
    double **A;          /* site tensors */
    double **L, **R;     /* environments (index 0..N) */
} ref_mps;

static void mps_free(ref_mps *m)
{
    if (m->A) for (int i = 0; i < m->N; ++i) free(m->A[i]);
    if (m->L) for (int i = 0; i <= m->N; ++i) free(m->L[i]);
    if (m->R) for (int i = 0; i <= m->N; ++i) free(m->R[i]);
    free(m->A); free(m->L); free(m->R); free(m->chi);
}

/* MLP features of bond i at visit `visit` (0-based count of controller steps). */
static void mlp_features(const ref_ctrl_state *st, int bond, int N, int sweep, int max_sweeps, double *x)
{
    int h = st->nhist;
    for (int j = 0; j < 8; ++j) {
        int idx = h - 8 + j;           /* pad with the oldest available value */
        if (idx < 0) idx = 0;
        x[j] = (h > 0) ? st->hist[idx] : 0.0;
    }
    x[8] = (double)(bond + 1) / (double)N;
    x[9] = (double)sweep / (double)(max_sweeps > 0 ? max_sweeps : 1);
}

/* Bond dimension chosen by the MLP, with the PID as fallback and arbiter:
 * chi = clamp(round(2^y), chi_min, chi_max); the PID choice is used if the
 * network output is not finite, or if the truncation error of the network's
 * chi exceeds 10x the PID's plus 1e-10.                                     */
static int mlp_choose(const double *P, const double *x, int chi_pid, const ref_params *p,
                      int r, const double *s, int *used_fallback)
{
    double y;
    ref_mlp_forward(P, 1, x, &y);
    double c = nearbyint(exp2(y));
    *used_fallback = 1;
    if (!isfinite(y)) return chi_pid;
    if (c < p->chi_min) c = p->chi_min;
    if (c > p->chi_max) c = p->chi_max;
    int chi_m = (int)c;
    int k_m = ref_trunc_k(r, s, chi_m, p->eps_trunc, p->multiplet_guard);
    int k_p = ref_trunc_k(r, s, chi_pid, p->eps_trunc, p->multiplet_guard);
    double *eps = malloc(sizeof(double) * (size_t)(r + 1));
    ref_entropy(r, s, eps);
    double em = eps[k_m], ep = eps[k_p];
    free(eps);
    if (em > 10.0 * ep + 1e-10) return chi_pid;
    *used_fallback = 0;
    return chi_m;
}

/*
 * Run adaptive two-site DMRG.
 *   W            N MPO tensors (D x D x d x d each), from ref_build_mpo.
 *   mps_init     Gaussian entries of the initial MPS, site after site, with
 *                chi_i = min(chi_init, d^i, d^(N-i)); right-canonicalised
 *                here (Householder LQ from the right) and normalised.
 *   ctrl_init    optional initial controller states (N-1), else zero state
 *                with chi = chi_min (Section 10).
 *   mlp_params   network parameters when ctrl == MLP (else NULL).
 * Outputs (per visit v of sweep t, index t*(2N-3)+v, bonds 0-based):
 *   rec_bond, rec_E, rec_S, rec_eps, rec_k, rec_chi, plus E_sweep[t] (Ritz
 *   value at the sweep's last bond) and the final chi profile (N+1).
 * Returns the number of sweeps run (stops early if |dE/E| < eps_conv and
 * stop_on_conv), or a negative error code.
 */
int ref_dmrg_run(int N, int d, int D, const double *W, const double *mps_init,
                 const ref_params *p, int n_sweeps, int stop_on_conv,
                 ref_ctrl_state *ctrl, const double *mlp_params,
                 double *E_sweep, int *rec_bond, double *rec_E, double *rec_S, double *rec_eps,
                 int *rec_k, int *rec_chi, int *chi_final, double *theta_final_norm)
{
    if (N < 2 || d != 2) return -REF_EINVAL;
    ref_mps m;
    memset(&m, 0, sizeof(m));
    m.N = N; m.d = d; m.D = D;
    m.chi = malloc(sizeof(int) * (size_t)(N + 1));
    m.A = calloc((size_t)N, sizeof(double *));
    m.L = calloc((size_t)N + 1, sizeof(double *));
    m.R = calloc((size_t)N + 1, sizeof(double *));
    if (!m.chi || !m.A || !m.L || !m.R) { mps_free(&m); return -REF_ENOMEM; }
    for (int i = 0; i <= N; ++i) {
        double lim = 1.0;
        int c = p->chi_init;
        for (int t = 0; t < i && lim < c; ++t) lim *= d;
        if (lim < c) c = (int)lim;
        double lim2 = 1.0;
        for (int t = 0; t < N - i && lim2 < c; ++t) lim2 *= d;
        if (lim2 < c) c = (int)lim2;
        m.chi[i] = c;
    }
    size_t off = 0;
    for (int i = 0; i < N; ++i) {
        size_t sz = (size_t)m.chi[i] * d * m.chi[i + 1];
        m.A[i] = malloc(sizeof(double) * sz);
        memcpy(m.A[i], mps_init + off, sizeof(double) * sz);
        off += sz;
    }
    /* right-canonicalise: M_i (chi_i x d chi_{i+1}) = Lf Q, A_i = Q, A_{i-1} <- A_{i-1} Lf */
    for (int i = N - 1; i >= 1; --i) {
        int rows = m.chi[i], cols = d * m.chi[i + 1];
        double *Mt = malloc(sizeof(double) * (size_t)rows * cols);
        double *Q = malloc(sizeof(double) * (size_t)rows * cols);
        double *Rf = malloc(sizeof(double) * (size_t)rows * rows);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) Mt[(size_t)c * rows + r] = m.A[i][(size_t)r * cols + c];
        ref_qr(cols, rows, Mt, Q, Rf);         /* M^T = Q Rf  ->  M = Rf^T Q^T */
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) m.A[i][(size_t)r * cols + c] = Q[(size_t)c * rows + r];
        int pr = m.chi[i - 1] * d;
        double *tmp = malloc(sizeof(double) * (size_t)pr * rows);
        double *RfT = malloc(sizeof(double) * (size_t)rows * rows);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < rows; ++c) RfT[(size_t)r * rows + c] = Rf[(size_t)c * rows + r];
        mm(pr, rows, rows, m.A[i - 1], RfT, tmp);
        memcpy(m.A[i - 1], tmp, sizeof(double) * (size_t)pr * rows);
        free(Mt); free(Q); free(Rf); free(tmp); free(RfT);
    }
    {
        size_t sz = (size_t)d * m.chi[1];
        double nn = 0.0;
        for (size_t x = 0; x < sz; ++x) nn += m.A[0][x] * m.A[0][x];
        nn = sqrt(nn);
        for (size_t x = 0; x < sz; ++x) m.A[0][x] /= nn;
    }
    /* boundary environments */
    m.L[0] = calloc((size_t)D, sizeof(double)); m.L[0][D - 1] = 1.0;
    m.R[N] = calloc((size_t)D, sizeof(double)); m.R[N][0] = 1.0;
    for (int i = N - 1; i >= 2; --i) {
        m.R[i] = malloc(sizeof(double) * (size_t)D * m.chi[i] * m.chi[i]);
        ref_env_right(m.chi[i], m.chi[i + 1], d, D, m.R[i + 1], W + (size_t)D * D * d * d * i, m.A[i], m.R[i]);
    }
    /* controllers */
    ref_ctrl_state *cs = ctrl;
    ref_ctrl_state *own = NULL;
    if (!cs) {
        own = calloc((size_t)(N - 1), sizeof(ref_ctrl_state));
        for (int b = 0; b < N - 1; ++b) own[b].chi = p->chi_min;
        cs = own;
    }
    /* global adaptive chi (Section 6): one controller on the mean of the
     * per-bond filtered entropies, stepped once per sweep, chi uniform */
    ref_ctrl_state gcs;
    memset(&gcs, 0, sizeof gcs);
    gcs.chi = p->chi_min;
    int visits_per_sweep = 2 * N - 3;
    double E_prev = 0.0;
    int sweeps_done = 0;
    int status = 0;
    size_t Wsz = (size_t)D * D * d * d;
    for (int t = 0; t < n_sweeps && status == 0; ++t) {
        int v = 0;
        double E_last = 0.0;
        for (int half = 0; half < 2; ++half) {
            int nb = (half == 0) ? N - 1 : N - 2;
            for (int q = 0; q < nb; ++q, ++v) {
                int k = (half == 0) ? q : N - 3 - q;     /* bond between sites k, k+1 */
                int cl = m.chi[k], cm = m.chi[k + 1], cr = m.chi[k + 2];
                int rows = cl * d, cols = d * cr;
                double *theta = malloc(sizeof(double) * (size_t)rows * cols);
                mm(rows, cols, cm, m.A[k], m.A[k + 1], theta);
                double E; int kused;
                ref_lanczos(cl, cr, d, D, m.L[k], W + Wsz * k, W + Wsz * (k + 1), m.R[k + 2], theta,
                            p->lanczos_steps, &E, &kused, NULL, NULL);
                int r = rows < cols ? rows : cols;
                double *U = malloc(sizeof(double) * (size_t)rows * r);
                double *s = malloc(sizeof(double) * (size_t)r);
                double *Vt = malloc(sizeof(double) * (size_t)r * cols);
                double *eps = malloc(sizeof(double) * (size_t)(r + 1));
                int sst = ref_svd(rows, cols, theta, U, s, Vt, p->jacobi_max_sweeps > 0 ? p->jacobi_max_sweeps : 60);
                if (sst != REF_OK) status = sst;
                double S = ref_entropy(r, s, eps);
                int chi_c;
                int do_ctrl = (p->pid_steps_per_sweep >= 2) || (half == 0);
                if (p->ctrl == CTRL_GLOBAL) {
                    int unused;
                    if (do_ctrl) ref_ctrl_step(&cs[k], S, p, &unused);   /* the bond's filter only */
                    chi_c = gcs.chi;
                } else if (do_ctrl) {
                    ref_ctrl_step(&cs[k], S, p, &chi_c);
                    if (p->ctrl == CTRL_MLP && mlp_params) {
                        double x[MLP_IN];
                        int fb;
                        mlp_features(&cs[k], k, N, t, p->max_sweeps, x);
                        chi_c = mlp_choose(mlp_params, x, chi_c, p, r, s, &fb);
                    }
                } else {
                    chi_c = cs[k].chi;
                }
                int kk = ref_trunc_k(r, s, chi_c, p->eps_trunc, p->multiplet_guard);
                /* renormalise the retained spectrum to unit norm */
                double z = 0.0;
                for (int j = 0; j < kk; ++j) z += s[j] * s[j];
                z = sqrt(z);
                int go_right = (half == 0 && k < N - 2);   /* centre moves right */
                free(m.A[k]); free(m.A[k + 1]);
                m.A[k] = malloc(sizeof(double) * (size_t)rows * kk);
                m.A[k + 1] = malloc(sizeof(double) * (size_t)kk * cols);
                for (int i = 0; i < rows; ++i)
                    for (int j = 0; j < kk; ++j)
                        m.A[k][(size_t)i * kk + j] = U[(size_t)i * r + j] * (go_right ? 1.0 : s[j] / z);
                for (int j = 0; j < kk; ++j)
                    for (int c = 0; c < cols; ++c)
                        m.A[k + 1][(size_t)j * cols + c] = Vt[(size_t)j * cols + c] * (go_right ? s[j] / z : 1.0);
                m.chi[k + 1] = kk;
                if (go_right) {
                    free(m.L[k + 1]);
                    m.L[k + 1] = malloc(sizeof(double) * (size_t)D * kk * kk);
                    ref_env_left(cl, kk, d, D, m.L[k], W + Wsz * k, m.A[k], m.L[k + 1]);
                } else if (k + 1 >= 2) {
                    free(m.R[k + 1]);
                    m.R[k + 1] = malloc(sizeof(double) * (size_t)D * kk * kk);
                    ref_env_right(kk, cr, d, D, m.R[k + 2], W + Wsz * (k + 1), m.A[k + 1], m.R[k + 1]);
                }
                size_t idx = (size_t)t * visits_per_sweep + v;
                if (rec_bond) rec_bond[idx] = k;
                if (rec_E) rec_E[idx] = E;
                if (rec_S) rec_S[idx] = S;
                if (rec_eps) rec_eps[idx] = eps[kk];
                if (rec_k) rec_k[idx] = kk;
                if (rec_chi) rec_chi[idx] = chi_c;
                E_last = E;
                free(theta); free(U); free(s); free(Vt); free(eps);
            }
        }
        if (p->ctrl == CTRL_GLOBAL) {
            /* S-bar(t) = (N-1)^-1 sum_i S-bar_i(t); the per-bond values are
             * already filtered, so the global controller takes it with alpha = 1 */
            double sum = 0.0;
            for (int b = 0; b < N - 1; ++b) sum += cs[b].Sbar;
            double mean = sum / (double)(N - 1);
            ref_params gp = *p;
            gp.alpha_ema = 1.0;
            int chi_g;
            ref_ctrl_step(&gcs, mean, &gp, &chi_g);
        }
        E_sweep[t] = E_last;
        sweeps_done = t + 1;
        if (stop_on_conv && t > 0 && fabs((E_last - E_prev) / E_last) < p->eps_conv) break;
        E_prev = E_last;
    }
    if (chi_final) for (int i = 0; i <= N; ++i) chi_final[i] = m.chi[i];
    if (theta_final_norm) {
        double nn = 0.0;
        size_t sz = (size_t)m.chi[0] * d * m.chi[1];
        for (size_t x = 0; x < sz; ++x) nn += m.A[0][x] * m.A[0][x];
        *theta_final_norm = sqrt(nn);
    }
    free(own);
    mps_free(&m);
    return status ? -status : sweeps_done;
}

/* ------------------------------------------------------------------------ */
/* Exact diagonalisation (independent of the MPO code): lowest eigenvalue of */
/* the spin chain in a basis of bit strings (bit i set = spin i up).         */
/*   model 0/1: XXZ / J1-J2 in the sector with n_up up spins (n_up < 0: all)  */
/*   model 2:   transverse-field Ising, full space (Pauli convention)        */
/* Plain Lanczos without reorthogonalisation (the lowest Ritz value is not   */
/* affected by loss of orthogonality); T's lowest eigenvalue by Sturm        */
/* bisection.  Stops when the estimate changes by < 1e-13 over 10 steps.    */
/* ------------------------------------------------------------------------ */
static int popcount64(uint64_t x) { int c = 0; while (x) { x &= x - 1; ++c; } return c; }

static int bsearch_u64(const uint64_t *a, size_t n, uint64_t key, size_t *pos)
{
    size_t lo = 0, hi = n;
    while (lo < hi) {
        size_t mid = (lo + hi) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    if (lo < n && a[lo] == key) { *pos = lo; return 1; }
    return 0;
}

static double sturm_lowest(int m, const double *a, const double *b)
{
    /* Gershgorin bounds */
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        if (a[i] - r < lo) lo = a[i] - r;
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 200; ++it) {
        double x = 0.5 * (lo + hi);
        /* count eigenvalues < x via the LDL^T pivots of T - x I */
        int cnt = 0;
        double q = a[0] - x;
        if (q < 0) cnt++;
        for (int i = 1; i < m; ++i) {
            if (q == 0.0) q = 1e-300;
            q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
            if (q < 0) cnt++;
        }
        if (cnt >= 1) hi = x; else lo = x;
        if (hi - lo <= 1e-15 * fabs(hi) + 1e-300) break;
    }
    return 0.5 * (lo + hi);
}

static void ed_apply(int model, int N, double J, double Delta, double J2, const uint64_t *basis,
                     size_t dim, int full, const double *x, double *y)
{
    for (size_t i = 0; i < dim; ++i) y[i] = 0.0;
    for (size_t i = 0; i < dim; ++i) {
        uint64_t st = full ? (uint64_t)i : basis[i];
        double xi = x[i];
        if (model == 2) {
            for (int q = 0; q + 1 < N; ++q) {
                int zq = ((st >> q) & 1) ? 1 : -1, zr = ((st >> (q + 1)) & 1) ? 1 : -1;
                y[i] += -J * zq * zr * xi;
            }
            for (int q = 0; q < N; ++q) {
                uint64_t f = st ^ ((uint64_t)1 << q);
                y[f] += -Delta * xi;
            }
            continue;
        }
        for (int range = 1; range <= (model == 1 ? 2 : 1); ++range) {
            double Jr = (range == 1) ? J : J2;
            double Dr = (range == 1) ? Delta : 1.0;
            if (Jr == 0.0) continue;
            for (int q = 0; q + range < N; ++q) {
                int r = q + range;
                int uq = (st >> q) & 1, ur = (st >> r) & 1;
                y[i] += Jr * Dr * ((uq == ur) ? 0.25 : -0.25) * xi;
                if (uq != ur) {
                    uint64_t f = st ^ ((uint64_t)1 << q) ^ ((uint64_t)1 << r);
                    size_t pos;
                    if (full) pos = (size_t)f;
                    else if (!bsearch_u64(basis, dim, f, &pos)) continue;
                    y[pos] += 0.5 * Jr * xi;
                }
            }
        }
    }
}

int ref_ed_ground(int model, int N, double J, double Delta, double J2, int n_up, int max_iter, double *E0)
{
    if (N < 2 || N > 30) return REF_EINVAL;
    int full = (model == 2) || (n_up < 0);
    size_t dim = 0;
    uint64_t *basis = NULL;
    if (full) {
        dim = (size_t)1 << N;
    } else {
        for (uint64_t s = 0; s < ((uint64_t)1 << N); ++s) if (popcount64(s) == n_up) dim++;
        basis = malloc(sizeof(uint64_t) * dim);
        size_t c = 0;
        for (uint64_t s = 0; s < ((uint64_t)1 << N); ++s) if (popcount64(s) == n_up) basis[c++] = s;
    }
    double *v0 = malloc(sizeof(double) * dim), *v1 = malloc(sizeof(double) * dim), *w = malloc(sizeof(double) * dim);
    double *a = malloc(sizeof(double) * (size_t)max_iter), *b = malloc(sizeof(double) * (size_t)max_iter);
    if (!v0 || !v1 || !w || !a || !b) return REF_ENOMEM;
    /* deterministic start vector with small irregular components */
    uint64_t h = 0x9E3779B97F4A7C15ull;
    double nn = 0.0;
    for (size_t i = 0; i < dim; ++i) {
        h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
        v1[i] = 1.0 + (double)(h >> 11) * (1.0 / 9007199254740992.0);
        nn += v1[i] * v1[i];
    }
    nn = sqrt(nn);
    for (size_t i = 0; i < dim; ++i) { v1[i] /= nn; v0[i] = 0.0; }
    double est = 0.0, prev = 1e300;
    int m = 0;
    double bprev = 0.0;
    for (int j = 0; j < max_iter; ++j) {
        ed_apply(model, N, J, Delta, J2, basis, dim, full, v1, w);
        double al = 0.0;
        for (size_t i = 0; i < dim; ++i) al += v1[i] * w[i];
        for (size_t i = 0; i < dim; ++i) w[i] -= al * v1[i] + bprev * v0[i];
        double bt = 0.0;
        for (size_t i = 0; i < dim; ++i) bt += w[i] * w[i];
        bt = sqrt(bt);
        a[j] = al; b[j] = bt;
        m = j + 1;
        if (m % 10 == 0 || bt < 1e-13) {
            est = sturm_lowest(m, a, b);
            if (fabs(est - prev) < 1e-13 * fabs(est) || bt < 1e-13) break;
            prev = est;
        }
        for (size_t i = 0; i < dim; ++i) { v0[i] = v1[i]; v1[i] = w[i] / bt; }
        bprev = bt;
    }
    est = sturm_lowest(m, a, b);
    *E0 = est;
    free(v0); free(v1); free(w); free(a); free(b); free(basis);
    return REF_OK;
}

/* Dense ED on the full space via ref_sym_eig (N <= 10): all eigenvalues.   */
int ref_ed_dense(int model, int N, double J, double Delta, double J2, double *evals)
{
    if (N > 10) return REF_EINVAL;
    size_t dim = (size_t)1 << N;
    double *H = calloc(dim * dim, sizeof(double)), *x = calloc(dim, sizeof(double)), *y = malloc(sizeof(double) * dim);
    double *Z = malloc(sizeof(double) * dim * dim);
    for (size_t c = 0; c < dim; ++c) {
        memset(x, 0, sizeof(double) * dim);
        x[c] = 1.0;
        ed_apply(model, N, J, Delta, J2, NULL, dim, 1, x, y);
        for (size_t r = 0; r < dim; ++r) H[r * dim + c] = y[r];
    }
    ref_sym_eig((int)dim, H, evals, Z);
    free(H); free(x); free(y); free(Z);
    return REF_OK;
}

/* Round-half-even check hook: exposes the rounding used by the controller. */
double ref_round_half_even(double x) { return nearbyint(x); }
int ref_rounding_mode_is_nearest(void) { return fegetround() == FE_TONEAREST; }

/* ------------------------------------------------------------------------ */
/* Circuit simulation with per-bond chi control (Section 8: circuit-level    */
/* bond dimension maps).                                                     */
/*                                                                           */
/* Qubit q of an N-qubit state is bit N-1-q of the basis index (qubit 0 the  */
/* most significant).  A two-qubit gate on (q, q+1) is a real 4 x 4 matrix    */
/* G[(s1' s2')][(s1 s2)], row-major, index 2 s1 + s2 with s1 the state of    */
/* qubit q.                                                                  */
/* ------------------------------------------------------------------------ */

/* Exact statevector: psi (2^N) <- G psi for each gate in order. */
int ref_statevector_apply(int N, double *psi, int n_gates, const int *pos, const double *gates)
{
    if (N < 2 || N > 30) return REF_EINVAL;
    const size_t dim = (size_t)1 << N;
    for (int g = 0; g < n_gates; ++g) {
        const int q = pos[g];
        if (q < 0 || q + 1 >= N) return REF_EINVAL;
        const double *G = gates + 16 * (size_t)g;
        const size_t b1 = (size_t)1 << (N - 1 - q), b2 = (size_t)1 << (N - 2 - q);
        for (size_t x = 0; x < dim; ++x) {
            if (x & (b1 | b2)) continue;          /* visit each group of four once */
            const size_t idx[4] = {x, x | b2, x | b1, x | b1 | b2};   /* s1 s2 = 00, 01, 10, 11 */
            double in[4], out[4];
            for (int i = 0; i < 4; ++i) in[i] = psi[idx[i]];
            for (int i = 0; i < 4; ++i) {
                double a = 0.0;
                for (int j = 0; j < 4; ++j) a += G[4 * i + j] * in[j];
                out[i] = a;
            }
            for (int i = 0; i < 4; ++i) psi[idx[i]] = out[i];
        }
    }
    return REF_OK;
}

/*
 * MPS circuit run.  The state starts as |0...0> (every bond dimension 1).
 * Layer l holds n_gates[l] gates on disjoint qubit pairs (brickwork); its
 * gates are gate_pos / gates from offset sum_{l' < l} n_gates[l'].  A layer is
 * one pass over the bonds, left to right for even l and right to left for
 * odd l, that moves the orthogonality centre across every bond: at bond k
 * theta = A_k A_{k+1}, the layer's gate on (k, k+1) if it has one, the SVD
 * (ref_svd), the entropy of the full spectrum (Eq. 5) and the truncation
 * (ref_trunc_k with the eps_trunc threshold), the split with the centre
 * moving in the pass direction and the retained spectrum renormalised.
 * At a gated bond the bond's controller takes a step on the entropy
 * (Algorithms 1-2 with Eqs. 8 and 16, ref_ctrl_step) and its chi bounds k;
 * with chi_warm (n_layers x (N-1), may be NULL) the gated bonds take chi from
 * it instead (a warm start from an earlier run's map).  A bond without a
 * gate keeps its spectrum (a gauge move: only the threshold applies).
 * Outputs: chi_map[l][b] = dimension of bond b (between qubits b, b+1) after
 * layer l; S_map[l][b] = the entropy at gated bonds (0 elsewhere); psi (2^N,
 * may be NULL) the final state contracted from the MPS (N <= 24).
 */
int ref_circuit_run(int N, int n_layers, const int *n_gates, const int *gate_pos, const double *gates,
                    const ref_params *p, const int *chi_warm, ref_ctrl_state *ctrl, int *chi_map, double *S_map,
                    double *psi)
{
    if (N < 2 || n_layers < 0) return -REF_EINVAL;
    const int d = 2;
    int *chi = calloc((size_t)N + 1, sizeof(int));
    double **A = calloc((size_t)N, sizeof(double *));
    ref_ctrl_state *own = NULL;
    if (!chi || !A) return -REF_ENOMEM;
    for (int i = 0; i <= N; ++i) chi[i] = 1;
    for (int i = 0; i < N; ++i) {
        A[i] = calloc(2, sizeof(double));
        A[i][0] = 1.0;                            /* |0> */
    }
    if (!ctrl) {
        own = calloc((size_t)(N - 1), sizeof(ref_ctrl_state));
        for (int b = 0; b < N - 1; ++b) own[b].chi = p->chi_min;
        ctrl = own;
    }
    int status = 0, off = 0;
    int *gate_at = malloc(sizeof(int) * (size_t)(N - 1));
    for (int l = 0; l < n_layers && status == 0; ++l) {
        for (int b = 0; b < N - 1; ++b) gate_at[b] = -1;
        for (int g = 0; g < n_gates[l]; ++g) {
            const int q = gate_pos[off + g];
            if (q < 0 || q >= N - 1 || gate_at[q] >= 0 || (q > 0 && gate_at[q - 1] >= 0) ||
                (q + 1 < N - 1 && gate_at[q + 1] >= 0)) { status = REF_EINVAL; break; }
            gate_at[q] = off + g;
        }
        if (status) break;
        const int go_right = (l % 2 == 0);
        for (int step = 0; step < N - 1; ++step) {
            const int k = go_right ? step : N - 2 - step;
            const int cl = chi[k], cm = chi[k + 1], cr = chi[k + 2];
            const int rows = cl * d, cols = d * cr;
            double *theta = malloc(sizeof(double) * (size_t)rows * cols);
            mm(rows, cols, cm, A[k], A[k + 1], theta);
            if (gate_at[k] >= 0) {
                const double *G = gates + 16 * (size_t)gate_at[k];
                double *t2 = malloc(sizeof(double) * (size_t)rows * cols);
                for (int a = 0; a < cl; ++a)
                    for (int qo = 0; qo < 4; ++qo)
                        for (int bb = 0; bb < cr; ++bb) {
                            double acc = 0.0;
                            for (int qi = 0; qi < 4; ++qi)
                                acc += G[4 * qo + qi] * theta[((size_t)a * 4 + qi) * cr + bb];
                            t2[((size_t)a * 4 + qo) * cr + bb] = acc;
                        }
                free(theta);
                theta = t2;
            }
            const int r = rows < cols ? rows : cols;
            double *U = malloc(sizeof(double) * (size_t)rows * r);
            double *s = malloc(sizeof(double) * (size_t)r);
            double *Vt = malloc(sizeof(double) * (size_t)r * cols);
            double *eps = malloc(sizeof(double) * (size_t)(r + 1));
            int sst = ref_svd(rows, cols, theta, U, s, Vt, p->jacobi_max_sweeps > 0 ? p->jacobi_max_sweeps : 60);
            if (sst != REF_OK) status = sst;
            const double S = ref_entropy(r, s, eps);
            int chi_c;
            if (gate_at[k] >= 0) {
                int c2;
                if (chi_warm) {
                    chi_c = chi_warm[(size_t)l * (N - 1) + k];
                } else {
                    ref_ctrl_step(&ctrl[k], S, p, &c2);
                    chi_c = c2;
                }
            } else {
                chi_c = p->chi_max;                   /* a gauge move keeps the spectrum */
            }
            if (S_map) S_map[(size_t)l * (N - 1) + k] = gate_at[k] >= 0 ? S : 0.0;
            int kk = ref_trunc_k(r, s, chi_c, p->eps_trunc, p->multiplet_guard);
            double z = 0.0;
            for (int j = 0; j < kk; ++j) z += s[j] * s[j];
            z = sqrt(z);
            free(A[k]); free(A[k + 1]);
            A[k] = malloc(sizeof(double) * (size_t)rows * kk);
            A[k + 1] = malloc(sizeof(double) * (size_t)kk * cols);
            for (int i = 0; i < rows; ++i)
                for (int j = 0; j < kk; ++j)
                    A[k][(size_t)i * kk + j] = U[(size_t)i * r + j] * (go_right ? 1.0 : s[j] / z);
            for (int j = 0; j < kk; ++j)
                for (int c = 0; c < cols; ++c)
                    A[k + 1][(size_t)j * cols + c] = Vt[(size_t)j * cols + c] * (go_right ? s[j] / z : 1.0);
            chi[k + 1] = kk;
            free(theta); free(U); free(s); free(Vt); free(eps);
        }
        if (chi_map) for (int b = 0; b < N - 1; ++b) chi_map[(size_t)l * (N - 1) + b] = chi[b + 1];
        off += n_gates[l];
    }
    if (psi && status == 0 && N <= 24) {
        /* contract: T (2^i x chi_i) <- T A_i reshaped, qubit 0 most significant */
        size_t rows = 1;
        double *T = malloc(sizeof(double));
        T[0] = 1.0;
        for (int i = 0; i < N; ++i) {
            const int ci = chi[i], cn = chi[i + 1];
            double *T2 = malloc(sizeof(double) * rows * (size_t)d * cn);
            mm((int)rows, d * cn, ci, T, A[i], T2);        /* (rows x ci) (ci x 2 cn) */
            free(T);
            T = T2;
            rows *= 2;                                      /* (rows*2) x cn, row = (prefix, s_i) */
        }
        memcpy(psi, T, sizeof(double) * rows);
        free(T);
    }
    for (int i = 0; i < N; ++i) free(A[i]);
    free(A); free(chi); free(own); free(gate_at);
    return status ? -status : REF_OK;
}
