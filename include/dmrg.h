/*
 * dmrg.h -- C ABI of the GB300 (sm_103a) adaptive two-site DMRG library.
 *
 * The library implements the per-bond local update of adaptive two-site DMRG
 * described in arXiv 2604.03960 ("Adaptive Tensor Network Simulation via
 * Entropy-Feedback PID Control and GPU-Accelerated SVD"): the effective
 * Hamiltonian eigenproblem of Eq. (19) solved by Lanczos, the SVD of the
 * two-site tensor (Eq. 20), the von Neumann entropy (Eq. 5), the EMA ->
 * predictor -> PID choice of the bond dimension (Eqs. 8-11, 16; Algorithms
 * 1-2), truncation (Eq. 4, Section 10) and the environment update.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - All tensors are FP64, row-major, last index fastest, spin-1/2 (d = 2).
 *  - MPO  W[i][wl][wr][s][s']   (N sites, D x D x 2 x 2 each; s = bra, s' = ket).
 *    The left boundary selects row D-1, the right boundary column 0.
 *  - MPS  A[i][a][s][b]          chi_i x 2 x chi_{i+1}.
 *  - Environments L[w][a'][a], R[w][b'][b] (D x chi x chi; a' bra, a ket).
 *  - Two-site tensor theta[a][s1][s2][b]; as a matrix it is (2 chi_l) x (2 chi_r).
 *  - Pointers named *_dev are device pointers owned by the caller (normally
 *    allocated by PyTorch); the library never frees or retains them beyond
 *    the call.  Pointers named *_host are host pointers.
 *  - All work is enqueued on the context's stream.  Calls that return host
 *    values synchronise that stream before returning.
 *  - Every call returns a dmrg_status.  Errors found on the device (a bounded
 *    wait that gave up, a non-finite value) are recorded in a device status
 *    word and reported by the next synchronising call or dmrg_get_status();
 *    no call traps or aborts.
 *  - The library allocates its own workspace (device arena) inside
 *    dmrg_create/dmrg_state_create and frees it in the matching destroy.
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_ctx dmrg_ctx;
typedef struct dmrg_state dmrg_state;

typedef enum {
    DMRG_OK = 0,
    DMRG_EINVAL = 1,       /* bad argument (null pointer, size out of range) */
    DMRG_ENOMEM = 2,       /* device allocation failed                        */
    DMRG_ENOCONV = 3,      /* Jacobi SVD did not converge in jacobi_max_sweeps */
    DMRG_ENAN = 4,         /* non-finite value detected                       */
    DMRG_ETIMEOUT = 5,     /* a bounded device-side wait gave up              */
    DMRG_ECUDA = 6,        /* a CUDA runtime call failed                      */
    DMRG_EUNSUPPORTED = 7  /* option not available (e.g. precision on this device) */
} dmrg_status;

typedef enum { DMRG_XXZ = 0, DMRG_J1J2 = 1, DMRG_TFIM = 2 } dmrg_model;

typedef enum {
    DMRG_PREC_FP64 = 0,    /* every contraction in FP64                                  */
    DMRG_PREC_3XTF32 = 1,  /* theta and H_eff contractions as 3xTF32 tcgen05 GEMMs with
                              FP32 accumulation; environment updates in FP64 (option
                              "mixed_env_tc" moves them to the tensor cores); SVD as an
                              FP32 Jacobi whose retained isometry is re-orthonormalised
                              in FP64; Lanczos vectors, tridiagonal solve and entropy FP64 */
    DMRG_PREC_BF16X3 = 2   /* reserved: split-BF16 contractions                           */
} dmrg_precision;

typedef enum {
    DMRG_CTRL_PID = 0,       /* EMA -> predictor -> PID (Algorithm 2, Eqs. 8, 16)       */
    DMRG_CTRL_DIRECT = 1,    /* chi = clamp(ceil(gamma exp(Sbar))) (Algorithm 1)         */
    DMRG_CTRL_FIXED = 2,     /* chi = chi_fixed                                          */
    DMRG_CTRL_THRESHOLD = 3, /* chi = chi_max; the eps_trunc threshold decides (Sec. 10) */
    DMRG_CTRL_MLP = 4,       /* learned scheduler with the PID as fallback               */
    DMRG_CTRL_GLOBAL = 5,    /* global adaptive chi (Section 6): one PID on the mean of the
                                per-bond filtered entropies, stepped once per sweep (with
                                alpha = 1: the inputs are already filtered); every bond is
                                truncated to the same chi, which starts at chi_min        */
    DMRG_CTRL_HOLD = 6,      /* no controller step: every bond keeps the chi its controller
                                holds (no counterpart in the paper; with
                                dmrg_state_set_params it converges a run at the schedule
                                the controller reached)                                   */
    DMRG_CTRL_REPLAY = 7     /* the chi of every visit of dmrg_sweep comes from the schedule
                                set by dmrg_state_set_schedule (no counterpart in the
                                paper: runs another precision on a recorded schedule)     */
} dmrg_ctrl_mode;

/* Parameters of the local update and of the controller. */
typedef struct {
    double alpha_ema;   /* EMA smoothing alpha, Eq. (8)                               */
    double gamma;       /* margin gamma of the direct map, Eq. (7)                    */
    double S_target;    /* target entropy, Eq. (9)                                    */
    double Kp, Ki, Kd;  /* PID gains, Eq. (10)                                        */
    double beta;        /* predictor aggressiveness, Eq. (16)                         */
    double eps_trunc;   /* drop s_j / |s| <= eps_trunc (Section 10)                   */
    double eps_conv;    /* stop when |dE/E| < eps_conv (Section 10)                   */
    int chi_min, chi_max;
    int lanczos_steps;  /* Krylov steps per bond (K)                                   */
    int max_sweeps;     /* sweep horizon (feature scaling of the learned scheduler)   */
    int jacobi_max_sweeps;
    int prec;           /* dmrg_precision                                              */
    int ctrl;           /* dmrg_ctrl_mode                                              */
    int ema_init_zero;  /* 1: first EMA value alpha*S (Section 10) instead of S (Sec. 4) */
    int multiplet_guard;/* 1: never truncate inside a group of equal singular values  */
    int pid_steps_per_sweep; /* 2: controller step on every visit; 1: L->R visits only */
    int chi_init;       /* bond dimension of the random initial MPS                   */
    int chi_fixed;      /* chi for DMRG_CTRL_FIXED                                    */
    int second_order;   /* 1: second-order predictor (Section 7, curvature term)      */
} dmrg_params;

typedef struct {
    int N;              /* number of sites                                             */
    double J;           /* nearest-neighbour coupling (TFIM: zz coupling)              */
    double Delta;       /* XXZ anisotropy (TFIM: transverse field h)                   */
    double J2;          /* next-nearest-neighbour coupling (J1-J2 only)               */
} dmrg_model_params;

/* Per-bond controller state (device-resident; same meaning as Algorithm 2's
 * inputs plus the predictor's and the learned scheduler's history). */
typedef struct {
    double Sbar, Sbar_prev, Sbar_prev2, e_prev, I;
    double hist[8];
    int chi, initialized, nhist, pad;
} dmrg_ctrl_state;

/* One record per sweep, filled by dmrg_sweep (host memory). */
typedef struct {
    double E;              /* Ritz value at the last bond of the sweep                 */
    double max_trunc_err;  /* max over visits of eps (Eq. 4)                           */
    double mean_chi;       /* mean retained bond dimension over the sweep's visits     */
    double seconds;        /* device time of the sweep (CUDA events)                   */
    double flops;          /* algorithmic flops of the sweep (realised shapes)         */
    int max_chi;           /* largest retained bond dimension                          */
    int n_visits;          /* bond visits (2N - 3)                                     */
    int jacobi_sweeps;     /* total Jacobi sweeps over the sweep's SVDs                */
    int lanczos_steps;     /* total Lanczos steps over the sweep                        */
} dmrg_sweep_record;

/* Per-visit record (bond, Ritz value, entropy, truncation error, retained k,
 * controller chi), filled by dmrg_sweep when requested. */
typedef struct {
    int bond, k, chi_ctrl, direction;
    double E, S, trunc_err;
    int jacobi_sweeps;     /* Jacobi sweeps of the visit's SVD (negative: not converged) */
    int lanczos_steps;     /* Krylov steps taken                                          */
    float feat[10];        /* learned-scheduler features after this visit's controller
                              step: last 8 EMA entropies, (bond+1)/N, sweep/max_sweeps   */
    int k_star;            /* smallest k with sum_{j>=k} p_j <= eps_target^2 (context
                              option "mlp_eps_target"): the training label source       */
    int mlp_used;          /* 1 if the learned scheduler's chi was taken this visit       */
} dmrg_visit_record;

/* ---------------------------------------------------------------------- */
/* Context                                                                */
/* ---------------------------------------------------------------------- */
/* Create a context on `device` that enqueues all work on `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  *out receives the handle. */
dmrg_status dmrg_create(dmrg_ctx **out, int device, void *cuda_stream);
void dmrg_destroy(dmrg_ctx *ctx);
/* Device status word: DMRG_OK or the first device-side error since the last
 * call (then cleared).  Synchronises the stream. */
dmrg_status dmrg_get_status(dmrg_ctx *ctx);
const char *dmrg_status_string(dmrg_status s);
/* Tuning knobs of a context (no counterpart in the paper): "tc_force" (1: use
 * the tensor cores even for tiny products), "tc_min_work" (M N K below
 * which 3xTF32 requests run on the FP32 CUDA-core kernel with compensated
 * sums; 2^24 by default), "tc_bn" (0, 64, 128 or 256: tile width of the
 * tensor-core GEMM, 0 = heuristic), "tc_split_kb"
 * (tensor-core GEMM: most 32-wide blocks of the 3 K split products one FP32
 * accumulator sums, 8; beyond, K is split and the slices added in FP64;
 * 0 = never split), "cjac32" (1, default: the FP32 Jacobi of the mixed form
 * runs on one thread-block cluster of 8 CTAs, or 16 where 8 CTAs' shared
 * memory cannot hold the blocks, vectors in blocks in the CTAs' shared
 * memory and moved between them through distributed shared memory, for
 * problems of at least "cjac_min_r" (32) vectors with at most 32 vectors a
 * block and length <= 512; 0: the kernels below), "tc_presplit" (1, default:
 * the matvec's L and R are split into TF32 parts once per local update and
 * the Lanczos vector and mix output by the kernels that make them; 0: every
 * product splits its operands), "lz_fused" (1, default: one cooperative
 * launch per Lanczos step for both Gram-Schmidt passes; 0: five launches),
 * "lz_cluster_n" (the fused step on one thread-block cluster, with cluster
 * barriers instead of grid barriers, for vectors up to this length; 4096
 * by default, 0 = never),
 * "f64_fill" (1, default: FP64 GEMMs that would leave SMs idle take 32 x 32
 * tiles and split K), "f32_fill" (1, default: the same for the FP32
 * small products of the mixed form), "gjac32" (grouped block
 * FP32 Jacobi: 0 never (default),
 * 1 for problems that fit one CTA's shared memory, 2 always), "gjac_nv" / "gjac_groups" (its vectors per block pair, 16 or
 * 32, and groups per CTA, 1-4; 0 = by size / autotuner), "jacobi64_gram"
 * (1: FP64 Jacobi on the grouped kernel, 0: one warp per pair),
 * "jacobi64_precond" (1: FP32 preconditioning pass before the FP64
 * Jacobi), "jacobi32_tol" (FP32 Jacobi: rotate while a pair's cosine exceeds
 * this, 1e-6), "mixed_svd64" (1: the 3xTF32 form takes the FP64 SVD and split, so
 * only its contractions are in reduced precision), "prof_mask"
 * (bit k set: dmrg_profile brackets the launches of kind k; default all 9
 * kinds; bracketing one kind keeps the events off every other launch),
 * "mlp_eps_target" (truncation-error target of the k_star label, 1e-5),
 * "mixed_env_tc" (1: environment updates of the 3xTF32 form on the tensor
 * cores instead of FP64), "svd_prec" (standalone svd_truncate: 0 FP64 Jacobi,
 * 1 mixed: FP32 Jacobi, FP64-re-orthonormalised isometry, tensor-core
 * projection for the other factor; values below 2^-22 s_0 are not resolved),
 * "bjac_pairs" / "bjac_inner" (blocked FP32 Jacobi: target block pairs per
 * round, inner sweeps per block pair), "bjac_gram" (1: the blocked FP32
 * Jacobi takes its inner sweep on the block pair's Gram matrix and applies
 * the accumulated rotation once; 0: rotations of the vectors themselves),
 * "tjac" (FP32 Jacobi of the mixed form: 64 or 128 = blocked one-sided
 * Jacobi with pairs of that many vectors, whose Gram blocks G = P P^T and
 * block rotations P <- Q^T P are 3xTF32 tcgen05 GEMMs around one Jacobi sweep
 * of each G in a CTA; 0 = off; default 128), "tjac_min_r" (from this many
 * vectors on, ahead of the other FP32 kernels; default 3072; not taken
 * while the stream is captured, since it reads a convergence counter on the
 * host once per outer sweep), "jacobi_max_sweeps" (standalone
 * svd_truncate and svd_truncate_batched), "batched_inner" (svd_truncate_batched:
 * Jacobi sweeps on each 32 x 32 block-pair Gram matrix, 4), "batched_floor32"
 * (FP32 svd_truncate_batched: vectors with norm below this x |A|_F take no
 * rotation, 2^-23).  DMRG_EINVAL for an unknown name or value. */
dmrg_status dmrg_set_option(dmrg_ctx *ctx, const char *name, double value);
/* Bond dimension D of the MPO of `model` (5, 8, 3), or -1. */
int dmrg_mpo_dim(int model);

/* ---------------------------------------------------------------------- */
/* Hot-path entry points                                                  */
/* ---------------------------------------------------------------------- */

/* MPO of the paper's benchmark Hamiltonians: XXZ (Eq. 18 at Delta = 1),
 * J1-J2 and transverse-field Ising (Table 5), written on the device into
 * W_dev (N * D * D * 4 doubles, caller-owned, layout above). */
dmrg_status dmrg_build_mpo(dmrg_ctx *ctx, dmrg_model model, const dmrg_model_params *mp, double *W_dev);

/* Create a DMRG state for N sites: copies W_dev (N*D*D*4) and the Gaussian
 * entries of the initial MPS (mps_init_dev, site after site, chi_i =
 * min(chi_init, 2^i, 2^(N-i)), "random initial state" of Section 10), brings
 * it to right-canonical form on the device, builds every right environment
 * and sets each bond's controller to chi = chi_min, S-bar = I = 0
 * (Section 10).  Memory for the MPS, environments and workspace is sized for
 * chi_max and owned by the state.  The parameter block is copied. */
dmrg_status dmrg_state_create(dmrg_ctx *ctx, int D, const dmrg_model_params *mp, const double *W_dev,
                              const dmrg_params *p, const double *mps_init_dev, dmrg_state **out);
void dmrg_state_destroy(dmrg_state *st);

/* Run n_sweeps two-site sweeps (Section 10): left to right over bonds
 * 0..N-2, right to left over N-3..0, a local update at each visit.
 * rec_host (n_sweeps entries) receives one record per sweep; visits_host
 * (optional, n_sweeps*(2N-3) entries) one record per bond visit.  If
 * stop_on_conv, stops once |dE/E| < eps_conv; *sweeps_done (optional)
 * receives the number of sweeps run. */
dmrg_status dmrg_sweep(dmrg_ctx *ctx, dmrg_state *st, int n_sweeps, int stop_on_conv,
                       dmrg_sweep_record *rec_host, dmrg_visit_record *visits_host, int *sweeps_done);

/* Advance n_chains independent chains (batched bond steps, Section 10's
 * sweep on each) by n_sweeps sweeps each.  Chain c is states[c] on ctxs[c];
 * every chain needs a context of its own, with a stream of its own (a
 * context's workspace serves one chain at a time).  The bond steps are
 * interleaved: the first phase of the current bond step of every live chain
 * (two-site tensor, Lanczos, SVD, entropy, controller) is enqueued, then the
 * second phase of each (truncation, split, environment update) after its
 * retained k has reached the host, so the chains' kernels overlap on the
 * device; chains of different lengths finish at different steps.  Results
 * are those of dmrg_sweep on each chain alone.  rec_host (host, may be NULL)
 * receives n_chains x n_sweeps records, chain-major; their `seconds` is 0
 * (the chains share the device), and *seconds_out (may be NULL) gets the
 * wall time of the whole call. */
dmrg_status dmrg_sweep_chains(int n_chains, dmrg_ctx *const *ctxs, dmrg_state *const *states, int n_sweeps,
                              dmrg_sweep_record *rec_host, double *seconds_out);
/* One local update at `bond` (sites bond, bond+1) in `direction` (+1: the
 * orthogonality centre moves right, -1: left).  The state's centre must
 * be at that bond (as it is at every visit of dmrg_sweep).  *E_out (host)
 * receives the Ritz value (Eq. 19); *k_out (optional) the retained chi. */
dmrg_status bond_update(dmrg_ctx *ctx, dmrg_state *st, int bond, int direction, double *E_out, int *k_out);

/* SVD of the m x n row-major matrix theta_dev (Eq. 20), by one-sided
 * (Hestenes) Jacobi on the device, then truncation (Section 10):
 *   k = min(chi_max, rank, #{s_j/|s| > eps}), k >= 1.
 * Outputs (caller-owned device buffers, r = min(m, n)):
 *   U_dev  m x r, s_dev r (descending), Vt_dev r x n  -- the full factors;
 *   the retained factors are their first k columns/values/rows.
 * Host outputs: *k_out, *S_out (Eq. 5 entropy of the full spectrum),
 * *trunc_err_out (Eq. 4 on the normalised spectrum).  Any host output may
 * be NULL.  Synchronises the stream.  Returns DMRG_ENOCONV if the Jacobi
 * iteration did not converge within the context's jacobi_max_sweeps (60). */
dmrg_status svd_truncate(dmrg_ctx *ctx, const double *theta_dev, int m, int n, int chi_max, double eps,
                         double *U_dev, double *s_dev, double *Vt_dev, int *k_out, double *S_out,
                         double *trunc_err_out);

/* svd_truncate for callers that cannot allocate device memory (no
 * counterpart in the paper).  Same inputs, outputs and results as
 * svd_truncate in its default FP64 form, limited to m, n <= 256.  Some
 * callers cannot call cudaMalloc: code whose device memory is owned by
 * another component (a framework's caching pool that must see every
 * allocation, or a budget fixed ahead of time), and time-critical loops in
 * which an allocation, which can synchronise the whole device, is not
 * acceptable.  This call allocates nothing: its scratch is a file-scope
 * device array of about 1.06 MiB (1088 KiB reserved) that every GPU which
 * loads the library holds until the process exits.
 *  - The first call on a device looks up that array's device address with
 *    that device current (with CUDA's lazy module loading this lookup also
 *    loads the library's device code, which creates the array), so only the
 *    calls after the first are free of any device-memory growth; make this
 *    first call before any stream capture.
 *  - Every call on a device shares the one array, and it keeps the last
 *    call's contents (the call clears what must start at zero).  Calls that
 *    overlap on the GPU (other streams, other threads, other contexts on the
 *    same device) race on it: serialise them.
 *  - The SVD is always the FP64 Jacobi of svd_truncate's default form,
 *    whatever the context's "svd_prec" option says.
 *  - The call synchronises the context's stream before it returns (it reads
 *    k, S and the truncation error back to the host).
 *  - Sizes above 256 return DMRG_EINVAL with a message on stderr. */
dmrg_status svd_truncate_noalloc(dmrg_ctx *ctx, const double *theta_dev, int m, int n, int chi_max, double eps,
                                 double *U_dev, double *s_dev, double *Vt_dev, int *k_out, double *S_out,
                                 double *trunc_err_out);

/* Batched SVD + entropy + truncation of `batch` independent matrices (the
 * uneven isolated-SVD workload; Eqs. 4-5, 20).  Matrix b is m[b] x n[b]
 * (host arrays), row-major at theta_dev + off_in[b]; U_b (m x r), s_b (r,
 * descending) and Vt_b (r x n), r = min(m, n), go to U_dev + off_U[b],
 * s_dev + off_s[b], Vt_dev + off_Vt[b] (host offset arrays, counted in
 * doubles).  k_dev[b], S_dev[b], err_dev[b] (device) receive k = min(chi_max,
 * rank, #{s_j/|s| > eps}), the entropy and the truncation error.  prec:
 * DMRG_PREC_FP64, or DMRG_PREC_3XTF32 for FP32 Jacobi (factors orthogonal to
 * ~1e-5; values below 2^-22 s_0 unresolved).  One CTA per matrix.  No host
 * synchronisation; the descriptors are staged in the context's pinned
 * memory, so after a first call of the same shapes the call can be captured
 * with dmrg_graph_begin/end and replayed with dmrg_graph_launch (a batched
 * call of other shapes on the same context between capture and replay
 * changes what the graph replays).  sweeps_dev (device, batch ints, may be
 * NULL) receives the Jacobi sweeps of each matrix, negative if it did not
 * converge within "jacobi_max_sweeps" (the status word then holds
 * DMRG_ENOCONV). */
dmrg_status svd_truncate_batched(dmrg_ctx *ctx, int prec, int batch, const int *m, const int *n,
                                 const double *theta_dev, const long long *off_in, double *U_dev,
                                 const long long *off_U, double *s_dev, const long long *off_s, double *Vt_dev,
                                 const long long *off_Vt, int chi_max, double eps, int *k_dev, double *S_dev,
                                 double *err_dev, int *sweeps_dev);
/* Autotuner (no counterpart in the paper): times, on this context's device
 * and stream, the launch choices of the hot path and keeps the fastest in the
 * context, where the launchers consult it before their heuristics.
 * dmrg_autotune_gemm: for each M x N x K (host arrays of n_shapes), the
 * 3xTF32 tensor-core GEMM with 64-, 128- and 256-column tiles at split
 * depths 4 and 8 (K blocks of 32 per FP32 accumulator; depth 8 is the
 * default, 4 accumulates less); the choice applies to the shape's bucket
 * (ceil log2 of each dimension).  At a given depth the result bits do not
 * depend on the tile width.  dmrg_autotune_svd: for each n (host array), the
 * mixed-precision SVD of an n x n matrix: the cluster FP32 Jacobi on 8 and on
 * 16 CTAs (where the vectors fit; this sets its block width ceil(n / 2C)),
 * and the other kernels (with the grouped FP32 Jacobi, option "gjac32", its
 * block-pair width, 16 or 32 vectors, and groups per CTA, 1, 2 or 4; else
 * the blocked kernel's block-pair target in {24, 48, 96, 152} and 1 or 2
 * inner sweeps), and from n = 256 on the blocked Jacobi whose Gram blocks
 * and block rotations are tcgen05 GEMMs with pairs of 64 and of 128 vectors;
 * the fastest applies to the (ceil log2 n, ceil log2 n)
 * bucket.  Inputs are generated on the device; `reps` timed calls follow one
 * warm-up call.  These calls allocate and free device memory and
 * synchronise.  dmrg_autotune_save / _load write and read the tables as JSON
 * (format "dmrg-autotune-4"; load also reads formats 1 to 3) and load
 * replaces the tables; DMRG_EINVAL for a file that is missing or in none of
 * these formats.
 * dmrg_autotune_entries: number of GEMM (which = 0) or SVD (1) entries. */
dmrg_status dmrg_autotune_gemm(dmrg_ctx *ctx, int n_shapes, const int *M, const int *N, const int *K, int reps);
dmrg_status dmrg_autotune_svd(dmrg_ctx *ctx, int n_sizes, const int *n, int reps);
dmrg_status dmrg_autotune_clear(dmrg_ctx *ctx);
dmrg_status dmrg_autotune_save(const dmrg_ctx *ctx, const char *path);
dmrg_status dmrg_autotune_load(dmrg_ctx *ctx, const char *path);
int dmrg_autotune_entries(const dmrg_ctx *ctx, int which);

/* CUDA-graph capture of a context's stream (which must not be the legacy
 * default stream): begin, end (instantiates into *graph_exec), launch, destroy. */
dmrg_status dmrg_graph_begin(dmrg_ctx *ctx);
dmrg_status dmrg_graph_end(dmrg_ctx *ctx, void **graph_exec);
dmrg_status dmrg_graph_launch(dmrg_ctx *ctx, void *graph_exec);
dmrg_status dmrg_graph_destroy(void *graph_exec);

/* One controller step for each of n_bonds bonds (Algorithms 1-2 with
 * Eqs. 8 and 16): S_raw_dev[i] is bond i's raw entropy, st_dev[i] its
 * state (updated in place), chi_out_dev[i] receives the new chi.  All
 * arithmetic is FP64 without fused multiply-add, in a fixed order, so a
 * recorded entropy sequence reproduces the integer chi schedule exactly. */
dmrg_status entropy_pid_step(dmrg_ctx *ctx, int n_bonds, const double *S_raw_dev, dmrg_ctrl_state *st_dev,
                             const dmrg_params *p_host, int *chi_out_dev);

/* ---------------------------------------------------------------------- */
/* Circuit-level bond dimension maps (Section 8)                          */
/* ---------------------------------------------------------------------- */
/* An MPS of N qubits (|0...0> at creation, every bond dimension 1) under
 * layers of two-qubit gates, with one controller per bond.  Qubit q is the
 * q-th site; amplitudes index qubit 0 as the most significant bit.
 * Parameters: chi_min/chi_max, eps_trunc, multiplet_guard and the controller
 * (ctrl = PID, DIRECT, FIXED or THRESHOLD, else DMRG_EINVAL) as in
 * dmrg_params; the state owns its device memory (sized for chi_max). */
typedef struct dmrg_circ dmrg_circ;
dmrg_status dmrg_circ_create(dmrg_ctx *ctx, int N, const dmrg_params *p, dmrg_circ **out);
void dmrg_circ_destroy(dmrg_circ *c);
/* Apply one layer: gate g acts on qubits (pos_host[g], pos_host[g] + 1) with
 * the real 4 x 4 matrix gates_host + 16 g, row-major G[(s1' s2')][(s1 s2)],
 * index 2 s1 + s2, s1 the state of the first qubit; the pairs must be
 * disjoint (DMRG_EINVAL otherwise).  The layer is one pass over the bonds,
 * left to right for the even-numbered layers of the state and right to left
 * for the odd ones, that moves the orthogonality centre across every bond:
 * theta, the gate if the bond has one, the SVD (Eq. 20), the entropy of the
 * full spectrum (Eq. 5), the truncation and the split.  At a gated bond the
 * bond's controller steps on the entropy (Algorithms 1-2, Eqs. 8 and 16) and
 * its chi bounds the retained dimension, or, with chi_warm_host (N - 1
 * entries, host, may be NULL), the recorded chi of an earlier run does (warm
 * start); a bond without a gate keeps its spectrum above eps_trunc.
 * chi_row_host (N - 1, may be NULL) receives the bond dimensions after the
 * layer (one row of the map chi_i^(l)), S_row_host (N - 1, may be NULL) the
 * entropies of the gated bonds (0 elsewhere).  Synchronises the stream. */
dmrg_status dmrg_circ_apply_layer(dmrg_circ *c, int n_gates, const int *pos_host, const double *gates_host,
                                  const int *chi_warm_host, int *chi_row_host, double *S_row_host);
/* The state's 2^N amplitudes (N <= 22) into the caller's device buffer
 * psi_dev.  Allocates a 2^N scratch in the context and synchronises. */
dmrg_status dmrg_circ_state(dmrg_circ *c, double *psi_dev);

/* ---------------------------------------------------------------------- */
/* Building blocks exposed for sampled parity checks and benchmarks       */
/* ---------------------------------------------------------------------- */

/* Eq. (5) entropy and Eq. (4) truncation errors of one spectrum:
 * S_dev[0] = -sum p ln p, eps_dev[k] = sqrt(sum_{j>=k} p_j), k = 0..n
 * (eps_dev optional, n+1 entries).  FP64 with compensated summation. */
dmrg_status dmrg_entropy(dmrg_ctx *ctx, int n, const double *s_dev, double *S_dev, double *eps_dev);

/* y = H_eff theta (Eq. 19) for environments L_dev (D x cl x cl), R_dev
 * (D x cr x cr), MPO tensors W1_dev, W2_dev (D x D x 2 x 2) and
 * theta_dev (cl x 2 x 2 x cr), in precision `prec` (dmrg_precision). */
dmrg_status dmrg_heff_apply(dmrg_ctx *ctx, int prec, int D, int cl, int cr, const double *L_dev,
                            const double *W1_dev, const double *W2_dev, const double *R_dev,
                            const double *theta_dev, double *y_dev);

/* Environment updates of a bond step: left L_new (D x ck x ck) from L
 * (D x cl x cl), W and a left-canonical site A (cl x 2 x ck); right R_new
 * (D x ck x ck) from R (D x cr x cr), W and a right-canonical B (ck x 2 x cr). */
dmrg_status dmrg_env_left(dmrg_ctx *ctx, int prec, int D, int cl, int ck, const double *L_dev,
                          const double *W_dev, const double *A_dev, double *Lnew_dev);
dmrg_status dmrg_env_right(dmrg_ctx *ctx, int prec, int D, int ck, int cr, const double *R_dev,
                           const double *W_dev, const double *B_dev, double *Rnew_dev);

/* K-step Lanczos for the lowest eigenpair of H_eff (Eq. 19): theta_dev is
 * the start vector on entry and the normalised Ritz vector on return;
 * *E_out (host) the Ritz value, *steps_out (host, optional) the steps taken. */
dmrg_status dmrg_lanczos(dmrg_ctx *ctx, int prec, int D, int cl, int cr, const double *L_dev,
                         const double *W1_dev, const double *W2_dev, const double *R_dev,
                         double *theta_dev, int K, double *E_out, int *steps_out);

/* C (M x N) = A (M x K) B (K x N), all row-major FP64 device buffers, in
 * precision `prec`; the contraction engine behind every step above.  With
 * prec = DMRG_PREC_3XTF32 each operand is split into two TF32 parts and the
 * product runs on the tcgen05 tensor cores with FP32 accumulation; products
 * smaller than 2^22 multiply-adds use the FP64 kernel unless force_tc != 0. */
dmrg_status dmrg_gemm(dmrg_ctx *ctx, int prec, int force_tc, int M, int N, int K, const double *A_dev,
                      const double *B_dev, double *C_dev);

/* Accessors of a state (device buffers owned by the state; valid until the
 * next call that modifies it). */
dmrg_status dmrg_state_chi(dmrg_state *st, int *chi_host /* N+1 */);
dmrg_status dmrg_state_site(dmrg_state *st, int i, const double **A_dev);
/* Copy environment k (left: L_k, else R_k) in the layout above into the
 * caller's buffer E_out_dev (D x chi_k x chi_k); synchronises the stream. */
dmrg_status dmrg_state_env(dmrg_state *st, int left, int k, double *E_out_dev);
dmrg_status dmrg_state_ctrl(dmrg_state *st, dmrg_ctrl_state **ctrl_dev /* N-1 */);
/* Checkpoint / restore of the MPS (no counterpart in the paper): the site
 * tensors at the current bond dimensions, concatenated site after site
 * (sum_i chi_i * 2 * chi_{i+1} doubles, see dmrg_state_mps_size).  `out` /
 * `in` may be host (pageable or pinned) or device memory.  put_mps requires
 * the same bond dimensions and gauge as the matching get_mps (environments
 * are kept); both synchronise the stream. */
long long dmrg_state_mps_size(dmrg_state *st);
dmrg_status dmrg_state_get_mps(dmrg_state *st, double *out);
dmrg_status dmrg_state_put_mps(dmrg_state *st, const double *in);
/* Failure detection without a fault (no counterpart in the paper): runs the
 * bounded grid barrier of the cooperative kernels with two co-resident
 * blocks.  With absent = 1 one block never arrives; the other polls the
 * barrier spin_limit times, records DMRG_ETIMEOUT in the context's status
 * word and returns (no trap).  Returns the status read back (DMRG_ETIMEOUT
 * when absent = 1, DMRG_OK when both blocks arrive); the context stays
 * usable.  Allocates and frees 64 bytes and synchronises. */
dmrg_status dmrg_wait_selftest(dmrg_ctx *ctx, long long spin_limit, int absent);
/* Kernels launched by this library since it was loaded (all contexts). */
long long dmrg_launch_count(void);
/* Outer Jacobi sweeps of the context's last standalone svd_truncate (Eq. 20):
 * positive if the iteration converged, minus the count if it stopped at the
 * sweep limit, 0 before the first call.  Host read only; no GPU work. */
int dmrg_svd_last_sweeps(const dmrg_ctx *ctx);
/* Live timing of the heavy kernels (no counterpart in the paper): with
 * profiling on, CUDA events on the context stream bracket every launch of
 * kind 0 (tensor-core GEMM), 1 (FP32 Jacobi sweeps), 2 (FP64 Jacobi sweeps),
 * 3 (FP64 GEMM), 4 (H_eff / environment mixing), 5 (FP32 SIMT GEMM of small
 * products), 6 (QR preconditioning), 7 (Lanczos vector operations), 8 (the
 * entropy/controller/truncation decision).  dmrg_profile(ctx, on) resets the counters;
 * dmrg_profile_read returns the summed device time (ms), the launches and
 * their algorithmic flops and bytes. */
dmrg_status dmrg_profile(dmrg_ctx *ctx, int on);
dmrg_status dmrg_profile_read(dmrg_ctx *ctx, int kind, double *ms, long long *launches, double *flops, double *bytes);
/* Replace the state's controller and truncation parameters between sweeps
 * (no counterpart in the paper), e.g. DMRG_CTRL_HOLD to finish a run at the
 * chi the per-bond controllers reached.  chi_max, prec and lanczos_steps
 * must equal the state's (its memory is sized for them): DMRG_EINVAL
 * otherwise.  The controllers' device state is kept. */
dmrg_status dmrg_state_set_params(dmrg_state *st, const dmrg_params *p);
/* Schedule of DMRG_CTRL_REPLAY: chi_host[v] (host, n = 2N - 3 entries in
 * [1, chi_max]) bounds the retained dimension at visit v of every following
 * dmrg_sweep (k = min(chi, rank, threshold count)), until replaced.  The
 * schedule is copied.  bond_update is not available in that mode
 * (DMRG_EINVAL); a sweep without a schedule returns DMRG_EINVAL. */
dmrg_status dmrg_state_set_schedule(dmrg_state *st, const int *chi_host, int n);
/* Set the learned scheduler's parameters (4929 FP32 values, layout of
 * dmrg_mlp_forward) used when ctrl == DMRG_CTRL_MLP. */
dmrg_status dmrg_state_set_mlp(dmrg_state *st, const float *params_dev);

/* ---------------------------------------------------------------------- */
/* Learned scheduler (not in the paper): MLP 10 -> 64 -> 64 -> 1 with     */
/* exact-erf GELU, FP32.  Parameter layout: W1[64][10], b1[64],           */
/* W2[64][64], b2[64], W3[64], b3[1] (4929 floats).                       */
/* ---------------------------------------------------------------------- */
dmrg_status dmrg_mlp_forward(dmrg_ctx *ctx, const float *params_dev, int B, const float *X_dev, float *y_dev);
/* loss_dev[0] = mean_b (y_b - t_b)^2 and grad_dev = d loss / d params. */
dmrg_status dmrg_mlp_loss_grad(dmrg_ctx *ctx, const float *params_dev, int B, const float *X_dev,
                               const float *t_dev, float *loss_dev, float *grad_dev);
/* Train the network on (X_dev [B][10], t_dev [B]) for `steps` full-batch
 * Adam steps (lr, betas 0.9/0.999, eps 1e-8) starting at Adam step
 * first_step; m_dev, v_dev are the moment buffers (4929 floats each, zero
 * for a fresh start).  Every step runs dmrg_mlp_loss_grad's kernels and the
 * Adam kernel on the device; *loss_host (optional) receives the loss before
 * the last step. */
dmrg_status dmrg_mlp_train(dmrg_ctx *ctx, float *params_dev, int B, const float *X_dev, const float *t_dev,
                           float *m_dev, float *v_dev, int first_step, int steps, float lr, float *loss_host);
/* One Adam step (step is 1-based) on n parameters; m, v are moment buffers. */
dmrg_status dmrg_mlp_adam(dmrg_ctx *ctx, int n, float *params_dev, const float *grad_dev, float *m_dev,
                          float *v_dev, int step, float lr, float beta1, float beta2, float eps);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_GB300_H */
