/*
 * chase_gb300.h -- C ABI of a single-GPU (GB300, sm_103a) Chebyshev-accelerated
 * subspace iteration eigensolver (ChASE, Algorithm 1 of the paper).
 *
 * Problem (Section "Distributed eigensolvers", Eq. AV = V Lambda): the nev
 * lowest eigenpairs of a dense n x n complex Hermitian or real symmetric A.
 *
 * Conventions for every entry point
 *   - Matrices are column-major with an explicit leading dimension (elements).
 *     Complex matrices are interleaved (re, im) doubles (C99 double complex /
 *     cuDoubleComplex / torch.complex128 layout); real ones are doubles.
 *   - Pointers named *_dev are device pointers on the context's device; the
 *     caller owns them and they must stay valid for the duration of the call.
 *     Pointers named *_host are host pointers.
 *   - All work is enqueued on the context's stream.  Calls that return results
 *     to the host synchronise that stream; the others are asynchronous unless
 *     stated.
 *   - Every call returns a chase_status.  Nothing throws across the ABI.  On a
 *     non-OK status chase_last_error() holds a one-line description.  An
 *     asynchronous device error surfaces as CHASE_ERR_CUDA at the next call.
 *   - A is read-only: the Chebyshev shift (A - cI) is fused into the product
 *     epilogue and never applied to A in place (the paper shifts in place).
 */
#ifndef CHASE_GB300_H
#define CHASE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chase_ctx chase_ctx;

typedef enum {
  CHASE_OK = 0,
  CHASE_ERR_ARG = 1,          /* invalid argument (sizes, null pointer, mode) */
  CHASE_ERR_OOM = 2,          /* workspace does not fit in device memory */
  CHASE_ERR_NOCONV = 3,       /* maxiter outer iterations without locking nev pairs */
  CHASE_ERR_QR_BREAKDOWN = 4, /* Cholesky-QR failed even after the shifted fallback */
  CHASE_ERR_NAN = 5,          /* a NaN/Inf appeared (e.g. in A or the start block) */
  CHASE_ERR_CUDA = 6,         /* a CUDA runtime/driver error */
  CHASE_ERR_STATE = 7,        /* call out of order (e.g. eigvals before solve) */
  CHASE_ERR_TIMEOUT = 8,      /* a bounded device-side loop hit its iteration cap */
  CHASE_ERR_UNSUPPORTED = 9   /* mode not available on this device */
} chase_status;

typedef enum { CHASE_R64 = 0, CHASE_C128 = 1 } chase_dtype;

/* Arithmetic of the Chebyshev filter products (Algorithm 1, line 4).
 * QR, Rayleigh-Ritz, the small eigensolve, residuals and Lanczos always run with
 * FP64 accuracy. */
typedef enum {
  CHASE_FP64 = 0,       /* FP64-accurate products: split-BF16 tensor-core products
                           with exact FP32 partial sums, combined in integer/FP64 */
  CHASE_FP64_NATIVE = 1,/* plain DFMA kernels (reference path; slow on this chip) */
  CHASE_BF16x3 = 2,     /* mixed: 2-slice split-BF16 (3 products) bulk filter, then
                           FP64 sweeps once residuals reach the bulk precision */
  CHASE_BF16x6 = 3      /* mixed: 3-slice split-BF16 (6 products) bulk filter */
} chase_mode;

typedef struct {
  int maxdeg;          /* largest filter degree per vector (default 36) */
  int lanczos_steps;   /* Lanczos steps per run (default 25) */
  int lanczos_runs;    /* independent Lanczos runs (default 4) */
  int maxiter;         /* outer iterations before CHASE_ERR_NOCONV (default 30) */
  int extra_deg;       /* constant added to the optimised degree (default 2) */
  int nfinal;          /* mixed modes: minimum FP64 sweeps at the end (default 1) */
  int oz_slices;       /* FP64 mode: BF16 slices per operand, 6 or 7 (default 7) */
  int native_below_mflop; /* products below this many MFLOP use DFMA kernels; 0: always
                             split tensor-core products (default 2000) */
  int batch_workers;   /* chase_solve_batched: host threads that run the per-problem stages (grouped
                          mode), or problems solved concurrently, each worker with its own stream and
                          workspace sized (n_max, ne_max) (worker-pool mode); default 1, at most 32 */
  int batch_grouped;   /* chase_solve_batched: 1 (default) grouped mode, 0 worker-pool mode; see there */
} chase_opts;

typedef struct {
  int iterations;      /* outer iterations of Algorithm 1 */
  int locked;          /* converged (locked) pairs */
  int64_t matvecs;     /* filter matrix-vector products: sum of degrees (footnote on Matvecs) */
  int64_t matvecs_lowp;/* of which were done in the mixed-precision bulk mode */
  int lowp_iterations; /* outer iterations that used the mixed-precision filter */
  double ms_total, ms_lanczos, ms_filter, ms_qr, ms_rr, ms_resid;  /* stage times (CUDA events) */
  double b_sup, mu_1, mu_ne, norm_est;   /* spectral bounds after Lanczos */
  double max_resid;    /* largest residual ratio abs(A v - lambda v) / norm_est over all locked pairs
                          (computed when each pair locked; bounds the returned pairs) */
  int qr_fallbacks;    /* shifted Cholesky-QR fallbacks taken */
  int filter_launches; /* filter product launches */
  double ms_filter_kernel;      /* CUDA-event time of the FP64 split-product filter kernels alone */
  int filter_kernel_launches;   /* launches timed in ms_filter_kernel */
  double ms_filter_kernel_lowp; /* same for the mixed-precision bulk filter kernels */
  double ms_backward;           /* time of the last chase_backward */
  int minres_iterations;        /* MINRES iterations of the last chase_backward */
  int rr_clusters;              /* eigenvalue clusters solved exactly in the Rayleigh-Ritz eigensolves */
  int rr_fallbacks;             /* Rayleigh-Ritz eigensolves that fell back to the FP64 Jacobi */
  int qr_householder;           /* QR steps whose block was numerically rank deficient for Cholesky-QR and
                                   went to the Householder QR */
  int filter_reorth;            /* orthonormalisations inside equal-degree filters whose amplification
                                   would exceed 1e7 (the filtered span is unchanged) */
  int rr_sweeps;                /* Jacobi sweeps of the Rayleigh-Ritz eigensolves (FP32 first passes and
                                   FP64 solves) */
} chase_stats_t;

/* Kernel launches made by this library in this process so far (all contexts). */
int64_t chase_kernel_launch_count(void);

/* Testing hook (not part of Algorithm 1): wall-clock limit, in nanoseconds, of every grid-barrier wait
 * of the persistent Jacobi sweep kernel of the Rayleigh-Ritz eigensolve, for launches made after the
 * call (process-wide).  0 restores the default of 2 s.  A wait that reaches the limit makes every block
 * of the launch return and the call that launched it return CHASE_ERR_TIMEOUT; the context stays
 * usable.  Lets a test make a wait expire without faulting or hanging the GPU. */
void chase_set_wait_limit_ns(uint64_t ns);

/* FP64 throughput probe (not part of Algorithm 1): the rate of this device's FP64 units, the
 * denominators the FP64 filter is compared against.  which = 0: DFMA (fma.rn.f64 on the CUDA cores),
 * which = 1: DMMA (mma.sync m8n8k4 f64 on the tensor cores).  One timed launch over every SM after a
 * warm-up launch (CUDA events); *tflops_out = 2 x FMAs / time, *ms_out (nullable) the launch time.
 * Runs on its own stream of the current device and returns when it has finished. */
chase_status chase_measure_fp64_peak(int which, double* tflops_out, double* ms_out);

/* tcgen05 issue-rate probe (not part of Algorithm 1): cycles per MMA of the FP64 split-product kernel's
 * per-k-block issue pattern (7 left slices, 28 digit pairs, 2 planes x 2 K-steps: 112 MMAs of M = 128,
 * width n_cols, K = 16, bf16 operands, FP32 accumulators), issued back to back by one thread of one CTA per
 * SM, zero operands.  variant 0: no synchronisation, n_cols in {16, 32, 64, 80, 96, 128, 256}; for n_cols = 80:
 * variant bits 1 = a tcgen05.commit after each slice, 2 = a distinct left tile per slice, 4 = an mbarrier
 * test (of a completed phase) before each slice, 8 = no A-collector hints (variants 1, 2, 3, 7, 8).  Cycles are
 * clock64 counts of the issuing thread from the first MMA to the completion of the last, averaged over the
 * SMs.  CHASE_ERR_UNSUPPORTED off sm_103; CHASE_ERR_ARG for other sizes or variants. */
chase_status chase_measure_mma_issue(int n_cols, int variant, double* cycles_per_mma);

/* Fill *opts with defaults. */
void chase_default_opts(chase_opts* opts);

/* Create a context on the current CUDA device.  Preallocates the whole
 * workspace for problems up to n_max x n_max with nev+nex <= ne_max (the
 * single-GPU form of Eq. GPU_mem plus split-product buffers); returns
 * CHASE_ERR_OOM early if it does not fit.  stream: the cudaStream_t all work of
 * the context is enqueued on; NULL is the legacy default stream.  opts may be NULL. */
chase_status chase_create(chase_ctx** ctx, int64_t n_max, int ne_max, chase_dtype dtype,
                          const chase_opts* opts, void* stream);
void chase_destroy(chase_ctx* ctx);
const char* chase_last_error(const chase_ctx* ctx);

/* Device memory the context would allocate for (n_max, ne_max, dtype, mode set),
 * in bytes; the single-GPU form of Eq. GPU_mem (n^2 term excluded: A is the
 * caller's) plus split-product buffers. */
int64_t chase_workspace_bytes(int64_t n_max, int ne_max, chase_dtype dtype, const chase_opts* opts);

/* Seeds of the start vectors the library draws when the caller passes none (chase_solve with V0 or L0
 * NULL): element (i, j) of the n x m block is the counter-based normal of counter i + j n under the seed,
 * SplitMix64 (Steele, Lea & Flood 2014) of seed ^ SplitMix64(2c) and of seed ^ SplitMix64(2c + 1) as two
 * 53-bit uniforms u1 = (a >> 11 + 1) 2^-53, u2 = (b >> 11) 2^-53, Box-Muller r = sqrt(-2 ln u1), t = 2 pi u2;
 * real: r cos t; complex: (r cos t + i r sin t) / sqrt(2).  A host program can reproduce the block. */
#define CHASE_SEED_V0 0x2205024910000001ull
#define CHASE_SEED_L0 0x2205024910000002ull

/* Algorithm 1 end to end.  A: n x n Hermitian (lda >= n).  V0: n x (nev+nex)
 * start block (ld n), or NULL: the library draws it (CHASE_SEED_V0 above; Algorithm 1 starts from a
 * random block).  L0: n x lanczos_runs Lanczos start vectors (ld n), or NULL: drawn the same way
 * (CHASE_SEED_L0).
 * A, V0 and L0 may be device pointers or host pointers (pinned or pageable):
 * host inputs are first copied to the device on the context's stream (pinned
 * memory is copied by DMA).  A host A needs a device copy of n x n elements,
 * allocated on the first such call and kept until chase_destroy
 * (CHASE_ERR_OOM if it does not fit).
 * Converged when the residual of each of the nev lowest Ritz pairs is
 * <= tol * ||A||_est (||A||_est: largest Lanczos Ritz value magnitude).
 * Synchronous: returns when the solve has finished; read the results with
 * chase_eigvals / chase_eigvecs (to host or device memory). */
chase_status chase_solve(chase_ctx* ctx, const void* A, int64_t n, int64_t lda, int nev, int nex,
                         double tol, int deg, int mode, const void* V0, const void* L0);

/* Batched / warm-start form: nprob independent problems (sizes <= the context's),
 * each from its own start block (warm start: pass the previous step's
 * eigenvectors padded to nev+nex).  With opts.batch_workers = W > 1 the context
 * holds W - 1 more workspaces, each with its own non-blocking stream; W host
 * threads take the problems in order of decreasing n (longest first) from one
 * queue, so small problems fill the SMs that large ones leave idle.  The call
 * first waits for the context's stream and returns when every problem has
 * finished.  Eigenpairs are written to the caller's arrays: eigvals_dev[p]
 * (nev[p] doubles), eigvecs_dev[p] (n[p] x (nev[p]+nex[p]), ld n[p]; on exit the
 * leading nev[p] columns are the eigenvectors and the rest the next start
 * block).  stats_host (nullable): nprob records.  On error the first failing
 * problem's status is returned and the other workers stop after their current
 * problem.  After the call, chase_eigvals/eigvecs/stats/backward refer to an
 * unspecified problem of the batch. */
chase_status chase_solve_batched(chase_ctx* ctx, int nprob, const void* const* A_dev, const int64_t* n,
                                 const int* nev, const int* nex, double tol, int deg, int mode,
                                 void* const* V_dev, const void* const* L0_dev, double* const* eigvals_dev,
                                 chase_stats_t* stats_host);

/* Results of the last solve: nev eigenvalues ascending; eigenvectors n x nev. */
chase_status chase_eigvals(chase_ctx* ctx, double* out, int on_device);
chase_status chase_eigvecs(chase_ctx* ctx, void* out, int64_t ldv, int on_device);
chase_status chase_stats(const chase_ctx* ctx, chase_stats_t* out);

/* Adjoint of (Lambda, V) = the last solve's eigenpairs, real symmetric only.
 * gbar_lambda_dev: nev doubles or NULL; gbar_V_dev: n x nev (ld ldg) or NULL;
 * gbar_A_dev: n x n output (ld ldga), symmetrised.  A_dev must be the matrix of
 * the last solve.  Abar = V (diag(gl) + F o (V^T Vbar)) V^T + X V^T with
 * F_ij = 1/(lambda_j - lambda_i) and X from projected MINRES on (A - lambda_j I). */
chase_status chase_backward(chase_ctx* ctx, const void* A_dev, int64_t lda, const double* gbar_lambda_dev,
                            const void* gbar_V_dev, int64_t ldg, void* gbar_A_dev, int64_t ldga,
                            double minres_tol, int minres_maxit);

/* ---------------------------------------------------------------------------
 * Step-level entry points (one step of Algorithm 1 each), used for per-step
 * parity checks and by advanced callers.  All device buffers are the caller's.
 * ------------------------------------------------------------------------- */

/* Algorithm 1, line 2: Lanczos bounds.  out_host[0..3] = {b_sup, mu_1, mu_ne, theta_max}. */
chase_status chase_lanczos(chase_ctx* ctx, const void* A_dev, int64_t n, int64_t lda, int ne,
                           const void* L0_dev, int runs, int steps, double* out_host);

/* Algorithm 1, line 4: filter ncols columns of V in place (ld ldv) with degrees
 * deg_host[a] (non-decreasing) using the scaled three-term recurrence with
 * c = (b_sup+mu_ne)/2, e = (b_sup-mu_ne)/2.  mode: a chase_mode. */
chase_status chase_filter(chase_ctx* ctx, const void* A_dev, int64_t n, int64_t lda, void* V_dev, int64_t ldv,
                          int ncols, const int* deg_host, double b_sup, double mu_1, double mu_ne, int mode);

/* Algorithm 1, line 5: orthonormalise X (n x ncols, ld ldx) in place by
 * Cholesky-QR2 (shifted Cholesky-QR3 fallback); the first nlocked columns are
 * assumed orthonormal and are left unchanged.  A block that is numerically
 * rank deficient for Cholesky-QR (a column's remainder after the columns before
 * it within the rounding of the Gram matrix) is first orthonormalised by a
 * blocked Householder QR (counted in chase_stats_t.qr_householder). */
chase_status chase_qr(chase_ctx* ctx, void* X_dev, int64_t n, int64_t ldx, int ncols, int nlocked);

/* Algorithm 1, lines 6-7: Rayleigh-Ritz on the ncols orthonormal columns Q
 * (in place: on exit the Ritz vectors), Ritz values ascending to ritz_host and
 * residual norms ||A v - lambda v||_2 to resid_host. */
chase_status chase_rayleigh_ritz(chase_ctx* ctx, const void* A_dev, int64_t n, int64_t lda, void* Q_dev,
                                 int64_t ldq, int ncols, double* ritz_host, double* resid_host);

/* Dense Hermitian eigensolve of G (k x k, ld ldg) on the device by parallel
 * cyclic Jacobi: eigenvalues ascending to w_host, eigenvectors to Z_dev (ld ldz). */
chase_status chase_heevj(chase_ctx* ctx, const void* G_dev, int64_t ldg, int k, double* w_host,
                         void* Z_dev, int64_t ldz);

/* Largest k accepted by chase_heevj_noalloc. */
#define CHASE_HEEVJ_NOALLOC_KMAX 256

/* chase_heevj for callers that cannot allocate device memory (a process whose
 * device memory is already reserved by a framework's caching allocator or its
 * own arena, or code that must not allocate because cudaMalloc can fail under
 * memory pressure and synchronises the device).  The paper has no counterpart:
 * this is a deployment variant of the Rayleigh-Ritz eigensolve.
 * Needs no context.  G_dev: k x k Hermitian (ld ldg) of type dtype, read only;
 * eigenvalues ascending to w_host (k doubles); eigenvectors to Z_dev (k x k,
 * ld ldz).  All work is enqueued on `stream` (NULL: legacy default stream) and
 * the call returns when it has finished.
 * Scratch is one fixed array in the library's device memory (about 2.1 MB per
 * device, held until the process exits): k > CHASE_HEEVJ_NOALLOC_KMAX returns
 * CHASE_ERR_ARG; calls that overlap on the GPU share it and race; it keeps the
 * previous call's contents (the solver writes all it reads).  The first call in
 * a CUDA context (normally a device's primary context) looks up the array's
 * address in that context and caches it per context; make it before any stream
 * capture.  Errors are returned as statuses only (no message). */
chase_status chase_heevj_noalloc(const void* G_dev, int64_t ldg, int k, chase_dtype dtype, double* w_host,
                                 void* Z_dev, int64_t ldz, void* stream);

/* Dense product C = A B (n x n times n x ncols) with the filter's product
 * arithmetic for the given mode; used to check the split-product kernels. */
chase_status chase_hemm(chase_ctx* ctx, const void* A_dev, int64_t n, int64_t lda, const void* B_dev,
                        int64_t ldb, int ncols, void* C_dev, int64_t ldc, int mode);

/* Input generator (not part of Algorithm 1): A = Q diag(lam) Q^H with Q a
 * product of k Householder reflectors, from the compact-WY factors U, B = U T
 * and D = B (U^H diag(lam) U) (each n x k, ld n, host-computed).  Writes an
 * exactly Hermitian A (ld lda). */
chase_status chase_generate(chase_ctx* ctx, void* A_dev, int64_t n, int64_t lda, const double* lam_dev,
                            const void* U_dev, const void* B_dev, const void* D_dev, int k);

/* Input generator for correlated sequences (not part of Algorithm 1): A += eps * H with
 * H = s (G + G^H)/2, G_ij standard (complex) Gaussian from a counter-based generator
 * (SplitMix64 hash of the seed and the element's counter, Box-Muller), s = 1/sqrt(2n) the
 * semicircle-edge estimate of 1/||(G+G^H)/2||_2 (real: G_ij ~ N(0,1), same s).  Keeps A
 * exactly Hermitian.  The same generator is available on the host for parity checks. */
chase_status chase_perturb(chase_ctx* ctx, void* A_dev, int64_t n, int64_t lda, double eps, uint64_t seed);

#ifdef __cplusplus
}
#endif
#endif /* CHASE_GB300_H */
