/*
 * spd.h -- C ABI of libspd, a GB300 (sm_103a) solver for dense symmetric
 * positive-definite systems  A X = B  (Section 3, eqs. (problemSingleRHS)
 * and (problemMultipleRHS) of Klavik, Malossi, Bekas, Curioni, "Changing
 * Computing Paradigms Towards Power Efficiency", arXiv:1405.4644).
 *
 * The library implements the two mixed-precision refinement schemes of
 * Section 3: Cholesky with iterative refinement (Algorithm 1) and conjugate
 * gradients with iterative refinement (Algorithm 2), plus batched and
 * preconditioned variants.  Low-precision work (factorisation, triangular
 * solves, CG matrix-vector products) runs in the precision the caller picks;
 * residuals, solution updates, norms and convergence tests run in float64.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory   All matrix and vector arguments are DEVICE pointers unless the
 *          name ends in _host.  They are float64, column-major, with a
 *          leading dimension >= the row count.  A is symmetric and both
 *          triangles must hold it: the factorisation reads only the lower
 *          triangle (i >= j) and the float64 residual streams the whole
 *          matrix.  Buffers belong to the caller; the library never frees
 *          them.  The library owns its handle, factor objects and workspace,
 *          released by the matching *_destroy call.
 * Streams  Every call is ordered on the stream given to spd_create and
 *          returns after that stream has drained (the report is filled on
 *          the host), unless stated otherwise.
 * Errors   Every call returns an spd_status; no exception or signal crosses
 *          the ABI.  spd_last_error_string(h) describes the last failure on
 *          a handle.  On SPD_ERR_NOT_SPD, report.info holds the 1-based
 *          column of the first non-positive pivot (LAPACK potrf
 *          convention).  On SPD_ERR_NO_CONVERGENCE, X holds the best iterate.
 *          On SPD_ERR_TIMEOUT a bounded device wait gave up and the context
 *          is still usable.  NaN or Inf in A gives SPD_ERR_ARG.
 * Sizes    n, m >= 0 (n = 0 or m = 0 is a no-op returning SPD_OK).
 *          int is 32-bit; n * lda must fit in 63 bits.
 */
#ifndef SPD_H
#define SPD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spd_status {
    SPD_OK = 0,
    SPD_ERR_ARG = 1,            /* invalid argument or non-finite input        */
    SPD_ERR_NOT_SPD = 2,        /* factorisation broke down (report.info)      */
    SPD_ERR_NO_CONVERGENCE = 3, /* refinement / CG did not reach the tolerance */
    SPD_ERR_TIMEOUT = 4,        /* a bounded device-side wait expired          */
    SPD_ERR_CUDA = 5,           /* a CUDA runtime call failed                  */
    SPD_ERR_OOM = 6,            /* device allocation failed                    */
    SPD_ERR_UNSUPPORTED = 7,    /* precision / mode not available              */
    SPD_ERR_SCRATCH = 8         /* problem too large for spd_residual_static's
                                   fixed scratch array                         */
} spd_status;

/* Precision of the low-precision work (Section 3.1, "~" quantities).
 * FP64 is the plain baseline: the whole factorisation in float64.
 * FP32 keeps the factor in float32 and computes its trailing updates to
 * float32 accuracy on the tensor cores, each float32 operand split into
 * three bf16 slices (see spd_gemm_update); SPD_FACTOR_CUDA_CORES runs them
 * as plain float32 products on the CUDA cores instead.
 * TF32/BF16/FP16/FP8 keep the factor in float32 but feed the trailing
 * updates to the tensor cores with operands rounded (RNE) to that type and
 * float32 accumulation; FP8 is OCP E4M3 with one fixed power-of-two operand
 * scale (2^8: every entry of the scaled factor has magnitude <= 1).  AUTO
 * picks per matrix (see spd_factor). */
typedef enum spd_prec {
    SPD_PREC_FP64 = 0,
    SPD_PREC_FP32 = 1,
    SPD_PREC_TF32 = 2,
    SPD_PREC_BF16 = 3,
    SPD_PREC_FP16 = 4,
    SPD_PREC_FP8 = 5,
    SPD_PREC_AUTO = 6
} spd_prec;

/* Stopping rules (Alg. 1 and Alg. 2 print ||r||_2 >= tolerance; the
 * normwise backward error is the accuracy target of this library). */
typedef enum spd_crit {
    SPD_CRIT_BERR = 0, /* ||b - A x||_inf / (||A||_inf ||x||_inf) <= tol */
    SPD_CRIT_REL2 = 1, /* ||b - A x||_2 <= tol * ||b||_2               */
    SPD_CRIT_ABS2 = 2  /* ||b - A x||_2 <  tol   (as printed, Alg. 1/2)  */
} spd_crit;

/* Preconditioners for spd_cg. */
typedef enum spd_precond {
    SPD_PC_NONE = 0,   /* Algorithm 2 as printed                           */
    SPD_PC_JACOBI = 1, /* M = diag(A)^{-1}                                  */
    SPD_PC_FACTOR = 2, /* M = (R~^T R~)^{-1} from an spd_factor object      */
    SPD_PC_LOWRANK = 3 /* learned M = S (Dh + Uh Uh^T)^{-1} S (spd_lowrank)  */
} spd_precond;

/* Arithmetic of the float64-accurate residual r = b - A x. */
typedef enum spd_resid {
    SPD_RESID_FP64 = 0, /* float64 fused multiply-adds                        */
    SPD_RESID_DF32 = 1, /* refinement loops: residuals of spd_residual_df32 (float32
                           units, about 48-bit accurate) while the largest
                           backward error is above 2^-36 and, below that,
                           while each sweep still shrinks it fourfold;
                           float64 residuals from there on; a column is only
                           ever accepted as
                           converged on a float64 residual, so the stopping
                           rule and its guarantee are those of SPD_RESID_FP64.
                           The float64 products of the CG fallback use
                           spd_residual_df32's arithmetic throughout.        */
    SPD_RESID_TC = 2,   /* every residual (and every float64 product of the
                           CG fallback) from spd_residual_tc: exact products
                           of bf16 digits on the tensor cores; columns may be
                           accepted on it.  The digit planes of A (20 bytes
                           per entry of A) are formed once per solve and stay
                           in the handle's workspace.                        */
    SPD_RESID_AUTO = 3  /* SPD_RESID_FP64 for one right-hand side (8 bytes
                           per entry of A, bound by HBM), SPD_RESID_TC for
                           m >= 2 (float64 fused multiply-adds are then bound
                           by the FP64 rate)                                  */
} spd_resid;

/* Flags of spd_factor. */
#define SPD_SCALE_DIAG 1u /* factor D^{-1/2} A D^{-1/2} (D = diag A); default */
#define SPD_FACTOR_CUDA_CORES 2u /* run the trailing updates of a FP32/TF32/
                                    BF16/FP16 factor on the CUDA cores (same
                                    rounded operands, float32 accumulation;
                                    plain float32 products for FP32): a
                                    reference engine for validation       */
#define SPD_FACTOR_RECURSIVE 4u  /* tensor-core factors: recursive blocking
                                    (large updates, many small panels) instead
                                    of the default left-looking 128-column
                                    schedule                                */
#define SPD_FACTOR_SHIFT 16u     /* if the factorisation breaks down, factor
                                    the scaled matrix plus sigma I instead,
                                    sigma = 2 u (u the unit roundoff of the
                                    update operands: the size of the updates'
                                    rounding relative to the unit diagonal),
                                    raised fourfold until it succeeds (at
                                    most sigma = 1); refinement then sees a
                                    perturbation of norm <= sigma and, when it
                                    stagnates, hands over to the factor-
                                    preconditioned CG fallback (Section 3.1,
                                    eq. (iterref): the inner solver only has
                                    to contract).  report.shift gives sigma */
#define SPD_FACTOR_BLOCK_SWEEPS 32u /* float32 factors: apply the factor
                                    with the sweeps over 128-row blocks.  By
                                    default a factor of at least 16 blocks
                                    also holds the inverses of its diagonal
                                    super-blocks (8 blocks each, formed once,
                                    4 (1024)^2 bytes each) and is applied with
                                    the super-block sweeps */
#define SPD_FACTOR_SERIAL 8u     /* left-looking schedule without its
                                    look-ahead: every kernel on the handle's
                                    stream in order (kernels then run alone,
                                    e.g. to time them)                      */

typedef struct spd_opts {
    double tol;      /* stopping threshold (default 1e-14)                    */
    int crit;        /* spd_crit (default SPD_CRIT_BERR)                      */
    int maxit;       /* max refinement sweeps / outer CG steps (default 50)   */
    int maxit_inner; /* spd_cg: max inner steps per outer step (default 2000) */
    double eta;      /* spd_cg: inner stop at ||r_in|| <= eta ||r|| (1e-4)    */
    int band;        /* spd_cg: half bandwidth of the inner matrix, -1 dense  */
    int fallback;    /* spd_solve_ir: on stagnation switch to factor-
                        preconditioned CG in float64 (default 1)              */
    int resid;       /* spd_resid (default SPD_RESID_FP64)                    */
    int polish;      /* spd_solve_ir: extra sweeps after a column first meets
                        the rule, to bring its forward error to the float64
                        floor (default 1)                                     */
    int matvec_cores;/* spd_cg with FP32 products (step C1): spd_mv_cores
                        (default SPD_MV_AUTO)                                 */
} spd_opts;

/* Where spd_cg computes its FP32 products z = A~ p (Section 3.2, step C1).
 * On the tensor cores, A~ (float32) and p (float32) enter as three bf16
 * slices each and the six slice products of order <= 2 accumulate in float32
 * tensor memory, so the product keeps the float32 product's accuracy; A~ is
 * then held as three bf16 planes (6 n^2 bytes) instead of one float32 copy
 * (4 n^2 bytes).  On the CUDA cores, float32 fused multiply-adds. */
typedef enum spd_mv_cores {
    SPD_MV_AUTO = 0,    /* tensor cores when m >= 8, else CUDA cores */
    SPD_MV_CUDA = 1,    /* CUDA cores for every m                    */
    SPD_MV_TENSOR = 2   /* tensor cores for every m                  */
} spd_mv_cores;

typedef struct spd_report {
    int status;      /* spd_status of the call                               */
    int info;        /* SPD_ERR_NOT_SPD: 1-based failing column              */
    int iters_low;   /* low-precision iterations (solves or inner CG steps)  */
    int iters_high;  /* float64 residual evaluations after the first         */
    int prec_used;   /* spd_prec actually used                               */
    int fell_back;   /* 1 if the stagnation fallback ran                     */
    double berr;     /* final max-over-columns normwise backward error       */
    double rel_resid;/* final max-over-columns ||r||_2 / ||b||_2             */
    double time_ms;  /* device time of the call (CUDA events)                */
    double cond_est; /* spd_factor with AUTO: estimated 1-norm condition
                        number of the scaled matrix (Hager's estimator);
                        -1 when the FP16 factor broke down before it could
                        be estimated; 0 when no FP16 factor ran (the
                        pre-check below ruled it out) and for the other
                        precisions                                          */
    double shift;    /* spd_factor with SPD_FACTOR_SHIFT: the sigma of the
                        factor actually kept (0 = no shift was needed)      */
    double cond_lower; /* spd_factor with AUTO and n >= 4096: a lower bound
                        on the 2-norm condition number of the scaled matrix
                        from at most 16 Lanczos steps before any factor
                        (Ritz values lie inside the spectrum); above 512
                        (kappa u_fp16 > 1/4, eq. (iterref)) no FP16 factor
                        is attempted.  +inf when the float32 products do
                        not resolve the smallest eigenvalue; 0 when not
                        taken                                               */
} spd_report;

typedef struct spd_handle spd_handle;
typedef struct spd_factor_t spd_factor_t;

/* ---- handle ------------------------------------------------------------ */
/* Create a handle bound to the current CUDA device and `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The handle also owns
 * a second, non-blocking stream at the default (lowest) priority, on which
 * the factorisation's look-ahead issues its bulk trailing updates; every
 * call joins it back into `stream` before returning.  Callers that run
 * several handles concurrently get the most throughput when their own
 * streams have a higher priority: each solve's critical chain then goes
 * ahead of the other solves' bulk updates. */
spd_status spd_create(spd_handle **h, void *stream);
spd_status spd_destroy(spd_handle *h);
/* Text of the last failure on h (static storage owned by h; never NULL). */
const char *spd_last_error_string(const spd_handle *h);
/* Fill *o with the defaults listed in spd_opts. */
void spd_opts_default(spd_opts *o);

/* ---- Algorithm 1, step 1: low-precision Cholesky --------------------------
 * Factor A ~= R~^T R~ (Section 3.1, eq. (cholesky), Alg. 1 line 1) in
 * precision `prec`, after the symmetric diagonal scaling D^{-1/2} A D^{-1/2}
 * when flags has SPD_SCALE_DIAG.  Blocked Cholesky over 128-column block
 * columns: 128x128 diagonal-block factorisations, panel triangular solves
 * and trailing updates (A22 -= L21 L21^T, as block-column updates).  The
 * tensor-core precisions use a left-looking schedule whose bulk updates run
 * one block column ahead on the handle's second stream (SPD_FACTOR_SERIAL:
 * the same schedule on one stream, bit-identical; SPD_FACTOR_RECURSIVE:
 * right-looking recursive blocking); FP64 and the CUDA-core engine use the
 * recursive form.
 * A: n x n, lda >= n, read-only, lower triangle read.  On success *F owns
 * the factor (release with spd_factor_destroy).  AUTO keeps the cheapest
 * factor whose estimated ||A^{-1} dA|| keeps refinement convergent
 * (eq. (iterref)): FP16 first;
 * if its factor breaks down, or kappa_1 / sqrt(n) * 2^-11 > 1/4 with
 * kappa_1 the 1-norm condition number of the scaled matrix estimated by
 * Hager's method through the FP16 factor, FP32; if that breaks down, FP64.
 * rep may be NULL. */
spd_status spd_factor(spd_handle *h, int n, const double *A, int lda, int prec,
                      unsigned flags, spd_factor_t **F, spd_report *rep);
/* Releases the factor's memory, ordered on the handle's stream (no
 * device-wide synchronisation; factors come from the device's stream-ordered
 * pool, which spd_create sets to keep freed blocks cached).  The factor must
 * not be in use on another stream at that point. */
spd_status spd_factor_destroy(spd_factor_t *F);

/* Order and precision of a factor (either output may be NULL). */
spd_status spd_factor_info(const spd_factor_t *F, int *n, int *prec);

/* Copy a factor out for inspection: L receives n rows of the working
 * matrix, row-major with leading dimension ldl >= n (float32, or float64
 * for SPD_PREC_FP64 factors); its lower triangle is R~^T of the scaled
 * matrix diag(d) A diag(d), the upper triangle is scratch.  d receives the
 * n scaling factors.  L and d may be host or device pointers (either may
 * be NULL).  Synchronous. */
spd_status spd_factor_copy(const spd_factor_t *F, void *L, int ldl, double *d);

/* ---- Algorithm 1, lines 2-7: refinement --------------------------------
 * Solve A X = B with the factor F: X = R~^{-1} R~^{-T} B (line 2), then
 * repeat r = B - A X in float64 (lines 3, 7), Z = R~^{-1} R~^{-T} r in
 * low precision (line 5), X += Z in float64 (line 6) until every column
 * meets opts->crit/tol.  Converged columns are frozen.  When the error
 * stagnates (two sweeps each shrinking it by less than half) and
 * opts->fallback is set, the remaining columns continue with conjugate
 * gradients on A in float64 preconditioned by F.
 * B: n x m (ldb); X: n x m (ldx) output.  opts may be NULL (defaults). */
spd_status spd_solve_ir(spd_handle *h, const spd_factor_t *F, int n, int m,
                        const double *A, int lda, const double *B, int ldb,
                        double *X, int ldx, const spd_opts *opts, spd_report *rep);

/* Algorithm 1 with the loop's stop decision on the device, for CUDA graph
 * capture (no passage of the paper beyond Alg. 1 itself).  The call only
 * enqueues work on h's stream and returns: line 2, the first residual, then
 * opts->maxit refinement sweeps whose triangular solves and residuals
 * return at once on the device once every column meets opts->crit/tol
 * (each such sweep then costs a few microseconds of launches), and finally
 * a kernel that writes *rep (DEVICE memory).  The residual is
 * SPD_RESID_TC when opts->resid asks for it, else float64 (SPD_RESID_DF32
 * is taken as float64: its switch needs host decisions); there is no
 * stagnation fallback (rep->stagnated counts the columns that stalled:
 * solve those with spd_solve_ir).  FP64 factors are not accepted.
 * Capture: make one call with the same n, m and opts outside any capture
 * first (it sizes h's workspace and allocates the device epoch counter);
 * later calls allocate nothing and contain no host synchronisation.  The
 * sweeps' block flags take their epochs from a device counter the solve
 * itself advances, so a captured graph may be replayed any number of
 * times; replays must not overlap each other or other cooperative work of
 * the process (the sweeps are cooperative launches).
 * A, B, X, F, *rep stay owned by the caller and must stay valid until the
 * work has run. */
typedef struct spd_report_dev {
    int status;       /* SPD_OK if every column met the rule, SPD_ERR_NO_CONVERGENCE
                         if not, SPD_ERR_TIMEOUT / SPD_ERR_CUDA on a device error */
    int active;       /* columns above the tolerance at the end                     */
    int sweeps;       /* refinement sweeps applied (max over columns)               */
    int stagnated;    /* columns whose error stopped shrinking                      */
    int dev_flags;    /* the handle's device status word at the end                 */
    int pad;
    double berr;      /* max-over-columns normwise backward error                   */
    double rel_resid; /* max-over-columns ||r||_2 / ||b||_2                         */
} spd_report_dev;
spd_status spd_solve_ir_async(spd_handle *h, const spd_factor_t *F, int n, int m,
                              const double *A, int lda, const double *B, int ldb,
                              double *X, int ldx, const spd_opts *opts, spd_report_dev *rep);

/* Factor and refine in one call on HOST buffers: copies A and B to the
 * device, runs spd_factor + spd_solve_ir, copies X back (column-major,
 * lda/ldb/ldx >= n).  The device copies of A, B and X are the handle's: they
 * grow to the largest call and stay allocated until spd_destroy, so repeated
 * calls neither allocate nor free device memory for them.  Host buffers in
 * pinned memory copy at the link's full rate.  Returns after X is on the host. */
spd_status spd_solve_ir_host(spd_handle *h, int n, int m, const double *A_host, int lda,
                             const double *B_host, int ldb, double *X_host, int ldx,
                             int prec, const spd_opts *opts, spd_report *rep);

/* Z = R~^{-1} R~^{-T} R (Alg. 1 line 5): the two low-precision triangular
 * solves with F, including the diagonal scaling.  R, Z: n x m. */
spd_status spd_factor_solve(spd_handle *h, const spd_factor_t *F, int n, int m,
                            const double *R, int ldr, double *Z, int ldz);

/* R = B - A X in float64 (Alg. 1 lines 3/7, Alg. 2 line 2), plus per-column
 * norms written to colnorms (device, 3*m float64, may be NULL):
 * [||r_c||_inf, ||r_c||_2, ||x_c||_inf] for column c at 3c..3c+2. */
spd_status spd_residual(spd_handle *h, int n, int m, const double *A, int lda,
                        const double *B, int ldb, const double *X, int ldx,
                        double *R, int ldr, double *colnorms);

/* The residual of spd_residual computed on the float32 units (the
 * high-precision residual of Alg. 1 lines 3/7 and Alg. 2 line 2, emulated;
 * Section 3.1 only asks that it be more accurate than the factor).
 * A's float64 entries are split by bit operations into two float32 parts
 * (|a - ah - am| <= 2^-47 |a|), each column of X is scaled by a power of
 * two and split into two float32 parts, the leading product ah*xh is kept
 * exactly (FMA), the sums are float32 pairs updated by TwoSum and folded
 * into float64 every 64 terms.  This is 48-bit arithmetic (float64: 53):
 * products err by about 2^-47 |a_ij||x_j| and each run of 64 pair
 * additions by up to ~2^-43 of its largest partial sum, so
 * |computed - exact| stays below 2^-40 (|A||x|)_i per entry -- accurate
 * enough to drive refinement, not to certify a 1e-14 backward error
 * (SPD_RESID_DF32 hands that to a float64 residual).  Entries with |a| outside [2^-100, 2^100)
 * (and Inf/NaN) take float64 FMAs; non-finite X gives NaN.  Same arguments,
 * layout, ownership and errors as spd_residual. */
spd_status spd_residual_df32(spd_handle *h, int n, int m, const double *A, int lda,
                             const double *B, int ldb, const double *X, int ldx,
                             double *R, int ldr, double *colnorms);

/* The residual of spd_residual from exact integer products on the bf16
 * tensor cores (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
 * 2012; Section 3.1 asks only for a residual more accurate than the
 * factor).  Row i of A is cut into ten signed 7-bit digits below 2^e_i
 * (e_i = ilogb(max_j |a_ij|) + 2), column c of X likewise (f_c); entries
 * lose only their bits below 2^{e_i - 70} (2^{f_c - 70}).  The 55 digit
 * products of total weight <= 11 are summed exactly (float32 on the tensor
 * cores over 64-wide chunks of j, each sum an integer of magnitude < 2^22,
 * then integers), combined with their power-of-two scales in double-double,
 * and b - (A x) is rounded once.  The dropped digit products and the
 * truncation add less than 2^-64.5 max_j|a_ij| max|x_c| per term, so
 *   |computed - exact| <= 2^-53 |r_i| + n 2^-64 max_j |a_ij| max_j |x_jc|
 * (at n = 16384, 2^-50 ||A||_inf ||x||_inf at worst).  Rows of A with a
 * non-finite entry and columns of X with one give NaN.  Workspace: 20 bytes
 * per entry of A for the digit planes, plus O(n m).  Same arguments,
 * layout, ownership and errors as spd_residual. */
spd_status spd_residual_tc(spd_handle *h, int n, int m, const double *A, int lda,
                           const double *B, int ldb, const double *X, int ldx,
                           double *R, int ldr, double *colnorms);

/* The same float64 residual and norms as spd_residual, for callers that may
 * not allocate device memory at all (host callbacks, allocator hooks,
 * processes with a fixed memory budget, real-time loops).  It takes no
 * handle and calls no allocator: its partial sums live in a fixed 16 MiB
 * scratch array compiled into the library, which every GPU that loads the
 * library keeps until exit.  Limit: n*m + 3*m*ceil(n/256) float64 values
 * must fit in that array (n*m up to about 2.09 million); larger problems
 * return SPD_ERR_SCRATCH.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps
 * it for the life of the process; make that first call before any stream
 * capture, and do not call this entry point on a device after a
 * cudaDeviceReset of it.  All calls share the array and it keeps the last
 * call's contents (no part of it has to start at zero); calls that overlap
 * on the GPU race on it and must be serialised by the caller.  Ordered on
 * `stream` (a cudaStream_t, NULL = legacy default stream); returns after
 * that stream has drained.  This entry point has no counterpart in the
 * paper. */
spd_status spd_residual_static(void *stream, int n, int m, const double *A, int lda,
                               const double *B, int ldb, const double *X, int ldx, double *R,
                               int ldr, double *colnorms);

/* ---- Algorithm 2: CG with iterative refinement ---------------------------
 * Outer ("high") steps: r = B - A X in float64, stop when opts->crit/tol
 * holds.  Inner ("low") steps: Algorithm 2's loop on A e = r with the
 * matrix-vector product z = A~ p taken with A~ = A stored in `matvec_prec`
 * (SPD_PREC_FP32, SPD_PREC_BF16 or SPD_PREC_FP64) -- banded to
 * |i - j| <= opts->band when band >= 0 (Section 4.1) -- and rho, alpha,
 * beta and the vector updates in float64; then X += e.  beta is the
 * Fletcher-Reeves quotient r'^T r' / rho.  pc selects the preconditioner;
 * pc_data is the spd_factor_t* for SPD_PC_FACTOR, the spd_lowrank* for
 * SPD_PC_LOWRANK, else NULL.  X starts
 * from zero.  The m columns are independent CG runs sharing each pass
 * over A~. */
spd_status spd_cg(spd_handle *h, int n, int m, const double *A, int lda, int matvec_prec,
                  int pc, const void *pc_data, const double *B, int ldb, double *X, int ldx,
                  const spd_opts *opts, spd_report *rep);

/* ---- learned diagonal-plus-low-rank preconditioner for PCG -------------------
 * (No passage of the paper: an extension of Algorithm 2's CG.)  A small
 * network maps per-row features of A to Dh (diagonal, > 0) and Uh (n x 32),
 * defining the SPD preconditioner  M = S (Dh + Uh Uh^T)^{-1} S  with
 * S = diag(A)^{-1/2}, applied through the Woodbury identity in O(32 n).
 * The network is 16 -> H -> H -> 33 with SiLU activations; with bf16 set,
 * the forward products take bf16-rounded operands and activations
 * (float32 accumulation and float32 master weights).  Training minimises
 *   L = (1/p) sum_c ||A M z_c - z_c||^2 / ||z_c||^2
 *       + w_sup ||M z_0 - t_0||^2 / ||t_0||^2
 * over probe vectors z_c (device, n x p, column-major, ld n), where
 * t_0 = A^{-1} z_0 comes from the system's own Cholesky factor (optional).
 * All kernels (features, layers, loss, gradient, Adam, apply) run on the
 * GPU.  Buffers are device pointers unless stated. */
typedef struct spd_mlp spd_mlp;
typedef struct spd_lowrank spd_lowrank;
spd_status spd_mlp_create(spd_handle *h, int hidden, unsigned long long seed, int bf16, spd_mlp **net);
spd_status spd_mlp_destroy(spd_mlp *net);
/* Copy the flat float32 parameter vector out (out), in (in) and the
 * gradient of the last spd_mlp_loss_grad out (grad_out); host or device
 * pointers, each may be NULL; *count receives the parameter count. */
spd_status spd_mlp_params(spd_mlp *net, float *out, const float *in, float *grad_out, long *count);
/* F (n x 16 float32, row-major) = row features of A: point coordinates
 * (coords, n x 2 float64 row-major), log ell, log nugget, Fourier terms of
 * the coordinates, mean/rms/max-off-diagonal of the scaled row, 1. */
spd_status spd_learned_features(spd_handle *h, int n, const double *A, int lda, const double *coords,
                                double ell, double nugget, float *F);
/* Loss L (host *loss) and its gradient with respect to every parameter
 * (kept in the network for spd_mlp_adam).  T may be NULL (w_sup unused). */
spd_status spd_mlp_loss_grad(spd_mlp *net, int n, const double *A, int lda, const float *F, int p,
                             const double *Z, const double *T, double w_sup, double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
spd_status spd_mlp_adam(spd_mlp *net, double lr);
/* Inference: build the preconditioner of A from its features. */
spd_status spd_lowrank_build(spd_mlp *net, int n, const double *A, int lda, const float *F,
                             spd_lowrank **P);
/* Z = M R for m columns (float64, column-major). */
spd_status spd_lowrank_apply(spd_lowrank *P, int m, const double *R, int ldr, double *Z, int ldz);
spd_status spd_lowrank_destroy(spd_lowrank *P);
/* Checkpoint of a network (the survey's "weights and training-data
 * manifest" item; no passage of the paper): spd_learned_save writes
 * <path>.json (format, features, hidden width, outputs, bf16, parameter
 * count, Adam step), <path>.bin (the float32 parameters, little endian, in
 * the order W1 b1 W2 b2 W3 b3) and <path>.adam.bin (the two Adam moments);
 * spd_learned_load creates a network on h from them (Adam state restored
 * when <path>.adam.bin is present), so that training resumes or inference
 * runs in another process.  A manifest that does not match this library's
 * feature and output counts, or a short file, gives SPD_ERR_ARG. */
spd_status spd_learned_save(spd_mlp *net, const char *path);
spd_status spd_learned_load(spd_handle *h, const char *path, spd_mlp **net);
/* PCG on A in float64 with the learned M (spd_cg with SPD_PC_LOWRANK, at
 * most opts->maxit_inner steps); if it misses the tolerance, float32
 * Cholesky with iterative refinement takes over (report.fell_back = 1). */
spd_status spd_solve_learned(spd_handle *h, const spd_lowrank *P, int n, int m, const double *A,
                             int lda, const double *B, int ldb, double *X, int ldx,
                             const spd_opts *opts, spd_report *rep);

/* ---- batched solves ----------------------------------------------------------
 * Many independent systems A_i x_i = b_i (1 <= n_i <= 512, one right-hand
 * side each) solved in ONE persistent launch, replayed from a CUDA graph.
 * Each CTA takes whole systems from a shared counter over the systems
 * sorted by decreasing n, so results do not depend on the schedule.
 *   SPD_BATCH_CHOL_IR     Algorithm 1 per system: scaled Cholesky in float32
 *                         (with the trailing-update operands rounded to
 *                         `prec`: FP32, BF16 or FP16), float32 triangular
 *                         solves, float64 residual and update; stops at
 *                         opts->tol on the normwise backward error (plus
 *                         opts->polish sweeps), at most opts->maxit sweeps.
 *   SPD_BATCH_PCG_JACOBI  conjugate gradients in float64 with M = diag(A)^-1,
 *                         x0 = 0, at most opts->maxit_inner steps.
 * spd_batch_create copies the descriptors (host arrays of DEVICE pointers:
 * A_i column-major with lda_i, b_i, x_i) into a plan; the plan may be
 * solved any number of times (the buffers' contents may change between
 * solves, the pointers may not).  The first solve of a method times the
 * CTA-size candidates (256, 512 threads) and keeps the fastest.  Per-system
 * results go to the optional host arrays status/berr/iters (count each);
 * summary gets the worst backward error and the device time of the launch.
 * Returns SPD_ERR_NOT_SPD if any system broke down, SPD_ERR_NO_CONVERGENCE
 * if any missed the tolerance (per-system status tells which). */
#define SPD_BATCH_CHOL_IR 0
#define SPD_BATCH_PCG_JACOBI 1
typedef struct spd_batch spd_batch;
spd_status spd_batch_create(spd_handle *h, int count, const int *n, const double *const *A,
                            const int *lda, const double *const *B, double *const *X,
                            spd_batch **plan);
spd_status spd_batch_solve(spd_batch *plan, int method, int prec, const spd_opts *opts,
                           spd_report *summary, int *status, double *berr, int *iters);
/* The solve of spd_batch_solve as a CUDA graph the caller launches: after
 * spd_batch_graph (which tunes the CTA size on first use and captures a
 * counter reset plus the one persistent launch), *graph_exec is a
 * cudaGraphExec_t owned by the plan -- valid until spd_batch_destroy or the
 * next spd_batch_graph/spd_batch_solve of the same method and precision with
 * other opts; launch it on any stream with spd_graph_launch (or
 * cudaGraphLaunch), as often as wanted; launches of one plan must not
 * overlap.  spd_batch_results reads the last launch's per-system results
 * (as spd_batch_solve returns them; time_ms 0) after the caller has
 * synchronised the launching stream; it also drains the handle's stream. */
spd_status spd_batch_graph(spd_batch *plan, int method, int prec, const spd_opts *opts,
                           void **graph_exec);
spd_status spd_batch_results(spd_batch *plan, int method, int prec, spd_report *summary, int *status,
                             double *berr, int *iters);
/* cudaGraphLaunch(graph_exec, stream) through this library's CUDA runtime. */
spd_status spd_graph_launch(void *graph_exec, void *stream);
/* Tuned CTA size (0 before the first solve), CTA count and the timed
 * candidates (ms for 256 and 512 threads; tune_ms may be NULL). */
spd_status spd_batch_info(const spd_batch *plan, int method, int *threads_per_cta, int *ctas,
                          float *tune_ms);
spd_status spd_batch_destroy(spd_batch *plan);

/* ---- the trailing update as a standalone operation -------------------------
 * C -= A B^T (step A3 of the factorisation, eq. (cholesky)'s O(n^3) part) on
 * the tensor cores: A (M x K) and B (N x K) float32 row-major are rounded
 * (RNE) to `prec` (SPD_PREC_TF32, BF16, FP16 or FP8 -- FP8 multiplies the
 * operands by 2^8 before rounding, so |entries| <= 1.75 stay in range)
 * and multiplied with float32 accumulation; C is float32 row-major
 * (ldc >= N).  With SPD_GEMM_LOWER (requires A == B, M == N, lda == ldb)
 * only entries with row >= column are updated.  SPD_PREC_FP32 splits each
 * operand into three bf16 slices (s0 = bf16(x), s1 = bf16(x - s0), s2 =
 * bf16(x - s0 - s1), together x's 24 significant bits) and accumulates the
 * six slice products of order <= 2 in float32, the five small ones and
 * s0*t0 in separate accumulators added at the end: float32-class accuracy
 * (the dropped products are below 2^-23 |a||b|, the slices' last rounding
 * below 2^-24 |x|) at one sixth of the bf16 tensor-core rate.
 * flags: SPD_GEMM_LOWER as above; SPD_GEMM_STREAM_K schedules the tiles'
 * K loops over all SMs in equal contiguous ranges of (tile, K tile) units
 * ("stream-K", the schedule the factorisation picks for its long bulk
 * updates; the pieces of shared tiles are added to C in K order, so the
 * result does not depend on timing).  Device pointers; synchronous. */
#define SPD_GEMM_LOWER 1
#define SPD_GEMM_STREAM_K 2
#define SPD_GEMM_NARROW 4  /* SPD_PREC_FP32 only, not with LOWER: tiles of
                              128 x 32 (N <= 32) or 128 x 64 whose pipeline
                              stages hold all three slices of both operand
                              tiles -- the skinny products of spd_cg with
                              several right-hand sides (Section 3.2) */
spd_status spd_gemm_update(spd_handle *h, int prec, int M, int N, int K, const float *A, int lda,
                           const float *B, int ldb, float *C, int ldc, int flags);

/* ---- resource limits and failure checks -------------------------------------
 * (No passage of the paper: the library's own failure handling.)
 * spd_set_wait_limit bounds every spin-wait of h's kernels on a flag that
 * another CTA sets (the triangular sweeps' block flags and slot table;
 * default 1 s, allowed (0, 60] s).  A wait that runs out raises
 * SPD_ERR_TIMEOUT from the call, which winds down without fault; the handle
 * and the CUDA context stay usable.
 * spd_set_memory_cap caps the device memory one call on h may request
 * (a factor's arrays, the workspace, spd_solve_ir_host's device copies);
 * a larger request returns SPD_ERR_OOM before anything is allocated.
 * 0 (the default) means no cap.
 * spd_wait_probe launches one kernel that waits, with h's wait limit, on a
 * device flag that nothing sets: it returns SPD_ERR_TIMEOUT after that
 * limit, through the same device status word and error mapping as a real
 * expired wait.  For callers that test their handling of SPD_ERR_TIMEOUT. */
spd_status spd_set_wait_limit(spd_handle *h, double seconds);
spd_status spd_set_memory_cap(spd_handle *h, size_t bytes);
spd_status spd_wait_probe(spd_handle *h);

/* ---- phase timing ---------------------------------------------------------
 * Code-phase markers in the spirit of the paper's instrumentation library
 * (Section 2): when enabled, every launch of a hot-path kernel on h's
 * stream is bracketed by CUDA events and tagged with its phase and its
 * algorithmic work (flops and minimum HBM bytes).  Enabling clears the
 * statistics; reading synchronises the stream and sums the event times. */
typedef enum spd_phase {
    SPD_PHASE_CONVERT = 0,  /* A0: scaling + conversion                  */
    SPD_PHASE_LEAF = 1,     /* A1: diagonal-block factorisations         */
    SPD_PHASE_TRAILING = 2, /* A3: trailing updates (GEMM/SYRK)          */
    SPD_PHASE_SOLVE = 3,    /* A4: low-precision triangular solves       */
    SPD_PHASE_RESID = 4,    /* A5/C3: float64 residual / products        */
    SPD_PHASE_MATVEC = 5,   /* C1: low-precision CG products             */
    SPD_PHASE_VECTOR = 6,   /* A6/C2: float64 vector updates and dots    */
    SPD_PHASE_PANEL = 7,    /* A2: panel triangular solves (leaf TRSM)   */
    SPD_PHASE_BATCH = 8,    /* B1: persistent batched solves             */
    SPD_PHASE_TRAILING_X3 = 9, /* A3 of an FP32 factor: three bf16 slices
                                  on the tensor cores (flops counted once) */
    SPD_PHASE_RESID_DF32 = 10, /* A5/C3 on the float32 units (float32 pairs) */
    SPD_PHASE_RESID_TC = 11,   /* A5/C3 on the tensor cores (bf16 digits)     */
    SPD_PHASE_TRAILING_LAST = 12, /* A3: the rank-128 updates on the
                                     factorisation's critical path (the
                                     last update of each block column before
                                     its diagonal block is factored)        */
    SPD_PHASE_INVERSES = 13,      /* once per factor: inverses of the diagonal
                                     blocks and super-blocks, and the
                                     128-block sweeps' couplings (A4)        */
    SPD_PHASE_ESTIMATE = 14,      /* AUTO: the Lanczos condition bound before
                                     any factor (symmetric products of the
                                     scaled float32 matrix)                 */
    SPD_PHASE_COUNT = 15
} spd_phase;

spd_status spd_profile_enable(spd_handle *h, int on);
/* launches, summed device milliseconds, flops and bytes of one phase. */
spd_status spd_profile_read(spd_handle *h, int phase, int *launches, double *ms, double *flops,
                            double *bytes);
/* Total kernels launched through h since it was created (every phase). */
spd_status spd_launch_count(const spd_handle *h, long long *count);

#ifdef __cplusplus
}
#endif
#endif /* SPD_H */
