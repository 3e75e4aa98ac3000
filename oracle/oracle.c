/*
 * CPU oracle for the mixed-precision SPD solver -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct float64 C code for what the solver must
 * compute.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the product path never does.  It shares
 * no code, header or constant with the CUDA path.
 *
 * Conventions: every matrix is column-major with a leading dimension; an SPD
 * matrix A is read through its lower triangle (i >= j) only, except in the
 * residual, which applies the plain definition r = b - A x to the whole
 * stored matrix.  The loops are the textbook ones, with no blocking.
 *
 * What each routine follows:
 *   oracle_potrf       Section 3.1, eq. (cholesky): A = R^T R, R upper.
 *   oracle_potrs       Section 3.1, eq. (cholesky): X = R^{-1} R^{-T} B.
 *   oracle_potrf_f32   the same factorisation carried out in IEEE single
 *                      (the "low precision" of Section 3.1).
 *   oracle_potrs_f32   the same solve in IEEE single.
 *   oracle_residual    R = B - A X (Alg. 1 residual step, high precision).
 *   oracle_chol_ir     Algorithm 1 (Cholesky with iterative refinement) with a
 *                      given low-precision factor; solves in single,
 *                      residual and update in double.
 *   oracle_cg          textbook conjugate gradients in double.
 *   oracle_cg_ir       Algorithm 2 (CG with iterative refinement) in its
 *                      nested reading: the inner loop is Algorithm 2 with a
 *                      single-precision matrix (optionally banded), the
 *                      outer loop recomputes the true residual in double.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* --------------------------------------------------------------------------
 * Cholesky factorisation A = R^T R (R upper triangular), Section 3.1.
 * Column-by-column (Cholesky-Crout) order:
 *   R_jj = sqrt(A_jj - sum_{k<j} R_kj^2)
 *   R_ji = (A_ij - sum_{k<j} R_kj R_ki) / R_jj        for i > j
 * Returns 0 on success, or the 1-based column whose pivot is not positive.
 * The strictly lower part of R is set to zero.
 * ------------------------------------------------------------------------ */
int oracle_potrf(int n, const double *A, long lda, double *R, long ldr)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            R[IDX(i, j, ldr)] = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = A[IDX(j, j, lda)];
        const double *Rj = R + IDX(0, j, ldr);
        for (int k = 0; k < j; ++k)
            s -= Rj[k] * Rj[k];
        if (!(s > 0.0))
            return j + 1;
        double rjj = sqrt(s);
        R[IDX(j, j, ldr)] = rjj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            const double *Ri = R + IDX(0, i, ldr);
            double t = A[IDX(i, j, lda)];
            for (int k = 0; k < j; ++k)
                t -= Rj[k] * Ri[k];
            R[IDX(j, i, ldr)] = t / rjj;
        }
    }
    return 0;
}

/* X = R^{-1} R^{-T} B: forward substitution R^T y = b, then back substitution
 * R x = y, column by column of B. */
void oracle_potrs(int n, int m, const double *R, long ldr,
                  const double *B, long ldb, double *X, long ldx)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < m; ++c) {
        double *x = X + IDX(0, c, ldx);
        const double *b = B + IDX(0, c, ldb);
        for (int i = 0; i < n; ++i)
            x[i] = b[i];
        /* R^T y = b: y_i = (b_i - sum_{k<i} R_ki y_k) / R_ii */
        for (int i = 0; i < n; ++i) {
            const double *Ri = R + IDX(0, i, ldr);
            double t = x[i];
            for (int k = 0; k < i; ++k)
                t -= Ri[k] * x[k];
            x[i] = t / Ri[i];
        }
        /* R x = y, by columns: x_i = y_i / R_ii, then y_k -= R_ki x_i */
        for (int i = n - 1; i >= 0; --i) {
            const double *Ri = R + IDX(0, i, ldr);
            x[i] /= Ri[i];
            for (int k = 0; k < i; ++k)
                x[k] -= Ri[k] * x[i];
        }
    }
}

/* The same factorisation in IEEE single: A is rounded to float on input and
 * every operation is a float operation.  R is float. */
int oracle_potrf_f32(int n, const double *A, long lda, float *R, long ldr)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            R[IDX(i, j, ldr)] = 0.0f;
    for (int j = 0; j < n; ++j) {
        float s = (float)A[IDX(j, j, lda)];
        const float *Rj = R + IDX(0, j, ldr);
        for (int k = 0; k < j; ++k)
            s -= Rj[k] * Rj[k];
        if (!(s > 0.0f))
            return j + 1;
        float rjj = sqrtf(s);
        R[IDX(j, j, ldr)] = rjj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            const float *Ri = R + IDX(0, i, ldr);
            float t = (float)A[IDX(i, j, lda)];
            for (int k = 0; k < j; ++k)
                t -= Rj[k] * Ri[k];
            R[IDX(j, i, ldr)] = t / rjj;
        }
    }
    return 0;
}

/* z = R^{-1} R^{-T} r carried out in IEEE single (r rounded on input). */
static void potrs_f32_one(int n, const float *R, long ldr, const double *r, double *z, float *w)
{
    for (int i = 0; i < n; ++i)
        w[i] = (float)r[i];
    for (int i = 0; i < n; ++i) {
        const float *Ri = R + IDX(0, i, ldr);
        float t = w[i];
        for (int k = 0; k < i; ++k)
            t -= Ri[k] * w[k];
        w[i] = t / Ri[i];
    }
    for (int i = n - 1; i >= 0; --i) {
        const float *Ri = R + IDX(0, i, ldr);
        w[i] /= Ri[i];
        for (int k = 0; k < i; ++k)
            w[k] -= Ri[k] * w[i];
    }
    for (int i = 0; i < n; ++i)
        z[i] = (double)w[i];
}

void oracle_potrs_f32(int n, int m, const float *R, long ldr,
                      const double *B, long ldb, double *X, long ldx)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < m; ++c) {
        float *w = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
        potrs_f32_one(n, R, ldr, B + IDX(0, c, ldb), X + IDX(0, c, ldx), w);
        free(w);
    }
}

/* R = B - A X over the whole stored matrix A (plain definition). */
void oracle_residual(int n, int m, const double *A, long lda,
                     const double *B, long ldb, const double *X, long ldx,
                     double *Rr, long ldr)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < m; ++c) {
            double t = B[IDX(i, c, ldb)];
            for (int j = 0; j < n; ++j)
                t -= A[IDX(i, j, lda)] * X[IDX(j, c, ldx)];
            Rr[IDX(i, c, ldr)] = t;
        }
    }
}

/* ||A||_inf = max_i sum_j |A_ij| over the whole stored matrix. */
double oracle_norm_inf(int n, const double *A, long lda)
{
    double best = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            s += fabs(A[IDX(i, j, lda)]);
        if (s > best)
            best = s;
    }
    return best;
}

static double vnorm2(int n, const double *x)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += x[i] * x[i];
    return sqrt(s);
}

static double vnorm_inf(int n, const double *x)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        if (fabs(x[i]) > s)
            s = fabs(x[i]);
    return s;
}

/* Normwise backward error of column c: ||b - A x||_inf / (||A||_inf ||x||_inf).
 * Writes one value per column; returns the largest. */
double oracle_berr(int n, int m, const double *A, long lda,
                   const double *B, long ldb, const double *X, long ldx, double *per_col)
{
    double anorm = oracle_norm_inf(n, A, lda);
    double *r = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m > 0 ? m : 1));
    oracle_residual(n, m, A, lda, B, ldb, X, ldx, r, n);
    double worst = 0.0;
    for (int c = 0; c < m; ++c) {
        double rn = vnorm_inf(n, r + IDX(0, c, n));
        double xn = vnorm_inf(n, X + IDX(0, c, ldx));
        double e = (xn > 0.0 && anorm > 0.0) ? rn / (anorm * xn) : rn;
        if (per_col)
            per_col[c] = e;
        if (e > worst)
            worst = e;
    }
    free(r);
    return worst;
}

/* --------------------------------------------------------------------------
 * Algorithm 1 -- Cholesky with iterative refinement, one column at a time.
 * The low-precision factor Rt (float, upper) is supplied by the caller.
 *   x = Rt^{-1} Rt^{-T} b          [single]
 *   r = b - A x                    [double]
 *   while not converged:
 *       z = Rt^{-1} Rt^{-T} r      [single]
 *       x = x + z                  [double]
 *       r = b - A x                [double]
 * Stopping rule: crit == 0 -> ||r||_2 < tol (as printed in Alg. 1);
 *                crit == 1 -> ||r||_inf / (||A||_inf ||x||_inf) <= tol.
 * iters[c] counts the refinement sweeps (executions of the loop body).
 * Returns 0 if every column met the rule within maxit sweeps, else 1.
 * ------------------------------------------------------------------------ */
int oracle_chol_ir(int n, int m, const double *A, long lda, const float *Rt, long ldr,
                   const double *B, long ldb, double *X, long ldx,
                   double tol, int crit, int maxit, int *iters, double *final_err)
{
    double anorm = oracle_norm_inf(n, A, lda);
    int failed = 0;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    float *w = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < m; ++c) {
        double *x = X + IDX(0, c, ldx);
        const double *b = B + IDX(0, c, ldb);
        potrs_f32_one(n, Rt, ldr, b, x, w);
        oracle_residual(n, 1, A, lda, b, n, x, n, r, n);
        int it = 0;
        double err = 0.0;
        for (;;) {
            err = (crit == 0) ? vnorm2(n, r)
                              : vnorm_inf(n, r) / (anorm * (vnorm_inf(n, x) > 0 ? vnorm_inf(n, x) : 1.0));
            if ((crit == 0 && err < tol) || (crit == 1 && err <= tol))
                break;
            if (it >= maxit) {
                failed = 1;
                break;
            }
            potrs_f32_one(n, Rt, ldr, r, z, w);
            for (int i = 0; i < n; ++i)
                x[i] += z[i];
            oracle_residual(n, 1, A, lda, b, n, x, n, r, n);
            ++it;
        }
        if (iters)
            iters[c] = it;
        if (final_err)
            final_err[c] = err;
    }
    free(r);
    free(z);
    free(w);
    return failed;
}

/* Same loop with a double-precision perturbed factor (Fig. 3b experiment):
 * solves with Rp in double, residual in double, stop on backward error. */
int oracle_chol_ir_f64(int n, int m, const double *A, long lda, const double *Rp, long ldr,
                       const double *B, long ldb, double *X, long ldx,
                       double tol, int maxit, int *iters, double *final_err)
{
    double anorm = oracle_norm_inf(n, A, lda);
    int failed = 0;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < m; ++c) {
        double *x = X + IDX(0, c, ldx);
        const double *b = B + IDX(0, c, ldb);
        oracle_potrs(n, 1, Rp, ldr, b, n, x, n);
        oracle_residual(n, 1, A, lda, b, n, x, n, r, n);
        int it = 0;
        double err;
        for (;;) {
            double xn = vnorm_inf(n, x);
            err = vnorm_inf(n, r) / (anorm * (xn > 0 ? xn : 1.0));
            if (err <= tol)
                break;
            if (it >= maxit) {
                failed = 1;
                break;
            }
            oracle_potrs(n, 1, Rp, ldr, r, n, z, n);
            for (int i = 0; i < n; ++i)
                x[i] += z[i];
            oracle_residual(n, 1, A, lda, b, n, x, n, r, n);
            ++it;
        }
        if (iters)
            iters[c] = it;
        if (final_err)
            final_err[c] = err;
    }
    free(r);
    free(z);
    return failed;
}

/* --------------------------------------------------------------------------
 * Textbook conjugate gradients in double, x0 = 0, per column:
 *   r = b, p = r, rho = r^T r
 *   repeat: z = A p; alpha = rho / p^T z; x += alpha p; r -= alpha z;
 *           rho' = r^T r; beta = rho'/rho; p = r + beta p
 * until ||r||_2 <= tol_rel ||b||_2 or maxit.  A is read through its lower
 * triangle.  iters[c] = iterations taken; relres[c] = final ||r||/||b||
 * with r the recursively updated residual.
 * ------------------------------------------------------------------------ */
static double sym_at(const double *A, long lda, int i, int j)
{
    return (i >= j) ? A[IDX(i, j, lda)] : A[IDX(j, i, lda)];
}

static void symv(int n, const double *A, long lda, const double *p, double *z)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double t = 0.0;
        for (int j = 0; j < n; ++j)
            t += sym_at(A, lda, i, j) * p[j];
        z[i] = t;
    }
}

int oracle_cg(int n, int m, const double *A, long lda, const double *B, long ldb,
              double *X, long ldx, double tol_rel, int maxit, int *iters, double *relres)
{
    int failed = 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(sizeof(double) * nn);
    double *p = (double *)malloc(sizeof(double) * nn);
    double *z = (double *)malloc(sizeof(double) * nn);
    for (int c = 0; c < m; ++c) {
        double *x = X + IDX(0, c, ldx);
        const double *b = B + IDX(0, c, ldb);
        for (int i = 0; i < n; ++i) {
            x[i] = 0.0;
            r[i] = b[i];
            p[i] = b[i];
        }
        double bnorm = vnorm2(n, b);
        double rho = 0.0;
        for (int i = 0; i < n; ++i)
            rho += r[i] * r[i];
        int it = 0;
        while (sqrt(rho) > tol_rel * bnorm) {
            if (it >= maxit) {
                failed = 1;
                break;
            }
            symv(n, A, lda, p, z);
            double pz = 0.0;
            for (int i = 0; i < n; ++i)
                pz += p[i] * z[i];
            double alpha = rho / pz;
            for (int i = 0; i < n; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * z[i];
            }
            double rho_new = 0.0;
            for (int i = 0; i < n; ++i)
                rho_new += r[i] * r[i];
            double beta = rho_new / rho;
            for (int i = 0; i < n; ++i)
                p[i] = r[i] + beta * p[i];
            rho = rho_new;
            ++it;
        }
        if (iters)
            iters[c] = it;
        if (relres)
            relres[c] = (bnorm > 0) ? sqrt(rho) / bnorm : sqrt(rho);
    }
    free(r);
    free(p);
    free(z);
    return failed;
}

/* --------------------------------------------------------------------------
 * Algorithm 2 -- CG with iterative refinement, nested reading, per column.
 *   outer ("high"): r = b - A x in double over the full A; stop when the
 *                   rule holds; else run the inner loop on A z = r, x += z.
 *   inner ("low"):  Algorithm 2's loop with z = At p computed in IEEE single
 *                   (At is the single-precision matrix, p rounded to single,
 *                   float accumulation); rho, alpha, beta and the vector
 *                   updates in double.  Stops when the recursively updated
 *                   ||r_in||_2 <= max(eta ||r_outer||_2, tol_abs) or after
 *                   maxit_in steps.
 *   beta is r'^T r' / rho (Fletcher-Reeves form of the printed quotient).
 * Matrix At: full n x n float (column-major, ldat), or banded when band >= 0:
 * then only |i-j| <= band entries of At are used.
 * Stopping rule: crit == 0 -> ||r||_2 < tol; crit == 1 -> ||r||_2 <= tol ||b||_2.
 * iters_low[c] / iters_high[c]: inner steps in total / outer residuals
 * after the first.  Returns 0 if every column met the rule.
 * ------------------------------------------------------------------------ */
static void matvec_f32(int n, const float *At, long ldat, int band, const double *p, double *z, float *pw)
{
    for (int j = 0; j < n; ++j)
        pw[j] = (float)p[j];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        float t = 0.0f;
        int j0 = 0, j1 = n;
        if (band >= 0) {
            j0 = i - band < 0 ? 0 : i - band;
            j1 = i + band + 1 > n ? n : i + band + 1;
        }
        for (int j = j0; j < j1; ++j)
            t += At[IDX(i, j, ldat)] * pw[j];
        z[i] = (double)t;
    }
}

int oracle_cg_ir(int n, int m, const double *A, long lda, const float *At, long ldat, int band,
                 const double *B, long ldb, double *X, long ldx,
                 double tol, int crit, double eta, int maxit_in, int maxit_out,
                 int *iters_low, int *iters_high, double *final_err)
{
    int failed = 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(sizeof(double) * nn);
    double *ri = (double *)malloc(sizeof(double) * nn);
    double *p = (double *)malloc(sizeof(double) * nn);
    double *z = (double *)malloc(sizeof(double) * nn);
    double *e = (double *)malloc(sizeof(double) * nn);
    float *pw = (float *)malloc(sizeof(float) * nn);
    for (int c = 0; c < m; ++c) {
        double *x = X + IDX(0, c, ldx);
        const double *b = B + IDX(0, c, ldb);
        double bnorm = vnorm2(n, b);
        double target = (crit == 0) ? tol : tol * bnorm;
        for (int i = 0; i < n; ++i)
            x[i] = 0.0;
        int low = 0, high = -1;
        double rn;
        for (;;) {
            oracle_residual(n, 1, A, lda, b, n, x, n, r, n);
            ++high;
            rn = vnorm2(n, r);
            int ok = (crit == 0) ? (rn < target) : (rn <= target);
            if (ok)
                break;
            if (high >= maxit_out) {
                failed = 1;
                break;
            }
            /* inner: Algorithm 2 on A e = r from e = 0 */
            for (int i = 0; i < n; ++i) {
                e[i] = 0.0;
                ri[i] = r[i];
                p[i] = r[i];
            }
            double stop = eta * rn;
            if (stop < target)
                stop = target;
            double rho = 0.0;
            for (int i = 0; i < n; ++i)
                rho += ri[i] * ri[i];
            int k = 0;
            while (sqrt(rho) > stop && k < maxit_in) {
                matvec_f32(n, At, ldat, band, p, z, pw);
                double pz = 0.0;
                for (int i = 0; i < n; ++i)
                    pz += p[i] * z[i];
                double alpha = rho / pz;
                for (int i = 0; i < n; ++i) {
                    e[i] += alpha * p[i];
                    ri[i] -= alpha * z[i];
                }
                double rho_new = 0.0;
                for (int i = 0; i < n; ++i)
                    rho_new += ri[i] * ri[i];
                double beta = rho_new / rho;
                for (int i = 0; i < n; ++i)
                    p[i] = ri[i] + beta * p[i];
                rho = rho_new;
                ++k;
            }
            low += k;
            for (int i = 0; i < n; ++i)
                x[i] += e[i];
        }
        if (iters_low)
            iters_low[c] = low;
        if (iters_high)
            iters_high[c] = high;
        if (final_err)
            final_err[c] = rn;
    }
    free(r);
    free(ri);
    free(p);
    free(z);
    free(e);
    free(pw);
    return failed;
}
