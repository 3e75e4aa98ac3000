// k_resid.cuh -- step A5: the float64 residual R = B - A X of Algorithm 1
// (lines 3, 7) and Algorithm 2 (line 2), and float64 products Q = A P for
// the float64 CG fallback; plus per-column norms and the convergence test
// (A7).  All reductions run in a fixed order, so results are bitwise
// reproducible run to run.
//
// Pass 1 (k_resid_partial): grid (row blocks of 256) x (S column splits);
//   thread i accumulates sum_{j in split} A[i + j lda] X[j, c] for MT
//   columns in float64 registers; X rows are staged through shared memory.
//   A is read once per launch (coalesced along i), optionally with the
//   float32 row sums of |A| for ||A||_inf.
// Pass 2 (k_resid_final): R = B - sum_s P_s (or Q = sum_s P_s), per-block
//   partial norms.  Pass 3 (k_colnorms): per-column norms.
#pragma once
#include "common.cuh"
#include "tc_ptx.cuh"

#define RESID_ROWS 256
#define RESID_JT 64

template <int MT>
static __global__ void __launch_bounds__(RESID_ROWS) k_resid_partial(const double* __restrict__ A, long lda, int n,
                                                              const double* __restrict__ X, long ldx, int c0,
                                                              int mc, int jchunk, int mtot,
                                                              double* __restrict__ P, float* __restrict__ rowabs,
                                                              const int* __restrict__ gate = nullptr) {
    __shared__ __align__(16) double xs[RESID_JT][MT];
    if (gate && *gate == 0) return;  // refinement over: nothing to do (capturable solves)
    const int tid = threadIdx.x;
    const int i = blockIdx.x * RESID_ROWS + tid;
    const int s = blockIdx.y;
    const int j0 = s * jchunk;
    const int j1 = min(n, j0 + jchunk);
    double acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[c] = 0.0;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;  // MT == 1: the interleaved accumulators
    float asum = 0.f;
    const double* Ai = A + (i < n ? i : 0);
    for (int jb = j0; jb < j1; jb += RESID_JT) {
        const int jn = min(RESID_JT, j1 - jb);
        __syncthreads();
        for (int e = tid; e < RESID_JT * MT; e += RESID_ROWS) {
            int jj = e % RESID_JT, c = e / RESID_JT;
            xs[jj][c] = (jj < jn && c < mc) ? X[(long)(c0 + c) * ldx + jb + jj] : 0.0;
        }
        __syncthreads();
        if (i < n) {
            const double* ap = Ai + (long)jb * lda;
            if (MT == 1 && jn == RESID_JT && !rowabs) {
                // one column: four interleaved accumulators (column jj into
                // accumulator jj % 4) and sixteen loads in flight per thread,
                // added in a fixed order below
#pragma unroll 4
                for (int jj = 0; jj < RESID_JT; jj += 4) {
                    const double a0 = __ldg(ap + (long)jj * lda), a1 = __ldg(ap + (long)(jj + 1) * lda);
                    const double a2 = __ldg(ap + (long)(jj + 2) * lda), a3 = __ldg(ap + (long)(jj + 3) * lda);
                    q0 = fma(a0, xs[jj][0], q0);
                    q1 = fma(a1, xs[jj + 1][0], q1);
                    q2 = fma(a2, xs[jj + 2][0], q2);
                    q3 = fma(a3, xs[jj + 3][0], q3);
                }
            } else if (jn == RESID_JT) {
#pragma unroll 4
                for (int jj = 0; jj < RESID_JT; ++jj) {
                    double a = __ldg(ap + (long)jj * lda);
                    if (rowabs) asum += fabsf((float)a);
#pragma unroll
                    for (int c = 0; c < MT; ++c) acc[c] = fma(a, xs[jj][c], acc[c]);
                }
            } else {
                for (int jj = 0; jj < jn; ++jj) {
                    double a = __ldg(ap + (long)jj * lda);
                    if (rowabs) asum += fabsf((float)a);
#pragma unroll
                    for (int c = 0; c < MT; ++c) acc[c] = fma(a, xs[jj][c], acc[c]);
                }
            }
        }
    }
    if (i < n) {
        if (MT == 1) acc[0] += (q0 + q1) + (q2 + q3);
#pragma unroll
        for (int c = 0; c < MT; ++c)
            if (c < mc) P[((long)s * mtot + c0 + c) * n + i] = acc[c];
        if (rowabs) rowabs[(long)s * n + i] = asum;
    }
}

// mode 0: R = B - sum_s P_s ; mode 1: R = sum_s P_s.  Block partial norms
// NP[(blk * m + c) * 3 + {0,1,2}] = max|r|, sum r^2, max|x| (x from X; if X
// is NULL the third entry is 0).
static __global__ void __launch_bounds__(256) k_resid_final(const double* __restrict__ B, long ldb, int n, int m,
                                                     const double* __restrict__ P, int S,
                                                     double* __restrict__ R, long ldr,
                                                     const double* __restrict__ X, long ldx,
                                                     double* __restrict__ NP, int mode,
                                                     const int* __restrict__ gate = nullptr) {
    __shared__ double red[3][8];
    if (gate && *gate == 0) return;
    const int c = blockIdx.y;
    const int i = blockIdx.x * 256 + threadIdx.x;
    double rmax = 0.0, r2 = 0.0, xmax = 0.0;
    if (i < n) {
        double s = 0.0;
        for (int k = 0; k < S; ++k) s += P[((long)k * m + c) * n + i];
        double r = (mode == 0) ? B[(long)c * ldb + i] - s : s;
        R[(long)c * ldr + i] = r;
        rmax = fabs(r);
        r2 = r * r;
        if (X) xmax = fabs(X[(long)c * ldx + i]);
    }
    rmax = warp_max(rmax);
    r2 = warp_sum(r2);
    xmax = warp_max(xmax);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = rmax;
        red[1][w] = r2;
        red[2][w] = xmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, x = 0.0;
        for (int k = 0; k < 8; ++k) {
            a = fmax(a, red[0][k]);
            b += red[1][k];
            x = fmax(x, red[2][k]);
        }
        double* o = NP + ((long)blockIdx.x * m + c) * 3;
        o[0] = a;
        o[1] = b;
        o[2] = x;
    }
}

// colnorms[3c..3c+2] = ||r_c||_inf, ||r_c||_2, ||x_c||_inf from G block partials.
static __global__ void __launch_bounds__(256) k_colnorms(const double* __restrict__ NP, int G, int m,
                                                  double* __restrict__ colnorms) {
    __shared__ double red[3][8];
    const int c = blockIdx.x;
    double a = 0.0, b = 0.0, x = 0.0;
    for (int g = threadIdx.x; g < G; g += 256) {
        const double* o = NP + ((long)g * m + c) * 3;
        a = fmax(a, o[0]);
        b += o[1];
        x = fmax(x, o[2]);
    }
    a = warp_max(a);
    b = warp_sum(b);
    x = warp_max(x);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A_ = 0.0, B_ = 0.0, X_ = 0.0;
        for (int k = 0; k < 8; ++k) {
            A_ = fmax(A_, red[0][k]);
            B_ += red[1][k];
            X_ = fmax(X_, red[2][k]);
        }
        colnorms[3 * c + 0] = A_;
        colnorms[3 * c + 1] = sqrt(B_);
        colnorms[3 * c + 2] = X_;
    }
}

// ||A||_inf = max_i sum_s rowabs[s][i]  (single CTA, fixed order)
static __global__ void __launch_bounds__(1024) k_anorm(const float* __restrict__ rowabs, int S, int n,
                                                double* __restrict__ anorm) {
    __shared__ double red[32];
    double best = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) {
        double s = 0.0;
        for (int k = 0; k < S; ++k) s += (double)rowabs[(long)k * n + i];
        best = fmax(best, s);
    }
    best = warp_max(best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < 32; ++k) b = fmax(b, red[k]);
        *anorm = b;
    }
}

// ||b_c||_2 for m columns (one CTA per column, fixed order)
static __global__ void __launch_bounds__(256) k_col_nrm2(const double* __restrict__ B, long ldb, int n,
                                                  double* __restrict__ out) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        double v = B[(long)c * ldb + i];
        s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        out[c] = sqrt(t);
    }
}

// Convergence bookkeeping for the refinement loops (A7).
struct IrCol {
    double err;       // current value of the stopping quantity
    double prev;      // previous value
    int conv;         // 1 once the column met the rule (frozen)
    int stall;        // consecutive sweeps that shrank err by less than half
    int iters;        // sweeps applied to this column
    int extra;        // polish sweeps still owed once the rule holds
};
struct IrSummary {
    int active;       // columns not yet converged
    int stagnated;    // columns whose stall count reached 2
    double max_berr;  // max over columns of the backward error
    double max_rel;   // max over columns of ||r||_2 / ||b||_2
    int pending;      // columns that met the rule on a residual not allowed to accept
};

// One CTA: update per-column state from colnorms; crit as spd_crit.
static __global__ void k_ir_check(const double* __restrict__ colnorms, const double* __restrict__ anorm,
                           const double* __restrict__ b2, int m, int crit, double tol,
                           IrCol* __restrict__ cols, IrSummary* __restrict__ sum, int count_sweep, int polish,
                           int accept = 1, int restart = 0) {
    __shared__ int s_active, s_stag, s_pend;
    __shared__ double s_berr, s_rel;
    if (threadIdx.x == 0) {
        s_active = 0;
        s_stag = 0;
        s_pend = 0;
        s_berr = 0.0;
        s_rel = 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        IrCol st = cols[c];
        double rinf = colnorms[3 * c], r2 = colnorms[3 * c + 1], xinf = colnorms[3 * c + 2];
        double an = *anorm;
        double berr = (an > 0.0 && xinf > 0.0) ? rinf / (an * xinf) : rinf;
        double rel = (b2[c] > 0.0) ? r2 / b2[c] : r2;
        double err = (crit == 0) ? berr : (crit == 1 ? rel : r2);
        if (!st.conv) {
            if (count_sweep) st.iters += 1;
            bool ok = (crit == 2) ? (err < tol) : (err <= tol);
            if (ok && !accept) {
                // a residual that may not decide convergence (float32 pairs):
                // the next sweep, judged by a float64 residual, doubles as
                // the polish sweep
                st.stall = 0;
                st.extra = 0;
                atomicAdd(&s_pend, 1);
            } else if (ok) {
                if (st.extra > 0) st.extra -= 1;  // meets the rule: polish once more
                else st.conv = 1;
                st.stall = 0;
            } else {
                st.extra = polish;
                // restart: the first residual of another arithmetic is not
                // compared with the last one of the previous arithmetic
                if (restart) st.stall = 0;
                else if (count_sweep) st.stall = (err > 0.5 * st.prev) ? st.stall + 1 : 0;
            }
            st.prev = err;
            st.err = err;
        }
        cols[c] = st;
        if (!st.conv) atomicAdd(&s_active, 1);
        if (!st.conv && st.stall >= 2) atomicAdd(&s_stag, 1);
        // max of non-negative doubles through their bit patterns (order-independent)
        atomicMax((unsigned long long*)&s_berr, (unsigned long long)__double_as_longlong(berr));
        atomicMax((unsigned long long*)&s_rel, (unsigned long long)__double_as_longlong(rel));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sum->active = s_active;
        sum->stagnated = s_stag;
        sum->pending = s_pend;
        sum->max_berr = s_berr;
        sum->max_rel = s_rel;
    }
}

// frozen[c] = cols[c].conv
static __global__ void k_frozen_from_cols(const IrCol* __restrict__ cols, int m, int* __restrict__ frozen) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) frozen[c] = cols[c].conv;
}

// ---------------------------------------------------------------------------
// The same residual in float32 arithmetic, float64-accurate ("DF32"): the
// float64 pipe of this GPU is a small fraction of its float32 pipe, so the
// products run on the float32 units with error-free transformations.
//
// * Each float64 entry a of A is split by integer operations on its bits:
//   ah = its 24 leading significand bits (truncated), am = the next 23 bits
//   rounded to nearest, so |a - ah - am| <= 2^-47 |a|.  Entries outside
//   [2^-100, 2^100) in magnitude (and Inf/NaN) are not split: they take a
//   float64 FMA (a branch no ordinary matrix takes; zeros split to 0, 0).
// * Column c of X is scaled by a power of two sc_c (max |x| in [1/2, 1))
//   and each entry split as xh = fl32(x), xm = fl32(x - xh).
// * a x = ah xh + (am xh + ah xm) + dropped terms below 2^-46 |a||x|; the
//   leading product is kept exactly as p + e (e by FMA).
// * Running sums are unevaluated float32 pairs (S, C): S <- S + p by
//   TwoSum (exact), C collects the TwoSum errors, e and the cross terms;
//   every RESID_FOLD terms the pair is added into a float64 accumulator, and
//   the result is scaled back by 1/sc_c.  Each addition into C rounds at
//   2^-24 |C| with |C| up to ~k 2^-25 |S| after k terms, so a run of 64
//   terms errs by up to ~2^-43 of its largest partial sum: 48-bit pairs, not
//   float64 (2^-53 per operation).
// All float32 operations use explicit round-to-nearest intrinsics, so the
// compiler cannot fuse a product into a sum and break the TwoSum.
// ---------------------------------------------------------------------------
#define RESID_FOLD 64

// Split a float64 into two float32 values; returns false when a must take
// the float64 path (|a| outside [2^-100, 2^100) and a != 0, or Inf/NaN).
__device__ __forceinline__ bool df32_split(double a, float& ah, float& am) {
    const unsigned hi = (unsigned)__double2hiint(a), lo = (unsigned)__double2loint(a);
    const unsigned ex = (hi >> 20) & 0x7ffu;
    const unsigned sg = hi & 0x80000000u;
    if (ex - 923u >= 200u) {
        ah = 0.f;
        am = 0.f;
        return ((hi & 0x7fffffffu) | lo) == 0u;
    }
    // ah: biased float32 exponent ex - 1023 + 127, mantissa = the 23 bits
    // after the leading one
    ah = __uint_as_float(sg | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    // am: the remaining 29 bits rounded to 23 (a carry out simply bumps the
    // exponent), built as (2^23 + r) 2^(E-150) - 2^23 2^(E-150), E = ex - 919
    const unsigned r = ((lo & 0x1fffffffu) + 32u) >> 6;
    const unsigned eb = (ex - 919u) << 23;
    am = __fsub_rn(__uint_as_float(sg | (eb + r)), __uint_as_float(sg | eb));
    return true;
}

// sc[c] = 2^-e_c and sc[m + c] = 2^e_c with max_i |X[i, c]| = f 2^e_c,
// f in [1/2, 1); 1 for an all-zero or non-finite column.
static __global__ void __launch_bounds__(256) k_xscale(const double* __restrict__ X, long ldx, int n, int m,
                                                double* __restrict__ sc) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) mx = fmax(mx, fabs(X[(long)c * ldx + i]));
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < 8; ++k) v = fmax(v, red[k]);
        int e = 0;
        if (v > 0.0 && isfinite(v)) {
            frexp(v, &e);
            e = max(-1000, min(1000, e));
        }
        sc[c] = ldexp(1.0, -e);
        sc[m + c] = ldexp(1.0, e);
    }
}

// A reaches shared memory in 16-column chunks by bulk copies (one 2 KB copy
// per column of the CTA's 256 rows, double-buffered, completing on an
// mbarrier), so the loads in flight no longer depend on registers.  A CTA
// whose rows are ragged (the last row block) or whose columns are not 16-byte
// aligned reads A directly instead.
#define DF_DJ 16
template <int MT>
constexpr size_t df32_smem() {
    return (size_t)2 * DF_DJ * RESID_ROWS * sizeof(double)       // A chunks
           + (size_t)RESID_JT * (MT + 1) * sizeof(float2)          // (xh, xm)
           + (size_t)RESID_JT * (MT + 1) * sizeof(double) + 64;   // scaled X, barriers
}

template <int MT>
__device__ __forceinline__ void df32_madd(double a, const float2* xfj, const double* xdj, float (&S)[MT],
                                          float (&C)[MT], double (&acc)[MT], float& asum, bool with_abs) {
    float ah, am;
    if (!df32_split(a, ah, am)) {
#pragma unroll
        for (int c = 0; c < MT; ++c) acc[c] = fma(a, xdj[c], acc[c]);
        if (with_abs) asum += fabsf(__double2float_rn(a));
    }
    if (with_abs) asum += fabsf(ah);
#pragma unroll
    for (int c = 0; c < MT; ++c) {
        const float2 x = xfj[c];
        const float p = __fmul_rn(ah, x.x);
        const float e = __fmaf_rn(ah, x.x, -p);
        const float cr = __fmaf_rn(ah, x.y, __fmaf_rn(am, x.x, e));
        const float s = __fadd_rn(S[c], p);
        const float bp = __fsub_rn(s, S[c]);
        const float t = __fadd_rn(__fsub_rn(S[c], __fsub_rn(s, bp)), __fsub_rn(p, bp));
        S[c] = s;
        C[c] = __fadd_rn(C[c], __fadd_rn(t, cr));
    }
}

template <int MT>
static __global__ void __launch_bounds__(RESID_ROWS, 2)
    k_resid_partial_df32(const double* __restrict__ A, long lda, int n, const double* __restrict__ X, long ldx,
                         int c0, int mc, int jchunk, int mtot, const double* __restrict__ sc,
                         double* __restrict__ P, float* __restrict__ rowabs, DevStatus* st) {
    extern __shared__ __align__(128) unsigned char df_smem[];
    double* Ast = reinterpret_cast<double*>(df_smem);                                   // [2][DF_DJ][256]
    float2* xf = reinterpret_cast<float2*>(Ast + 2 * DF_DJ * RESID_ROWS);              // [JT][MT+1]
    double* xd = reinterpret_cast<double*>(xf + RESID_JT * (MT + 1));                   // [JT][MT+1]
    uint64_t* bar = reinterpret_cast<uint64_t*>(xd + RESID_JT * (MT + 1));              // [2]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 2);
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * RESID_ROWS, i = i0 + tid;
    const int j0 = blockIdx.y * jchunk;
    const int j1 = min(n, j0 + jchunk);
    const bool bulk = (i0 + RESID_ROWS <= n) && ((reinterpret_cast<uintptr_t>(A + i0) & 15) == 0) &&
                      ((lda * (long)sizeof(double)) % 16 == 0);
    const int nchunks = (j1 - j0 + DF_DJ - 1) / DF_DJ;
    float S[MT], C[MT];
    double acc[MT];
#pragma unroll
    for (int c = 0; c < MT; ++c) {
        S[c] = 0.f;
        C[c] = 0.f;
        acc[c] = 0.0;
    }
    float asum = 0.f;
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    // issue chunk g (columns j0 + 16 g ..) into buffer g & 1
    auto issue = [&](int g) {
        const int jc = j0 + g * DF_DJ, w = min(DF_DJ, j1 - jc);
        uint64_t* b = &bar[g & 1];
        tc::mbar_arrive_expect_tx(b, (uint32_t)(w * RESID_ROWS * sizeof(double)));
        for (int q = 0; q < w; ++q)
            tc::bulk_g2s(Ast + ((g & 1) * DF_DJ + q) * RESID_ROWS, A + (long)(jc + q) * lda + i0,
                         RESID_ROWS * sizeof(double), b);
    };
    if (bulk && tid == 0) {
        if (nchunks > 0) issue(0);
        if (nchunks > 1) issue(1);
    }
    const double* Ai = A + (i < n ? i : 0);
    bool ok = true;
    int g = 0;
    for (int jb = j0; jb < j1; jb += RESID_JT) {
        const int jn = min(RESID_JT, j1 - jb);
        __syncthreads();
        for (int e = tid; e < RESID_JT * MT; e += RESID_ROWS) {
            const int jj = e % RESID_JT, c = e / RESID_JT;
            double v = 0.0;
            if (jj < jn && c < mc) v = X[(long)(c0 + c) * ldx + jb + jj] * sc[c0 + c];
            const float hx = __double2float_rn(v);
            xd[jj * (MT + 1) + c] = v;
            xf[jj * (MT + 1) + c] = make_float2(hx, __double2float_rn(v - (double)hx));
        }
        __syncthreads();
        for (int jf = 0; jf < jn; jf += DF_DJ, ++g) {
            const int je = min(jn, jf + DF_DJ);
            if (bulk) {
                ok = ok && tc::mbar_wait(&bar[g & 1], (uint32_t)((g >> 1) & 1), abort_flag, 2000000000ull);
                if (ok) {
                    const double* ac = Ast + (g & 1) * DF_DJ * RESID_ROWS + tid;
#pragma unroll 4
                    for (int jj = jf; jj < je; ++jj)
                        df32_madd<MT>(ac[(jj - jf) * RESID_ROWS], xf + jj * (MT + 1), xd + jj * (MT + 1), S, C, acc,
                                      asum, rowabs != nullptr);
                }
                __syncthreads();  // every thread is done with buffer g & 1
                if (tid == 0 && ok && !*abort_flag && g + 2 < nchunks) issue(g + 2);
            } else if (i < n) {
                const double* ap = Ai + (long)jb * lda;
#pragma unroll 2
                for (int jj = jf; jj < je; ++jj)
                    df32_madd<MT>(__ldg(ap + (long)jj * lda), xf + jj * (MT + 1), xd + jj * (MT + 1), S, C, acc,
                                  asum, rowabs != nullptr);
            }
            if ((jf + DF_DJ) % RESID_FOLD == 0 || jf + DF_DJ >= jn) {  // fold the float32 pairs
#pragma unroll
                for (int c = 0; c < MT; ++c) {
                    acc[c] += (double)S[c] + (double)C[c];
                    S[c] = 0.f;
                    C[c] = 0.f;
                }
            }
        }
    }
    if (bulk && !ok && tid == 0) atomicOr(&st->flags, SPD_DEV_TIMEOUT);
    if (i < n) {
#pragma unroll
        for (int c = 0; c < MT; ++c)
            if (c < mc) P[((long)blockIdx.y * mtot + c0 + c) * n + i] = acc[c] * sc[mtot + c0 + c];
        if (rowabs) rowabs[(long)blockIdx.y * n + i] = asum;
    }
}
