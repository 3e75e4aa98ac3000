// k_cg.cuh -- steps C1/C2 of Algorithm 2 (CG with iterative refinement):
// the low-precision product z = A~ p (C1) and the float64 scalar/vector
// work rho, alpha, x += alpha p, r -= alpha z, beta, p = r + beta p (C2).
// m right-hand sides are m independent CG runs that share each pass over
// A~.  Dots are reduced in a fixed order (per-CTA partials, then every
// consumer CTA sums them in the same order), so runs are reproducible.
#pragma once
#include "common.cuh"

#define MV_ROWS_PER_WARP 4
#define MV_ROWS (8 * MV_ROWS_PER_WARP)
#define MV_JCH 512

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// Q[:, c0:c0+mc] = A~ Pf (float32 products and sums), A~ row-major n x ldt
// (ldt a multiple of 4, padding columns zero), Pf float32 n x m (ld n).
// One warp per row group; lanes stride the row 4 elements at a time.
template <typename T, int MC>
static __global__ void __launch_bounds__(256) k_matvec_lp(const T* __restrict__ At, long ldt, int n,
                                                   const float* __restrict__ Pf, int c0, int mc,
                                                   double* __restrict__ Q, const int* __restrict__ done) {
    __shared__ __align__(16) float ps[MC][MV_JCH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rbase = blockIdx.x * MV_ROWS + warp * MV_ROWS_PER_WARP;
    float acc[MV_ROWS_PER_WARP][MC];
#pragma unroll
    for (int r = 0; r < MV_ROWS_PER_WARP; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[r][c] = 0.f;
    for (int jb = 0; jb < n; jb += MV_JCH) {
        const int jn = min(MV_JCH, n - jb);
        __syncthreads();
        for (int e = tid; e < MC * MV_JCH; e += 256) {
            int c = e / MV_JCH, jj = e % MV_JCH;
            ps[c][jj] = (c < mc && jj < jn) ? Pf[(long)(c0 + c) * n + jb + jj] : 0.f;
        }
        __syncthreads();
        const int jlim = (jn + 3) & ~3;  // padding columns of A~ are zero
#pragma unroll
        for (int r = 0; r < MV_ROWS_PER_WARP; ++r) {
            const int row = rbase + r;
            if (row >= n) break;
            const T* arow = At + (long)row * ldt + jb;
            for (int jj = lane * 4; jj < jlim; jj += 128) {
                float4 a = ld4(arow + jj);
#pragma unroll
                for (int c = 0; c < MC; ++c) {
                    float4 p = *reinterpret_cast<const float4*>(&ps[c][jj]);
                    acc[r][c] = fmaf(a.x, p.x, fmaf(a.y, p.y, fmaf(a.z, p.z, fmaf(a.w, p.w, acc[r][c]))));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < MV_ROWS_PER_WARP; ++r) {
        const int row = rbase + r;
#pragma unroll
        for (int c = 0; c < MC; ++c) {
            float v = warp_sum(acc[r][c]);
            if (lane == 0 && row < n && c < mc) Q[(long)(c0 + c) * n + row] = (double)v;
        }
    }
}

// The tensor-core product of C1 for m > 1 right-hand sides: A~ and the
// float32 P enter the tensor cores as three bf16 slices each (x = s0 + s1 +
// s2, the float32 value to within a last rounding below 2^-24 |x|), and the
// six slice products of order <= 2 accumulate in float32, so the product
// carries the float32 product's accuracy.  The narrow GEMM computes
// C -= A~ P^T on a zeroed float32 C (n x ldc, row-major); Q = -C.
//
// Slice planes of A~ (plane stride `plane`): row j, column i = the slices of
// fl32(A(i, j)) (A symmetric), zero in the padding columns n <= i < Kp.
static __global__ void k_convert_x3(const double* __restrict__ A, long lda, int n, int Kp,
                                    __nv_bfloat16* __restrict__ M, long ldo, long plane, DevStatus* st) {
    const long total = (long)n * Kp;
    bool bad = false;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long j = e / Kp, i = e - j * Kp;  // column j of A = row j of the planes: coalesced both ways
        float v = 0.f;
        if (i < n) {
            const double a = A[j * lda + i];
            if (!isfinite(a)) bad = true;
            v = (float)a;
        }
        __nv_bfloat16 s0, s1, s2;
        split_bf16x3(v, s0, s1, s2);
        __nv_bfloat16* q = M + j * ldo + i;
        q[0] = s0;
        q[plane] = s1;
        q[2 * plane] = s2;
    }
    if (bad) dev_raise(st, SPD_DEV_NONFINITE);
}

// Rows c < m of P^T's slice planes: row c, column k = the slices of Pf[c n + k]
// (padding rows and columns stay zero from the setup).
static __global__ void k_p_x3(const float* __restrict__ Pf, int n, int m, __nv_bfloat16* __restrict__ Pm, long ldo,
                              long plane) {
    const long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long c = e / n, k = e - c * n;
        __nv_bfloat16 s0, s1, s2;
        split_bf16x3(Pf[e], s0, s1, s2);
        __nv_bfloat16* q = Pm + c * ldo + k;
        q[0] = s0;
        q[plane] = s1;
        q[2 * plane] = s2;
    }
}

// Q[c n + i] = -C[i ldc + c] (float64, column-major) from the narrow GEMM's C
static __global__ void k_cf_to_q(const float* __restrict__ Cf, long ldc, int n, int m, double* __restrict__ Q) {
    const long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long c = e / n, i = e - c * n;
        Q[e] = -(double)Cf[i * ldc + c];
    }
}

// Banded product with the diagonal-major band Ab[(o+band)*n + i] = A~(i, i+o).
static __global__ void k_matvec_band(const float* __restrict__ Ab, int n, int band, const float* __restrict__ Pf,
                              int m, double* __restrict__ Q) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int c = (int)(e / n), i = (int)(e % n);
        const float* p = Pf + (long)c * n;
        float acc = 0.f;
        for (int o = -band; o <= band; ++o) {
            int j = i + o;
            if (j >= 0 && j < n) acc = fmaf(Ab[(long)(o + band) * n + i], p[j], acc);
        }
        Q[(long)c * n + i] = (double)acc;
    }
}

// Per-block partial dots: block (x, c) sums rows [x r, (x + 1) r) of column
// c (r = ceil(n / gridDim.x)): part[(x m + c) 2 + {0, 1}] = sum a1.b1,
// sum a2.b2 (a2/b2 may be NULL).  Every column reduces at once; the row
// chunks per column shrink as m grows, so that the consumers' fixed-order
// sums over gridDim.x partials stay short.
static __global__ void __launch_bounds__(256) k_dot2(const double* __restrict__ a1, const double* __restrict__ b1,
                                              const double* __restrict__ a2, const double* __restrict__ b2,
                                              int n, int m, double* __restrict__ part) {
    __shared__ double red[2][8];
    const int c = blockIdx.y;
    const int rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * rows_per, i1 = min(n, i0 + rows_per);
    double s1 = 0.0, s2 = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += 256) {
        const long k = (long)c * n + i;
        s1 += a1[k] * b1[k];
        if (a2) s2 += a2[k] * b2[k];
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < 8; ++k) {
            t1 += red[0][k];
            t2 += red[1][k];
        }
        part[((long)blockIdx.x * m + c) * 2 + 0] = t1;
        part[((long)blockIdx.x * m + c) * 2 + 1] = t2;
    }
}

// The G partials of column c (which = 0 or 1) summed by one warp: lane l adds
// partials l, l + 32, ... in order, then a fixed shuffle tree; every lane
// returns lane 0's total, so every CTA that sums them gets the same value.
__device__ __forceinline__ double warp_sum_parts(const double* part, int G, int m, int c, int which, int lane) {
    double s = 0.0;
    for (int g = lane; g < G; g += 32) s += part[((long)g * m + c) * 2 + which];
    s = warp_sum(s);
    return __shfl_sync(0xffffffffu, s, 0);
}

// Per-column CG state (inner loop of Algorithm 2).
struct CgCol {
    double rho[2];    // r^T z, double-buffered by iteration parity
    double alpha;
    double stop;      // stop when ||r_in||_2 <= stop
    double rr;        // latest r^T r
    int done;         // 1 once the column stopped
    int iters;        // inner steps taken in the current outer step
    int total;        // inner steps over all outer steps
    int pad;
};

// alpha_c = rho_c / (p^T q)_c (every CTA computes it identically from the
// partials); e += alpha p; r -= alpha q; with Jacobi z = dinv .* r.
static __global__ void __launch_bounds__(256) k_cg_update(const double* __restrict__ part, int G, int n, int m,
                                                   CgCol* __restrict__ cols, int parity,
                                                   double* __restrict__ E, double* __restrict__ Rr,
                                                   const double* __restrict__ P, const double* __restrict__ Qv,
                                                   const double* __restrict__ dinv, double* __restrict__ Z) {
    __shared__ double s_alpha[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int cb = 0; cb < m; cb += 64) {
        const int cn = min(64, m - cb);
        __syncthreads();
        for (int c = warp; c < cn; c += blockDim.x >> 5) {  // one warp per column
            const double pq = warp_sum_parts(part, G, m, cb + c, 0, lane);
            if (lane == 0) {
                const CgCol& st = cols[cb + c];
                s_alpha[c] = st.done ? 0.0 : st.rho[parity] / pq;
            }
        }
        __syncthreads();
        long total = (long)n * cn;
        for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
            int cl = (int)(e / n), i = (int)(e % n);
            int c = cb + cl;
            double a = s_alpha[cl];
            long k = (long)c * n + i;
            if (a != 0.0) {
                E[k] = fma(a, P[k], E[k]);
                Rr[k] = fma(-a, Qv[k], Rr[k]);
            }
            if (dinv) Z[k] = dinv[i] * Rr[k];
        }
        if (blockIdx.x == 0 && threadIdx.x < cn) cols[cb + threadIdx.x].alpha = s_alpha[threadIdx.x];
    }
}

// rho'_c = (r^T z)_c, rr_c = (r^T r)_c from partials; beta = rho'/rho;
// p = z + beta p, pf = fl32(p); CTA 0 records rho' and the stop test.
static __global__ void __launch_bounds__(256) k_cg_pupdate(const double* __restrict__ part, int G, int n, int m,
                                                    CgCol* __restrict__ cols, int parity, int* __restrict__ active,
                                                    double* __restrict__ P, float* __restrict__ Pf,
                                                    const double* __restrict__ Z) {
    __shared__ double s_beta[64];
    __shared__ int s_done[64];
    __shared__ int s_active;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_active = 0;
    for (int cb = 0; cb < m; cb += 64) {
        const int cn = min(64, m - cb);
        __syncthreads();
        for (int c = warp; c < cn; c += blockDim.x >> 5) {  // one warp per column
            const double rz = warp_sum_parts(part, G, m, cb + c, 0, lane);
            const double rr = warp_sum_parts(part, G, m, cb + c, 1, lane);
            if (lane != 0) continue;
            CgCol st = cols[cb + c];
            bool was_done = st.done;
            bool stop = was_done || (sqrt(rr) <= st.stop);
            s_beta[c] = stop ? 0.0 : rz / st.rho[parity];
            s_done[c] = stop;
            if (blockIdx.x == 0) {
                if (!was_done) {
                    st.iters += 1;
                    st.total += 1;
                    st.rho[parity ^ 1] = rz;
                    st.rr = rr;
                }
                st.done = stop;
                cols[cb + c] = st;
                if (!stop) atomicAdd(&s_active, 1);
            }
        }
        __syncthreads();
        long total = (long)n * cn;
        for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
            int cl = (int)(e / n), i = (int)(e % n);
            if (s_done[cl]) continue;
            long k = (long)(cb + cl) * n + i;
            double p = fma(s_beta[cl], P[k], Z[k]);
            P[k] = p;
            Pf[k] = (float)p;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *active = s_active;
}

// Start of an inner loop: e = 0, r_in = r, z = M r (Jacobi or identity),
// p = z, pf = fl32(p).
static __global__ void k_cg_start(int n, int m, const double* __restrict__ R, long ldr, double* __restrict__ E,
                           double* __restrict__ Rr, double* __restrict__ Z, double* __restrict__ P,
                           float* __restrict__ Pf, const double* __restrict__ dinv, int set_pz) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int c = (int)(e / n), i = (int)(e % n);
        double r = R[(long)c * ldr + i];
        E[e] = 0.0;
        Rr[e] = r;
        double z = dinv ? dinv[i] * r : r;
        if (dinv) Z[e] = z;
        if (set_pz) {
            P[e] = z;
            Pf[e] = (float)z;
        }
    }
}

// p = z, pf = fl32(z) (after a preconditioner applied outside).
static __global__ void k_copy_p(int n, int m, const double* __restrict__ Z, double* __restrict__ P, float* __restrict__ Pf) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        P[e] = Z[e];
        Pf[e] = (float)Z[e];
    }
}

// Initialise the per-column CG state for one inner loop:
// rho[0] = (r^T z), rr = r^T r, stop = max(eta * ||r||_2, target_c).
static __global__ void k_cg_init_cols(const double* __restrict__ part, int G, int m, CgCol* __restrict__ cols,
                               const int* __restrict__ frozen, double eta, const double* __restrict__ target) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < m; c += gridDim.x * wpb) {  // one warp per column
        const double rz = warp_sum_parts(part, G, m, c, 0, lane);
        const double rr = warp_sum_parts(part, G, m, c, 1, lane);
        if (lane != 0) continue;
        CgCol st = cols[c];
        st.rho[0] = rz;
        st.rho[1] = rz;
        st.rr = rr;
        st.stop = fmax(eta * sqrt(rr), target[c]);
        st.iters = 0;
        st.done = (frozen && frozen[c]) || !(sqrt(rr) > st.stop);
        cols[c] = st;
    }
}

// X += E on columns not frozen.
static __global__ void k_add_cols(double* __restrict__ X, long ldx, const double* __restrict__ E, int n, int m,
                           const int* __restrict__ frozen) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int c = (int)(e / n), i = (int)(e % n);
        if (frozen && frozen[c]) continue;
        X[(long)c * ldx + i] += E[e];
    }
}

// target_c for the inner stop: crit ABS2 -> tol, REL2 -> tol * ||b_c||,
// BERR -> tol * ||A||_inf * ||x_c||_inf (a 2-norm proxy of the rule).
static __global__ void k_inner_target(const double* __restrict__ b2, const double* __restrict__ colnorms,
                               const double* __restrict__ anorm, int m, int crit, double tol, int n,
                               double* __restrict__ target) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        double t;
        if (crit == 2) t = tol;
        else if (crit == 1) t = tol * b2[c];
        else t = tol * (*anorm) * fmax(colnorms[3 * c + 2], 1e-300);
        target[c] = t;
    }
}

// dinv_i = 1 / A_ii
static __global__ void k_jacobi_dinv(const double* __restrict__ A, long lda, int n, double* __restrict__ dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / A[(long)i * lda + i];
}

// ---- learned preconditioner (Woodbury form) fused into the inner step -------
// M r = S (Dh^{-1} s - Dh^{-1} Uh Ci Uh^T Dh^{-1} s) with s = S r, Ci the
// inverse of the 32 x 32 core, rows in 256-row chunks x.

// The update of k_cg_update for block (x, c) = rows [256 x, 256 x + 256) of
// column c (alpha from the partials of p^T q), then the chunk's partial
// projection wpart[(x m + c) 32 + k] = sum_i Uh_ik q_i, q = sdg .* r ./ dh:
// warp w takes rows 32 w .. 32 w + 31, lane k column k, the eight warps'
// sums added in warp order.
static __global__ void __launch_bounds__(256) k_cg_update_wb(const double* __restrict__ part, int G2, int n, int m,
                                                      CgCol* __restrict__ cols, int parity, double* __restrict__ E,
                                                      double* __restrict__ Rr, const double* __restrict__ P,
                                                      const double* __restrict__ Qv, const double* __restrict__ sdg,
                                                      const double* __restrict__ dh, const double* __restrict__ Uh,
                                                      double* __restrict__ wpart) {
    static_assert(LOWRANK_RANK == 32, "one lane per column of Uh");
    __shared__ double s_alpha;
    __shared__ double qs[256];
    __shared__ double red[8][LOWRANK_RANK];
    const int c = blockIdx.y, x = blockIdx.x, i0 = 256 * x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {
        const double pq = warp_sum_parts(part, G2, m, c, 0, lane);
        if (lane == 0) {
            const CgCol& st = cols[c];
            s_alpha = st.done ? 0.0 : st.rho[parity] / pq;
        }
    }
    __syncthreads();
    const double a = s_alpha;
    {
        const int i = i0 + threadIdx.x;
        double q = 0.0;
        if (i < n) {
            const long k = (long)c * n + i;
            double r = Rr[k];
            if (a != 0.0) {
                E[k] = fma(a, P[k], E[k]);
                r = fma(-a, Qv[k], r);
                Rr[k] = r;
            }
            q = sdg[i] * r / dh[i];
        }
        qs[threadIdx.x] = q;
    }
    __syncthreads();
    double u[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = i0 + 32 * w + r;
        u[r] = i < n ? Uh[(long)i * LOWRANK_RANK + lane] : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < 32; ++r) acc = fma(u[r], qs[32 * w + r], acc);
    red[w][lane] = acc;
    __syncthreads();
    if (threadIdx.x < LOWRANK_RANK) {
        double s = 0.0;
#pragma unroll
        for (int wv = 0; wv < 8; ++wv) s += red[wv][threadIdx.x];
        wpart[((long)x * m + c) * LOWRANK_RANK + threadIdx.x] = s;
    }
    if (x == 0 && threadIdx.x == 0) cols[c].alpha = a;
}

// The apply for block (x, c): w = column c's G partial projections (chunk
// order within eight groups, then group order), y = Ci w, z_i = s_i (q_i -
// (Uh_i . y) / dh_i) for the chunk's rows, and the chunk's partials of r^T z
// and r^T r into dpart[(x m + c) 2 + {0, 1}] (the layout k_cg_pupdate reads).
static __global__ void __launch_bounds__(256) k_wb_apply_dot(const double* __restrict__ Rr, const double* __restrict__ sdg,
                                                      const double* __restrict__ dh, const double* __restrict__ Uh,
                                                      const double* __restrict__ Lc, const double* __restrict__ wpart,
                                                      int G, int n, int m, double* __restrict__ Z,
                                                      double* __restrict__ dpart) {
    __shared__ double red[8][LOWRANK_RANK];
    __shared__ double ws[LOWRANK_RANK], ys[LOWRANK_RANK];
    __shared__ double rd[2][8];
    const int c = blockIdx.y, x = blockIdx.x, k = threadIdx.x & 31, g = threadIdx.x >> 5;
    {
        double s = 0.0;
        for (int xx = g; xx < G; xx += 8) s += wpart[((long)xx * m + c) * LOWRANK_RANK + k];
        red[g][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < LOWRANK_RANK) {
        double s = 0.0;
#pragma unroll
        for (int gv = 0; gv < 8; ++gv) s += red[gv][threadIdx.x];
        ws[threadIdx.x] = s;
    }
    __syncthreads();
    {   // y_k = sum_j Ci[k][j] w_j: group g takes j = 4 g .. 4 g + 3
        const double* ci = Lc + LOWRANK_RANK * LOWRANK_RANK + k * LOWRANK_RANK + 4 * g;
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) y = fma(ci[j], ws[4 * g + j], y);
        red[g][k] = y;
    }
    __syncthreads();
    if (threadIdx.x < LOWRANK_RANK) {
        double y = 0.0;
#pragma unroll
        for (int gv = 0; gv < 8; ++gv) y += red[gv][threadIdx.x];
        ys[threadIdx.x] = y;
    }
    __syncthreads();
    const int i = 256 * x + threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    if (i < n) {
        const long kk = (long)c * n + i;
        const double r = Rr[kk];
        const double q = sdg[i] * r / dh[i];
        double u = 0.0;
#pragma unroll
        for (int j = 0; j < LOWRANK_RANK; ++j) u = fma(Uh[(long)i * LOWRANK_RANK + j], ys[j], u);
        const double z = sdg[i] * (q - u / dh[i]);
        Z[kk] = z;
        s1 = r * z;
        s2 = r * r;
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) {
        rd[0][threadIdx.x >> 5] = s1;
        rd[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int q = 0; q < 8; ++q) {
            t1 += rd[0][q];
            t2 += rd[1][q];
        }
        dpart[((long)x * m + c) * 2 + 0] = t1;
        dpart[((long)x * m + c) * 2 + 1] = t2;
    }
}
