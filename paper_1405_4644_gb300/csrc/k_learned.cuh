// k_learned.cuh -- the learned diagonal-plus-low-rank preconditioner for
// PCG: per-row features (K12), a 3-layer MLP forward/backward with Adam
// (K13), and the preconditioner M = S (Dh + Uh Uh^T)^{-1} S applied through
// the Woodbury identity (K14), S = diag(A)^{-1/2}.
#pragma once
#include "common.cuh"

#define LR_RANK 32
#define LR_FEAT 16

// ---- K12: per-row features ----------------------------------------------
// f[i] = [x, y, log ell, log nugget, sin/cos(pi x), sin/cos(pi y),
//         sin/cos(2 pi x), sin/cos(2 pi y), mean |Ah_i,:|, rms Ah_i,:,
//         max_{j != i} |Ah_ij|, 1], Ah = S A S.  One warp per row.
// sdiag (s_i = A_ii^{-1/2}) must be filled before the launch.
static __global__ void k_features(const double* __restrict__ A, long lda, int n, const double* __restrict__ coords,
                                  double ell, double nugget, float* __restrict__ F, const double* __restrict__ sdiag) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i >= n) return;
    const double si = sdiag[i];
    double s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int j = lane; j < n; j += 32) {  // row i read as column i (symmetric): coalesced
        const double v = fabs(A[(long)i * lda + j] * si * sdiag[j]);
        s1 += v;
        s2 += v * v;
        if (j != i) mx = fmax(mx, v);
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    mx = warp_max(mx);
    if (lane == 0) {
        const double x = coords[2 * i], y = coords[2 * i + 1];
        const double pi = 3.14159265358979323846;
        float* f = F + (long)i * LR_FEAT;
        f[0] = (float)x;
        f[1] = (float)y;
        f[2] = (float)log(ell);
        f[3] = (float)log(nugget);
        f[4] = (float)sin(pi * x);
        f[5] = (float)cos(pi * x);
        f[6] = (float)sin(pi * y);
        f[7] = (float)cos(pi * y);
        f[8] = (float)sin(2 * pi * x);
        f[9] = (float)cos(2 * pi * x);
        f[10] = (float)sin(2 * pi * y);
        f[11] = (float)cos(2 * pi * y);
        f[12] = (float)(s1 / n);
        f[13] = (float)sqrt(s2 / n);
        f[14] = (float)mx;
        f[15] = 1.0f;
    }
}

// ---- K13: dense layers --------------------------------------------------
// Generic strided SIMT GEMM: C[m][n] = alpha * sum_k A(m,k) B(k,n) + beta C
// with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]; optional bf16
// rounding of both operands (mixed-precision training).  64x64 tiles.
static __global__ void __launch_bounds__(256) k_gemm_strided(int M, int N, int K, const float* __restrict__ A,
                                                             long sam, long sak, const float* __restrict__ B,
                                                             long sbk, long sbn, float* __restrict__ C, long ldc,
                                                             float alpha, float beta, int bf16) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int gm = m0 + mm, gk = k0 + kk;
            float va = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.f;
            const int gn = n0 + mm;
            float vb = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : 0.f;
            if (bf16) {
                va = __bfloat162float(__float2bfloat16_rn(va));
                vb = __bfloat162float(__float2bfloat16_rn(vb));
            }
            As[kk][mm] = va;
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gm = m0 + ty * 4 + p, gn = n0 + tx * 4 + q;
            if (gm < M && gn < N) {
                float* c = C + (long)gm * ldc + gn;
                *c = alpha * acc[p][q] + (beta != 0.f ? beta * *c : 0.f);
            }
        }
}

__device__ __forceinline__ float silu(float x) { return x / (1.f + __expf(-x)); }
__device__ __forceinline__ float silu_grad(float x) {
    const float s = 1.f / (1.f + __expf(-x));
    return s * (1.f + x * (1.f - s));
}

// Z (pre-activation, rows x N) += bias; H = silu(Z) (act = 1) or Z, optionally
// rounded to bf16.  H may be Z (the output layer works in place), so neither
// is restrict-qualified.
static __global__ void k_bias_act(float* Z, const float* __restrict__ b, float* H, int rows, int N, int act,
                                  int bf16) {
    long total = (long)rows * N;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int c = (int)(e % N);
        float z = Z[e] + b[c];
        Z[e] = z;
        float h = act ? silu(z) : z;
        if (bf16) h = __bfloat162float(__float2bfloat16_rn(h));
        H[e] = h;
    }
}

// dZ = dH * silu'(Z)
static __global__ void k_act_back(const float* __restrict__ Z, float* __restrict__ dH, long total) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x)
        dH[e] *= silu_grad(Z[e]);
}

// db[c] = sum_r dZ[r][c]  (one thread per column, fixed order)
static __global__ void k_colsum(const float* __restrict__ dZ, int rows, int N, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dZ[(long)r * N + c];
    db[c] = s;
}

// Adam on a flat parameter vector (float32 master weights)
static __global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                              float* __restrict__ m2, long count, float lr, float b1, float b2, float eps, float c1,
                              float c2) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < count; e += (long)gridDim.x * blockDim.x) {
        const float gr = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gr;
        const float b = b2 * m2[e] + (1.f - b2) * gr * gr;
        m1[e] = a;
        m2[e] = b;
        p[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// ---- K14: preconditioner from the network output -------------------------
// O (n x 33): dh_i = softplus(O_i0) + 1e-3, Uh_ik = O_i,1+k.
static __global__ void k_out_to_dU(const float* __restrict__ O, int n, double* __restrict__ dh, double* __restrict__ Uh) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float* o = O + (long)i * (1 + LR_RANK);
        const float z = o[0];
        dh[i] = (double)((z > 20.f ? z : log1pf(__expf(z))) + 1e-3f);
        for (int k = 0; k < LR_RANK; ++k) Uh[(long)i * LR_RANK + k] = (double)o[1 + k];
    }
}

// Cc = I + Uh^T Dh^{-1} Uh (32 x 32, float64), then its Cholesky factor Lc
// (lower, row-major) -- one CTA of 1024 threads: thread (a, b) sums over n.
// Writes Lc (the core's Cholesky factor, row-major) and, after it, Ci = the
// core's inverse Lc^{-T} Lc^{-1} (the Woodbury apply multiplies by it).
// The core's Gram term over row chunks: block x (1024 threads) stages rows
// [CORE_ROWS x, CORE_ROWS (x + 1)) of Uh and 1/dh in shared memory; thread
// (a, b) writes part[x][a][b] = sum over the chunk's rows, in row order, of
// Uh_ia Uh_ib (1/dh_i).
#define CORE_ROWS 128
static __global__ void __launch_bounds__(1024) k_core_gram(const double* __restrict__ dh, const double* __restrict__ Uh,
                                                           int n, double* __restrict__ part) {
    __shared__ double Us[CORE_ROWS][LR_RANK];
    __shared__ double rd[CORE_ROWS];
    const int i0 = blockIdx.x * CORE_ROWS, rows = min(CORE_ROWS, n - i0);
    for (int e = threadIdx.x; e < CORE_ROWS * LR_RANK; e += 1024) {
        const int r = e / LR_RANK, k = e % LR_RANK;
        Us[r][k] = r < rows ? Uh[(long)(i0 + r) * LR_RANK + k] : 0.0;
    }
    if (threadIdx.x < CORE_ROWS) rd[threadIdx.x] = threadIdx.x < rows ? 1.0 / dh[i0 + threadIdx.x] : 0.0;
    __syncthreads();
    const int a = threadIdx.x / LR_RANK, b = threadIdx.x % LR_RANK;
    double s = 0.0;
#pragma unroll 8
    for (int r = 0; r < CORE_ROWS; ++r) s = fma(Us[r][a] * Us[r][b], rd[r], s);
    part[(long)blockIdx.x * LR_RANK * LR_RANK + threadIdx.x] = s;
}

// Cc = I + the G chunk partials (in chunk order), then its Cholesky factor Lc
// and the inverse Ci = Lc^{-T} Lc^{-1}.
static __global__ void __launch_bounds__(1024) k_core_chol(const double* __restrict__ part, int G,
                                                           double* __restrict__ Lc, int* __restrict__ bad) {
    __shared__ double Cs[LR_RANK][LR_RANK + 1];
    __shared__ double Li[LR_RANK][LR_RANK + 1];
    const int a = threadIdx.x / LR_RANK, b = threadIdx.x % LR_RANK;
    double s = (a == b) ? 1.0 : 0.0;
    for (int x = 0; x < G; ++x) s += part[(long)x * LR_RANK * LR_RANK + threadIdx.x];
    Cs[a][b] = s;
    __syncthreads();
    if (threadIdx.x < 32) {  // warp 0: Cholesky of Cs in place, lane = row
        const int r = threadIdx.x;
        for (int j = 0; j < LR_RANK; ++j) {
            if (r == j) {
                double v = Cs[j][j];
                for (int k = 0; k < j; ++k) v -= Cs[j][k] * Cs[j][k];
                if (!(v > 0.0)) {
                    *bad = 1;
                    v = 1.0;
                }
                Cs[j][j] = sqrt(v);
            }
            __syncwarp();
            if (r > j) {
                double v = Cs[r][j];
                for (int k = 0; k < j; ++k) v -= Cs[r][k] * Cs[j][k];
                Cs[r][j] = v / Cs[j][j];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    Lc[a * LR_RANK + b] = (b <= a) ? Cs[a][b] : 0.0;
    if (threadIdx.x < 32) {  // lane b: column b of Lc^{-1} by forward substitution
        const int bb = threadIdx.x;
        for (int r = 0; r < LR_RANK; ++r) {
            double v = (r == bb) ? 1.0 : 0.0;
            for (int k = bb; k < r; ++k) v -= Cs[r][k] * Li[k][bb];
            Li[r][bb] = (r >= bb) ? v / Cs[r][r] : 0.0;
        }
    }
    __syncthreads();
    double ci = 0.0;
    for (int k = max(a, b); k < LR_RANK; ++k) ci += Li[k][a] * Li[k][b];
    Lc[LR_RANK * LR_RANK + a * LR_RANK + b] = ci;
}

// Woodbury apply, p columns (float64, n x p, ld n):
// out = s .* (q - Dh^{-1} Uh Cc^{-1} Uh^T q),  q = Dh^{-1} (s .* r)
// step 1 (k_wb_proj): partial projections, block (x, c) over rows
// [256 x, 256 x + 256): wpart[(x p + c) R + k] = sum_i Uh_ik q_i.  Warp w
// takes rows 32 w .. 32 w + 31 of the chunk, lane k column k (each row of Uh
// one coalesced 256-byte load across the warp); the eight warps' sums are
// added in warp order.
static __global__ void __launch_bounds__(256) k_wb_proj(const double* __restrict__ R, long ldr, const double* __restrict__ sdg,
                                                        const double* __restrict__ dh, const double* __restrict__ Uh, int n,
                                                        int p, double* __restrict__ wpart) {
    static_assert(LR_RANK == 32, "one lane per column of Uh");
    __shared__ double qs[256];
    __shared__ double red[8][LR_RANK];
    const int c = blockIdx.y, i0 = blockIdx.x * 256, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        const int i = i0 + threadIdx.x;
        qs[threadIdx.x] = i < n ? sdg[i] * R[(long)c * ldr + i] / dh[i] : 0.0;
    }
    __syncthreads();
    double u[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = i0 + 32 * w + r;
        u[r] = i < n ? Uh[(long)i * LR_RANK + lane] : 0.0;
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < 32; ++r) acc = fma(u[r], qs[32 * w + r], acc);
    red[w][lane] = acc;
    __syncthreads();
    if (threadIdx.x < LR_RANK) {
        double s = 0.0;
#pragma unroll
        for (int wv = 0; wv < 8; ++wv) s += red[wv][threadIdx.x];
        wpart[((long)blockIdx.x * p + c) * LR_RANK + threadIdx.x] = s;
    }
}

// step 2: w = the G partials (in chunk order within each of eight groups,
// then group order), y = Ci w (Ci = Cc^{-1}, after Lc), then
// out_i = s_i (q_i - (Uh_i . y) / dh_i).  Every CTA forms w and y itself
// with all 256 threads: thread (g, k) = (tid / 32, tid % 32).
static __global__ void __launch_bounds__(256) k_wb_apply(const double* __restrict__ R, long ldr, const double* __restrict__ sdg,
                                                         const double* __restrict__ dh, const double* __restrict__ Uh,
                                                         const double* __restrict__ Lc, const double* __restrict__ wpart,
                                                         int G, int n, int p, double* __restrict__ out, long ldo) {
    __shared__ double red[8][LR_RANK];
    __shared__ double ws[LR_RANK], ys[LR_RANK];
    const int c = blockIdx.y, k = threadIdx.x & 31, g = threadIdx.x >> 5;
    {
        double s = 0.0;
        for (int x = g; x < G; x += 8) s += wpart[((long)x * p + c) * LR_RANK + k];
        red[g][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < LR_RANK) {
        double s = 0.0;
#pragma unroll
        for (int gv = 0; gv < 8; ++gv) s += red[gv][threadIdx.x];
        ws[threadIdx.x] = s;
    }
    __syncthreads();
    {   // y_k = sum_j Ci[k][j] w_j: group g takes j = 4 g .. 4 g + 3
        const double* ci = Lc + LR_RANK * LR_RANK + k * LR_RANK + 4 * g;
        double y = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) y = fma(ci[j], ws[4 * g + j], y);
        red[g][k] = y;
    }
    __syncthreads();
    if (threadIdx.x < LR_RANK) {
        double y = 0.0;
#pragma unroll
        for (int gv = 0; gv < 8; ++gv) y += red[gv][threadIdx.x];
        ys[threadIdx.x] = y;
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double q = sdg[i] * R[(long)c * ldr + i] / dh[i];
        double u = 0.0;
#pragma unroll
        for (int kk = 0; kk < LR_RANK; ++kk) u = fma(Uh[(long)i * LR_RANK + kk], ys[kk], u);
        out[(long)c * ldo + i] = sdg[i] * (q - u / dh[i]);
    }
}

// ---- gradient of the probe loss with respect to (dh, Uh) -------------------
// With yh = Mh sh (sh = s .* z), wh = Mh gh (gh = s .* g):
//   dL/ddh_i = -sum_c wh_ic yh_ic,
//   dL/dUh_ik = -sum_c (wh_ic (Uh^T yh)_kc + yh_ic (Uh^T wh)_kc).
// Yh/Wh are the unscaled Woodbury outputs (out / s); PY = Uh^T yh, PW = Uh^T wh.
// Writes dO (n x 33) including the softplus chain rule for column 0.
static __global__ void k_loss_grad_out(const double* __restrict__ Yh, const double* __restrict__ Wh, int n, int p,
                                       const double* __restrict__ Uh, const double* __restrict__ PY,
                                       const double* __restrict__ PW, const float* __restrict__ O, float* __restrict__ dO) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double gd = 0.0;
        double gu[LR_RANK];
#pragma unroll
        for (int k = 0; k < LR_RANK; ++k) gu[k] = 0.0;
        for (int c = 0; c < p; ++c) {
            const double y = Yh[(long)c * n + i], w = Wh[(long)c * n + i];
            gd -= w * y;
#pragma unroll
            for (int k = 0; k < LR_RANK; ++k) gu[k] -= w * PY[c * LR_RANK + k] + y * PW[c * LR_RANK + k];
        }
        const float z = O[(long)i * (1 + LR_RANK)];
        const float sg = 1.f / (1.f + __expf(-z));  // softplus'
        float* d = dO + (long)i * (1 + LR_RANK);
        d[0] = (float)(gd * sg);
#pragma unroll
        for (int k = 0; k < LR_RANK; ++k) d[1 + k] = (float)gu[k];
    }
}
