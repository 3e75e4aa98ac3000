// k_lanczos.cuh -- a lower bound on the 2-norm condition number of the
// scaled matrix As = D A D, taken before any factor, for the AUTO choice of
// the factor precision (eq. (iterref): the refinement converges only while
// kappa u_f stays below one).
//
// k steps of Lanczos with full reorthogonalisation on As give the tridiagonal
// T_k = Q_k^T As Q_k; its eigenvalues (Ritz values) lie in [lambda_min,
// lambda_max] of As (Cauchy interlacing for an orthonormal Q_k), so
// theta_max / theta_min <= kappa_2(As) up to the float32 rounding of the
// products.  The bound can only rule a precision out, never in.
//
// Kernels (As from the float32 scaled lower triangle the factorisation has
// just written; Lanczos vectors float32, every reduction in float64 and in a
// fixed order, so the result does not depend on scheduling):
//   k_lz_symv_tiles   partials of y = As x over 128 x 128 tiles of the lower
//                     triangle, each tile read once: P[I][J] = W_IJ x_J and,
//                     below the diagonal, P[J][I] = W_IJ^T x_I
//   k_lz_symv_reduce  y_I = sum_J P[I][J] in J order
//   k_lz_dots         partial dot products Q_i . y over row chunks
//   k_lz_orth         h_i from the partials, y -= sum_i h_i Q_i, partial ||y||^2
//   k_lz_normalize    beta = ||y||, Q_{j+1} = y / beta; alpha_j = h_j, beta_j
#pragma once
#include "common.cuh"

#define LZ_T 128        // tile order of the symmetric product
#define LZ_CHUNKS 64    // row chunks of the vector reductions
#define LZ_MAXK 16      // Lanczos steps at most

// tile t of the lower triangle, row-major over (I, J <= I)
__device__ __forceinline__ void lz_tile(long t, int& I, int& J) {
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long)(i + 1) * (i + 2) / 2 <= t) ++i;
    while ((long)i * (i + 1) / 2 > t) --i;
    I = i;
    J = (int)(t - (long)i * (i + 1) / 2);
}

// The sixteen row sums of a warp (v[k]: this lane's part of row k) with 16
// shuffles instead of 5 per row: at each step a lane keeps half of its
// values, sends the other half to the partner (lane ^ 16, 8, 4, 2) and adds
// what it receives; lane L ends with the total of row (L >> 1) & 15 (the
// same in both lanes of a pair: the last addition is commutative).
__device__ __forceinline__ float lz_reduce16(const float (&v)[16], int lane) {
    float a8[8], a4[4], a2[2];
    {
        const bool b = (lane >> 4) & 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float s = b ? v[i] : v[i + 8], k = b ? v[i + 8] : v[i];
            a8[i] = k + __shfl_xor_sync(0xffffffffu, s, 16);
        }
    }
    {
        const bool b = (lane >> 3) & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float s = b ? a8[i] : a8[i + 4], k = b ? a8[i + 4] : a8[i];
            a4[i] = k + __shfl_xor_sync(0xffffffffu, s, 8);
        }
    }
    {
        const bool b = (lane >> 2) & 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float s = b ? a4[i] : a4[i + 2], k = b ? a4[i + 2] : a4[i];
            a2[i] = k + __shfl_xor_sync(0xffffffffu, s, 4);
        }
    }
    const bool b = (lane >> 1) & 1;
    const float s = b ? a2[0] : a2[1], k = b ? a2[1] : a2[0];
    const float a1 = k + __shfl_xor_sync(0xffffffffu, s, 2);
    return a1 + __shfl_xor_sync(0xffffffffu, a1, 1);
}

// 256 threads: warp w takes rows w, w + 8, .. of the tile (16 rows), lane l
// the four columns 4l .. 4l + 3.  Entries outside the matrix (c >= n, r >= n)
// and above the diagonal are masked, never read as data: the factor's
// padding columns hold no values.  Interior tiles below the diagonal (every
// row and column inside the matrix) take a path without masks.
__global__ void __launch_bounds__(256, 3) k_lz_symv_tiles(const float* __restrict__ W, long ldw, int n, int nb,
                                                     const float* __restrict__ x, float* __restrict__ P) {
    __shared__ float xs_i[LZ_T];
    __shared__ float ps[LZ_T];
    __shared__ float qs[8][LZ_T];
    int I, J;
    lz_tile(blockIdx.x, I, J);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = I * LZ_T, c0 = J * LZ_T;
    if (tid < LZ_T) xs_i[tid] = (r0 + tid < n) ? x[r0 + tid] : 0.f;
    const int c4 = c0 + 4 * lane;
    float xj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xj[q] = (c4 + q < n) ? x[c4 + q] : 0.f;
    __syncthreads();
    const bool diag = (I == J);
    float4 w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int r = r0 + warp + 8 * k;
        // c4 < n keeps the float4 inside the row's ldw (a multiple of 64 >= n)
        w[k] = (r < n && c4 < n) ? *reinterpret_cast<const float4*>(W + (long)r * ldw + c4)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float qa[4] = {0.f, 0.f, 0.f, 0.f};
    float pk[16];
    if (!diag && r0 + LZ_T <= n && c0 + LZ_T <= n) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float xi = xs_i[warp + 8 * k];
            pk[k] = fmaf(w[k].x, xj[0], fmaf(w[k].y, xj[1], fmaf(w[k].z, xj[2], w[k].w * xj[3])));
            qa[0] = fmaf(w[k].x, xi, qa[0]);
            qa[1] = fmaf(w[k].y, xi, qa[1]);
            qa[2] = fmaf(w[k].z, xi, qa[2]);
            qa[3] = fmaf(w[k].w, xi, qa[3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int rl = warp + 8 * k, r = r0 + rl;
            float v[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
            float p = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c4 + q;
                const bool in = (c < n) && (!diag || c <= r);  // r >= n rows were loaded as zeros
                const float a = in ? v[q] : 0.f;
                p = fmaf(a, xj[q], p);
                // the transposed part: strictly below the diagonal only
                const float at = (diag && c == r) ? 0.f : a;
                qa[q] = fmaf(at, xs_i[rl], qa[q]);
            }
            pk[k] = p;
        }
    }
    {
        const float p = lz_reduce16(pk, lane);
        if ((lane & 1) == 0) ps[warp + 8 * ((lane >> 1) & 15)] = p;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) qs[warp][4 * lane + q] = qa[q];
    __syncthreads();
    if (tid < LZ_T) {
        float q = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) q += qs[w8][tid];
        if (diag) {
            P[((long)I * nb + I) * LZ_T + tid] = ps[tid] + q;
        } else {
            P[((long)I * nb + J) * LZ_T + tid] = ps[tid];
            P[((long)J * nb + I) * LZ_T + tid] = q;
        }
    }
}

// y[I*128 + t] = sum_J P[I][J][t]: one CTA of 128 x 8 per I, thread (t, w)
// sums J = w, w + 8, .. (several loads in flight), then the eight partials
// are added in w order
__global__ void __launch_bounds__(LZ_T * 8) k_lz_symv_reduce(const float* __restrict__ P, int n, int nb,
                                                           float* __restrict__ y) {
    __shared__ double part[8][LZ_T];
    const int I = blockIdx.x, t = threadIdx.x, w = threadIdx.y;
    const float* row = P + (long)I * nb * LZ_T + t;
    double s = 0.0;
#pragma unroll 4
    for (int J = w; J < nb; J += 8) s += (double)row[(long)J * LZ_T];
    part[w][t] = s;
    __syncthreads();
    if (w == 0) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) a += part[q][t];
        if (I * LZ_T + t < n) y[I * LZ_T + t] = (float)a;
    }
}

__device__ __forceinline__ void lz_chunk(int n, int g, int& lo, int& hi) {
    const int len = (n + LZ_CHUNKS - 1) / LZ_CHUNKS;
    lo = min(n, g * len);
    hi = min(n, lo + len);
}

__device__ __forceinline__ double lz_block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// grid (LZ_CHUNKS, j + 1), 256 threads: dpart[i][g] = Q_i . y over chunk g
__global__ void __launch_bounds__(256) k_lz_dots(const float* __restrict__ Q, long ldq, const float* __restrict__ y,
                                               int n, double* __restrict__ dpart) {
    __shared__ double red[8];
    const int g = blockIdx.x, i = blockIdx.y;
    int lo, hi;
    lz_chunk(n, g, lo, hi);
    double s = 0.0;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) s += (double)Q[(long)i * ldq + r] * (double)y[r];
    s = lz_block_sum(s, red);
    if (threadIdx.x == 0) dpart[i * LZ_CHUNKS + g] = s;
}

// grid LZ_CHUNKS, 256 threads: h_i = sum_g dpart[i][g] (i <= j, g ascending),
// y -= sum_i h_i Q_i on chunk g, npart[g] = ||y||^2 on chunk g; chunk 0
// stores alpha_j = h_j.  j = -1: no projection (the start vector).
__global__ void __launch_bounds__(256) k_lz_orth(const float* __restrict__ Q, long ldq, float* __restrict__ y, int n,
                                               int j, const double* __restrict__ dpart, double* __restrict__ npart,
                                               double* __restrict__ alpha) {
    __shared__ double h[LZ_MAXK + 1];
    __shared__ double red[8];
    const int g = blockIdx.x;
    if ((int)threadIdx.x <= j) {
        double s = 0.0;
        for (int q = 0; q < LZ_CHUNKS; ++q) s += dpart[threadIdx.x * LZ_CHUNKS + q];
        h[threadIdx.x] = s;
    }
    __syncthreads();
    if (g == 0 && threadIdx.x == 0 && j >= 0) alpha[j] = h[j];
    int lo, hi;
    lz_chunk(n, g, lo, hi);
    double s2 = 0.0;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        double v = (double)y[r];
        for (int i = 0; i <= j; ++i) v -= h[i] * (double)Q[(long)i * ldq + r];
        const float f = (float)v;
        y[r] = f;
        s2 += (double)f * (double)f;
    }
    s2 = lz_block_sum(s2, red);
    if (threadIdx.x == 0) npart[g] = s2;
}

// grid LZ_CHUNKS: beta = sqrt(sum_g npart[g]); Q_{j+1} = y / beta on chunk g
// (zero when beta vanishes: an invariant subspace, which the host sees in
// beta_j); chunk 0 stores beta_j (j = -1: the start vector, not stored).
__global__ void __launch_bounds__(256) k_lz_normalize(const float* __restrict__ y, float* __restrict__ qn, int n, int j,
                                                    const double* __restrict__ npart, double* __restrict__ beta) {
    double s = 0.0;
    for (int q = 0; q < LZ_CHUNKS; ++q) s += npart[q];
    const double b = sqrt(s);
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && j >= 0) beta[j] = b;
    int lo, hi;
    lz_chunk(n, blockIdx.x, lo, hi);
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) qn[r] = (float)((double)y[r] * inv);
}

// start vector: entries in [-1, 1) from a 32-bit integer hash of the index
// (a fixed, seedless choice: any vector with components along the extreme
// eigenvectors serves)
__global__ void k_lz_start(float* __restrict__ y, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    unsigned v = (unsigned)r * 0x9E3779B1u + 0x7F4A7C15u;
    v ^= v >> 16;
    v *= 0x85EBCA6Bu;
    v ^= v >> 13;
    v *= 0xC2B2AE35u;
    v ^= v >> 16;
    y[r] = (float)((double)v * 0x1p-31 - 1.0);
}
