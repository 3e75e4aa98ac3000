// k_leaf32.cuh -- float32 leaves of the low-precision factorisation (steps
// A1/A2 of Section 3.1's Cholesky), built around the full inverse of each
// 128x128 diagonal block:
//
//   k_potrf_leaf32  factors W[k:k+nb, k:k+nb] = L L^T (four 32x32 sub-steps,
//                   warp-level pivots) and forms X = L^{-1} by block rows,
//                   X_i = I_ii (E_i - sum_{j<i} L_ij X_j), I_ii the 32x32
//                   inverses; stores L (and its operand mirror) and X^T.
//   k_trsm_leaf32   panel solve X L^T = B as the product B (L^{-1})^T, one
//                   register-tiled 64 x 128 block of rows per CTA.
//
// The float64 baseline keeps the sub-block kernels of k_leaf.cuh.
#pragma once
#include "common.cuh"

#define LD32 129

constexpr size_t potrf_leaf32_smem() { return (size_t)(2 * 128 * LD32 + 96 * 33) * sizeof(float); }

// Linv_T for block b lives at LinvT + b * 128 * 128, row-major:
// LinvT[l][c] = (L^{-1})[c][l]  (upper triangular).
__global__ void __launch_bounds__(256, 1) k_potrf_leaf32(float* __restrict__ W, long ldw, int k, int nb,
                                                      float* __restrict__ LinvT, Mirror mir, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* S = reinterpret_cast<float*>(smem_raw);  // [128][129] the block, then L
    float* X = S + 128 * LD32;                      // [128][129] L^{-1}
    float* Tmp = X + 128 * LD32;                    // [96][33] or [32][97] scratch
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;

    if (nb == 128) {
        // 16 float4 per thread, all loads in flight before the stores
        float4 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            v[q] = *reinterpret_cast<const float4*>(W + (long)(k + r) * ldw + k + c4);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            float* d = S + r * LD32 + c4;
            d[0] = (c4 + 0 <= r) ? v[q].x : 0.f;
            d[1] = (c4 + 1 <= r) ? v[q].y : 0.f;
            d[2] = (c4 + 2 <= r) ? v[q].z : 0.f;
            d[3] = (c4 + 3 <= r) ? v[q].w : 0.f;
        }
    } else {
        for (int e = tid; e < 128 * 128; e += 256) {
            int r = e >> 7, c = e & 127;
            float v;
            if (r < nb && c < nb) v = (c <= r) ? W[(long)(k + r) * ldw + k + c] : 0.f;
            else v = (r == c) ? 1.f : 0.f;
            S[r * LD32 + c] = v;
        }
    }
    for (int e = tid; e < 128 * 128; e += 256) X[(e >> 7) * LD32 + (e & 127)] = 0.f;
    if (tid == 0) s_bad = 0;
    __syncthreads();

    for (int J = 0; J < 4; ++J) {
        const int o = J * 32;
        if (warp == 0) {
            float a[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) a[c] = S[(o + lane) * LD32 + o + c];
            int badj = -1;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float piv = __shfl_sync(0xffffffffu, a[j], j);
                if (!(piv > 0.f)) {
                    if (badj < 0) badj = j;
                    piv = 1.f;
                }
                const float dj = sqrtf(piv);
                const float inv = 1.f / dj;
                a[j] = (lane == j) ? dj : (lane > j ? a[j] * inv : a[j]);
#pragma unroll
                for (int l = 0; l < 32; ++l) {  // constant bounds: fully unrolled, a[] stays in registers
                    if (l > j) {
                        const float t = __shfl_sync(0xffffffffu, a[j], l);
                        a[l] = (lane >= l) ? fmaf(-a[j], t, a[l]) : a[l];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) S[(o + lane) * LD32 + o + c] = (c <= lane) ? a[c] : 0.f;
            if (badj >= 0 && lane == 0 && o + badj < nb) {
                s_bad = 1;
                atomicMin(&st->info, k + o + badj + 1);
                dev_raise(st, SPD_DEV_BREAKDOWN);
            }
            __syncwarp();
            // lane c: column c of the 32x32 inverse, by forward substitution;
            // row i of L is broadcast from shared memory
            float x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float* li = S + (o + i) * LD32 + o;
                float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
                for (int l = 0; l < 32; ++l)
                    if (l < i) s = fmaf(-li[l], x[l], s);
                x[i] = s / li[i];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) X[(o + i) * LD32 + o + lane] = x[i];
        }
        __syncthreads();
        if (s_bad) return;
        const int rows = 128 - (o + 32);
        if (rows == 0) break;
        // sub-panel below: L_iJ = A_iJ I_JJ^T, 4 outputs per thread-iteration
        for (int e = tid; e < rows * 8; e += 256) {
            const int i = e >> 3, c4 = (e & 7) * 4;
            const float* brow = S + (o + 32 + i) * LD32 + o;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (int l = 0; l <= c4 + 3; ++l) {
                const float b = brow[l];
                s0 += b * X[(o + c4 + 0) * LD32 + o + l];
                s1 += b * X[(o + c4 + 1) * LD32 + o + l];
                s2 += b * X[(o + c4 + 2) * LD32 + o + l];
                s3 += b * X[(o + c4 + 3) * LD32 + o + l];
            }
            float* t = Tmp + i * 33 + c4;
            t[0] = s0;
            t[1] = s1;
            t[2] = s2;
            t[3] = s3;
        }
        __syncthreads();
        for (int e = tid; e < rows * 32; e += 256) {
            const int i = e >> 5, c = e & 31;
            S[(o + 32 + i) * LD32 + o + c] = Tmp[i * 33 + c];
        }
        __syncthreads();
        // trailing update of the rest of the leaf: 2x2 outputs per thread-iteration
        const int base = o + 32;
        const int hr = rows >> 1;
        for (int e = tid; e < hr * hr; e += 256) {
            const int bi = e / hr, bj = e - bi * hr;
            if (bj > bi) continue;
            const int i = base + 2 * bi, j = base + 2 * bj;
            const float* r0 = S + i * LD32 + o;
            const float* r1 = r0 + LD32;
            const float* q0 = S + j * LD32 + o;
            const float* q1 = q0 + LD32;
            float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const float a0 = r0[l], a1 = r1[l], b0 = q0[l], b1 = q1[l];
                s00 += a0 * b0;
                s01 += a0 * b1;
                s10 += a1 * b0;
                s11 += a1 * b1;
            }
            S[i * LD32 + j] -= s00;
            S[(i + 1) * LD32 + j] -= s10;
            S[(i + 1) * LD32 + j + 1] -= s11;
            if (j + 1 <= i) S[i * LD32 + j + 1] -= s01;
        }
        __syncthreads();
    }
    // off-diagonal blocks of X = L^{-1}, block row by block row:
    // T = L_i,0:i X_0:i,0:i  (into Tmp as [32][97]), then X_i,0:i = -I_ii T
    for (int i = 1; i < 4; ++i) {
        const int ri = i * 32, w = i * 32;  // rows ri..ri+31 of X, columns 0..w-1
        for (int e = tid; e < 32 * w; e += 256) {
            const int r = e / w, c = e - r * w;
            const float* lr = S + (ri + r) * LD32;
            float s = 0.f;
            for (int l = (c >> 5) << 5; l < ri; ++l) s += lr[l] * X[l * LD32 + c];
            Tmp[r * 97 + c] = s;
        }
        __syncthreads();
        for (int e = tid; e < 32 * w; e += 256) {
            const int r = e / w, c = e - r * w;
            const float* ir = X + (ri + r) * LD32 + ri;
            float s = 0.f;
            for (int l = 0; l <= r; ++l) s += ir[l] * Tmp[l * 97 + c];
            X[(ri + r) * LD32 + c] = -s;
        }
        __syncthreads();
    }
    // X^T to global: LinvT[l][c] = X[c][l]
    float* out = LinvT + (long)(k / 128) * 128 * 128;
    for (int e = tid; e < 128 * 128; e += 256) {
        const int l = e >> 7, c = e & 127;
        out[e] = X[c * LD32 + l];
    }
    for (int e = tid; e < 128 * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        if (r < nb && c <= r) {
            float v = S[r * LD32 + c];
            W[(long)(k + r) * ldw + k + c] = v;
            mirror_store(mir, (long)(k + r), (long)(k + c), v);
        }
    }
}

// Panel solve for rows [r0, r0 + m) against the factored diagonal block at
// column c0 (order 128): X = B (L^{-1})^T, i.e. X[r][c] = sum_{l<=c} B[r][l]
// LinvT[l][c].  CTA = 64 rows; thread = 4 rows x 8 columns; warp w covers
// columns 16w..16w+15, so its loop stops at l = 16w + 15 (the inverse is
// lower triangular).
constexpr size_t trsm_leaf32_smem() { return (size_t)(128 * 68 + 128 * 132) * sizeof(float); }

__global__ void __launch_bounds__(256) k_trsm_leaf32(float* __restrict__ W, long ldw, int r0, int m, int c0,
                                                     const float* __restrict__ LinvT, Mirror mir,
                                                     const DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Bt = reinterpret_cast<float*>(smem_raw);  // [128][68]  Bt[l][r] = B[r][l]
    float* Lt = Bt + 128 * 68;                       // [128][132] LinvT
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;
    const int tid = threadIdx.x;
    const int rb0 = r0 + blockIdx.x * 64;
    const float* Lg = LinvT + (long)(c0 / 128) * 128 * 128;
    {
        float4 vb[8], vl[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // B: 64 rows x 128 columns
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            vb[q] = (rb0 + r < r0 + m) ? *reinterpret_cast<const float4*>(W + (long)(rb0 + r) * ldw + c0 + c4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + q * 256, l = e >> 5, c4 = (e & 31) * 4;
            vl[q] = *reinterpret_cast<const float4*>(Lg + l * 128 + c4);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            Bt[(c4 + 0) * 68 + r] = vb[q].x;
            Bt[(c4 + 1) * 68 + r] = vb[q].y;
            Bt[(c4 + 2) * 68 + r] = vb[q].z;
            Bt[(c4 + 3) * 68 + r] = vb[q].w;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + q * 256, l = e >> 5, c4 = (e & 31) * 4;
            *reinterpret_cast<float4*>(Lt + l * 132 + c4) = vl[q];
        }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int cb = warp * 16 + (lane >> 4) * 8;  // 8 columns
    const int rr = (lane & 15) * 4;              // 4 rows
    const int lmax = warp * 16 + 16;
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int l = 0; l < lmax; ++l) {
        const float4 a = *reinterpret_cast<const float4*>(Bt + l * 68 + rr);
        const float4 b0 = *reinterpret_cast<const float4*>(Lt + l * 132 + cb);
        const float4 b1 = *reinterpret_cast<const float4*>(Lt + l * 132 + cb + 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long row = rb0 + rr + i;
        if (row >= r0 + m) continue;
        float* dst = W + row * ldw + c0 + cb;
        *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(dst + 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
#pragma unroll
        for (int j = 0; j < 8; ++j) mirror_store(mir, row, (long)(c0 + cb + j), acc[i][j]);
    }
}
