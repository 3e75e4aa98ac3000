// k_leaf32.cuh -- float32 leaves of the low-precision factorisation (steps
// A1/A2 of Section 3.1's Cholesky) and the per-block inverses the
// triangular sweeps use:
//
//   k_potrf_leaf32   factors W[k:k+nb, k:k+nb] = L L^T in four 32-column
//                    steps: one warp factors the 32x32 diagonal block
//                    (warp-level pivots) and inverts it by right-looking
//                    substitution with the pivots' reciprocals; all warps
//                    form the sub-panel below it with that inverse and
//                    update the rest of the block; only the next diagonal
//                    block's part of that update precedes the next pivot
//                    step, and while warp 0 factors it the other warps
//                    store the finished block column of L (and its operand
//                    mirror) and finish the update.  Also stores the four
//                    32x32 inverses.
//   k_trsm_leaf32    panel solve X L^T = B for 64 rows per CTA in four
//                    32-column steps with the same 32x32 inverses.
//   k_block_inverse  after the whole factorisation, off the critical path
//                    and one CTA per block: the full (L_JJ^{-1})^T of every
//                    128x128 diagonal block, for the sweeps.
//
// The float64 baseline keeps the sub-block kernels of k_leaf.cuh.
#pragma once
#include "common.cuh"

#define LD32 129

// Dinv32 for block b lives at Dinv32 + b * 4096: four row-major 32x32
// blocks, D_s[i][c] = (L_ss^{-1})[i][c] (lower triangular).
constexpr size_t potrf_leaf32_smem() { return (size_t)(128 * LD32 + 32 * 33 + 96 * 33) * sizeof(float); }

// Entries of L in columns [c0, c0 + 32), rows c0 .. nb - 1, from the leaf's
// shared copy S to W and its mirror, four columns per store; thread t of nt.
__device__ __forceinline__ void leaf_store_cols(const float* S, float* W, long ldw, int k, int nb, int c0,
                                                const Mirror& mir, int t, int nt) {
    for (int e = t; e < (128 - c0) * 8; e += nt) {
        const int r = c0 + (e >> 3), c4 = c0 + (e & 7) * 4;
        if (r >= nb || c4 > r) continue;
        const float* sr = S + r * LD32 + c4;
        float v[4] = {sr[0], sr[1], sr[2], sr[3]};
        float* dst = W + (long)(k + r) * ldw + k + c4;
        if (c4 + 3 <= r) {
            const float4 f = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst) = f;
            mirror_store4(mir, (long)(k + r), (long)(k + c4), f);
        } else {
            for (int q = 0; c4 + q <= r; ++q) {
                dst[q] = v[q];
                mirror_store(mir, (long)(k + r), (long)(k + c4 + q), v[q]);
            }
        }
    }
}

// Part of the leaf's trailing update after step o: S[i][j] -= sum_{l<32}
// S[i][o+l] S[j][o+l] for the 2x2 blocks (bi, bj), bj <= bi, of the region
// from row/column base = o + 32 with bi in [bi0, bi1) (bi1 <= (128 - base) /
// 2); thread t of nt.
__device__ __forceinline__ void leaf_trailing(float* S, int o, int bi0, int bi1, int t, int nt) {
    const int base = o + 32;
    const int nc = bi1;  // columns bj < bi1 cover every bj <= bi
    for (int e = t; e < (bi1 - bi0) * nc; e += nt) {
        const int bi = bi0 + e / nc, bj = e % nc;
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
}

__global__ void __launch_bounds__(256, 1) k_potrf_leaf32(float* __restrict__ W, long ldw, int k, int nb,
                                                      float* __restrict__ Dinv32, Mirror mir, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* S = reinterpret_cast<float*>(smem_raw);  // [128][129] the block, then L
    float* Dj = S + 128 * LD32;                     // [32][33] inverse of the current 32x32 diagonal block
    float* Tmp = Dj + 32 * 33;                      // [96][33] sub-panel scratch
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();  // the update of this diagonal block is the previous kernel
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
    } else {  // ragged last block: identity beyond nb
        for (int e = tid; e < 128 * 128; e += 256) {
            int r = e >> 7, c = e & 127;
            float v;
            if (r < nb && c < nb) v = (c <= r) ? W[(long)(k + r) * ldw + k + c] : 0.f;
            else v = (r == c) ? 1.f : 0.f;
            S[r * LD32 + c] = v;
        }
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    float* Dout = Dinv32 + (long)(k / 128) * 4096;

    for (int J = 0; J < 4; ++J) {
        const int o = J * 32;
        if (J == 2 && tid == 0) pdl_trigger();  // the panel solve may start loading its rows
        if (warp == 0) {
            // lane r holds row o + r of the diagonal block
            float a[32], rd[32];
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
                // one MUFU op on the pivot chain: 1/sqrt, then sqrt = piv / sqrt
                const float inv = rsqrtf(piv);
                const float dj = piv * inv;
                rd[j] = inv;
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
            // lane c: column c of the inverse, right-looking: x_i = s_i / L_ii,
            // then s_r -= L_ri x_i for r > i (independent updates, short chain)
            float x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                x[i] *= rd[i];
#pragma unroll
                for (int r = i + 1; r < 32; ++r) x[r] = fmaf(-S[(o + r) * LD32 + o + i], x[i], x[r]);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                Dj[i * 33 + lane] = x[i];
                Dout[J * 1024 + i * 32 + lane] = x[i];
            }
        } else if (J > 0) {
            // while warp 0 factors this diagonal block, the other warps write
            // out block column J - 1 (final) and finish step J - 1's trailing
            // update below this diagonal block (rows o + 32 .., read only
            // after the next barrier)
            leaf_store_cols(S, W, ldw, k, nb, o - 32, mir, tid - 32, 224);
            leaf_trailing(S, o - 32, 16, (128 - o) >> 1, tid - 32, 224);
        }
        __syncthreads();
        if (s_bad) return;
        const int rows = 128 - (o + 32);
        if (rows == 0) break;
        // sub-panel below: L_iJ = A_iJ D_J^T, 4 outputs per thread-iteration
        for (int e = tid; e < rows * 8; e += 256) {
            const int i = e >> 3, c4 = (e & 7) * 4;
            const float* brow = S + (o + 32 + i) * LD32 + o;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (int l = 0; l <= c4 + 3; ++l) {
                const float b = brow[l];
                s0 = fmaf(b, Dj[(c4 + 0) * 33 + l], s0);
                s1 = fmaf(b, Dj[(c4 + 1) * 33 + l], s1);
                s2 = fmaf(b, Dj[(c4 + 2) * 33 + l], s2);
                s3 = fmaf(b, Dj[(c4 + 3) * 33 + l], s3);
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
        // trailing update of the next diagonal block only (rows and columns
        // o + 32 .. o + 63); the rest of it runs during the next diagonal step
        leaf_trailing(S, o, 0, 16, tid, 256);
        __syncthreads();
    }
    // the last block column (the others went out during the next diagonal step)
    leaf_store_cols(S, W, ldw, k, nb, 96, mir, tid, 256);
}

// Panel solve for rows [r0, r0 + m) against the factored diagonal block at
// column c0 (order 128): X L^T = B, in four 32-column steps s:
//   X_s = B_s D_s^T,   B_s' -= X_s L_s's^T  (s' > s),
// with D_s the 32x32 inverses the leaf stored.  CTA = 64 rows; each thread
// owns a 4-row by (2 | 6 - 2 s)-column register tile of each step.
constexpr size_t trsm_leaf32_smem() { return (size_t)(64 * 132 + 96 * LD32 + 4 * 32 * 33) * sizeof(float); }

// b_ready: the previous kernel in the stream (the leaf) does not write B,
// so B is loaded before waiting for it (programmatic dependent launch).
__global__ void __launch_bounds__(256, 2) k_trsm_leaf32(float* __restrict__ W, long ldw, int r0, int m, int c0,
                                                     const float* __restrict__ Dinv32, Mirror mir,
                                                     const DevStatus* st, int b_ready) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Bs = reinterpret_cast<float*>(smem_raw);  // [64][132] B, becoming X
    float* Ls = Bs + 64 * 132;                       // [96][129] rows 32..127 of L_kk, columns 0..95
    float* Ds = Ls + 96 * LD32;                      // [4][32][33] D_s
    const int tid = threadIdx.x;
    const int rb0 = r0 + blockIdx.x * 64;
    {
        if (!b_ready) pdl_wait();
        float4 vb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // B: 64 rows x 128 columns
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            vb[q] = (rb0 + r < r0 + m) ? *reinterpret_cast<const float4*>(W + (long)(rb0 + r) * ldw + c0 + c4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (b_ready) pdl_wait();  // L_kk and its inverses come from the previous kernel
        if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;
        // the strictly-below-diagonal 32-blocks of L_kk (rows 32..127, columns
        // 0..95) and the four 32x32 inverses: every load in flight first
        float4 vl[9], vd[4];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int e = tid + q * 256, r = e / 24, c4 = (e - r * 24) * 4;
            vl[q] = *reinterpret_cast<const float4*>(W + (long)(c0 + 32 + r) * ldw + c0 + c4);
        }
        const float4* dg = reinterpret_cast<const float4*>(Dinv32 + (long)(c0 / 128) * 4096);
#pragma unroll
        for (int q = 0; q < 4; ++q) vd[q] = __ldg(dg + tid + q * 256);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int e = tid + q * 256, r = e / 24, c4 = (e - r * 24) * 4;
            float* d = Ls + r * LD32 + c4;
            d[0] = (c4 + 0 < r + 32) ? vl[q].x : 0.f;
            d[1] = (c4 + 1 < r + 32) ? vl[q].y : 0.f;
            d[2] = (c4 + 2 < r + 32) ? vl[q].z : 0.f;
            d[3] = (c4 + 3 < r + 32) ? vl[q].w : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = (tid + q * 256) * 4, i = e >> 5, c = e & 31;
            float* d = Ds + i * 33 + c;
            d[0] = vd[q].x;
            d[1] = vd[q].y;
            d[2] = vd[q].z;
            d[3] = vd[q].w;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + q * 256, r = e >> 5, c4 = (e & 31) * 4;
            *reinterpret_cast<float4*>(Bs + r * 132 + c4) = vb[q];
        }
    }
    __syncthreads();
    // thread tile: rows tr..tr+3 (16 row groups) x a column group (16 groups)
    const int tr = (tid >> 4) * 4, cgp = tid & 15;
    for (int s = 0; s < 4; ++s) {
        const int o = s * 32;
        const float* D = Ds + s * 32 * 33;
        // X_s, columns o + c, o + c + 1 (D[c][l] = 0 for l > c)
        const int c = 2 * cgp;
        float x[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j][0] = x[j][1] = 0.f;
        for (int l = 0; l <= c + 1; ++l) {
            const float d0 = D[c * 33 + l], d1 = D[(c + 1) * 33 + l];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float b = Bs[(tr + j) * 132 + o + l];
                x[j][0] = fmaf(b, d0, x[j][0]);
                x[j][1] = fmaf(b, d1, x[j][1]);
            }
        }
        __syncthreads();  // every read of B_s done
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Bs[(tr + j) * 132 + o + c] = x[j][0];
            Bs[(tr + j) * 132 + o + c + 1] = x[j][1];
        }
        __syncthreads();
        if (s == 3) break;
        // B_s' -= X_s L_s's^T for the 96 - 32 s columns to the right: CW each
        const int CW = 6 - 2 * s;
        const int cb = o + 32 + cgp * CW;  // first column (= row of L) of this thread
        float acc[4][6];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[j][q] = 0.f;
#pragma unroll 2
        for (int l = 0; l < 32; ++l) {
            float xv[4], lv[6];
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = Bs[(tr + j) * 132 + o + l];
#pragma unroll
            for (int q = 0; q < 6; ++q) lv[q] = (q < CW) ? Ls[(cb + q - 32) * LD32 + o + l] : 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[j][q] = fmaf(xv[j], lv[q], acc[j][q]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (q < CW) Bs[(tr + j) * 132 + cb + q] -= acc[j][q];
        __syncthreads();
    }
    for (int e = tid; e < 64 * 32; e += 256) {
        const int rr = e >> 5, c4 = (e & 31) * 4;
        const long row = rb0 + rr;
        if (row >= r0 + m) continue;
        const float4 v = *reinterpret_cast<const float4*>(Bs + rr * 132 + c4);
        *reinterpret_cast<float4*>(W + row * ldw + c0 + c4) = v;
        mirror_store4(mir, row, (long)(c0 + c4), v);
    }
}

// (L_JJ^{-1})^T of every 128x128 diagonal block (one CTA per block, after
// the factorisation): X = L^{-1} by block rows, X_ii = D_i (the leaf's 32x32
// inverses) and X_i,0:i = -D_i (L_i,0:i X_0:i,0:i); LinvT[l][c] = X[c][l].
// Rows past n are the identity, as in the leaf.
constexpr size_t block_inverse_smem() { return (size_t)(2 * 128 * LD32 + 32 * 97) * sizeof(float); }

__global__ void __launch_bounds__(256) k_block_inverse(const float* __restrict__ W, long ldw, int n,
                                                       const float* __restrict__ Dinv32, float* __restrict__ LinvT) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* S = reinterpret_cast<float*>(smem_raw);  // [128][129] L_JJ
    float* X = S + 128 * LD32;                      // [128][129] L_JJ^{-1}
    float* Tmp = X + 128 * LD32;                    // [32][97]
    const int tid = threadIdx.x;
    const int J = blockIdx.x;
    const long k = (long)J * 128;
    const int nb = (int)min((long)128, n - k);
    const float* dg = Dinv32 + (long)J * 4096;
    for (int e = tid; e < 128 * 128; e += 256) {
        const int r = e >> 7, c = e & 127;
        float v;
        if (r < nb && c < nb) v = (c <= r) ? W[(k + r) * ldw + k + c] : 0.f;
        else v = (r == c) ? 1.f : 0.f;
        S[r * LD32 + c] = v;
        const int br = r >> 5, bc = c >> 5;
        X[r * LD32 + c] = (br == bc) ? dg[br * 1024 + (r & 31) * 32 + (c & 31)] : 0.f;
    }
    __syncthreads();
    for (int i = 1; i < 4; ++i) {
        const int ri = i * 32, w = i * 32;  // rows ri..ri+31 of X, columns 0..w-1
        for (int e = tid; e < 32 * w; e += 256) {
            const int rr = e / w, c = e - rr * w;
            const float* lr = S + (ri + rr) * LD32;
            float s0 = 0.f, s1 = 0.f;
            int l = (c >> 5) << 5;
            for (; l + 1 < ri; l += 2) {  // two chains: shorter dependency
                s0 = fmaf(lr[l], X[l * LD32 + c], s0);
                s1 = fmaf(lr[l + 1], X[(l + 1) * LD32 + c], s1);
            }
            if (l < ri) s0 = fmaf(lr[l], X[l * LD32 + c], s0);
            Tmp[rr * 97 + c] = s0 + s1;
        }
        __syncthreads();
        for (int e = tid; e < 32 * w; e += 256) {
            const int rr = e / w, c = e - rr * w;
            const float* ir = X + (ri + rr) * LD32 + ri;
            float s = 0.f;
            for (int l = 0; l <= rr; ++l) s = fmaf(ir[l], Tmp[l * 97 + c], s);
            X[(ri + rr) * LD32 + c] = -s;
        }
        __syncthreads();
    }
    float* out = LinvT + (long)J * 16384;
    for (int e = tid; e < 128 * 128; e += 256) {
        const int l = e >> 7, c = e & 127;
        out[e] = X[c * LD32 + l];
    }
}
