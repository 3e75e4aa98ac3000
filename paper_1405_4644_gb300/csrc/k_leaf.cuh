// k_leaf.cuh -- steps A1 (diagonal-block Cholesky) and A2 (panel triangular
// solve) of the blocked right-looking factorisation (Section 3.1, eq.
// (cholesky)), on 128x128 diagonal blocks ("leaves").
//
// Storage: W is row-major with leading dimension ldw; its lower triangle
// holds the (scaled) matrix on entry and L = R~^T on exit.  Inside a leaf
// the work is split into four 32x32 sub-blocks: warp 0 factors a diagonal
// sub-block in registers (one row per lane, shuffles for the column
// broadcasts) and inverts it; the CTA then solves the sub-panel below and
// updates the rest of the leaf.  The inverses of the 32x32 diagonal
// sub-blocks are kept (Dinv) for the panel solves and the triangular
// solves of the refinement loop.
#pragma once
#include "common.cuh"

#define LDS_LEAF 129

template <typename T>
__device__ __forceinline__ T leaf_load(const T* W, long ldw, int base, int nb, int r, int c) {
    if (r < nb && c < nb) return (c <= r) ? W[(long)(base + r) * ldw + base + c] : T(0);
    return (r == c) ? T(1) : T(0);  // identity padding beyond the matrix
}

template <typename T>
constexpr size_t potrf_leaf_smem() {
    return (size_t)(128 * LDS_LEAF + 96 * 33 + 32 * 33) * sizeof(T);
}

// Factor the diagonal block W[k:k+nb, k:k+nb] (nb <= 128) in place.
// Dinv receives the 4 inverses of its 32x32 diagonal sub-blocks (row-major
// 32x32 each, at Dinv + ((k + 32 s) / 32) * 1024).  Finalised entries are
// also written to the operand mirror.  A non-positive pivot raises
// SPD_DEV_BREAKDOWN with the 1-based global column in st->info.
template <typename T>
__global__ void __launch_bounds__(256, 1) k_potrf_leaf(T* __restrict__ W, long ldw, int k, int nb,
                                                    T* __restrict__ Dinv, Mirror mir, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);  // [128][129]
    T* Tmp = S + 128 * LDS_LEAF;             // [96][33]
    T* Inv = Tmp + 96 * 33;                  // [32][33]
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;

    for (int e = tid; e < 128 * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        S[r * LDS_LEAF + c] = leaf_load(W, ldw, k, nb, r, c);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();

    for (int J = 0; J < 4; ++J) {
        const int o = J * 32;
        if (warp == 0) {
            T a[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) a[c] = S[(o + lane) * LDS_LEAF + o + c];
            int badj = -1;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                T piv = __shfl_sync(0xffffffffu, a[j], j);
                if (!(piv > T(0))) {  // uniform across the warp
                    if (badj < 0) badj = j;
                    piv = T(1);
                }
                T dj = dsqrt(piv);
                T inv = T(1) / dj;
                a[j] = (lane == j) ? dj : (lane > j ? a[j] * inv : a[j]);
#pragma unroll
                for (int l = 0; l < 32; ++l) {  // constant bounds keep a[] in registers
                    if (l > j) {
                        T t = __shfl_sync(0xffffffffu, a[j], l);
                        a[l] = (lane >= l) ? a[l] - a[j] * t : a[l];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) S[(o + lane) * LDS_LEAF + o + c] = (c <= lane) ? a[c] : T(0);
            if (badj >= 0 && lane == 0 && o + badj < nb) {
                s_bad = 1;
                atomicMin(&st->info, k + o + badj + 1);
                dev_raise(st, SPD_DEV_BREAKDOWN);
            }
            __syncwarp();
            // lane c: column c of the inverse, x_i = (delta_ic - sum_{l<i} L_il x_l) / L_ii
            T x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const T* li = S + (o + i) * LDS_LEAF + o;
                T s = (i == lane) ? T(1) : T(0);
#pragma unroll
                for (int l = 0; l < 32; ++l)
                    if (l < i) s -= li[l] * x[l];
                x[i] = s / li[i];
            }
            T* Dg = Dinv + (long)((k + o) / 32) * 1024;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                Inv[i * 33 + lane] = x[i];
                Dg[i * 32 + lane] = x[i];
            }
        }
        __syncthreads();
        if (s_bad) return;
        const int rows = 128 - (o + 32);
        if (rows == 0) break;
        // sub-panel: L_iJ = A_iJ * Inv^T   (X[i][c] = sum_{l<=c} B[i][l] Inv[c][l])
        for (int e = tid; e < rows * 32; e += 256) {
            int i = e >> 5, c = e & 31;
            const T* brow = S + (o + 32 + i) * LDS_LEAF + o;
            T s = T(0);
            for (int l = 0; l <= c; ++l) s += brow[l] * Inv[c * 33 + l];
            Tmp[i * 33 + c] = s;
        }
        __syncthreads();
        for (int e = tid; e < rows * 32; e += 256) {
            int i = e >> 5, c = e & 31;
            S[(o + 32 + i) * LDS_LEAF + o + c] = Tmp[i * 33 + c];
        }
        __syncthreads();
        // trailing update of the rest of the leaf (lower part)
        const int base = o + 32;
        for (int e = tid; e < rows * rows; e += 256) {
            int i = e / rows, j = e - i * rows;
            if (j > i) continue;
            const T* ri = S + (base + i) * LDS_LEAF + o;
            const T* rj = S + (base + j) * LDS_LEAF + o;
            T s = T(0);
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += ri[l] * rj[l];
            S[(base + i) * LDS_LEAF + base + j] -= s;
        }
        __syncthreads();
    }
    for (int e = tid; e < 128 * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        if (r < nb && c <= r) {
            T v = S[r * LDS_LEAF + c];
            W[(long)(k + r) * ldw + k + c] = v;
            mirror_store(mir, (long)(k + r), (long)(k + c), v);
        }
    }
}

template <typename T, int RB>
constexpr size_t trsm_leaf_smem() {
    return (size_t)(RB * LDS_LEAF + 128 * LDS_LEAF + 4 * 32 * 33 + RB * 33) * sizeof(T);
}

// Panel solve X L^T = B for rows [r0, r0+m) and the factored diagonal block
// at (c0, c0) of order kb <= 128:  X = B L^{-T}, done 32 columns at a time,
// X_j = (B_j - sum_{s<j} X_s L_js^T) Inv_jj^T.  RB rows per CTA.
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_trsm_leaf(T* __restrict__ W, long ldw, int r0, int m, int c0,
                                                   int kb, const T* __restrict__ Dinv, Mirror mir,
                                                   const DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Bs = reinterpret_cast<T*>(smem_raw);  // [RB][129]
    T* Ls = Bs + RB * LDS_LEAF;                 // [128][129]
    T* Iv = Ls + 128 * LDS_LEAF;                // [4][32][33]
    T* Tm = Iv + 4 * 32 * 33;                   // [RB][33]
    const int tid = threadIdx.x;
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;
    const int rb0 = r0 + blockIdx.x * RB;
    const int nsub = (kb + 31) / 32;

    for (int e = tid; e < RB * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        T v = T(0);
        if (rb0 + r < r0 + m && c < kb) v = W[(long)(rb0 + r) * ldw + c0 + c];
        Bs[r * LDS_LEAF + c] = v;
    }
    for (int e = tid; e < nsub * 32 * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        Ls[r * LDS_LEAF + c] = leaf_load(W, ldw, c0, kb, r, c);
    }
    for (int e = tid; e < nsub * 1024; e += 256) {
        int s = e >> 10, i = (e >> 5) & 31, c = e & 31;
        Iv[(s * 32 + i) * 33 + c] = Dinv[(long)(c0 / 32 + s) * 1024 + i * 32 + c];
    }
    __syncthreads();

    for (int j = 0; j < nsub; ++j) {
        for (int e = tid; e < RB * 32; e += 256) {
            int r = e >> 5, c = e & 31;
            const T* br = Bs + r * LDS_LEAF;
            const T* lr = Ls + (j * 32 + c) * LDS_LEAF;
            T s = br[j * 32 + c];
            for (int l = 0; l < j * 32; ++l) s -= br[l] * lr[l];
            Tm[r * 33 + c] = s;
        }
        __syncthreads();
        const T* Ij = Iv + j * 32 * 33;
        for (int e = tid; e < RB * 32; e += 256) {
            int r = e >> 5, c = e & 31;
            T s = T(0);
            for (int l = 0; l <= c; ++l) s += Tm[r * 33 + l] * Ij[c * 33 + l];
            Bs[r * LDS_LEAF + j * 32 + c] = s;
        }
        __syncthreads();
    }
    for (int e = tid; e < RB * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        if (rb0 + r < r0 + m && c < kb) {
            T v = Bs[r * LDS_LEAF + c];
            W[(long)(rb0 + r) * ldw + c0 + c] = v;
            mirror_store(mir, (long)(rb0 + r), (long)(c0 + c), v);
        }
    }
}
