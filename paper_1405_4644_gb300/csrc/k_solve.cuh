// k_solve.cuh -- step A4: the low-precision triangular solves of Algorithm 1
// (lines 2 and 5), z = R~^{-1} R~^{-T} r, with R~^T = L stored row-major
// (lower) in float32 (float64 for the baseline) and the scaling d:  z = d * L^{-T} L^{-1} (d * r).
//
// Forward sweep  y_J = L_JJ^{-1} (y_J - sum_{K<J} L_JK y_K)
// Backward sweep z_J = L_JJ^{-T} (y_J - sum_{K>J} L_KJ^T z_K)
// on 128-row blocks, right-looking: step J pushes the finished block J into
// every later (forward) / earlier (backward) block, one CTA per target
// block; the CTA of the next block then finishes it with the 32x32
// diagonal sub-block inverses.  Vectors are float32, column-major with
// leading dimension n; a launch handles up to 32 (float32) or 16 (float64)
// columns [c0, c0+mc).  The float64 instance serves the float64 baseline.
#pragma once
#include "common.cuh"

#define LDL 129

// columns per launch: 32 for float32, 16 for float64 (shared-memory budget)
template <typename T> constexpr int solve_mc() { return sizeof(T) == 4 ? 32 : 16; }

template <typename T>
constexpr size_t solve_smem_bytes() {
    return (size_t)(128 * LDL + 2 * 128 * (solve_mc<T>() + 1) + 4 * 32 * 33 + 32 * (solve_mc<T>() + 1)) * sizeof(T);
}

template <typename T>
__device__ __forceinline__ T lsolve_val(const T* W, long ldw, int n, int r, int c, bool diag) {
    if (r < n && c < n) return W[(long)r * ldw + c];
    return (diag && r == c) ? T(1) : T(0);
}

// Ys <- L_KK^{-1} Ys  (forward, sub-block by sub-block)
template <typename T, int MC>
__device__ void diag_fwd(const T* Ls, T* Ys, const T* Iv, T* Tm, int mc) {
    constexpr int LDY = MC + 1;
    const int tid = threadIdx.x;
    for (int s = 0; s < 4; ++s) {
        for (int e = tid; e < 32 * MC; e += 256) {
            int i = e & 31, c = e >> 5;
            if (c >= mc) continue;
            const T* lr = Ls + (s * 32 + i) * LDL;
            T acc = Ys[(s * 32 + i) * LDY + c];
            for (int l = 0; l < s * 32; ++l) acc -= lr[l] * Ys[l * LDY + c];
            Tm[i * LDY + c] = acc;
        }
        __syncthreads();
        const T* I = Iv + s * 32 * 33;
        for (int e = tid; e < 32 * MC; e += 256) {
            int i = e & 31, c = e >> 5;
            if (c >= mc) continue;
            T acc = T(0);
            for (int l = 0; l <= i; ++l) acc += I[i * 33 + l] * Tm[l * LDY + c];
            Ys[(s * 32 + i) * LDY + c] = acc;
        }
        __syncthreads();
    }
}

// Ys <- L_KK^{-T} Ys  (backward)
template <typename T, int MC>
__device__ void diag_bwd(const T* Ls, T* Ys, const T* Iv, T* Tm, int mc) {
    constexpr int LDY = MC + 1;
    const int tid = threadIdx.x;
    for (int s = 3; s >= 0; --s) {
        for (int e = tid; e < 32 * MC; e += 256) {
            int i = e & 31, c = e >> 5;
            if (c >= mc) continue;
            T acc = Ys[(s * 32 + i) * LDY + c];
            for (int l = (s + 1) * 32; l < 128; ++l) acc -= Ls[l * LDL + s * 32 + i] * Ys[l * LDY + c];
            Tm[i * LDY + c] = acc;
        }
        __syncthreads();
        const T* I = Iv + s * 32 * 33;
        for (int e = tid; e < 32 * MC; e += 256) {
            int i = e & 31, c = e >> 5;
            if (c >= mc) continue;
            T acc = T(0);
            for (int l = i; l < 32; ++l) acc += I[l * 33 + i] * Tm[l * LDY + c];
            Ys[(s * 32 + i) * LDY + c] = acc;
        }
        __syncthreads();
    }
}

template <typename T, int MC>
__device__ __forceinline__ void load_y(const T* Y, int n, int c0, int mc, int blk, T* Ys) {
    constexpr int LDY = MC + 1;
    for (int e = threadIdx.x; e < 128 * MC; e += 256) {
        int i = e & 127, c = e >> 7;
        int r = blk * 128 + i;
        Ys[i * LDY + c] = (c < mc && r < n) ? Y[(long)(c0 + c) * n + r] : T(0);
    }
}
template <typename T, int MC>
__device__ __forceinline__ void store_y(T* Y, int n, int c0, int mc, int blk, const T* Ys) {
    constexpr int LDY = MC + 1;
    for (int e = threadIdx.x; e < 128 * MC; e += 256) {
        int i = e & 127, c = e >> 7;
        int r = blk * 128 + i;
        if (c < mc && r < n) Y[(long)(c0 + c) * n + r] = Ys[i * LDY + c];
    }
}
template <typename T>
__device__ __forceinline__ void load_tile(const T* W, long ldw, int n, int rb, int cb, bool diag, T* Ls) {
    for (int e = threadIdx.x; e < 128 * 128; e += 256) {
        int r = e >> 7, c = e & 127;
        int gr = rb * 128 + r, gc = cb * 128 + c;
        T v = (diag && c > r) ? T(0) : lsolve_val(W, ldw, n, gr, gc, diag);
        Ls[r * LDL + c] = v;
    }
}
template <typename T>
__device__ __forceinline__ void load_inv(const T* Dinv, int blk, T* Iv) {
    for (int e = threadIdx.x; e < 4 * 1024; e += 256) {
        int s = e >> 10, i = (e >> 5) & 31, c = e & 31;
        Iv[(s * 32 + i) * 33 + c] = Dinv[(long)(blk * 4 + s) * 1024 + i * 32 + c];
    }
}

// Forward step J (J = -1 .. NB-2): CTA b updates block K = J+1+b with the
// finished block J; CTA 0 then finishes block J+1.
template <typename T, int MC>
static __global__ void __launch_bounds__(256) k_trsv_fwd_step(const T* __restrict__ W, long ldw, int n,
                                                       const T* __restrict__ Dinv, T* __restrict__ Y,
                                                       int c0, int mc, int J) {
    constexpr int LDY = MC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ls = reinterpret_cast<T*>(smem_raw);
    T* Yk = Ls + 128 * LDL;
    T* Yj = Yk + 128 * LDY;
    T* Iv = Yj + 128 * LDY;
    T* Tm = Iv + 4 * 32 * 33;
    const int K = J + 1 + blockIdx.x;
    load_y<T, MC>(Y, n, c0, mc, K, Yk);
    if (J >= 0) {
        load_y<T, MC>(Y, n, c0, mc, J, Yj);
        load_tile(W, ldw, n, K, J, false, Ls);
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * MC; e += 256) {
            int i = e & 127, c = e >> 7;
            if (c >= mc) continue;
            const T* lr = Ls + i * LDL;
            T acc = T(0);
#pragma unroll 8
            for (int l = 0; l < 128; ++l) acc += lr[l] * Yj[l * LDY + c];
            Yk[i * LDY + c] -= acc;
        }
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        load_tile(W, ldw, n, K, K, true, Ls);
        load_inv(Dinv, K, Iv);
        __syncthreads();
        diag_fwd<T, MC>(Ls, Yk, Iv, Tm, mc);
    }
    __syncthreads();
    store_y<T, MC>(Y, n, c0, mc, K, Yk);
}

// Backward step J (J = NB .. 1): CTA b updates block K = J-1-b with the
// finished block J (when J < NB); CTA 0 then finishes block J-1.
template <typename T, int MC>
static __global__ void __launch_bounds__(256) k_trsv_bwd_step(const T* __restrict__ W, long ldw, int n, int NB,
                                                       const T* __restrict__ Dinv, T* __restrict__ Y,
                                                       int c0, int mc, int J) {
    constexpr int LDY = MC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Ls = reinterpret_cast<T*>(smem_raw);
    T* Yk = Ls + 128 * LDL;
    T* Yj = Yk + 128 * LDY;
    T* Iv = Yj + 128 * LDY;
    T* Tm = Iv + 4 * 32 * 33;
    const int K = J - 1 - blockIdx.x;
    load_y<T, MC>(Y, n, c0, mc, K, Yk);
    if (J < NB) {
        load_y<T, MC>(Y, n, c0, mc, J, Yj);
        load_tile(W, ldw, n, J, K, false, Ls);  // L_JK: rows of block J, columns of block K
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * MC; e += 256) {
            int l = e & 127, c = e >> 7;
            if (c >= mc) continue;
            T acc = T(0);
#pragma unroll 8
            for (int r = 0; r < 128; ++r) acc += Ls[r * LDL + l] * Yj[r * LDY + c];
            Yk[l * LDY + c] -= acc;
        }
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        load_tile(W, ldw, n, K, K, true, Ls);
        load_inv(Dinv, K, Iv);
        __syncthreads();
        diag_bwd<T, MC>(Ls, Yk, Iv, Tm, mc);
    }
    __syncthreads();
    store_y<T, MC>(Y, n, c0, mc, K, Yk);
}

// y = fl(d .* r) for columns [0, m)
template <typename T>
static __global__ void k_scale_to(const double* __restrict__ R, long ldr, const double* __restrict__ d, int n, int m,
                           T* __restrict__ Y) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        long c = e / n, i = e - c * n;
        Y[e] = (T)(d[i] * R[c * ldr + i]);
    }
}

// mode 0: X = d .* y ; mode 1: X += d .* y on columns whose frozen flag is 0
template <typename T>
static __global__ void k_apply_correction(double* __restrict__ X, long ldx, const double* __restrict__ d,
                                   const T* __restrict__ Y, int n, int m, const int* __restrict__ frozen,
                                   int mode) {
    long total = (long)n * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        long c = e / n, i = e - c * n;
        if (frozen && frozen[c]) continue;
        double z = d[i] * (double)Y[e];
        if (mode == 0) X[c * ldx + i] = z;
        else X[c * ldx + i] += z;
    }
}
