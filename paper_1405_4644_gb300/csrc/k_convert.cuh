// k_convert.cuh -- step A0: symmetric diagonal scaling and conversion of the
// float64 input into the working matrix of the factorisation.
#pragma once
#include "common.cuh"

// d_i = 1/sqrt(A_ii) (or 1 when scaling is off).  A non-positive or
// non-finite diagonal entry raises SPD_DEV_BADDIAG / SPD_DEV_NONFINITE and
// records the 1-based index in st->info.
static __global__ void k_diag_scale(const double* __restrict__ A, long lda, int n, int scale,
                             double* __restrict__ d, DevStatus* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = A[(long)i * lda + i];
    if (!isfinite(a)) {
        dev_raise(st, SPD_DEV_NONFINITE);
        atomicMin(&st->info, i + 1);
        d[i] = 1.0;
        return;
    }
    if (!(a > 0.0)) {
        dev_raise(st, SPD_DEV_BADDIAG);
        atomicMin(&st->info, i + 1);
        d[i] = 1.0;
        return;
    }
    d[i] = scale ? 1.0 / sqrt(a) : 1.0;
}

// |x| = m 2^e for a finite, nonzero float64 x (magnitude bits b): m in [1, 2]
// is the mantissa rounded to 24 bits (half up), formed with integer
// operations only (subnormal x normalised first)
__device__ __forceinline__ float f64_mant24(unsigned long long b, int& e) {
    int ef = (int)(b >> 52);
    unsigned long long M = b & 0xFFFFFFFFFFFFFull;
    if (ef == 0) {  // subnormal: shift the leading one to bit 52
        const int sh = __clzll((long long)M) - 11;
        M = (M << sh) & 0xFFFFFFFFFFFFFull;
        ef = 1 - sh;
    }
    e = ef - 1023;
    const uint32_t m = (uint32_t)((M + (1ull << 28)) >> 29);  // 2^23 carries to 2.0
    return __uint_as_float(0x3F800000u + m);
}

// d_i a d_j rounded to float32 without float64 arithmetic, which runs at a
// small fraction of the float32 rate on this part: the three 24-bit
// mantissas are multiplied in float32 and the exponents added (scalbnf).
// Five roundings of 2^-24 at most: |error| <= 2^-21.6 |d_i a d_j| for normal
// results.
__device__ __forceinline__ float scaled_f32(double a, double di, double dj) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    if (mag == 0ull) return (b >> 63) ? -0.f : 0.f;
    int ea, ei, ej;
    const float ma = f64_mant24(mag, ea);
    const float mi = f64_mant24((unsigned long long)__double_as_longlong(di), ei);
    const float mj = f64_mant24((unsigned long long)__double_as_longlong(dj), ej);
    const float v = scalbnf(ma * mi * mj, ea + ei + ej);
    return (b >> 63) ? -v : v;
}


// W[i][i] += sigma: the shifted factorisation of SPD_FACTOR_SHIFT.
template <typename T>
static __global__ void k_add_diag(T* __restrict__ W, long ldw, int n, double sigma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) W[(long)i * ldw + i] += (T)sigma;
}

// Full low-precision copy A~ = fl(A) for the CG matrix-vector product:
// row-major n x lda_out (A is symmetric, so this is also its column-major
// copy).  T is float or __nv_bfloat16.
template <typename T>
static __global__ void k_convert_full(const double* __restrict__ A, long lda, int n,
                               T* __restrict__ At, long ldt, DevStatus* st) {
    long total = (long)n * n;
    bool bad = false;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        long j = e / n, i = e - j * n;  // column-major walk: coalesced reads
        double v = A[j * lda + i];
        if (!isfinite(v)) bad = true;
        // symmetric: A(i, j) = A(j, i); write row j, column i of the copy
        At[j * ldt + i] = (T)(float)v;
    }
    if (bad) dev_raise(st, SPD_DEV_NONFINITE);
}

// Banded low-precision copy in diagonal-major layout:
// Ab[(o + band) * n + i] = fl(A(i, i + o)) for |o| <= band (0 outside).
static __global__ void k_convert_band(const double* __restrict__ A, long lda, int n, int band,
                               float* __restrict__ Ab, DevStatus* st) {
    long total = (long)(2 * band + 1) * n;
    bool bad = false;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        int o = (int)(e / n) - band;
        int i = (int)(e % n);
        int j = i + o;
        float v = 0.0f;
        if (j >= 0 && j < n) {
            double a = A[(long)j * lda + i];
            if (!isfinite(a)) bad = true;
            v = (float)a;
        }
        Ab[e] = v;
    }
    if (bad) dev_raise(st, SPD_DEV_NONFINITE);
}

// W (row-major, ldw) lower triangle <- d_i A_ij d_j for i >= j, rounded to
// T.  A is column-major (lda); element (i, j) lives at A[i + j*lda].  Only
// the 64 x 64 tiles of the lower triangle are launched (a triangular grid:
// block t -> tile (bi, bj), bj <= bi).  Thread (tx, ty) = (tid % 32, tid / 32)
// reads rows i0 + tx and i0 + 32 + tx of the columns j0 + ty + 8 k (coalesced
// in A), all sixteen loads in flight before any is converted; the tile goes
// back along W's rows (coalesced in W) through shared memory.  Non-finite
// entries raise SPD_DEV_NONFINITE.  For float32 W the scaling avoids float64
// arithmetic (scaled_f32; d is positive and normal).
template <typename T>
static __global__ void __launch_bounds__(256) k_scale_convert(const double* __restrict__ A, long lda, int n,
                                                                const double* __restrict__ d, T* __restrict__ W,
                                                                long ldw, DevStatus* st) {
    __shared__ T tile[64][65];  // tile[i_local][j_local]
    const long t = blockIdx.x;
    int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while ((long)bi * (bi + 1) / 2 > t) --bi;
    const int bj = (int)(t - (long)bi * (bi + 1) / 2);
    const int i0 = bi * 64, j0 = bj * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double a[16];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + 32 * h + tx, j = j0 + ty + 8 * k;
            a[2 * k + h] = (i < n && j < n && j <= i) ? A[(long)j * lda + i] : 0.0;
        }
    const double di0 = (i0 + tx < n) ? d[i0 + tx] : 0.0;
    const double di1 = (i0 + 32 + tx < n) ? d[i0 + 32 + tx] : 0.0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int j = j0 + ty + 8 * k;
        const double dj = j < n ? d[j] : 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + 32 * h + tx;
            const double v = a[2 * k + h];
            T w = T(0);
            if (i < n && j < n && j <= i) {
                if (((unsigned long long)__double_as_longlong(v) & 0x7FF0000000000000ull) == 0x7FF0000000000000ull)
                    bad = true;
                const double di = h ? di1 : di0;
                if constexpr (sizeof(T) == 8) w = di * v * dj;
                else w = scaled_f32(v, di, dj);
            }
            tile[32 * h + tx][ty + 8 * k] = w;
        }
    }
    if (bad) dev_raise(st, SPD_DEV_NONFINITE);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + ty + 8 * k, j = j0 + 32 * h + tx;
            if (i < n && j < n && j <= i) W[(long)i * ldw + j] = tile[ty + 8 * k][32 * h + tx];
        }
}
