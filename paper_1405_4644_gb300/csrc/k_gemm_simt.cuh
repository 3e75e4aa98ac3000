// k_gemm_simt.cuh -- step A3 (trailing update) on the CUDA cores, used by the
// float32 and float64 factorisations:
//     W[r0+r][c0+c] -= sum_k Op[r0+r][k0+k] * Op[c0+c][k0+k]
// for r < M, c < N, k < K.  Op is W itself (float32 / float64 factor) or
// the factor's operand mirror (entries already rounded to a lower type),
// row-major with the panel rows K-contiguous; products and sums are in T.
// With `lower` set (a SYRK on a diagonal block, r0 == c0) only entries with
// r >= c are updated and tiles entirely above the diagonal are skipped.
// W and Op may be the same array: the columns written, [c0, c0 + N), and the
// columns read, [k0, k0 + K), are disjoint (the panel lies left of the block
// it updates, k0 + K <= c0), so no element is reached through both
// restrict-qualified pointers.
#pragma once
#include "common.cuh"

template <typename OpT> __device__ __forceinline__ float op_to_f(OpT v) { return (float)v; }
template <> __device__ __forceinline__ float op_to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float op_to_f<__half>(__half v) { return __half2float(v); }

template <typename T, typename OpT> __device__ __forceinline__ T op_load(const OpT* p) { return (T)op_to_f(*p); }
template <> __device__ __forceinline__ double op_load<double, double>(const double* p) { return *p; }

template <typename T, typename OpT, int TM, int TN, int BK>
__global__ void __launch_bounds__(256) k_gemm_nt_simt(T* __restrict__ W, long ldw, const OpT* __restrict__ Op,
                                                      long ldo, int r0, int M, int c0, int N, int k0, int K,
                                                      int lower, const DevStatus* st) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    __shared__ __align__(16) T As[2][BK][BM + 4];
    __shared__ __align__(16) T Bs[2][BK][BN + 4];
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;
    const int bm = blockIdx.y, bn = blockIdx.x;
    const int rbase = bm * BM, cbase = bn * BN;
    if (lower && (r0 + rbase + BM - 1 < c0 + cbase)) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    constexpr int A_PER = BM * BK / 256, B_PER = BN * BK / 256;
    T ra[A_PER], rb[B_PER];

    auto load_tiles = [&](int kt) {
#pragma unroll
        for (int t = 0; t < A_PER; ++t) {
            int e = tid + t * 256, row = e / BK, kk = e % BK;
            int gr = rbase + row, gk = kt + kk;
            ra[t] = (gr < M && gk < K) ? op_load<T, OpT>(Op + (long)(r0 + gr) * ldo + k0 + gk) : T(0);
        }
#pragma unroll
        for (int t = 0; t < B_PER; ++t) {
            int e = tid + t * 256, row = e / BK, kk = e % BK;
            int gc = cbase + row, gk = kt + kk;
            rb[t] = (gc < N && gk < K) ? op_load<T, OpT>(Op + (long)(c0 + gc) * ldo + k0 + gk) : T(0);
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int t = 0; t < A_PER; ++t) {
            int e = tid + t * 256, row = e / BK, kk = e % BK;
            As[buf][kk][row] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < B_PER; ++t) {
            int e = tid + t * 256, row = e / BK, kk = e % BK;
            Bs[buf][kk][row] = rb[t];
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    load_tiles(0);
    store_tiles(0);
    __syncthreads();
    int buf = 0;
    for (int kt = 0; kt < K; kt += BK) {
        const bool more = kt + BK < K;
        if (more) load_tiles(kt + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
        }
        if (more) {
            store_tiles(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gr = rbase + ty * TM + i;
        if (gr >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gc = cbase + tx * TN + j;
            if (gc >= N) continue;
            if (lower && (r0 + gr < c0 + gc)) continue;
            W[(long)(r0 + gr) * ldw + c0 + gc] -= acc[i][j];
        }
    }
}
