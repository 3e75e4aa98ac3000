// k_trsv32.cuh -- step A4 (Algorithm 1, lines 2 and 5): the float32
// triangular sweeps y = L^{-1} y (forward) and z = L^{-T} z (backward) over
// 128-row blocks, in one persistent cooperative kernel per sweep.
//
// Block J is owned by CTA J mod G.  Its owner accumulates the contributions
// of the finished blocks in a fixed order (forward: K = 0..J-1 with
// L_JK y_K; backward: K = NB-1..J+1 with L_KJ^T z_K), waiting for each with a
// bounded acquire-load of ready[K], then finishes the block with the full
// inverse of the diagonal block (y_J = L_JJ^{-1} t, z_J = L_JJ^{-T} t) and
// publishes it with a release-store.  Owners take their blocks in sweep
// order, so a wait only ever targets an earlier block; the cooperative
// launch keeps all CTAs resident.  A wait that exceeds its limit raises
// SPD_DEV_TIMEOUT and the kernel winds down without publishing.
#pragma once
#include "common.cuh"

#define TV_LD 129

struct TrsvArgs {
    const float* W;      // factor rows (row-major, lower), ldw
    long ldw;
    int n, NB;
    const float* LinvT;  // per block: (L_JJ^{-1})^T, 128 x 128 row-major
    float* Y;            // n x m, column-major (ld n), in place
    int c0, mc;          // columns [c0, c0 + mc) in this pass
    int* ready;          // NB flags
    int epoch;           // value that marks a block finished in this sweep
    DevStatus* st;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t tv_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int MC>
constexpr size_t trsv32_smem() {
    return (size_t)(2 * 128 * TV_LD + 2 * 128 * MC) * sizeof(float);
}

// 128 x 128 tile (rows trow, columns tcol of L, zero outside the matrix) into
// 16 float4 registers per thread: every load is issued before any use.
__device__ __forceinline__ void tile_ld(float4* v, const TrsvArgs& a, int trow, int tcol) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * 256, r = e >> 5, c4 = (e & 31) * 4;
        const int gr = trow * 128 + r, gc = tcol * 128 + c4;
        v[q] = (gr < a.n && gc < a.n) ? *reinterpret_cast<const float4*>(a.W + (long)gr * a.ldw + gc)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        if (gc + 3 >= a.n) {  // columns past n hold scratch (ldw > n): zero them
            if (gc + 1 >= a.n) v[q].y = 0.f;
            if (gc + 2 >= a.n) v[q].z = 0.f;
            v[q].w = 0.f;
        }
    }
}
__device__ __forceinline__ void tile_ld_contig(float4* v, const float* src) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * 256;
        v[q] = reinterpret_cast<const float4*>(src)[e];
    }
}
__device__ __forceinline__ void tile_st(const float4* v, float* Ls) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int e = threadIdx.x + q * 256, r = e >> 5, c4 = (e & 31) * 4;
        float* d = Ls + r * TV_LD + c4;
        d[0] = v[q].x;
        d[1] = v[q].y;
        d[2] = v[q].z;
        d[3] = v[q].w;
    }
}

// acc[0..CPT) += x * p[0..CPT)  with vector shared-memory loads
template <int CPT>
__device__ __forceinline__ void axpy_row(float* acc, float x, const float* p) {
    if constexpr (CPT % 4 == 0) {
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(p)[q];
            acc[4 * q + 0] = fmaf(x, v.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(x, v.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(x, v.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(x, v.w, acc[4 * q + 3]);
        }
    } else if constexpr (CPT == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        acc[0] = fmaf(x, v.x, acc[0]);
        acc[1] = fmaf(x, v.y, acc[1]);
    } else {
        acc[0] = fmaf(x, p[0], acc[0]);
    }
}

template <int MC, bool FWD>
__global__ void __launch_bounds__(256, 1) k_trsv32(TrsvArgs a) {
    constexpr int LY = MC;                       // unpadded rows: vector reads of a thread's columns
    constexpr int CPT = MC >= 2 ? MC / 2 : 1;    // columns per thread
    constexpr int LSPLIT = MC >= 2 ? 1 : 2;      // the two threads of a row split l when MC == 1
    constexpr int YPT = (128 * MC + 255) / 256;  // y elements loaded per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Ls = reinterpret_cast<float*>(smem_raw);  // [128][129] L tile of the current contribution
    float* Lv = Ls + 128 * TV_LD;                    // [128][129] (L_JJ^{-1})^T
    float* Yk = Lv + 128 * TV_LD;                    // [128][MC]
    float* T = Yk + 128 * LY;                        // [128][MC]
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int i = tid >> 1, half = tid & 1;
    const int cbase = (MC >= 2) ? half * CPT : 0;
    const int l0 = (LSPLIT == 2) ? half * 64 : 0, l1 = (LSPLIT == 2) ? l0 + 64 : 128;
    if (tid == 0) s_abort = 0;
    __syncthreads();

    for (int t = blockIdx.x; t < a.NB; t += gridDim.x) {
        const int J = FWD ? t : a.NB - 1 - t;
        const int kcount = FWD ? J : a.NB - 1 - J;
        float4 pre[16];
        {  // (L_JJ^{-1})^T does not depend on any other block: fetch it first
            tile_ld_contig(pre, a.LinvT + (long)J * 128 * 128);
            tile_st(pre, Lv);
        }
        if (kcount > 0) {
            const int K = FWD ? 0 : a.NB - 1;
            tile_ld(pre, a, FWD ? J : K, FWD ? K : J);
        }
        float acc[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c] = 0.f;
        for (int q = 0; q < kcount; ++q) {
            const int K = FWD ? q : a.NB - 1 - q;
            if (tid == 0 && !s_abort) {
                if (ld_acquire(a.ready + K) != a.epoch) {
                    const uint64_t t0 = tv_globaltimer();
                    while (ld_acquire(a.ready + K) != a.epoch) {
                        __nanosleep(20);
                        if (tv_globaltimer() - t0 > 1000000000ull) {
                            s_abort = 1;
                            atomicOr(&a.st->flags, SPD_DEV_TIMEOUT);
                            break;
                        }
                    }
                }
                __threadfence();
            }
            __syncthreads();
            if (s_abort) break;
            float yv[YPT];
#pragma unroll
            for (int u = 0; u < YPT; ++u) {
                const int e = tid + u * 256, l = e & 127, c = e >> 7;
                const int r = K * 128 + l;
                yv[u] = (e < 128 * MC && c < a.mc && r < a.n) ? __ldcg(a.Y + (long)(a.c0 + c) * a.n + r) : 0.f;
            }
            tile_st(pre, Ls);
#pragma unroll
            for (int u = 0; u < YPT; ++u) {
                const int e = tid + u * 256, l = e & 127, c = e >> 7;
                if (e < 128 * MC) Yk[l * LY + c] = yv[u];
            }
            __syncthreads();
            if (q + 1 < kcount) {  // next tile in flight while this one is used
                const int Kn = FWD ? q + 1 : a.NB - 2 - q;
                tile_ld(pre, a, FWD ? J : Kn, FWD ? Kn : J);
            }
            if (FWD) {  // acc[c] += sum_l L_JK[i][l] y_K[l][c]
                const float* lr = Ls + i * TV_LD;
#pragma unroll 4
                for (int l = l0; l < l1; ++l) axpy_row<CPT>(acc, lr[l], Yk + l * LY + cbase);
            } else {  // acc[c] += sum_r L_KJ[r][i] z_K[r][c]
#pragma unroll 4
                for (int r = l0; r < l1; ++r) axpy_row<CPT>(acc, Ls[r * TV_LD + i], Yk + r * LY + cbase);
            }
            __syncthreads();
        }
        if (s_abort) break;
        if (LSPLIT == 2) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
        }
        // t = y_J - acc  (this CTA is the only writer of block J)
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int cc = cbase + c;
            const int r = J * 128 + i;
            if (half == 0 || MC >= 2) {
                float y = (cc < a.mc && r < a.n) ? __ldcg(a.Y + (long)(a.c0 + cc) * a.n + r) : 0.f;
                T[i * LY + cc] = y - acc[c];
            }
        }
        __syncthreads();
        float out[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[c] = 0.f;
        if (FWD) {  // y[i] = sum_{l<=i} Linv[i][l] t[l] = sum_l LinvT[l][i] t[l]
            const int lend = (LSPLIT == 2) ? min(l1, i + 1) : i + 1;
            for (int l = l0; l < lend; ++l) axpy_row<CPT>(out, Lv[l * TV_LD + i], T + l * LY + cbase);
        } else {  // z[i] = sum_{l>=i} Linv[l][i] t[l] = sum_l LinvT[i][l] t[l]
            const int lbeg = (LSPLIT == 2) ? max(l0, i) : i;
            const float* lr = Lv + i * TV_LD;
            for (int l = lbeg; l < l1; ++l) axpy_row<CPT>(out, lr[l], T + l * LY + cbase);
        }
        if (LSPLIT == 2) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) out[c] += __shfl_xor_sync(0xffffffffu, out[c], 1);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int cc = cbase + c;
            const int r = J * 128 + i;
            if ((half == 0 || MC >= 2) && cc < a.mc && r < a.n) a.Y[(long)(a.c0 + cc) * a.n + r] = out[c];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.ready + J, a.epoch);
    }
}
