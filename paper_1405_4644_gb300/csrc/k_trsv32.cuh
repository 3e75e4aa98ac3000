// k_trsv32.cuh -- step A4 (Algorithm 1, lines 2 and 5): the float32
// triangular sweeps y = L^{-1} y (forward) and z = L^{-T} z (backward) over
// 128-row blocks, in one persistent cooperative kernel per sweep.
//
// Block J (in sweep order t) is owned by the CTA of rank t mod G among the G
// CTAs ordered by SM id, which takes its blocks in sweep order.
// Forward, with t_J = y_J - sum_{K < J-2} L_JK y_K and u_J = L_JJ^{-1} t_J,
//
//   y_J = u_J - P_J y_{J-2} - M_J y_{J-1},
//   M_J = L_JJ^{-1} L_{J,J-1},  P_J = L_JJ^{-1} L_{J,J-2},
//
// and backward, with v_J = L_JJ^{-T} (z_J - sum_{K > J+2} L_KJ^T z_K),
//
//   z_J = v_J - Q_J z_{J+2} - N_J z_{J+1},
//   N_J = L_JJ^{-T} L_{J+1,J}^T,  Q_J = L_JJ^{-T} L_{J+2,J}^T,
//
// the couplings being formed once per factor (k_trsv_couplings).  The far
// sum and the diagonal solve happen while the two nearest blocks are still
// being solved; once block J-2 is published one product is left before
// block J-1 can be taken, and one sweep step on the critical path is:
// acquire the neighbour's flag, one 128x128 by 128xMC product, publish.  The
// far contributions are summed in a fixed order (forward K = 0..J-3,
// backward K = NB-1..J+3); each waits with a bounded acquire-load of
// ready[K].  A wait that exceeds its limit raises SPD_DEV_TIMEOUT and the
// kernel winds down without publishing.
//
// Thread (i, h) (i = tid / 2, h = tid % 2) owns row i of the block and the
// half h of the reduction index: its 64 tile entries go from global memory
// straight into registers (double-buffered across tiles), the right-hand
// sides are broadcast from shared memory, and the two halves meet through a
// shuffle.
#pragma once
#include "common.cuh"

#define TV_LD 132

struct TrsvArgs {
    const float* W;      // factor rows (row-major, lower), ldw
    long ldw;
    int n, NB;
    const float* LinvT;  // per block: (L_JJ^{-1})^T, 128 x 128 row-major
    const float* Cpl;    // couplings: M_J, N_J, P_J, Q_J at (J, NB + J, 2 NB + J, 3 NB + J) * 16384
    float* Y;            // n x m, column-major (ld n), in place
    int c0, mc;          // columns [c0, c0 + mc) in this pass
    int* ready;          // NB flags
    int epoch;           // value that marks a block finished in this sweep
    DevStatus* st;
    unsigned long long* slots;  // one per CTA: (epoch << 32) | SM id of the CTA in this sweep
    unsigned long long wait_ns; // bound of every wait on another CTA's flag or slot
    const int* gate;            // (may be NULL) return at once when *gate == 0
    const int* epoch_base;      // (may be NULL) epoch = 2^30 + *epoch_base + epoch
};

// largest grid of the sweeps (CTAs), the size of the slot table
#define TV_SLOTS 1024

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t tv_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// row stride of the staged right-hand sides: the eight reduction slices read
// rows s + 8 l' (s = 0..7) in one instruction; with this stride those rows
// fall in distinct banks
template <int MC>
__host__ __device__ constexpr int tv_ys() { return MC >= 8 ? MC + 4 : MC; }

template <int MC>
constexpr size_t trsv32_smem() {
    return (size_t)(128 * TV_LD + 128 * tv_ys<MC>() + 128 * MC) * sizeof(float);
}

// ---------------------------------------------------------------------------
// couplings, once per factor
// ---------------------------------------------------------------------------
// Couplings at distance d = 1 (blockIdx.y 0, 1) and d = 2 (blockIdx.y 2, 3):
//   forward  (y even): C[i][l] = sum_k LinvT_J[k][i] L_{J,J-d}[k][l],  J = blockIdx.x + d
//            (M_J for d = 1, P_J for d = 2);
//   backward (y odd):  C[i][l] = sum_k LinvT_J[i][k] L_{J+d,J}[l][k],  J = blockIdx.x
//            (N_J for d = 1, Q_J for d = 2).
// Stored at Cpl + (y NB + J) 16384.  Rows of L past n are zero.  Thread: row
// i = tid / 2, columns 64 (tid % 2) + 0..63.
constexpr size_t trsv_couplings_smem() { return (size_t)(2 * 128 * 129) * sizeof(float); }

static __global__ void __launch_bounds__(256) k_trsv_couplings(const float* __restrict__ W, long ldw, int n, int NB,
                                                        const float* __restrict__ LinvT, float* __restrict__ Cpl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Li = reinterpret_cast<float*>(smem_raw);  // [128][129] LinvT_J
    float* Bt = Li + 128 * 129;                      // [128][129] Bt[k][l]
    const bool fwd = (blockIdx.y & 1) == 0;
    const int d = (int)(blockIdx.y >> 1) + 1;
    const int J = fwd ? (int)blockIdx.x + d : (int)blockIdx.x;
    if ((fwd ? J : J + d) > NB - 1) return;
    const int tid = threadIdx.x;
    const float* lg = LinvT + (long)J * 16384;
    for (int e = tid; e < 16384; e += 256) Li[(e >> 7) * 129 + (e & 127)] = lg[e];
    for (int e = tid; e < 16384; e += 256) {
        const int r = e >> 7, c = e & 127;
        if (fwd) {  // Bt[k][l] = L_{J,J-d}[k][l]: row J*128 + r, column (J-d)*128 + c
            const long gr = (long)J * 128 + r;
            Bt[r * 129 + c] = gr < n ? W[gr * ldw + (long)(J - d) * 128 + c] : 0.f;
        } else {    // Bt[k][l] = L_{J+d,J}[l][k]: row (J+d)*128 + r (= l), column J*128 + c (= k)
            const long gr = (long)(J + d) * 128 + r;
            Bt[c * 129 + r] = gr < n ? W[gr * ldw + (long)J * 128 + c] : 0.f;
        }
    }
    __syncthreads();
    const int i = tid >> 1, lb = (tid & 1) * 64;
    float acc[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) acc[q] = 0.f;
    for (int k = 0; k < 128; ++k) {
        const float a = fwd ? Li[k * 129 + i] : Li[i * 129 + k];
        const float* b = Bt + k * 129 + lb;
#pragma unroll
        for (int q = 0; q < 64; ++q) acc[q] = fmaf(a, b[q], acc[q]);
    }
    float* out = Cpl + ((long)(blockIdx.y * NB + J) * 128 + i) * 128 + lb;
#pragma unroll
    for (int q = 0; q < 64; q += 4) *reinterpret_cast<float4*>(out + q) = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
}

// ---------------------------------------------------------------------------
// the sweeps
// ---------------------------------------------------------------------------
// Wait (thread 0, bounded) until ready[K] carries this sweep's epoch; then
// the whole CTA may read block K.  Returns false once the CTA has given up.
__device__ __forceinline__ bool tv_wait(const TrsvArgs& a, int K, int* s_abort) {
    if (threadIdx.x == 0 && !*s_abort) {
        if (ld_acquire(a.ready + K) != a.epoch) {
            const uint64_t t0 = tv_globaltimer();
            while (ld_acquire(a.ready + K) != a.epoch) {
                if (tv_globaltimer() - t0 > a.wait_ns) {
                    *s_abort = 1;
                    atomicOr(&a.st->flags, SPD_DEV_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !*s_abort;
}

// Tile products use a 4-row register tile: thread (q, s) = (tid / 8, tid % 8)
// owns rows 4q..4q+3 of the block and the reduction slice l = s + 8 l'
// (l' = 0..15); each right-hand-side row read from shared memory feeds 4 MC
// multiply-adds, and the eight slices of a row quad (eight adjacent lanes)
// meet by shuffles.
//
// 64 tile entries into registers, v[j * 16 + l'] = entry (row 4q + j,
// column s + 8 l'): forward, rows of L_JK (eight adjacent lanes read 32
// contiguous bytes); backward, L_KJ^T, i.e. v[j * 16 + l'] =
// L_KJ[s + 8 l'][4 q + j] (float4 loads along a row of L_KJ).  Zero past n.
template <bool FWD>
__device__ __forceinline__ void tv_tile(float (&v)[64], const float* W, long ldw, int n, int J, int K, int q, int s) {
    if (FWD) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long gr = (long)J * 128 + 4 * q + j;
            const float* src = W + gr * ldw + (long)K * 128 + s;
#pragma unroll
            for (int l = 0; l < 16; ++l) v[j * 16 + l] = gr < n ? __ldg(src + 8 * l) : 0.f;
        }
    } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            const long gr = (long)K * 128 + s + 8 * l;
            const float4 t = gr < n ? __ldg(reinterpret_cast<const float4*>(W + gr * ldw + (long)J * 128 + 4 * q))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            v[l] = t.x;
            v[16 + l] = t.y;
            v[32 + l] = t.z;
            v[48 + l] = t.w;
        }
    }
}

// the coupling rows 4q..4q+3, slice s, of a row-major 128x128 matrix
__device__ __forceinline__ void tv_rows(float (&v)[64], const float* C, int q, int s) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float* src = C + (4 * q + j) * 128 + s;
#pragma unroll
        for (int l = 0; l < 16; ++l) v[j * 16 + l] = __ldg(src + 8 * l);
    }
}

// Yk[l][c] = Y[K*128 + l, c0 + c] (zero past n or past mc); all loads first
template <int MC>
__device__ __forceinline__ void tv_stage(float* Yk, const TrsvArgs& a, int K) {
    constexpr int PER = (128 * MC + 255) / 256;
    float v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
        const int r = K * 128 + l;
        v[u] = (e < 128 * MC && c < a.mc && r < a.n) ? __ldcg(a.Y + (long)(a.c0 + c) * a.n + r) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
        if (e < 128 * MC) Yk[l * tv_ys<MC>() + c] = v[u];
    }
}

// acc[j][c] += sum_l' v[j * 16 + l'] Yk[s + 8 l'][c]  (fully unrolled)
template <int MC>
__device__ __forceinline__ void tv_dot(float (&acc)[4][MC], const float (&v)[64], const float* Yk, int s) {
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        const float* y = Yk + (s + 8 * l) * tv_ys<MC>();
        float yv[MC];
        if constexpr (MC % 4 == 0) {
#pragma unroll
            for (int c = 0; c < MC; c += 4) {
                const float4 t = *reinterpret_cast<const float4*>(y + c);
                yv[c] = t.x;
                yv[c + 1] = t.y;
                yv[c + 2] = t.z;
                yv[c + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < MC; ++c) yv[c] = y[c];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[j][c] = fmaf(v[j * 16 + l], yv[c], acc[j][c]);
    }
}

// sum over the eight reduction slices (adjacent lanes): every lane of the
// group ends with the total
template <int MC>
__device__ __forceinline__ void tv_reduce8(float (&acc)[4][MC]) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < MC; ++c) {
            float x = acc[j][c];
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            x += __shfl_xor_sync(0xffffffffu, x, 4);
            acc[j][c] = x;
        }
}

template <int MC, bool FWD>
__global__ void __launch_bounds__(256, 1) k_trsv32(TrsvArgs a) {
    constexpr int CPT = MC >= 2 ? MC / 2 : 1;  // columns per thread in the diagonal step
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Lv = reinterpret_cast<float*>(smem_raw);  // [128][TV_LD] (L_JJ^{-1})^T
    float* Yk = Lv + 128 * TV_LD;                    // [128][tv_ys] right-hand sides of a finished block
    float* T = Yk + 128 * tv_ys<MC>();               // [128][MC] t_J, then u_J
    __shared__ int s_abort, s_rank;
    __shared__ unsigned s_sm;
    const int tid = threadIdx.x;
    const int tq = tid >> 3, ts = tid & 7;            // tile products: row quad, reduction slice
    const int i = tid >> 1, half = tid & 1;           // diagonal step: row, column half
    const int cbase = (MC >= 2) ? half * CPT : 0;
    // a capturable solve: nothing to do once its refinement is over, and the
    // epoch comes from the device counter the solve advanced (every CTA reads
    // the same values: both were written by earlier kernels in the stream)
    if (a.gate && *a.gate == 0) return;
    if (a.epoch_base) a.epoch += (1 << 30) + *a.epoch_base;
    if (tid == 0) {
        s_abort = 0;
        s_rank = 0;
        unsigned sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        s_sm = sm;
        st_release64(a.slots + blockIdx.x, ((unsigned long long)(unsigned)a.epoch << 32) | sm);
    }
    __syncthreads();
    // This CTA's rank among all CTAs ordered by SM id: blocks go to ranks in
    // sweep order, so consecutive blocks mostly run on neighbouring SMs (the
    // same TPC or GPC), where handing a finished block over is several times
    // faster than across the chip.  Every CTA is resident (cooperative
    // launch); the wait for the others' slots is bounded.
    {
        int before = 0;
        for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
            unsigned long long v = ld_acquire64(a.slots + b);
            if ((unsigned)(v >> 32) != (unsigned)a.epoch) {
                const uint64_t t0 = tv_globaltimer();
                while ((unsigned)((v = ld_acquire64(a.slots + b)) >> 32) != (unsigned)a.epoch) {
                    if (tv_globaltimer() - t0 > a.wait_ns) {
                        s_abort = 1;
                        atomicOr(&a.st->flags, SPD_DEV_TIMEOUT);
                        break;
                    }
                }
            }
            const unsigned smb = (unsigned)v;
            before += (smb < s_sm || (smb == s_sm && b < (int)blockIdx.x)) ? 1 : 0;
        }
        if (before) atomicAdd(&s_rank, before);
    }
    __syncthreads();
    if (s_abort) return;
    const int rank = s_rank;

    for (int t = rank; t < a.NB; t += gridDim.x) {
        const int J = FWD ? t : a.NB - 1 - t;
        const int nfar = FWD ? max(J - 2, 0) : max(a.NB - 3 - J, 0);
        const bool near = FWD ? J >= 1 : J <= a.NB - 2;   // a neighbour at distance 1
        const bool near2 = FWD ? J >= 2 : J <= a.NB - 3;  // and at distance 2
        float ra[64], rb[64];
        {  // (L_JJ^{-1})^T depends on no other block: into shared memory first
            const float4* src = reinterpret_cast<const float4*>(a.LinvT + (long)J * 16384);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = tid + u * 256, r = e >> 5, c4 = (e & 31) * 4;
                *reinterpret_cast<float4*>(Lv + r * TV_LD + c4) = __ldg(src + e);
            }
        }
        float acc[4][MC];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[j][c] = 0.f;
        // far contributions, two tiles per trip so that the register buffers
        // alternate without copies
        if (nfar > 0) tv_tile<FWD>(ra, a.W, a.ldw, a.n, J, FWD ? 0 : a.NB - 1, tq, ts);
        for (int q = 0; q < nfar; q += 2) {
            const int K = FWD ? q : a.NB - 1 - q;
            if (!tv_wait(a, K, &s_abort)) break;
            tv_stage<MC>(Yk, a, K);
            __syncthreads();
            if (q + 1 < nfar) tv_tile<FWD>(rb, a.W, a.ldw, a.n, J, FWD ? q + 1 : a.NB - 2 - q, tq, ts);
            tv_dot<MC>(acc, ra, Yk, ts);
            __syncthreads();
            if (q + 1 >= nfar) break;
            const int K1 = FWD ? q + 1 : a.NB - 2 - q;
            if (!tv_wait(a, K1, &s_abort)) break;
            tv_stage<MC>(Yk, a, K1);
            __syncthreads();
            if (q + 2 < nfar) tv_tile<FWD>(ra, a.W, a.ldw, a.n, J, FWD ? q + 2 : a.NB - 3 - q, tq, ts);
            tv_dot<MC>(acc, rb, Yk, ts);
            __syncthreads();
        }
        if (s_abort) break;
        // the coupling rows for the last two products do not depend on
        // anything still outstanding: start the first one's loads now
        const float* cp1 = a.Cpl + (long)(FWD ? J : a.NB + J) * 16384;           // M_J or N_J
        const float* cp2 = a.Cpl + (long)(FWD ? 2 * a.NB + J : 3 * a.NB + J) * 16384;  // P_J or Q_J
        if (near2) tv_rows(rb, cp2, tq, ts);
        else if (near) tv_rows(ra, cp1, tq, ts);
        tv_reduce8<MC>(acc);
        // t = y_J - far sum (this CTA is the only writer of block J)
        if (ts == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = J * 128 + 4 * tq + j;
#pragma unroll
                for (int c = 0; c < MC; ++c) {
                    const float y = (c < a.mc && r < a.n) ? __ldcg(a.Y + (long)(a.c0 + c) * a.n + r) : 0.f;
                    T[(4 * tq + j) * MC + c] = y - acc[j][c];
                }
            }
        }
        __syncthreads();
        // u = L_JJ^{-1} t (forward) or L_JJ^{-T} t (backward), CPT columns
        float out[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) out[c] = 0.f;
        if (MC >= 2) {
            if (FWD) {  // u[i] = sum_{l<=i} LinvT[l][i] t[l]
                for (int l = 0; l <= i; ++l) {
                    const float w = Lv[l * TV_LD + i];
#pragma unroll
                    for (int c = 0; c < CPT; ++c) out[c] = fmaf(w, T[l * MC + cbase + c], out[c]);
                }
            } else {    // u[i] = sum_{l>=i} LinvT[i][l] t[l]
                const float* lr = Lv + i * TV_LD;
                for (int l = i; l < 128; ++l) {
                    const float w = lr[l];
#pragma unroll
                    for (int c = 0; c < CPT; ++c) out[c] = fmaf(w, T[l * MC + cbase + c], out[c]);
                }
            }
        } else {  // one column: the two threads of a row split l
            const int l0 = half * 64, l1 = l0 + 64;
            if (FWD) {
                for (int l = l0; l < min(l1, i + 1); ++l) out[0] = fmaf(Lv[l * TV_LD + i], T[l], out[0]);
            } else {
                const float* lr = Lv + i * TV_LD;
                for (int l = max(l0, i); l < l1; ++l) out[0] = fmaf(lr[l], T[l], out[0]);
            }
            out[0] += __shfl_xor_sync(0xffffffffu, out[0], 1);
        }
        __syncthreads();  // every read of t done: T now takes u
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (half == 0 || MC >= 2) T[i * MC + cbase + c] = out[c];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[j][c] = 0.f;
        if (near2) {  // the neighbour at distance 2: acc = P_J y_{J-2} (Q_J z_{J+2})
            tv_rows(ra, cp1, tq, ts);
            const int K2 = FWD ? J - 2 : J + 2;
            if (!tv_wait(a, K2, &s_abort)) break;  // (its barrier also publishes u)
            tv_stage<MC>(Yk, a, K2);
            __syncthreads();
            tv_dot<MC>(acc, rb, Yk, ts);
        }
        if (near) {  // the step on the critical path: y_J = u - acc - C_J y_neighbour
            const int Kn = FWD ? J - 1 : J + 1;
            if (!tv_wait(a, Kn, &s_abort)) break;  // (its barrier also publishes u)
            tv_stage<MC>(Yk, a, Kn);
            __syncthreads();
            tv_dot<MC>(acc, ra, Yk, ts);
            tv_reduce8<MC>(acc);
        } else {
            __syncthreads();
        }
        if (ts == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = J * 128 + 4 * tq + j;
#pragma unroll
                for (int c = 0; c < MC; ++c)
                    if (c < a.mc && r < a.n) a.Y[(long)(a.c0 + c) * a.n + r] = T[(4 * tq + j) * MC + c] - acc[j][c];
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(a.ready + J, a.epoch);
    }
}
