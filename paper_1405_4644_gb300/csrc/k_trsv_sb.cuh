// k_trsv_sb.cuh -- step A4 (Algorithm 1, lines 2 and 5) over diagonal
// super-blocks: the float32 sweeps y = L^{-1} y and z = L^{-T} z with the
// explicit inverses X_I = L_II^{-1} of the diagonal super-blocks (SBB
// 128-blocks each, S = 128 SBB rows), formed once per factor.
//
// Forward, super-block by super-block (I = 0, 1, ...):
//   y_I = X_I r_I,   then   r_J -= L_JI y_I  for every 128-row block J below,
// backward (I = last, ..., 0):
//   z_I = X_I^T y_I, then   y_K -= L_IK^T z_I  for every 128-row block K above,
// i.e. block substitution with the diagonal solve replaced by a product with
// the inverse.  One persistent cooperative kernel per sweep runs three
// grid-wide phases per super-block, separated by bounded grid barriers:
//   F   the SBB (SBB + 1) / 2 tile products X_I[b][c] r_I[c] (c <= b; for the
//       backward sweep X_I[c][b]^T r_I[c], c >= b) into partial tiles; the
//       last tile of block row b to arrive (an atomic count) adds the row's
//       partials in a fixed order into y_I[b], written to the output vector
//       (never over r_I, which other tiles of the phase may still read); and
//       the fix-up of the previous panel update's split rows (below);
//   B   the panel update: units (J, c) = the tile L_{J, I c} (backward
//       L_{I c, J}^T) times y_I[c], J-major over every remaining 128-row block
//       J, in equal contiguous ranges over all CTAs ("stream-K"), so the
//       panel of L streams through every SM.  A CTA whose range covers a
//       whole block row subtracts its sum from r_J; the pieces of a row shared
//       by several CTAs go to partial slots (2g for CTA g's first piece, 2g+1
//       for its last), which the next phase F adds in CTA order (= c order):
//       folded into the staged rows of the next super-block's tile products,
//       subtracted from r_J for every other row.
// Every result is formed in an order fixed by the launch's grid, not by
// timing.  The chain of the 128-block sweeps (one cross-SM hand-over per 128
// rows) becomes two barriers per S rows.  The right-hand sides Y are reduced
// in place and the result goes to O (forward: Y = the caller's vectors, O =
// scratch; backward: Y = that scratch, O = the caller's vectors).  The product of a 128x128 tile
// with a 128 x MC block uses the register tiles of k_trsv32.cuh.
#pragma once
#include "k_trsv32.cuh"

struct SbArgs {
    const float* W;       // factor rows (row-major, lower), ldw
    long ldw;
    int n, NB;            // order and number of 128-blocks
    const float* X;       // super-block inverses: NS blocks of S x S floats, row-major
    int S, SBB, NS;       // super-block order (= 128 SBB), 128-blocks per super-block, super-blocks
    float* Y;             // right-hand sides, n x m column-major (ld n), reduced in place
    int c0, mc;           // columns [c0, c0 + mc) of Y in this pass
    float* O;             // the sweep's result, column-major (ld n), columns [oc0, oc0 + mc)
    int oc0;
    float* P;             // partial tiles of phase F: SBB (SBB + 1) / 2 x 128 x MC floats
    float* P2;            // partial slots of phase B: 2 gridDim.x x 128 x MC floats
    int* bar;             // [0] barrier arrivals, [1] abort, then NS SBB block-row tile counts (zero at launch)
    unsigned long long wait_ns;
    DevStatus* st;
    const int* gate;      // (may be NULL) return at once when *gate == 0
};

// Grid-wide barrier: the k-th barrier of a launch waits for k * gridDim.x
// arrivals (bounded; a CTA that gives up raises SPD_DEV_TIMEOUT and the abort
// flag, which releases the others).  Every write before it is visible after.
__device__ __forceinline__ bool sb_barrier(const SbArgs& a, int k, int* s_abort) {
    __syncthreads();
    if (threadIdx.x == 0 && !*s_abort) {
        __threadfence();
        atomicAdd(a.bar, 1);
        const int target = k * (int)gridDim.x;
        if (ld_acquire(a.bar) < target) {
            const uint64_t t0 = tv_globaltimer();
            while (ld_acquire(a.bar) < target) {
                if (ld_acquire(a.bar + 1)) {
                    *s_abort = 1;
                    break;
                }
                if (tv_globaltimer() - t0 > a.wait_ns) {
                    *s_abort = 1;
                    atomicOr(&a.st->flags, SPD_DEV_TIMEOUT);
                    atomicExch(a.bar + 1, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return !*s_abort;
}

// Geometry of one panel update (phase B): units u = (J - J0) nb + c for
// J0 <= J < J0 + rows, c < nb; CTA g < geff takes [g W / geff, (g+1) W / geff).
struct SbPanel {
    int J0, nb, geff;
    long W;
};
__device__ __forceinline__ long sb_ub(int g, long W, int G) { return (long)g * W / G; }

// The partial slots of block row J of panel pn in CTA order (= c order):
// returns their count (0: one CTA covered the row, nothing pending); slots
// are slot_lo, 2 (glo + 1), ..., 2 ghi.
__device__ __forceinline__ int sb_row_slots(const SbPanel& pn, int J, int& slot_lo, int& glo) {
    const long ut0 = (long)(J - pn.J0) * pn.nb, ut1 = ut0 + pn.nb;
    glo = (int)(((ut0 + 1) * pn.geff - 1) / pn.W);  // owner of the row's first unit
    const int ghi = (int)((ut1 * pn.geff - 1) / pn.W);
    if (glo == ghi) return 0;
    slot_lo = 2 * glo + (sb_ub(glo, pn.W, pn.geff) < ut0 ? 1 : 0);
    return ghi - glo + 1;
}

// Block row J's pending partial sum, for this thread's elements e = tid +
// 256 u (row l = e & 127, column c = e >> 7): the row's slots added in CTA
// order, each slot's loads issued together.
template <int MC, int PER>
__device__ __forceinline__ void sb_pending(const SbArgs& a, int ns, int slot_lo, int glo, float (&pend)[PER]) {
#pragma unroll
    for (int u = 0; u < PER; ++u) pend[u] = 0.f;
    for (int k = 0; k < ns; ++k) {
        const float* ps = a.P2 + (long)(k == 0 ? slot_lo : 2 * (glo + k)) * 128 * MC;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
            if (e < 128 * MC) pend[u] += __ldcg(ps + l * MC + c);
        }
    }
}

// Yk[l][c] = Y[r0 + l, c0 + c] (zero past n or past mc), minus the block
// row's pending partial sum when ns > 0
template <int MC>
__device__ __forceinline__ void sb_stage(float* Yk, const SbArgs& a, long r0, int ns = 0, int slot_lo = 0,
                                         int glo = 0) {
    constexpr int PER = (128 * MC + 255) / 256;
    float v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
        const long r = r0 + l;
        v[u] = (e < 128 * MC && c < a.mc && r < a.n) ? __ldcg(a.Y + (long)(a.c0 + c) * a.n + r) : 0.f;
    }
    if (ns > 0) {
        float pend[PER];
        sb_pending<MC>(a, ns, slot_lo, glo, pend);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
            if (e < 128 * MC && c < a.mc && r0 + l < a.n) v[u] -= pend[u];
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * 256, l = e & 127, c = e >> 7;
        if (e < 128 * MC) Yk[l * tv_ys<MC>() + c] = v[u];
    }
}

// Blocks [cs0, cs1) of y_I (from the output vector O) into YI (block c at
// YI + c 128 tv_ys), loads issued eight per thread at a time
template <int MC>
__device__ __forceinline__ void sb_stage_range(float* YI, const SbArgs& a, int jb0, int cs0, int cs1) {
    constexpr int BATCH = 8;
    const int total = (cs1 - cs0) * 128 * MC;
    for (int base = threadIdx.x; base < total; base += 256 * BATCH) {
        float v[BATCH];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int e = base + k * 256;
            v[k] = 0.f;
            if (e < total) {
                const int blk = cs0 + e / (128 * MC), rem = e - (blk - cs0) * 128 * MC;
                const int l = rem & 127, c = rem >> 7;
                const long row = (long)(jb0 + blk) * 128 + l;
                if (c < a.mc && row < a.n) v[k] = __ldcg(a.O + (long)(a.oc0 + c) * a.n + row);
            }
        }
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int e = base + k * 256;
            if (e < total) {
                const int blk = cs0 + e / (128 * MC), rem = e - (blk - cs0) * 128 * MC;
                YI[(blk * 128 + (rem & 127)) * tv_ys<MC>() + (rem >> 7)] = v[k];
            }
        }
    }
}

// Prefetch into L2 the 128 x 128 tile at rows r0.., columns k0.. of a
// row-major float matrix (ld floats, rows < nrows): 512 lines of 128 bytes,
// two per thread.  Nothing waits for it; the later loads find the lines in L2.
__device__ __forceinline__ void sb_prefetch_tile(const float* M, long ld, long nrows, long r0, long k0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int line = threadIdx.x + k * 256, r = line >> 2, part = line & 3;
        if (r0 + r < nrows) {
            const float* ptr = M + (r0 + r) * ld + k0 + part * 32;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
        }
    }
}

// The tile of unit u of panel pn (forward L_{J, jb0 + c}, backward
// L_{jb0 + c, J}), prefetched
template <bool FWD>
__device__ __forceinline__ void sb_prefetch_unit(const SbArgs& a, const SbPanel& pn, int jb0, long u) {
    const int J = pn.J0 + (int)(u / pn.nb), K = jb0 + (int)(u % pn.nb);
    if (FWD) sb_prefetch_tile(a.W, a.ldw, a.n, (long)J * 128, (long)K * 128);
    else sb_prefetch_tile(a.W, a.ldw, a.n, (long)K * 128, (long)J * 128);
}

// shared memory: y_I of one super-block (SPD_SB_BLOCKS staged 128 x MC blocks)
template <int MC>
constexpr size_t trsv_sb_smem() {
    return (size_t)SPD_SB_BLOCKS * 128 * tv_ys<MC>() * sizeof(float);
}

// tile index of the pair (p, q), q <= p, in the order (0,0), (1,0), (1,1), ...
__device__ __forceinline__ int sb_tri(int p, int q) { return p * (p + 1) / 2 + q; }

template <int MC, bool FWD>
__global__ void __launch_bounds__(256, 1) k_trsv_sb(SbArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* YI = reinterpret_cast<float*>(smem_raw);  // [SBB][128][tv_ys] staged blocks of y_I (F: one)
    constexpr int YB = 128 * tv_ys<MC>();           // floats per staged block
    __shared__ int s_abort, s_last;
    if (a.gate && *a.gate == 0) return;  // refinement over (capturable solves)
    const int tid = threadIdx.x;
    const int tq = tid >> 3, ts = tid & 7;
    const int G = gridDim.x, g = blockIdx.x;
    if (tid == 0) s_abort = 0;
    __syncthreads();
    int nbar = 0;
    float ra[64], rb[64];
    SbPanel prev{0, 1, 1, 0};  // the previous step's panel update (W = 0: none)
    for (int t = 0; t < a.NS; ++t) {
        const int I = FWD ? t : a.NS - 1 - t;
        const int jb0 = I * a.SBB;                    // first 128-block of the super-block
        const int nb = min(a.SBB, a.NB - jb0);        // its 128-blocks
        const float* XI = a.X + (long)I * a.S * a.S;  // its inverse, S x S row-major
        // F: partial tiles, and the previous panel's split rows outside this
        // super-block (forward: below it; backward: above it)
        const int ntile = nb * (nb + 1) / 2;
        const int nfix = prev.W == 0 ? 0 : (FWD ? a.NB - (jb0 + nb) : jb0);
        for (int task = g; task < ntile + nfix; task += G) {
            if (task >= ntile) {
                const int J = FWD ? jb0 + nb + (task - ntile) : task - ntile;
                int slot_lo, glo;
                const int ns = sb_row_slots(prev, J, slot_lo, glo);
                if (ns == 0) continue;  // block-uniform
                constexpr int PER = (128 * MC + 255) / 256;
                float pend[PER];
                sb_pending<MC>(a, ns, slot_lo, glo, pend);
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int e = tid + u * 256, l = e & 127, cc = e >> 7;
                    const long row = (long)J * 128 + l;
                    if (e < 128 * MC && cc < a.mc && row < a.n) {
                        float* y = a.Y + (long)(a.c0 + cc) * a.n + row;
                        *y = __ldcg(y) - pend[u];
                    }
                }
                continue;
            }
            int p = 0;
            while (sb_tri(p + 1, 0) <= task) ++p;
            const int q = task - sb_tri(p, 0);  // q <= p
            // forward: X[b][c] with b = p, c = q; backward: X[c][b]^T with b = q, c = p
            const int b = FWD ? p : q, c = FWD ? q : p;
            tv_tile<FWD>(ra, XI, a.S, a.S, b, c, tq, ts);
            int slot_lo = 0, glo = 0;
            const int ns = prev.W == 0 ? 0 : sb_row_slots(prev, jb0 + c, slot_lo, glo);
            sb_stage<MC>(YI, a, (long)(jb0 + c) * 128, ns, slot_lo, glo);
            __syncthreads();
            float acc[4][MC];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int cc = 0; cc < MC; ++cc) acc[j][cc] = 0.f;
            tv_dot<MC>(acc, ra, YI, ts);
            tv_reduce8<MC>(acc);
            if (ts == 0) {
                float* pt = a.P + (long)task * 128 * MC;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int cc = 0; cc < MC; ++cc) pt[(4 * tq + j) * MC + cc] = acc[j][cc];
            }
            __syncthreads();
            // the last tile of block row b to arrive adds the row's partials
            // in c order (forward c = 0..b, backward c = b..nb-1) into y_I[b]
            // in O, all of a thread's loads in flight together
            if (tid == 0) {
                __threadfence();
                const int cnt = FWD ? b + 1 : nb - b;
                s_last = atomicAdd(a.bar + 2 + t * a.SBB + b, 1) == cnt - 1;
                __threadfence();
            }
            __syncthreads();
            if (s_last) {
                constexpr int EPT = (128 * MC + 255) / 256;
                float v[SPD_SB_BLOCKS][EPT];
#pragma unroll
                for (int k = 0; k < SPD_SB_BLOCKS; ++k)
#pragma unroll
                    for (int i = 0; i < EPT; ++i) {
                        const int e = tid + 256 * i, c2 = FWD ? k : b + k;
                        const bool in = (FWD ? k <= b : c2 < nb) && e < 128 * MC;
                        v[k][i] = in ? __ldcg(a.P + (long)(FWD ? sb_tri(b, c2) : sb_tri(c2, b)) * 128 * MC + e) : 0.f;
                    }
#pragma unroll
                for (int i = 0; i < EPT; ++i) {
                    const int e = tid + 256 * i, r = e / MC, cc = e - r * MC;
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < SPD_SB_BLOCKS; ++k)
                        if (FWD ? k <= b : b + k < nb) s += v[k][i];
                    const long row = (long)(jb0 + b) * 128 + r;
                    if (e < 128 * MC && cc < a.mc && row < a.n) a.O[(long)(a.oc0 + cc) * a.n + row] = s;
                }
            }
        }
        if (t + 1 == a.NS) break;  // no rows left to update
        if (!sb_barrier(a, ++nbar, &s_abort)) return;
        // B: units (J, c) of every remaining 128-row block J (forward: below
        // the super-block, backward: above it), in equal ranges over the CTAs
        SbPanel pn;
        pn.J0 = FWD ? jb0 + nb : 0;
        pn.nb = nb;
        pn.W = (long)((FWD ? a.NB : jb0) - pn.J0) * nb;
        pn.geff = (int)min((long)G, pn.W);
        if (g < pn.geff) {
            const long u0 = sb_ub(g, pn.W, pn.geff), u1 = sb_ub(g + 1, pn.W, pn.geff);
            // the blocks of y_I this CTA's units multiply, staged once
            const bool all = (u1 - u0 >= nb) || (u0 / nb != (u1 - 1) / nb);
            const int cs0 = all ? 0 : (int)(u0 % nb), cs1 = all ? nb : (int)((u1 - 1) % nb) + 1;
            for (long v = u0; v < min(u1, u0 + 2); ++v) sb_prefetch_unit<FWD>(a, pn, jb0, v);
            sb_stage_range<MC>(YI, a, jb0, cs0, cs1);
            __syncthreads();
            for (long u = u0; u < u1;) {
                const int J = pn.J0 + (int)(u / nb), ca = (int)(u % nb);
                const int ce = (int)min((long)nb, ca + (u1 - u));
                float acc[4][MC];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int cc = 0; cc < MC; ++cc) acc[j][cc] = 0.f;
                // tiles L_{J, jb0 + c} (forward) or L_{jb0 + c, J}^T (backward),
                // two per trip so that the register buffers alternate: the
                // next tile's loads are in flight during this tile's products
                // (tiles two units ahead, across pieces, are prefetched into L2)
                tv_tile<FWD>(ra, a.W, a.ldw, a.n, J, jb0 + ca, tq, ts);
                for (int c = ca; c < ce; c += 2) {
                    const long uc = u + (c - ca);
                    if (uc + 2 < u1) sb_prefetch_unit<FWD>(a, pn, jb0, uc + 2);
                    if (c + 1 < ce) tv_tile<FWD>(rb, a.W, a.ldw, a.n, J, jb0 + c + 1, tq, ts);
                    tv_dot<MC>(acc, ra, YI + c * YB, ts);
                    if (c + 1 >= ce) break;
                    if (uc + 3 < u1) sb_prefetch_unit<FWD>(a, pn, jb0, uc + 3);
                    if (c + 2 < ce) tv_tile<FWD>(ra, a.W, a.ldw, a.n, J, jb0 + c + 2, tq, ts);
                    tv_dot<MC>(acc, rb, YI + (c + 1) * YB, ts);
                }
                tv_reduce8<MC>(acc);
                if (ts == 0) {
                    if (ca == 0 && ce == nb) {  // the whole row: subtract in place
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const long row = (long)J * 128 + 4 * tq + j;
#pragma unroll
                            for (int cc = 0; cc < MC; ++cc)
                                if (cc < a.mc && row < a.n) {
                                    float* y = a.Y + (long)(a.c0 + cc) * a.n + row;
                                    *y = __ldcg(y) - acc[j][cc];
                                }
                        }
                    } else {  // a piece of a shared row: partial slot
                        float* pt = a.P2 + (long)(2 * g + (u == u0 ? 0 : 1)) * 128 * MC;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int cc = 0; cc < MC; ++cc) pt[(4 * tq + j) * MC + cc] = acc[j][cc];
                    }
                }
                u += ce - ca;
            }
        }
        {   // the next super-block's inverse tiles this CTA will multiply in phase F
            const int In = FWD ? I + 1 : I - 1;
            const int nbn = min(a.SBB, a.NB - In * a.SBB), ntn = nbn * (nbn + 1) / 2;
            for (int task = g; task < ntn; task += G) {
                int p = 0;
                while (sb_tri(p + 1, 0) <= task) ++p;
                const int q = task - sb_tri(p, 0);
                const int b = FWD ? p : q, c = FWD ? q : p;
                const float* XN = a.X + (long)In * a.S * a.S;
                if (FWD) sb_prefetch_tile(XN, a.S, a.S, (long)b * 128, (long)c * 128);
                else sb_prefetch_tile(XN, a.S, a.S, (long)c * 128, (long)b * 128);
            }
        }
        prev = pn;
        if (!sb_barrier(a, ++nbar, &s_abort)) return;
    }
}

// ---------------------------------------------------------------------------
// the super-block inverses, once per factor
// ---------------------------------------------------------------------------
// X_I = L_II^{-1} by block forward substitution: X_cc = L_cc^{-1} (the
// transpose of LinvT's block), then for b = c+1 .. nb-1,
// X_bc = -L_bb^{-1} (sum_{k=c}^{b-1} L_bk X_kc).  A strip of 32 columns of
// block column c only needs the same strip of the blocks above it, so CTA
// (4 c + s, I) forms strip s of block column c of X_I on its own.  Rows of L
// past n are zero and LinvT's rows past n are the identity; those rows of X
// meet only right-hand-side rows past n, which the sweeps hold at zero.
// Products are 128 x 128 x 32 in float32 through shared memory, thread
// (ty, tx) = (tid / 8, tid % 8) owning a 4 x 4 block of the result.
constexpr int SB_STRIPS = 4;  // 32-column strips per block column
constexpr size_t sb_inverse_smem() { return (size_t)(128 * 33 + 32 * 36 + 128 * 36) * sizeof(float); }

static __global__ void __launch_bounds__(256) k_sb_inverse(const float* __restrict__ W, long ldw, int n, int NB,
                                                           const float* __restrict__ LinvT, int SBB,
                                                           float* __restrict__ X) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* As = reinterpret_cast<float*>(smem_raw);  // [128][33] a 128 x 32 slice of the left factor
    float* Bs = As + 128 * 33;                       // [32][36]  a 32 x 32 slice of the right factor
    float* Ts = Bs + 32 * 36;                        // [128][36] T = sum_k L_bk X_kc (this strip)
    const int c = blockIdx.x / SB_STRIPS, strip = blockIdx.x % SB_STRIPS;
    const int I = blockIdx.y, tid = threadIdx.x;
    const int S = SBB * 128;
    const int jb0 = I * SBB, nb = min(SBB, NB - jb0);
    if (c >= nb) return;
    float* XI = X + (long)I * S * S;
    const int x0 = c * 128 + strip * 32;  // first column of the strip in X_I
    const int ty = tid >> 3, tx = tid & 7;
    // X_cc (this strip) = (LinvT block)^T
    {
        const float* lt = LinvT + (long)(jb0 + c) * 16384;
        for (int e = tid; e < 128 * 32; e += 256) {
            const int r = e >> 5, col = e & 31;
            XI[(long)(c * 128 + r) * S + x0 + col] = lt[(strip * 32 + col) * 128 + r];
        }
    }
    __syncthreads();
    float acc[4][4];
    // chunk q of T's K loop: block k = c + q / 4, columns kk = 32 (q % 4);
    // the next chunk's entries wait in registers while this one is used
    float an[16], bn[4];
    auto load_chunk = [&](int b, int q) {
        const int k = c + (q >> 2), kk = (q & 3) * 32;
#pragma unroll
        for (int i = 0; i < 16; ++i) {  // As[r][q'] = L[row r of block b][col kk + q' of block k]
            const int e = tid + i * 256, r = e >> 5, qq = e & 31;
            const long gr = (long)(jb0 + b) * 128 + r;
            an[i] = gr < n ? W[gr * ldw + (long)(jb0 + k) * 128 + kk + qq] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // Bs[q'][col] = X_kc[kk + q'][strip col]
            const int e = tid + i * 256, qq = e >> 5, col = e & 31;
            bn[i] = __ldcg(XI + (long)(k * 128 + kk + qq) * S + x0 + col);
        }
    };
    for (int b = c + 1; b < nb; ++b) {
        // T = sum_{k=c}^{b-1} L_bk X_kc
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const int nq = (b - c) * 4;
        load_chunk(b, 0);
        for (int q = 0; q < nq; ++q) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = tid + i * 256;
                As[(e >> 5) * 33 + (e & 31)] = an[i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = tid + i * 256;
                Bs[(e >> 5) * 36 + (e & 31)] = bn[i];
            }
            __syncthreads();
            if (q + 1 < nq) load_chunk(b, q + 1);
#pragma unroll 8
            for (int qq = 0; qq < 32; ++qq) {
                float av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[(ty * 4 + i) * 33 + qq];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[qq * 36 + tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Ts[(ty * 4 + i) * 36 + tx * 4 + j] = acc[i][j];
        __syncthreads();
        // X_bc = -L_bb^{-1} T, L_bb^{-1}[r][q] = LinvT_b[q][r]
        const float* lt = LinvT + (long)(jb0 + b) * 16384;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int kk = 0; kk < 128; kk += 32) {
            for (int e = tid; e < 128 * 32; e += 256) {  // As[r][q] = L_bb^{-1}[r][kk + q]
                const int r = e >> 5, q = e & 31;
                As[r * 33 + q] = lt[(kk + q) * 128 + r];
            }
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                float av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[(ty * 4 + i) * 33 + q];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Ts[(kk + q) * 36 + tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                XI[(long)(b * 128 + ty * 4 + i) * S + x0 + tx * 4 + j] = -acc[i][j];
        __syncthreads();  // X_bc is read (through L2) by the next b
    }
}
