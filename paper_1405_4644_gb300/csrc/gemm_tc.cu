// gemm_tc.cu -- step A3 on the 5th-generation tensor cores: the trailing
// update C -= A B^T of the blocked Cholesky factorisation (Section 3.1,
// eq. (cholesky); the O(n^3) part that "stresses the components to their
// limits").
//
// One CTA computes a 128 x BNT tile of C (BNT = 256, or 128 for one block
// column).  Operand tiles (128 rows of A, BNT rows of B, 128 bytes of K each)
// are fetched by TMA into shared memory in the 128-byte swizzled K-major
// layout, through a multi-stage mbarrier pipeline: warp 0 (one thread) issues
// the loads, warp 1 (one thread) issues tcgen05.mma into float32
// accumulators in tensor memory and frees each stage with tcgen05.commit.
// The four warps then read the accumulators with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31, i.e. rows of the tile) and apply C -= scale * acc
// to float32 C in global memory.
//
// Float32 operands given as three bf16 slices (s0 + s1 + s2) are multiplied
// as the six slice products of order <= 2.  The products of one K tile are
// issued back to back (K outer, slice pair inner), so the three reloads of a
// slice tile within a K tile are served by L2 and each slice leaves HBM once;
// the five small products go to one accumulator and s0*t0 to a second one,
// added once in the epilogue, so no small product is ever rounded against
// the large partial sums.
//
// Epilogue: each warp brings its 32 rows of the C tile into the (now idle)
// stage buffers with TMA, as 32 x 32 boxes in the 128-byte swizzled layout
// (a thread's row is then read and written without bank conflicts),
// subtracts the accumulator and writes the boxes back with TMA stores.
// Split K: CTA z of a tile takes K tiles [z kslice, (z+1) kslice) and writes
// its raw accumulator to a partial buffer; k_reduce_parts, launched as a
// programmatic dependent of the GEMM, sums the partials of every entry in z
// order and updates C.
// Every wait is bounded; a wait that gives up raises SPD_DEV_TIMEOUT.
#include <cudaTypedefs.h>
#include <algorithm>
#include <cstring>
#include "gemm_tc.h"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128, BN = 256;
constexpr int A_STAGE = BM * 128;  // bytes: 128 rows x 128 B
// The tile width BNT is 256 (trailing updates) or 128 (one block column),
// with ST pipeline stages: 4 stages and one CTA per SM, or (128-wide tf32
// tiles, whose six-segment float32 updates are long) 3 stages of 32 KB and
// two CTAs per SM, so that one CTA's epilogue overlaps the other's main loop.
// Narrow tiles (BNT = 32 or 64, the skinny products A~ P of CG with m
// right-hand sides) take all three slices of an A tile and of a B tile in one
// stage (SL = 3 slices per stage, one TMA load each with a box three planes
// deep), so that each slice tile crosses from L2 to shared memory once per K
// tile and the six slice products are issued from the same stage.
template <int BNT> __host__ __device__ constexpr int b_stage() { return BNT * 128; }
template <int BNT, int SL = 1> __host__ __device__ constexpr int stage_bytes() {
    return SL * (A_STAGE + b_stage<BNT>());
}
template <int BNT, int ST, int SL = 1> constexpr size_t smem_bytes() {
    return (size_t)ST * stage_bytes<BNT, SL>() + 1024 + 256;
}
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait

template <int KIND> struct KindTraits;
template <> struct KindTraits<0> {  // fp16 / bf16
    static constexpr int BK = 64, KMMA = 16;
};
template <> struct KindTraits<1> {  // tf32
    static constexpr int BK = 32, KMMA = 8;
};
template <> struct KindTraits<2> {  // fp8 e4m3
    static constexpr int BK = 128, KMMA = 32;
};

// Without a tensor map of C (ldc * 4 bytes not a multiple of 16): v = acc
// (32 consecutive columns of one row of the tile) applied to C directly with
// the lower-triangle and ragged-edge masks, C[row][col0 + j] -= scale * v[j]
__device__ __forceinline__ void apply_chunk(float* __restrict__ crow, const float* v, int row, int col0, int N,
                                            int lower, float scale) {
    const bool full_chunk = (col0 + 32 <= N) && !(lower && row < col0 + 31) &&
                            ((reinterpret_cast<uintptr_t>(crow) & 15) == 0);
    if (full_chunk) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float4 c = reinterpret_cast<float4*>(crow)[q];
            c.x -= scale * v[4 * q + 0];
            c.y -= scale * v[4 * q + 1];
            c.z -= scale * v[4 * q + 2];
            c.w -= scale * v[4 * q + 3];
            reinterpret_cast<float4*>(crow)[q] = c;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = col0 + j;
            if (col < N && !(lower && row < col)) crow[j] -= scale * v[j];
        }
    }
}

// 32 columns (chunk ch) of the accumulator(s) of this thread's row: acc0
// (+ acc1); tacc addresses the warp's lane quadrant of the tile's accumulator
template <int NACC, int BNT>
__device__ __forceinline__ void load_acc(uint32_t tacc, int ch, float* v) {
    const uint32_t base = tacc + ch * 32;
    tc::tmem_ld_32x32b_x32(base, v);
    if constexpr (NACC == 2) {
        float w[32];
        tc::tmem_ld_32x32b_x32(base + BNT, w);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = v[j] + w[j];  // small products + s0*t0
    }
}

// C -= scale * acc (get(ch, v) gives 32 columns of this thread's row of the
// accumulator) for one warp's 32 rows through shared memory (the idle
// stage buffers, once the CTA's main loop is over): the rows as 32 x 32 boxes
// (4 KB each, 128-byte swizzle: 16-byte chunk q of box row r sits at chunk
// q ^ (r & 7), so a thread's row is read without bank conflicts), loaded by
// TMA, updated, stored back by TMA.  Rows >= M, columns >= N and (lower)
// entries above the diagonal keep their value: the boxes may reach past the
// update's block and every box entry is written back.  Returns false if the
// loads did not land in time.
template <int BNT, typename Get>
__device__ __forceinline__ bool epilogue_tma(unsigned char* base, uint64_t* cbar, volatile int* abort_flag,
                                             const CUtensorMap* mapC, Get get, int cx0, int cy0, int M, int N,
                                             int bm, int bn, int qd, int lane, int lower, float scale) {
    float* slab = reinterpret_cast<float*>(base) + qd * 32 * BNT;
    const int row_w = bm * BM + qd * 32, row = row_w + lane;
    int nbox = 0;
    uint32_t need = 0;  // boxes inside N and not wholly above the diagonal
    for (int ch = 0; ch < BNT / 32; ++ch) {
        const int col0 = bn * BNT + ch * 32;
        if (col0 >= N) break;
        nbox = ch + 1;
        if (!(lower && row_w + 31 < col0)) need |= 1u << ch;
    }
    if (!need) return true;
    if (lane == 0) {
        tc::mbar_arrive_expect_tx(&cbar[qd], 4096u * __popc(need));
        for (int ch = 0; ch < nbox; ++ch)
            if (need >> ch & 1u)
                tc::tma_load_2d(slab + ch * 1024, mapC, cx0 + bn * BNT + ch * 32, cy0 + row_w, &cbar[qd]);
    }
    bool landed = tc::mbar_wait(&cbar[qd], 0, abort_flag, WAIT_NS);
    if (!__all_sync(0xffffffffu, landed)) return false;
    const int lim = row < M ? (lower ? min(N - 1, row) : N - 1) : -1;  // last column to update
#pragma unroll
    for (int ch = 0; ch < BNT / 32; ++ch) {
        if (ch >= nbox) break;
        if (!(need >> ch & 1u)) continue;  // warp-uniform
        float v[32];
        get(ch, v);
        float4* rp = reinterpret_cast<float4*>(slab + ch * 1024 + lane * 32);
        const int col0 = bn * BNT + ch * 32;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float4 c = rp[q ^ (lane & 7)];
            const int cq = col0 + 4 * q;
            if (cq + 3 <= lim) {
                c.x -= scale * v[4 * q];
                c.y -= scale * v[4 * q + 1];
                c.z -= scale * v[4 * q + 2];
                c.w -= scale * v[4 * q + 3];
            } else {
                if (cq <= lim) c.x -= scale * v[4 * q];
                if (cq + 1 <= lim) c.y -= scale * v[4 * q + 1];
                if (cq + 2 <= lim) c.z -= scale * v[4 * q + 2];
            }
            rp[q ^ (lane & 7)] = c;
        }
    }
    tc::fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
        for (int ch = 0; ch < nbox; ++ch)
            if (need >> ch & 1u) tc::tma_store_2d(mapC, cx0 + bn * BNT + ch * 32, cy0 + row_w, slab + ch * 1024);
        tc::bulk_commit();
        tc::bulk_wait_all();
    }
    __syncwarp();
    return true;
}

// The launch covers T = tiles_m x tiles_n output tiles of 128 x BNT with nk
// K tiles each: W = T nk work units (tile t, K tile k) in tile-major order.
// CTA g takes units [g W / G, (g+1) W / G): with G = T each CTA owns one
// whole tile ("data-parallel"); with G < T ("stream-K") a CTA's range is cut
// by tile boundaries into pieces, and a piece that is not a whole tile can
// only be the CTA's first piece (partial slot 2g) or its last (slot 2g+1).
__device__ __forceinline__ long unit_begin(int g, long W, int G) { return (long)g * W / G; }

// Roles: warp 0 issues the TMA loads, warp 1 the MMAs, warps 2..5 run the
// epilogue (warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. those rows of the
// tile).  K loop of a piece: K tile kin, slice pair q inner; segment q
// multiplies slice (segs >> 4q) & 3 of A by slice (segs >> 4q+2) & 3 of B into
// accumulator (accsel >> q) & 1.  With one accumulator per tile (NACC = 1)
// the tensor memory holds two, so the epilogue of one piece overlaps the
// main loop of the next.
template <int KIND, int BNT, int ST, int NACC, int SL = 1>
__global__ void __launch_bounds__(192, (ST == 3 && SL == 1) ? 2 : 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapC, int use_map_c, float* __restrict__ C, long ldc, int cx0,
              int cy0, int M, int N, int a_row0, int b_row0, int k0, int lower, uint32_t idesc, float scale, int nseg,
              uint32_t segs, uint32_t accsel, int tiles_n, int nk, long W, int G, float* __restrict__ Cpart,
              DevStatus* st) {
    constexpr int BK = KindTraits<KIND>::BK;
    constexpr int B_STAGE = b_stage<BNT>();      // one slice of a B tile
    constexpr int STAGES = ST;
    constexpr int STAGE_BYTES = stage_bytes<BNT, SL>();
    constexpr int A_ST = SL * A_STAGE, B_ST = SL * B_STAGE;  // a stage's A and B parts
    // accumulator buffers: two per tile with one accumulator (the epilogue of
    // one piece overlaps the next); narrow tiles (SL = 3) promote every K
    // tile's sums to float32 registers, alternating two buffers
    constexpr int NBUF = (SL == 3 || NACC == 1) ? 2 : 1;
    constexpr uint32_t ACC_COLS = BNT * NACC;  // one tile's accumulator(s)
    constexpr uint32_t TMEM_COLS = ACC_COLS * NBUF;
    constexpr int MMA_PER_STAGE = BK / KindTraits<KIND>::KMMA;  // 32 bytes of K each
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + STAGES * A_ST;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accfull = empty + STAGES;  // [NBUF] MMA -> epilogue
    uint64_t* accempty = accfull + 2;    // [NBUF] epilogue -> MMA (4 arrivals)
    uint64_t* cbar = accempty + 2;       // [4] C boxes of a quadrant have landed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cbar + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;
    const int g = blockIdx.x;
    const long u0 = unit_begin(g, W, G), u1 = unit_begin(g + 1, W, G);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accfull[b], 1);
            tc::mbar_init(&accempty[b], 4);
        }
        for (int w = 0; w < 4; ++w) tc::mbar_init(&cbar[w], 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapB);
        if (use_map_c) tc::prefetch_tmap(&mapC);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    // pieces of [u0, u1): tile t, K tiles [kb, ke); tiles wholly above the
    // diagonal of a lower update are skipped by every role alike
#define SPD_FOR_PIECES                                                         \
    for (long u = u0, un = u0; u < u1; u = un)                                 \
        if (const int t = (int)(u / nk), kb = (int)(u - (long)t * nk),         \
            ke = (int)min((long)nk, kb + (u1 - u)), bm = t / tiles_n,          \
            bn = t - (t / tiles_n) * tiles_n;                                  \
            (un = u + (ke - kb)), (lower && (bm * BM + BM - 1 < bn * BNT)))    \
            ;                                                                  \
        else

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int kt = 0;
            SPD_FOR_PIECES {
                if constexpr (SL == 3) {  // one stage per K tile: every slice of both tiles
                    for (int kin = kb; kin < ke; ++kin, ++kt) {
                        const int s = kt % STAGES;
                        const uint32_t ph = (kt / STAGES) & 1u;
                        if (kt >= STAGES && !tc::mbar_wait(&empty[s], ph ^ 1u, abort_flag, WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                        tc::tma_load_3d(sA + s * A_ST, &mapA, k0 + kin * BK, a_row0 + bm * BM, 0, &full[s]);
                        tc::tma_load_3d(sB + s * B_ST, &mapB, k0 + kin * BK, b_row0 + bn * BNT, 0, &full[s]);
                    }
                    if (!ok) break;
                    continue;
                }
                for (int kin = kb; kin < ke && ok; ++kin)
                    for (int q = 0; q < nseg; ++q, ++kt) {
                        const int s = kt % STAGES;
                        const uint32_t ph = (kt / STAGES) & 1u;
                        const int za = (segs >> (4 * q)) & 3, zb = (segs >> (4 * q + 2)) & 3;
                        if (kt >= STAGES && !tc::mbar_wait(&empty[s], ph ^ 1u, abort_flag, WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                        tc::tma_load_3d(sA + s * A_ST, &mapA, k0 + kin * BK, a_row0 + bm * BM, za, &full[s]);
                        tc::tma_load_3d(sB + s * B_ST, &mapB, k0 + kin * BK, b_row0 + bn * BNT, zb, &full[s]);
                    }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            // first segment (in issue order) of each accumulator starts it from zero
            int first[2] = {-1, -1};
            for (int q = nseg - 1; q >= 0; --q) first[(accsel >> q) & 1] = q;
            int kt = 0, p = 0, pk = 0;
            SPD_FOR_PIECES {
                const int buf = p % NBUF;
                if (p >= NBUF) {  // the epilogue has drained this accumulator
                    if (!tc::mbar_wait(&accempty[buf], ((p / NBUF) - 1) & 1, abort_flag, WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                }
                if constexpr (SL == 3) {
                    // each K tile into a fresh accumulator pair (buffer pk & 1),
                    // which the epilogue adds to its float32 registers
                    for (int kin = kb; kin < ke; ++kin, ++kt, ++pk) {
                        const int b2 = pk & 1;
                        if (pk >= 2) {
                            if (!tc::mbar_wait(&accempty[b2], ((pk >> 1) - 1) & 1, abort_flag, WAIT_NS)) {
                                ok = false;
                                break;
                            }
                            tc::fence_after_sync();
                        }
                        const int s = kt % STAGES;
                        const uint32_t ph = (kt / STAGES) & 1u;
                        if (!tc::mbar_wait(&full[s], ph, abort_flag, WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        for (int q = 0; q < nseg; ++q) {
                            const int za = (segs >> (4 * q)) & 3, zb = (segs >> (4 * q + 2)) & 3;
                            const int a = (accsel >> q) & 1;
                            const uint64_t ad = tc::sdesc_kmajor_sw128(tc::smem_u32(sA + s * A_ST + za * A_STAGE));
                            const uint64_t bd = tc::sdesc_kmajor_sw128(tc::smem_u32(sB + s * B_ST + zb * B_STAGE));
                            const uint32_t d = tmem + (uint32_t)(b2 * ACC_COLS + a * BNT);
                            const bool fresh = q == first[a];
#pragma unroll
                            for (int k = 0; k < MMA_PER_STAGE; ++k)
                                tc::mma<KIND>(d, ad + 2 * k, bd + 2 * k, idesc, (fresh && k == 0) ? 0u : 1u);
                        }
                        tc::mma_commit(&empty[s]);
                        tc::mma_commit(&accfull[b2]);
                    }
                    if (!ok) break;
                    continue;
                }
                for (int kin = kb; kin < ke && ok; ++kin)
                    for (int q = 0; q < nseg; ++q, ++kt) {
                        const int s = kt % STAGES;
                        const uint32_t ph = (kt / STAGES) & 1u;
                        const int a = (accsel >> q) & 1;
                        if (!tc::mbar_wait(&full[s], ph, abort_flag, WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint64_t ad = tc::sdesc_kmajor_sw128(tc::smem_u32(sA + s * A_ST));
                        const uint64_t bd = tc::sdesc_kmajor_sw128(tc::smem_u32(sB + s * B_ST));
                        const uint32_t d = tmem + (uint32_t)(buf * ACC_COLS + a * BNT);
                        const bool fresh = kin == kb && q == first[a];
#pragma unroll
                        for (int k = 0; k < MMA_PER_STAGE; ++k)  // +32 bytes of K = +2 in the address field
                            tc::mma<KIND>(d, ad + 2 * k, bd + 2 * k, idesc, (fresh && k == 0) ? 0u : 1u);
                        tc::mma_commit(&empty[s]);
                    }
                if (!ok) break;
                tc::mma_commit(&accfull[buf]);
                ++p;
            }
        }
        __syncwarp();
    } else {  // epilogue warps
        const int qd = warp & 3;  // TMEM lane quadrant = rows 32 qd .. 32 qd + 31 of the tile
        int p = 0, pk = 0;
        // narrow tiles: the piece's sums, promoted K tile by K tile into
        // float32 registers (round to nearest) -- the tensor cores' own
        // float32 accumulation rounds toward zero, a bias that grows with K
        constexpr int NR = SL == 3 ? BNT : 1;
        float S0[NR], S1[NR];
        SPD_FOR_PIECES {
            const int buf = p % NBUF;
            uint32_t tacc = 0;
            if constexpr (SL == 3) {
#pragma unroll
                for (int j = 0; j < NR; ++j) S0[j] = S1[j] = 0.f;
                for (int kin = kb; kin < ke; ++kin, ++pk) {
                    const int b2 = pk & 1;
                    ok = tc::mbar_wait(&accfull[b2], (pk >> 1) & 1, abort_flag, WAIT_NS);
                    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t ta = tmem + (static_cast<uint32_t>(qd * 32) << 16) + (uint32_t)(b2 * ACC_COLS);
#pragma unroll
                    for (int ch = 0; ch < BNT / 32; ++ch) {
                        float v[32];
                        tc::tmem_ld_32x32b_x32(ta + ch * 32, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) S0[ch * 32 + j] += v[j];
                        tc::tmem_ld_32x32b_x32(ta + BNT + ch * 32, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) S1[ch * 32 + j] += v[j];
                    }
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&accempty[b2]);
                }
                if (!ok) break;
            } else {
                ok = tc::mbar_wait(&accfull[buf], (p / NBUF) & 1, abort_flag, WAIT_NS);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
                if (!ok) break;
                tc::fence_after_sync();
                tacc = tmem + (static_cast<uint32_t>(qd * 32) << 16) + (uint32_t)(buf * ACC_COLS);
            }
            // 32 columns (chunk ch) of this thread's row of the piece's sum
            auto get = [&](int ch, float* v) {
                if constexpr (SL == 3) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = S0[ch * 32 + j] + S1[ch * 32 + j];  // small + s0*t0
                } else {
                    load_acc<NACC, BNT>(tacc, ch, v);
                }
            };
            const bool last = un >= u1;
            if (last && warp == 2 && lane == 0) pdl_trigger();  // a dependent kernel may be scheduled
            const int row_w = bm * BM + qd * 32;  // first row of this warp's slab (local, warp-uniform)
            const int row = row_w + lane;
            if (!(kb == 0 && ke == nk) && !Cpart) {
                if (lane == 0) atomicOr(&st->flags, SPD_DEV_INTERNAL);  // a piece with nowhere to go
            } else if (!(kb == 0 && ke == nk)) {
                // part of a tile: raw accumulator into partial slot 2g (the
                // CTA's first piece) or 2g + 1 (its last)
                const int slot = 2 * g + (u == u0 ? 0 : 1);
                float* prow = Cpart + ((long)slot * BM + qd * 32 + lane) * BNT;
#pragma unroll
                for (int ch = 0; ch < BNT / 32; ++ch) {
                    if (bn * BNT + ch * 32 >= N) break;  // warp-uniform
                    float v[32];
                    get(ch, v);
                    if (row < M) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4*>(prow + ch * 32)[q] =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
            } else if (last && use_map_c) {
                if (row_w < M && !epilogue_tma<BNT>(base, cbar, abort_flag, &mapC, get, cx0, cy0, M, N, bm, bn, qd,
                                                    lane, lower, scale))
                    ok = false;
            } else {
#pragma unroll
                for (int ch = 0; ch < BNT / 32; ++ch) {
                    const int col0 = bn * BNT + ch * 32;
                    if (col0 >= N) break;                      // warp-uniform
                    if (lower && row_w + 31 < col0) continue;  // warp-uniform: chunk above the diagonal
                    float v[32];
                    get(ch, v);
                    if (row < M) apply_chunk(C + (long)row * ldc + col0, v, row, col0, N, lower, scale);
                }
            }
            ok = __all_sync(0xffffffffu, ok);
            if constexpr (SL != 3) {
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&accempty[buf]);
            }
            if (!ok) break;
            ++p;
        }
    }
#undef SPD_FOR_PIECES
    if (!ok && (lane == 0)) atomicOr(&st->flags, SPD_DEV_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return nullptr;
    }();
    return fn;
}

int elem_bytes(int kind) { return kind == 1 ? 4 : kind == 4 ? 1 : 2; }
int slices_of(int kind) { return kind == 5 ? 3 : 1; }

// 3-D map over `planes` row-major (rows x cols, ld elements) operand planes
// (plane stride rows*ld) with a box of (128 bytes of K) x box_rows x box_z
// (box_z = 1: one slice; 3: every slice of a float32 operand), 128-byte
// swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const void* base, int kind, long rows, long cols, long ld, int box_rows,
              int box_z = 1) {
    auto enc = get_encode();
    if (!enc) return false;
    CUtensorMapDataType dt = kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : (kind == 2 || kind == 5) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                             : kind == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                         : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const int es = elem_bytes(kind);
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)slices_of(kind)};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(rows * ld * es)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, (cuuint32_t)box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2-D map over a float32 row-major matrix (rows x cols, ld floats) with
// 32 x 32 boxes in the 128-byte swizzled layout: the epilogue's view of C.
bool make_map_c(CUtensorMap* map, float* C, long rows, long cols, long ld) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(float))};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

uint32_t idesc_for(int kind, int bn) {
    switch (kind) {
        case 1: return tc::idesc_f32acc(2, BM, bn);  // tf32
        case 2:
        case 5: return tc::idesc_f32acc(1, BM, bn);  // bf16 (and float32 as bf16 slices)
        case 3: return tc::idesc_f32acc(0, BM, bn);  // fp16
        default: return tc::idesc_f32acc(0, BM, bn); // e4m3 (kind::f8f6f4)
    }
}

template <int KIND, int BNT, int ST, int NACC, int SL = 1>
void set_smem() {
    cudaFuncSetAttribute(k_gemm_tc<KIND, BNT, ST, NACC, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_bytes<BNT, ST, SL>());
}

void set_attrs() {
    // once per process, thread-safe (function-local static)
    static const bool done = [] {
        set_smem<0, 256, 4, 1>();
        set_smem<1, 256, 4, 1>();
        set_smem<2, 256, 4, 1>();
        set_smem<0, 256, 4, 2>();
        set_smem<0, 128, 4, 1>();
        set_smem<1, 128, 4, 1>();
        set_smem<2, 128, 4, 1>();
        set_smem<0, 128, 3, 2>();
        set_smem<0, 32, 3, 2, 3>();
        set_smem<0, 64, 3, 2, 3>();
        return true;
    }();
    (void)done;
}

// Stream-K fix-up: for every entry of a tile that several CTAs share,
// C[i][j] -= scale * (sum of their partial slots in CTA order, i.e. in K
// order), only i >= j when lower.  Unit u belongs to CTA
// owner(u) = floor(((u + 1) G - 1) / W) (the largest g with g W / G <= u);
// tile t's piece of CTA g is g's first piece (slot 2g) when g's range starts
// inside tile t, else its last (slot 2g + 1).  Launched as a programmatic
// dependent of the GEMM: everything before pdl_wait overlaps its last CTAs.
__global__ void __launch_bounds__(256) k_reduce_parts(float* __restrict__ C, long ldc, int M, int N,
                                                      const float* __restrict__ P, int bnt, int tiles_n, int nk,
                                                      long W, int G, float scale, int lower) {
    // block (x, t): tile t = blockIdx.y, rows [x * RB, x * RB + RB) of it
    constexpr int RB = 16;
    const int t = blockIdx.y;
    const int bm = t / tiles_n, bn = t - bm * tiles_n;
    const long ut0 = (long)t * nk, ut1 = ut0 + nk;
    const int glo = (int)(((ut0 + 1) * G - 1) / W), ghi = (int)((ut1 * G - 1) / W);
    if (glo == ghi && unit_begin(glo, W, G) <= ut0 && unit_begin(glo + 1, W, G) >= ut1) return;  // one CTA's piece
    // slot of contributor glo: 2 glo + 1 when its range starts before the
    // tile, else 2 glo; every later contributor starts inside the tile (2g)
    const int slot_lo = 2 * glo + (unit_begin(glo, W, G) < ut0 ? 1 : 0);
    const int ncon = ghi - glo + 1;
    const int nq = bnt >> 2;  // float4 groups in a tile row
    pdl_wait();
    for (int e = threadIdx.x; e < RB * nq; e += blockDim.x) {
        const int r = blockIdx.x * RB + e / nq, c = (e % nq) * 4;
        const int i = bm * BM + r, j = bn * bnt + c;
        if (r >= BM || i >= M || j >= N || (lower && i < j)) continue;
        const float* pr = P + (long)r * bnt + c;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        // contributors in K order; loads issued eight at a time, added in order
        for (int k0 = 0; k0 < ncon; k0 += 8) {
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + q;
                const int slot = k == 0 ? slot_lo : 2 * (glo + k);
                v[q] = k < ncon ? __ldcg(reinterpret_cast<const float4*>(pr + (long)slot * BM * bnt))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (k0 + q < ncon) {
                    acc.x += v[q].x;
                    acc.y += v[q].y;
                    acc.z += v[q].z;
                    acc.w += v[q].w;
                }
        }
        float* cp = C + (long)i * ldc + j;
        const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q < N && !(lower && i < j + q)) cp[q] -= scale * a4[q];
    }
}

}  // namespace

struct TcGemm {
    CUtensorMap mapA, mapB, mapB128;  // box heights 128 (A), 256 and 128 (B)
    CUtensorMap mapC;                 // C in 32 x 32 boxes (when has_map_c)
    bool has_map_c;
    int narrow;                       // 32 or 64: narrow fused-slice tiles (maps three planes deep), else 0
    float* C;
    long ldc;
    int kind;
    int sms;
};

float tc_fp8_scale() { return SPD_FP8_SCALE; }

spd_status tc_gemm_create_maps(TcGemm** out, const void* Ah, long a_rows, long a_ld, const void* Bh, long b_rows,
                               long b_ld, long cols, float* C, long c_rows, long c_cols, long ldc, int kind) {
    *out = nullptr;
    if (kind < 1 || kind > 5) return SPD_ERR_UNSUPPORTED;
    TcGemm* g = new TcGemm();
    memset(g, 0, sizeof(*g));
    if (!make_map(&g->mapA, Ah, kind, a_rows, cols, a_ld, BM) || !make_map(&g->mapB, Bh, kind, b_rows, cols, b_ld, BN) ||
        !make_map(&g->mapB128, Bh, kind, b_rows, cols, b_ld, 128)) {
        delete g;
        return SPD_ERR_UNSUPPORTED;
    }
    // TMA needs 16-byte aligned rows of C; otherwise the epilogue writes C directly
    g->has_map_c = (ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0) &&
                   make_map_c(&g->mapC, C, c_rows, c_cols, ldc);
    g->C = C;
    g->ldc = ldc;
    g->kind = kind;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        g->sms = 148;
    set_attrs();
    *out = g;
    return SPD_OK;
}

spd_status tc_gemm_create_narrow(TcGemm** out, const void* Ah, long a_rows, long a_ld, const void* Bh, long b_rows,
                                 long b_ld, long cols, float* C, long c_rows, long c_cols, long ldc, int bnt) {
    *out = nullptr;
    if (bnt != 32 && bnt != 64) return SPD_ERR_ARG;
    TcGemm* g = new TcGemm();
    memset(g, 0, sizeof(*g));
    if (!make_map(&g->mapA, Ah, 5, a_rows, cols, a_ld, BM, 3) || !make_map(&g->mapB, Bh, 5, b_rows, cols, b_ld, bnt, 3)) {
        delete g;
        return SPD_ERR_UNSUPPORTED;
    }
    g->has_map_c = (ldc % 4 == 0) && (reinterpret_cast<uintptr_t>(C) % 16 == 0) &&
                   make_map_c(&g->mapC, C, c_rows, c_cols, ldc);
    g->C = C;
    g->ldc = ldc;
    g->kind = 5;
    g->narrow = bnt;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        g->sms = 148;
    set_attrs();
    *out = g;
    return SPD_OK;
}

spd_status tc_gemm_create(TcGemm** out, float* W, long ldw, void* Wh, long ldh, int kind, int n) {
    return tc_gemm_create_maps(out, Wh, n, ldh, Wh, n, ldh, n, W, n, n, ldw, kind);
}

namespace {

template <int BNT>
void launch_kind(TcGemm* g, cudaStream_t s, int G, int cx0, int cy0, int M, int N, int a_row0, int b_row0, int k0,
                 int lower, float scale, int nseg, uint32_t segs, uint32_t accsel, int tiles_n, int nk, long W,
                 float* Cpart, DevStatus* st) {
    const CUtensorMap& mb = (BNT == 128 && !g->narrow) ? g->mapB128 : g->mapB;
    const uint32_t idesc = idesc_for(g->kind, BNT);
    float* Cb = g->C + (long)cy0 * g->ldc + cx0;  // the block's origin (epilogue without a tensor map)
#define SPD_GEMM_ARGS                                                                                            \
    g->mapA, mb, g->mapC, g->has_map_c ? 1 : 0, Cb, g->ldc, cx0, cy0, M, N, a_row0, b_row0, k0, lower, idesc, \
        scale, nseg, segs, accsel, tiles_n, nk, W, G, Cpart, st
    if constexpr (BNT <= 64) {  // narrow tiles: float32 as bf16 slices, all slices in one stage
        k_gemm_tc<0, BNT, 3, 2, 3><<<G, 192, smem_bytes<BNT, 3, 3>(), s>>>(SPD_GEMM_ARGS);
    } else {
        switch (g->kind) {
            case 1: k_gemm_tc<1, BNT, 4, 1><<<G, 192, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS); break;
            case 5: {  // float32 as bf16 slices: two accumulators; two CTAs per SM on 128-wide tiles
                constexpr int ST = BNT == 128 ? 3 : 4;
                k_gemm_tc<0, BNT, ST, 2><<<G, 192, smem_bytes<BNT, ST>(), s>>>(SPD_GEMM_ARGS);
                break;
            }
            case 4: k_gemm_tc<2, BNT, 4, 1><<<G, 192, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS); break;
            default: k_gemm_tc<0, BNT, 4, 1><<<G, 192, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS);
        }
    }
#undef SPD_GEMM_ARGS
}

}  // namespace

spd_status tc_gemm_launch(TcGemm* g, cudaStream_t s, int cy0, int cx0, int M, int N, int K, int a_row0, int b_row0,
                          int k0, int lower, DevStatus* st, int splits, const TcSplit* sb) {
    const int bk = g->kind == 1 ? 32 : g->kind == 4 ? 128 : 64;
    if (M <= 0 || N <= 0 || K <= 0) return SPD_OK;
    if (K % bk != 0 || (k0 * elem_bytes(g->kind)) % 16 != 0 || cx0 % 4 != 0) return SPD_ERR_ARG;
    const float scale = g->kind == 4 ? 1.0f / (tc_fp8_scale() * tc_fp8_scale()) : 1.0f;
    // float32 as three bf16 slices: the six slice products of order <= 2 (A
    // slice in bits 4q..4q+1, B slice in bits 4q+2..4q+3 of segment q); the
    // five small ones into accumulator 0, s0*t0 into accumulator 1
    int nseg = 1;
    uint32_t segs = 0, accsel = 0;
    if (g->kind == 5) {
        const int pairs[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
        nseg = 6;
        for (int q = 0; q < 6; ++q) segs |= (uint32_t)(pairs[q][0] | (pairs[q][1] << 2)) << (4 * q);
        accsel = 1u << 5;
    }
    const int nk = K / bk;
    const int bnt = g->narrow ? g->narrow : (N <= 128) ? 128 : 256;
    const int tiles_n = (N + bnt - 1) / bnt, tiles_m = (M + BM - 1) / BM;
    const int T = tiles_n * tiles_m;
    const long W = (long)T * nk;
    // Data-parallel (one CTA per tile) or stream-K over `slots` CTAs, by an
    // estimate of the launch's length: waves x K tiles per CTA x the time of
    // one K tile, plus ~10 us of fix-up kernel for stream-K.  splits < 0
    // allows stream-K on -splits SMs (two CTAs per SM for the 128-wide
    // float32 tiles); splits = 1 keeps one CTA per tile.
    int G = T;
    if ((splits < 0 || splits == 0) && sb && sb->part && !(lower && tiles_n > 1)) {
        const int sms = splits < 0 ? -splits : g->sms;
        const int slots = (bnt == 128 && g->kind == 5 ? 2 : 1) * sms;
        int Gs = (int)std::min<long>(slots, W);
        // us per K tile (all segments); a narrow tile streams 48 KB of A
        // slices per K tile at about an SM's share of HBM bandwidth
        const double tk = g->narrow ? 1.0 : nseg * (bnt == 256 ? 0.40 : 0.25);
        const double dp = (double)((T + slots - 1) / slots) * nk * tk;
        // stream-K over Gc CTAs: the longest range, plus the fix-up: a launch
        // (~4 us) and its partial slots read at ~3 TB/s
        auto sk_us = [&](int Gc) {
            return (double)((W + Gc - 1) / Gc) * tk + 4.0 + 2.0 * Gc * BM * bnt * 4.0 / 3e6;
        };
        int best = Gs;
        for (int d = 2; d <= 16; d *= 2)
            if (Gs / d > T && sk_us(Gs / d) < sk_us(best)) best = Gs / d;
        // splits = 0: stream-K over all slots whenever it gives more CTAs than tiles
        const bool want = splits == 0 ? Gs > T : sk_us(best) < 0.9 * dp;
        if (splits != 0) Gs = best;
        if (want && Gs != T && (size_t)2 * Gs * BM * bnt <= sb->part_cap) G = Gs;
    }
    // stream-K (G != T: more or fewer CTAs than tiles) always writes partials
    float* part = (G != T) ? sb->part : nullptr;
    if (G != T && !part) return SPD_ERR_ARG;
    if (bnt == 32)
        launch_kind<32>(g, s, G, cx0, cy0, M, N, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, tiles_n, nk,
                        W, part, st);
    else if (bnt == 64)
        launch_kind<64>(g, s, G, cx0, cy0, M, N, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, tiles_n, nk,
                        W, part, st);
    else if (bnt == 128)
        launch_kind<128>(g, s, G, cx0, cy0, M, N, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, tiles_n, nk,
                         W, part, st);
    else
        launch_kind<256>(g, s, G, cx0, cy0, M, N, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, tiles_n, nk,
                         W, part, st);
    if (part) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(BM / 16, (unsigned)T);  // 16 rows of one tile per block
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        float* C = g->C + (long)cy0 * g->ldc + cx0;
        if (cudaLaunchKernelEx(&cfg, k_reduce_parts, C, g->ldc, M, N, (const float*)part, bnt, tiles_n, nk, W, G,
                               scale, lower) != cudaSuccess)
            return SPD_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? SPD_OK : SPD_ERR_CUDA;
}

spd_status tc_gemm_run(TcGemm* g, cudaStream_t s, int r0, int M, int c0, int N, int k0, int K, int lower,
                       DevStatus* st, int splits, const TcSplit* sb) {
    return tc_gemm_launch(g, s, r0, c0, M, N, K, r0, c0, k0, lower, st, splits, sb);
}

void tc_gemm_destroy(TcGemm* g) { delete g; }
