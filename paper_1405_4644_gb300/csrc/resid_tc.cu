// resid_tc.cu -- step A5 on the tensor cores: the float64-accurate residual
// of Algorithm 1 (lines 3, 7) and Algorithm 2 (line 2) from exact products of
// bf16 integer digits (scheme described in resid_tc.h).
//
// Kernels, in call order:
//   k_tcr_rowscan   bits of max_j |a_ij| per row (atomicMax) and partial row
//                   sums of |a_ij| for ||A||_inf; A read once, coalesced.
//   k_tcr_digits_a  64x64 tiles of column-major A transposed through shared
//                   memory into ten row-major digit planes.
//   k_tcr_digits_x  column exponent and ten digit planes of every column of X.
//   k_tcr_mma       persistent: work items (column block, row block, K chunk)
//                   in contiguous ranges per CTA.  Warp 0 feeds A and X digit
//                   tiles by TMA; warp 1 issues tcgen05.mma (M 128, K 16,
//                   N 16 (10 - p) for A's digit plane p against X's planes
//                   0 .. 9 - p stacked) for the 55 digit products with
//                   p + q <= 11, into ten group accumulators in tensor memory
//                   (two buffers, one per chunk parity); warps 2..9 move each finished chunk to
//                   32-bit integer sums and add them to 64-bit integer sums
//                   at the end of every (row block, column block) segment.
//   k_tcr_final     combines the groups with their scales in double-double,
//                   R = B - AX rounded once, block partial norms.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include "resid_tc.h"
#include "tc_ptx.cuh"

namespace {

constexpr int TCR_S = 10;           // digits per value (70 bits below 2^e)
constexpr int TCR_TMAX = 11;        // products of digits p, q (1-based) with p + q <= TCR_TMAX
constexpr int TCR_NG = TCR_TMAX - 1;  // groups t = 2..TCR_TMAX
constexpr int TCR_BK = 64;          // K per tile: 128 bytes of bf16
constexpr int TCR_KC = 1;           // K tiles per exactly accumulated chunk: 10 x 64^2 x 64 <= 2^22
constexpr int TCR_NA = 10;          // A ring: one digit plane tile (128 x 64) per stage
constexpr int TCR_NX = 2;           // X ring: ten plane tiles (16 x 64) per stage
constexpr int TCR_A_BYTES = 128 * 128;
constexpr int TCR_XP_BYTES = 16 * 128;
constexpr int TCR_X_BYTES = TCR_S * TCR_XP_BYTES;
constexpr int TCR_THREADS = 320;
constexpr uint32_t TCR_TMEM_COLS = 512;  // two buffers of 10 groups x 16 columns
constexpr size_t TCR_SMEM = (size_t)TCR_NA * TCR_A_BYTES + (size_t)TCR_NX * TCR_X_BYTES + 1024 + 256;
constexpr uint64_t TCR_WAIT_NS = 2000000000ull;
constexpr int TCR_RS = 64;          // column splits of the row scan
constexpr int TCR_NONFINITE = INT_MIN;
// 1.5 * 2^23: v + MAGIC has the integer v (|v| <= 2^22) in its low bits
constexpr float TCR_MAGIC = 12582912.0f;
constexpr uint32_t TCR_MAGIC_BITS = 0x4B400000u;

// exponent of a row or column from the bits of its largest magnitude: 2^e
// bounds every entry by a factor 4 (e = ilogb + 2); 0 for an all-zero row
// (integer operations only: float64 arithmetic is slow on this part)
__device__ __forceinline__ int tcr_exp(unsigned long long mx) {
    if (mx >= 0x7FF0000000000000ull) return TCR_NONFINITE;
    if (mx == 0ull) return 0;
    const int ef = (int)(mx >> 52);
    const int lg = ef > 0 ? ef - 1023 : (63 - __clzll((long long)mx)) - 1074;  // ilogb, subnormals included
    return lg + 2;
}

// |a| as a float from the bits of a (magnitude bits b), truncating the
// mantissa: no float64 arithmetic or conversion, which run at a small
// fraction of the float32 rate on this part; below 2^-126 counts as 0 and
// above float range as infinity (a row sum of |a| that large overflows anyway)
__device__ __forceinline__ float tcr_absf(unsigned long long b) {
    const uint32_t hi = (uint32_t)(b >> 32);
    const int e = (int)(hi >> 20);  // biased float64 exponent (sign already cleared)
    if (e < 1023 - 126) return 0.f;
    if (e > 1023 + 127) return __uint_as_float(0x7F800000u);
    return __uint_as_float(((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
}

// bf16 bits of a small integer (exact): through the float magic number
__device__ __forceinline__ uint32_t tcr_bf16(int v) {
    return __float_as_uint(__int_as_float((int)TCR_MAGIC_BITS + v) - TCR_MAGIC) >> 16;
}

// The ten signed digits of a / 2^e: a = 2^e sum_{p<10} d[p] 2^{-7(p+1)} up
// to the bits of a below 2^{e-70} (dropped, toward zero); |a| < 2^{e-1}.
// F = |a| 2^{70-e} < 2^69 is taken in four 21-bit fields (three digits
// each, the top one below 2^6); adding 64 at every digit position and
// subtracting it from every 7-bit field gives the balanced digits in
// [-64, 63] with the carries propagated, the top digit in [0, 64]; the sign
// of a then negates them all.  d[0] is the most significant digit.
// Two entries are done at a time and returned in bf16 pairs:
// pk[p] = bf16(d_p(a0)) | bf16(d_p(a1)) << 16.  The recoded 7-bit fields
// f = d + 64 of each 21-bit chunk are spread over bytes (tcr_fields); one
// byte permute puts field j of both entries into the mantissas of 0x4300
// (bf16 128 + f), and one packed bf16 FMA forms s (x - 192) = +-d exactly.
// The top digit (0..64) is converted directly.
__device__ __forceinline__ void tcr_fields(double a, int e, uint32_t (&u)[3], int& top, bool& neg) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    int ef = (int)((bits >> 52) & 0x7FF);
    unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
    if (ef) M |= 1ull << 52;
    else ef = 1;
    const int sh = ef - 1005 - e;
    unsigned long long lo = 0ull;
    uint32_t hi = 0;
    if (sh >= 64) {
        hi = (uint32_t)(M << (sh - 64));
    } else if (sh > 0) {
        lo = M << sh;
        hi = (uint32_t)(M >> (64 - sh));
    } else if (sh > -64) {
        lo = M >> (-sh);
    }
    const uint32_t c0 = (uint32_t)lo & 0x1FFFFFu, c1 = (uint32_t)(lo >> 21) & 0x1FFFFFu,
                   c2 = (uint32_t)(lo >> 42) & 0x1FFFFFu, c3 = (uint32_t)(lo >> 63) | (hi << 1);
    constexpr uint32_t K3 = 64u | (64u << 7) | (64u << 14);
    uint32_t t = c0 + K3;
    u[0] = (t & 0x7Fu) | ((t << 1) & 0x7F00u) | ((t << 2) & 0x7F0000u);
    t = c1 + K3 + (t >> 21);
    u[1] = (t & 0x7Fu) | ((t << 1) & 0x7F00u) | ((t << 2) & 0x7F0000u);
    t = c2 + K3 + (t >> 21);
    u[2] = (t & 0x7Fu) | ((t << 1) & 0x7F00u) | ((t << 2) & 0x7F0000u);
    top = (int)(c3 + (t >> 21));
    neg = (bits >> 63) != 0;
}

__device__ __forceinline__ void tcr_digits2(double a0, double a1, int e, uint32_t (&pk)[TCR_S]) {
    uint32_t u0[3], u1[3];
    int top0, top1;
    bool n0, n1;
    tcr_fields(a0, e, u0, top0, n0);
    tcr_fields(a1, e, u1, top1, n1);
    const uint32_t sb = (n0 ? 0xBF80u : 0x3F80u) | (n1 ? 0xBF800000u : 0x3F800000u);  // +-1
    const uint32_t cb = (n0 ? 0x4340u : 0xC340u) | (n1 ? 0x43400000u : 0xC3400000u);  // -+192
    const __nv_bfloat162 s2 = *reinterpret_cast<const __nv_bfloat162*>(&sb);
    const __nv_bfloat162 c2 = *reinterpret_cast<const __nv_bfloat162*>(&cb);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const uint32_t x = __byte_perm(u0[k], u1[k], (uint32_t)(j | (3 << 4) | ((4 + j) << 8) | (7 << 12))) |
                               0x43004300u;
            const __nv_bfloat162 r = __hfma2(*reinterpret_cast<const __nv_bfloat162*>(&x), s2, c2);
            pk[9 - 3 * k - j] = *reinterpret_cast<const uint32_t*>(&r);
        }
    pk[0] = (tcr_bf16(top0) ^ (n0 ? 0x8000u : 0u)) | ((tcr_bf16(top1) ^ (n1 ? 0x8000u : 0u)) << 16);
}

__global__ void __launch_bounds__(256) k_tcr_rowscan(const double* __restrict__ A, long lda, int n, int jchunk,
                                                     unsigned long long* __restrict__ rowmax,
                                                     float* __restrict__ rowabs) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n) return;
    const int j0 = s * jchunk, j1 = min(n, j0 + jchunk);
    // four independent chains, eight loads in flight per thread
    unsigned long long mx[4] = {0ull, 0ull, 0ull, 0ull};
    float asum[4] = {0.f, 0.f, 0.f, 0.f};
    const double* ap = A + i;
    int j = j0;
    for (; j + 8 <= j1; j += 8) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldg(ap + (long)(j + u) * lda);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(a[u]) & 0x7FFFFFFFFFFFFFFFull;
            mx[u & 3] = b > mx[u & 3] ? b : mx[u & 3];
            asum[u & 3] += tcr_absf(b);
        }
    }
    for (; j < j1; ++j) {
        const double a = __ldg(ap + (long)j * lda);
        const unsigned long long b = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
        mx[0] = b > mx[0] ? b : mx[0];
        asum[0] += tcr_absf(b);
    }
    const unsigned long long m01 = mx[0] > mx[1] ? mx[0] : mx[1], m23 = mx[2] > mx[3] ? mx[2] : mx[3];
    if (j1 > j0) atomicMax(rowmax + i, m01 > m23 ? m01 : m23);
    rowabs[(long)s * n + i] = (asum[0] + asum[1]) + (asum[2] + asum[3]);
}

// The same scan with A streamed by TMA: CTA (row block of 256, column
// chunk) loads 256 x 16 tiles (32 KB) into a 3-stage ring; thread t owns row
// t of the block.  Waits are bounded; a wait that gives up raises
// SPD_DEV_TIMEOUT and the CTA stops.
constexpr int TRS_COLS = 16, TRS_ST = 3;
constexpr int TRS_TILE = 256 * TRS_COLS * 8;
constexpr size_t TRS_SMEM = (size_t)TRS_ST * TRS_TILE + 128;
__global__ void __launch_bounds__(256) k_tcr_rowscan_tma(const __grid_constant__ CUtensorMap mapA, int n, int jchunk,
                                                         unsigned long long* __restrict__ rowmax,
                                                         float* __restrict__ rowabs, DevStatus* st) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const double* buf = reinterpret_cast<const double*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + TRS_ST * TRS_TILE);
    uint64_t* empty = full + TRS_ST;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + TRS_ST);
    const int tid = threadIdx.x, lane = tid & 31;
    const int i0 = blockIdx.x * 256, s = blockIdx.y;
    const int j0 = s * jchunk, j1 = min(n, j0 + jchunk);  // jchunk is a multiple of 16
    const int ntile = j1 > j0 ? (j1 - j0 + TRS_COLS - 1) / TRS_COLS : 0;
    if (tid == 0) {
        for (int k = 0; k < TRS_ST; ++k) {
            tc::mbar_init(&full[k], 1);
            tc::mbar_init(&empty[k], 8);
        }
        *abort_flag = 0;
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mapA);
        for (int t = 0; t < TRS_ST && t < ntile; ++t) {
            tc::mbar_arrive_expect_tx(&full[t], TRS_TILE);
            tc::tma_load_2d(smem_raw + t * TRS_TILE, &mapA, i0, j0 + t * TRS_COLS, &full[t]);
        }
    }
    __syncthreads();
    unsigned long long mx0 = 0ull, mx1 = 0ull;
    float as0 = 0.f, as1 = 0.f;
    for (int t = 0; t < ntile; ++t) {
        const int k = t % TRS_ST;
        const uint32_t ph = (t / TRS_ST) & 1u;
        if (!tc::mbar_wait(&full[k], ph, abort_flag, TCR_WAIT_NS)) break;
        const double* col = buf + (size_t)k * 256 * TRS_COLS + tid;
#pragma unroll
        for (int c = 0; c < TRS_COLS; c += 2) {
            const double a = col[c * 256], b = col[(c + 1) * 256];
            const unsigned long long ba = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long bb = (unsigned long long)__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFull;
            mx0 = ba > mx0 ? ba : mx0;
            mx1 = bb > mx1 ? bb : mx1;
            as0 += tcr_absf(ba);
            as1 += tcr_absf(bb);
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[k]);
        if (tid == 0 && t + TRS_ST < ntile) {  // refill this stage once every warp has read it
            if (!tc::mbar_wait(&empty[k], ph, abort_flag, TCR_WAIT_NS)) break;
            tc::mbar_arrive_expect_tx(&full[k], TRS_TILE);
            tc::tma_load_2d(smem_raw + k * TRS_TILE, &mapA, i0, j0 + (t + TRS_ST) * TRS_COLS, &full[k]);
        }
    }
    if (*abort_flag) {
        if (tid == 0) atomicOr(&st->flags, SPD_DEV_TIMEOUT);
        return;
    }
    const int i = i0 + tid;
    if (i < n) {
        if (ntile > 0) atomicMax(rowmax + i, mx0 > mx1 ? mx0 : mx1);
        rowabs[(long)s * n + i] = as0 + as1;
    }
}

// 64 x 64 tile: element (i0 + r, j0 + c) of column-major A goes to
// tile[r][c] (coalesced along r, odd pitch: conflict-free); warp w then
// takes rows w, w + 8, ... and lane l the columns 2 l, 2 l + 1, so each
// store writes 128 contiguous bytes of one plane row
__global__ void __launch_bounds__(256) k_tcr_digits_a(const double* __restrict__ A, long lda, int n,
                                                      const unsigned long long* __restrict__ rowmax,
                                                      uint16_t* __restrict__ Ad, long ldp) {
    __shared__ double tile[64][65];
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    const int tid = threadIdx.x;
#pragma unroll 4
    for (int e = tid; e < 64 * 64; e += 256) {
        const int c = e >> 6, r = e & 63;
        const int i = i0 + r, j = j0 + c;
        tile[r][c] = (i < n && j < n) ? __ldg(A + i + (long)j * lda) : 0.0;
    }
    __syncthreads();
    const int w = tid >> 5, lane = tid & 31;
    for (int r = w; r < 64; r += 8) {
        const int i = i0 + r;
        if (i >= n) break;
        const int e = tcr_exp(rowmax[i]);
        const bool zero = e == TCR_NONFINITE;
        uint32_t pk[TCR_S];
        tcr_digits2(zero ? 0.0 : tile[r][2 * lane], zero ? 0.0 : tile[r][2 * lane + 1], zero ? 0 : e, pk);
        // ldp is a multiple of 64, so the tile's columns are inside the row pitch
        uint32_t* dst = reinterpret_cast<uint32_t*>(Ad + (long)i * ldp + j0) + lane;
#pragma unroll
        for (int p = 0; p < TCR_S; ++p) dst[(long)p * n * ldp / 2] = pk[p];
    }
}

// one CTA per column of X: its exponent, then ten digit planes (row c of
// plane q holds the digits of column c)
__global__ void __launch_bounds__(256) k_tcr_digits_x(const double* __restrict__ X, long ldx, int n, int m,
                                                      int* __restrict__ xe, uint16_t* __restrict__ Xd, long ldp,
                                                      const int* __restrict__ gate) {
    __shared__ unsigned long long red[8];
    if (gate && *gate == 0) return;  // refinement over (capturable solves)
    const int c = blockIdx.x;
    const double* x = X + (long)c * ldx;
    unsigned long long mx = 0ull;
    for (int j = threadIdx.x; j < n; j += 256) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[j]) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0ull;
#pragma unroll
    for (int k = 0; k < 8; ++k) mx = red[k] > mx ? red[k] : mx;
    const int e = tcr_exp(mx);
    if (threadIdx.x == 0) xe[c] = e;
    const bool zero = e == TCR_NONFINITE;
    for (int j = 8 * threadIdx.x; j < n; j += 8 * 256) {
        uint32_t pk[TCR_S][4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            uint32_t pq[TCR_S];
            tcr_digits2((!zero && j + u < n) ? x[j + u] : 0.0, (!zero && j + u + 1 < n) ? x[j + u + 1] : 0.0,
                        zero ? 0 : e, pq);
#pragma unroll
            for (int p = 0; p < TCR_S; ++p) pk[p][u >> 1] = pq[p];
        }
#pragma unroll
        for (int p = 0; p < TCR_S; ++p)
            *reinterpret_cast<uint4*>(Xd + ((long)p * m + c) * ldp + j) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
    }
}

// ---------------------------------------------------------------------------
// the digit products
// ---------------------------------------------------------------------------
// Work item t: g = t / Nkc (segment: column block g / RB, row block g % RB)
// and K tile t % Nkc.  CTA b takes items [b T / G, (b+1) T / G).  At the end
// of each segment, and every TCR_FLUSH items, its 32-bit sums (at most
// TCR_FLUSH x 2^21.3 in magnitude) are added to the 64-bit integer sums
// part[g][group][column][row] (integer atomics: the order does not matter).
constexpr int TCR_FLUSH = 256;
__global__ void __launch_bounds__(TCR_THREADS, 1)
    k_tcr_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX, int n, int RB,
              int Nkc, long T, unsigned long long* __restrict__ part, DevStatus* st, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;  // before any barrier or tensor memory
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* sA = base;
    unsigned char* sX = base + TCR_NA * TCR_A_BYTES;
    uint64_t* afull = reinterpret_cast<uint64_t*>(sX + TCR_NX * TCR_X_BYTES);
    uint64_t* aempty = afull + TCR_NA;
    uint64_t* xfull = aempty + TCR_NA;
    uint64_t* xempty = xfull + TCR_NX;
    uint64_t* tfull = xempty + TCR_NX;  // [2] chunk accumulated (tcgen05.commit)
    uint64_t* tfree = tfull + 2;        // [2] chunk read out (8 epilogue warps)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long G = gridDim.x, b = blockIdx.x;
    const long t0 = b * T / G, t1 = (b + 1) * T / G;
    const int nitems = (int)(t1 - t0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TCR_NA; ++s) {
            tc::mbar_init(&afull[s], 1);
            tc::mbar_init(&aempty[s], 1);
        }
        for (int s = 0; s < TCR_NX; ++s) {
            tc::mbar_init(&xfull[s], 1);
            tc::mbar_init(&xempty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&tfull[s], 1);
            tc::mbar_init(&tfree[s], 8);
        }
        *abort_flag = 0;
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapX);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TCR_TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int ia = 0, ix = 0;
            bool ok = true;
            for (int u = 0; u < nitems && ok; ++u) {
                const long t = t0 + u;
                const long g = t / Nkc;
                const int kc = (int)(t - g * Nkc);
                const int cb = (int)(g / RB), rb = (int)(g - (long)cb * RB);
                for (int kt = 0; kt < TCR_KC && ok; ++kt) {
                    const int k = (kc * TCR_KC + kt) * TCR_BK;
                    if (k >= n) break;
                    {
                        const int s = ix % TCR_NX;
                        if (ix >= TCR_NX && !tc::mbar_wait(&xempty[s], ((ix / TCR_NX) & 1u) ^ 1u, abort_flag, TCR_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&xfull[s], TCR_X_BYTES);
#pragma unroll
                        for (int q = 0; q < TCR_S; ++q)
                            tc::tma_load_3d(sX + s * TCR_X_BYTES + q * TCR_XP_BYTES, &mapX, k, cb * 16, q, &xfull[s]);
                        ++ix;
                    }
                    for (int p = 0; p < TCR_S; ++p) {
                        const int s = ia % TCR_NA;
                        if (ia >= TCR_NA && !tc::mbar_wait(&aempty[s], ((ia / TCR_NA) & 1u) ^ 1u, abort_flag, TCR_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&afull[s], TCR_A_BYTES);
                        tc::tma_load_3d(sA + s * TCR_A_BYTES, &mapA, k, rb * 128, p, &afull[s]);
                        ++ia;
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int ia = 0, ix = 0;
            bool ok = true;
            for (int u = 0; u < nitems && ok; ++u) {
                const int buf = u & 1;
                if (u >= 2 && !tc::mbar_wait(&tfree[buf], ((u >> 1) - 1) & 1u, abort_flag, TCR_WAIT_NS)) break;
                tc::fence_after_sync();
                const uint32_t dbase = tmem + (uint32_t)(buf * TCR_NG * 16);
                const long t = t0 + u;
                const int kc = (int)(t % Nkc);
                for (int kt = 0; kt < TCR_KC && ok; ++kt) {
                    const int k = (kc * TCR_KC + kt) * TCR_BK;
                    if (k >= n) break;
                    const int sx = ix % TCR_NX;
                    if (!tc::mbar_wait(&xfull[sx], (ix / TCR_NX) & 1u, abort_flag, TCR_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    // the X stage holds planes q = 0..9 as one K-major tile of
                    // 160 rows (16 per plane); its first 16 (10 - p) rows
                    // against A plane p give the products (p, q), q <= 9 - p, as
                    // one N = 16 (10 - p) instruction whose columns are the
                    // accumulators of groups p .. 9 (group g at columns 16 g)
                    const uint64_t bd = tc::sdesc_kmajor_sw128(tc::smem_u32(sX + sx * TCR_X_BYTES));
                    for (int p = 0; p < TCR_S; ++p) {
                        const int sa = ia % TCR_NA;
                        if (!tc::mbar_wait(&afull[sa], (ia / TCR_NA) & 1u, abort_flag, TCR_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint64_t ad = tc::sdesc_kmajor_sw128(tc::smem_u32(sA + sa * TCR_A_BYTES));
                        const uint32_t idesc = tc::idesc_f32acc(1, 128, 16 * (TCR_TMAX - 1 - p));  // bf16 -> f32
#pragma unroll
                        for (int kk = 0; kk < TCR_BK / 16; ++kk)  // +32 bytes of K = +2 in the address field
                            tc::mma<0>(dbase + (uint32_t)(p * 16), ad + 2 * kk, bd + 2 * kk, idesc,
                                       (kt > 0 || p > 0 || kk > 0) ? 1u : 0u);
                        tc::mma_commit(&aempty[sa]);
                        ++ia;
                    }
                    if (!ok) break;
                    tc::mma_commit(&xempty[sx]);
                    ++ix;
                }
                if (!ok) break;
                tc::mma_commit(&tfull[buf]);
            }
        }
        __syncwarp();
    } else {  // warps 2..9: chunk read-out, lane quarter warp % 4, columns EW h .. EW h + EW - 1
        constexpr int EW = TCR_NG * 16 / 2;  // 80: groups 5 h .. 5 h + 4
        const int quarter = warp & 3, h = (warp - 2) >> 2;
        int acc[EW];
#pragma unroll
        for (int j = 0; j < EW; ++j) acc[j] = 0;
        int seg_items = 0;
        for (int u = 0; u < nitems; ++u) {
            const int buf = u & 1;
            bool ok = tc::mbar_wait(&tfull[buf], (u >> 1) & 1u, abort_flag, TCR_WAIT_NS) && !*abort_flag;
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
            if (!ok) break;
            tc::fence_after_sync();
            const uint32_t ta = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + (uint32_t)(buf * TCR_NG * 16 + h * EW);
#pragma unroll
            for (int q = 0; q < EW / 16; ++q) {
                float v[16];
                tc::tmem_ld_32x32b_x16(ta + q * 16, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[q * 16 + j] += __float_as_int(v[j] + TCR_MAGIC);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tfree[buf]);
            ++seg_items;
            const long t = t0 + u;
            if (u == nitems - 1 || (t + 1) % Nkc == 0 || seg_items == TCR_FLUSH) {
                // entry (group 5 h + j / 16, column j % 16, row r) at (h EW + j) 128 + r
                unsigned long long* out = part + (t / Nkc) * (TCR_NG * 16 * 128) + h * EW * 128 + quarter * 32 + lane;
                const uint32_t bias = (uint32_t)seg_items * TCR_MAGIC_BITS;
#pragma unroll
                for (int j = 0; j < EW; ++j) {
                    const long long v = (int)((uint32_t)acc[j] - bias);
                    atomicAdd(out + j * 128, (unsigned long long)v);
                    acc[j] = 0;
                }
                seg_items = 0;
            }
        }
    }
    if (*abort_flag && threadIdx.x == 0) atomicOr(&st->flags, SPD_DEV_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, TCR_TMEM_COLS);
}

// ---------------------------------------------------------------------------
// combination: R = B - A X (mode 0) or R = A X (mode 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tcr_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// thread: row i of column c = blockIdx.y; block partial norms as k_resid_final
__global__ void __launch_bounds__(256) k_tcr_final(const unsigned long long* __restrict__ rowmax,
                                                   const int* __restrict__ xe,
                                                   const unsigned long long* __restrict__ part, int n, int m, int RB,
                                                   const double* __restrict__ B, long ldb,
                                                   const double* __restrict__ X, long ldx, double* __restrict__ R,
                                                   long ldr, double* __restrict__ NP, int mode,
                                                   const int* __restrict__ gate) {
    __shared__ double red[3][8];
    if (gate && *gate == 0) return;
    const int c = blockIdx.y;
    const int i = blockIdx.x * 256 + threadIdx.x;
    double rmax = 0.0, r2 = 0.0, xmax = 0.0;
    if (i < n) {
        const int cb = c >> 4, cc = c & 15, rb = i >> 7, rr = i & 127;
        const long g = (long)cb * RB + rb;
        const unsigned long long* pp = part + g * (TCR_NG * 16 * 128) + cc * 128 + rr;
        long long gs[TCR_NG];
#pragma unroll
        for (int k = 0; k < TCR_NG; ++k) gs[k] = (long long)pp[k * 16 * 128];
        const int er = tcr_exp(rowmax[i]), fc = xe[c];
        double r;
        if (er == TCR_NONFINITE || fc == TCR_NONFINITE) {
            r = __longlong_as_double(0x7FF8000000000000ll);
        } else {
            // sum_t G_t 2^{-7t}, smallest group first, in double-double (each
            // term is exact: |G_t| < 2^53 for n < 2^30)
            double hi = 0.0, lo = 0.0;
#pragma unroll
            for (int k = TCR_NG - 1; k >= 0; --k) {  // 2^{-7(k+2)}: a constant, the product exact
                double e;
                tcr_two_sum(hi, (double)gs[k] * __longlong_as_double((long long)(1023 - 7 * (k + 2)) << 52), hi, e);
                lo += e;
            }
            hi = ldexp(hi, er + fc);
            lo = ldexp(lo, er + fc);
            if (mode == 0) {
                double s, e;
                tcr_two_sum(B[(long)c * ldb + i], -hi, s, e);
                r = s + (e - lo);
            } else {
                r = hi + lo;
            }
        }
        R[(long)c * ldr + i] = r;
        rmax = fabs(r);
        r2 = r * r;
        if (X) xmax = fabs(X[(long)c * ldx + i]);
    }
    rmax = warp_max(rmax);
    r2 = warp_sum(r2);
    xmax = warp_max(xmax);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = rmax;
        red[1][w] = r2;
        red[2][w] = xmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, s = 0.0, x = 0.0;
        for (int k = 0; k < 8; ++k) {
            a = fmax(a, red[0][k]);
            s += red[1][k];
            x = fmax(x, red[2][k]);
        }
        double* o = NP + ((long)blockIdx.x * m + c) * 3;
        o[0] = a;
        o[1] = s;
        o[2] = x;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tcr_encoder() {
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

// planes x rows x cols bf16 (row pitch ld elements), box 64 x box_rows x 1,
// 128-byte swizzle, zero fill outside
bool tcr_map(CUtensorMap* map, const void* base, long planes, long rows, long cols, long ld, int box_rows) {
    auto enc = tcr_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(rows * ld * 2)};
    cuuint32_t box[3] = {(cuuint32_t)TCR_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// column-major float64 A (n x n, ld lda) in 256-row x 16-column boxes; needs a
// 16-byte aligned A and lda a multiple of 2
bool tcr_map_a64(CUtensorMap* map, const double* A, int n, long lda) {
    auto enc = tcr_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(A) & 15) || (lda & 1)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(lda * 8)};
    cuuint32_t box[2] = {256, (cuuint32_t)TRS_COLS};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(A), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcrSchedule {
    int RB, CB, Nkc, G;
    long T;
};

TcrSchedule tcr_schedule(spd_handle* h, int n, int m) {
    TcrSchedule s;
    s.RB = ceil_div(n, 128);
    s.CB = ceil_div(m, 16);
    s.Nkc = ceil_div(n, TCR_BK * TCR_KC);
    s.T = (long)s.CB * s.RB * s.Nkc;
    s.G = (int)std::min<long>(std::max(1, h->sms), s.T);
    return s;
}

}  // namespace

size_t tc_resid_plan(WsPlan& p, spd_handle* h, int n, int m, size_t* off) {
    const long ldp = round_up(n, 64);
    const TcrSchedule s = tcr_schedule(h, n, m);
    off[0] = p.add<uint16_t>((size_t)TCR_S * n * ldp);
    off[1] = p.add<uint16_t>((size_t)TCR_S * m * ldp);
    off[2] = p.add<unsigned long long>((size_t)n);
    off[3] = p.add<float>((size_t)TCR_RS * n);
    off[4] = p.add<int>((size_t)m);
    off[5] = p.add<unsigned long long>((size_t)s.CB * s.RB * TCR_NG * 16 * 128);
    return p.bytes;
}

spd_status tc_resid_bind(spd_handle* h, TcResidWs* w, int n, int m, const size_t* off) {
    const TcrSchedule s = tcr_schedule(h, n, m);
    w->n = n;
    w->m = m;
    w->ldp = round_up(n, 64);
    w->Ad = ws_at<uint16_t>(h, off[0]);
    w->Xd = ws_at<uint16_t>(h, off[1]);
    w->rowmax = ws_at<unsigned long long>(h, off[2]);
    w->rowabs = ws_at<float>(h, off[3]);
    w->xe = ws_at<int>(h, off[4]);
    w->part = ws_at<unsigned long long>(h, off[5]);
    w->RS = TCR_RS;
    w->RB = s.RB;
    w->CB = s.CB;
    w->Nkc = s.Nkc;
    w->G = s.G;
    w->T = s.T;
    if (!tcr_map(&w->mapA, w->Ad, TCR_S, n, n, w->ldp, 128) || !tcr_map(&w->mapX, w->Xd, TCR_S, m, n, w->ldp, 16))
        return set_err(h, SPD_ERR_UNSUPPORTED, "tensor-core residual: tensor map encoding failed");
    return SPD_OK;
}

spd_status tc_resid_prepare(spd_handle* h, TcResidWs* w, const double* A, long lda) {
    cudaStream_t s = h->stream;
    const int n = w->n;
    CUDA_TRY(h, cudaMemsetAsync(w->rowmax, 0, sizeof(unsigned long long) * n, s));
    CUtensorMap mapA64;
    if (tcr_map_a64(&mapA64, A, n, lda)) {  // stream A by TMA
        static const bool attr = [] {  // once per process, thread-safe
            cudaFuncSetAttribute(k_tcr_rowscan_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRS_SMEM);
            return true;
        }();
        (void)attr;
        w->RS = 8;
        const int jchunk = (int)round_up(ceil_div(n, w->RS), TRS_COLS);
        ++(h)->launches, k_tcr_rowscan_tma<<<dim3(ceil_div(n, 256), w->RS), 256, TRS_SMEM, s>>>(
            mapA64, n, jchunk, w->rowmax, w->rowabs, h->dst);
    } else {
        w->RS = TCR_RS;
        const int jchunk = ceil_div(n, w->RS);
        ++(h)->launches, k_tcr_rowscan<<<dim3(ceil_div(n, 256), w->RS), 256, 0, s>>>(A, lda, n, jchunk, w->rowmax,
                                                                                    w->rowabs);
    }
    LAUNCH_CHECK(h);
    ++(h)->launches, k_tcr_digits_a<<<dim3(ceil_div(n, 64), ceil_div(n, 64)), 256, 0, s>>>(A, lda, n, w->rowmax,
                                                                                          w->Ad, w->ldp);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

spd_status tc_resid_run(spd_handle* h, const TcResidWs* w, const double* B, long ldb, const double* X, long ldx,
                        double* R, long ldr, double* NP, int mode, const int* gate) {
    static const bool attr = [] {  // once per process, thread-safe
        cudaFuncSetAttribute(k_tcr_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCR_SMEM);
        return true;
    }();
    (void)attr;
    cudaStream_t s = h->stream;
    const int n = w->n, m = w->m;
    ++(h)->launches, k_tcr_digits_x<<<m, 256, 0, s>>>(X, ldx, n, m, w->xe, w->Xd, w->ldp, gate);
    LAUNCH_CHECK(h);
    CUDA_TRY(h, cudaMemsetAsync(w->part, 0, sizeof(unsigned long long) * (size_t)w->CB * w->RB * TCR_NG * 16 * 128, s));
    ++(h)->launches, k_tcr_mma<<<w->G, TCR_THREADS, TCR_SMEM, s>>>(w->mapA, w->mapX, n, w->RB, w->Nkc, w->T, w->part,
                                                                   h->dst, gate);
    LAUNCH_CHECK(h);
    ++(h)->launches, k_tcr_final<<<dim3(ceil_div(n, 256), m), 256, 0, s>>>(
        w->rowmax, w->xe, w->part, n, m, w->RB, mode == 0 ? B : nullptr, ldb, X, ldx, R,
        ldr, NP, mode, gate);
    LAUNCH_CHECK(h);
    return SPD_OK;
}
