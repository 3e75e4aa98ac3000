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
template <int BNT> __host__ __device__ constexpr int b_stage() { return BNT * 128; }
template <int BNT> __host__ __device__ constexpr int stage_bytes() { return A_STAGE + b_stage<BNT>(); }
template <int BNT, int ST> constexpr size_t smem_bytes() { return (size_t)ST * stage_bytes<BNT>() + 1024 + 256; }
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

// 32 columns of the accumulator(s) of this thread's row: acc0 (+ acc1)
template <int NACC, int BNT>
__device__ __forceinline__ void load_acc(uint32_t tmem, int warp, int ch, float* v) {
    const uint32_t base = tmem + (static_cast<uint32_t>(warp * 32) << 16) + ch * 32;
    tc::tmem_ld_32x32b_x32(base, v);
    if constexpr (NACC == 2) {
        float w[32];
        tc::tmem_ld_32x32b_x32(base + BNT, w);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = v[j] + w[j];  // small products + s0*t0
    }
}

// K loop: K tile kin of this CTA's share, slice pair q inner.  Segment q
// multiplies slice (segs >> 4q) & 3 of A by slice (segs >> 4q+2) & 3 of B
// into accumulator (accsel >> q) & 1.
template <int KIND, int BNT, int ST, int NACC>
__global__ void __launch_bounds__(128, ST == 3 ? 2 : 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapC, float* __restrict__ C, long ldc, int cx0, int cy0, int M,
              int N, int K, int a_row0, int b_row0, int k0, int lower, uint32_t idesc, float scale, int nseg,
              uint32_t segs, uint32_t accsel, int kslice, float* __restrict__ Cpart, long ldp, DevStatus* st) {
    constexpr int BK = KindTraits<KIND>::BK;
    constexpr int B_STAGE = b_stage<BNT>();
    constexpr int STAGES = ST;
    constexpr int STAGE_BYTES = stage_bytes<BNT>();
    constexpr uint32_t TMEM_COLS = BNT * NACC;
    constexpr int MMA_PER_STAGE = BK / KindTraits<KIND>::KMMA;  // 4: 32 bytes of K each
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + STAGES * A_STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;
    uint64_t* cbar = accf + 1;  // one per warp: its C boxes have landed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cbar + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bm = blockIdx.y, bn = blockIdx.x;
    if (lower && (bm * BM + BM - 1 < bn * BNT)) return;  // whole tile above the diagonal
    if (st->flags & (SPD_DEV_BREAKDOWN | SPD_DEV_NONFINITE | SPD_DEV_BADDIAG)) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accf, 1);
        for (int w = 0; w < 4; ++w) tc::mbar_init(&cbar[w], 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapB);
        if (!Cpart && !C) tc::prefetch_tmap(&mapC);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int nk_all = K / BK;  // K tiles per segment
    const int kb = kslice > 0 ? (int)blockIdx.z * kslice : 0;
    const int nk = kslice > 0 ? max(0, min(nk_all, kb + kslice) - kb) : nk_all;  // this CTA's share
    const int ntiles = nk * nseg;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            for (int kt = 0; kt < ntiles; ++kt) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1u;
                const int kin = kt / nseg, q = kt - kin * nseg;
                const int za = (segs >> (4 * q)) & 3, zb = (segs >> (4 * q + 2)) & 3;
                if (kt >= STAGES && !tc::mbar_wait(&empty[s], ph ^ 1u, abort_flag, WAIT_NS)) break;
                tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tc::tma_load_3d(sA + s * A_STAGE, &mapA, k0 + (kb + kin) * BK, a_row0 + bm * BM, za, &full[s]);
                tc::tma_load_3d(sB + s * B_STAGE, &mapB, k0 + (kb + kin) * BK, b_row0 + bn * BNT, zb, &full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            // first segment (in issue order) of each accumulator starts it from zero
            int first[2] = {-1, -1};
            for (int q = nseg - 1; q >= 0; --q) first[(accsel >> q) & 1] = q;
            for (int kt = 0; kt < ntiles; ++kt) {
                const int s = kt % STAGES;
                const uint32_t ph = (kt / STAGES) & 1u;
                const int kin = kt / nseg, q = kt - kin * nseg;
                const int a = (accsel >> q) & 1;
                if (!tc::mbar_wait(&full[s], ph, abort_flag, WAIT_NS)) break;
                tc::fence_after_sync();
                const uint64_t ad = tc::sdesc_kmajor_sw128(tc::smem_u32(sA + s * A_STAGE));
                const uint64_t bd = tc::sdesc_kmajor_sw128(tc::smem_u32(sB + s * B_STAGE));
                const uint32_t d = tmem + (uint32_t)(a * BNT);
                const bool fresh = kin == 0 && q == first[a];
#pragma unroll
                for (int k = 0; k < MMA_PER_STAGE; ++k)  // +32 bytes of K = +2 in the address field
                    tc::mma<KIND>(d, ad + 2 * k, bd + 2 * k, idesc, (fresh && k == 0) ? 0u : 1u);
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(accf);
        }
        __syncwarp();
    }

    // epilogue: TMEM -> registers -> C -= scale * acc
    bool ok = tc::mbar_wait(accf, 0, abort_flag, WAIT_NS) && !*abort_flag;
    if (threadIdx.x == 0) pdl_trigger();  // a dependent kernel (the next leaf) may be scheduled
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
    tc::fence_after_sync();
    const int row = bm * BM + warp * 32 + lane;
    const int row_w = bm * BM + warp * 32;  // first row of this warp's slab (warp-uniform)
    if (Cpart) {
        // split K: this CTA's raw accumulator (zero for an empty share)
        if (ok) {
            for (int ch = 0; ch < BNT / 32; ++ch) {
                const int col0 = bn * BNT + ch * 32;
                if (col0 >= N) break;
                float v[32];
                if (ntiles > 0) load_acc<NACC, BNT>(tmem, warp, ch, v);
                else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
                if (row < M) {
                    float* prow = Cpart + ((long)blockIdx.z * M + row) * ldp + col0;
                    if (col0 + 32 <= N && ((reinterpret_cast<uintptr_t>(prow) & 15) == 0)) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4*>(prow)[q] =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < N) prow[j] = v[j];
                    }
                }
            }
        }
    } else if (ok && C) {  // C given directly (no tensor map): C is the block's origin
        for (int ch = 0; ch < BNT / 32; ++ch) {
            const int col0 = bn * BNT + ch * 32;
            if (col0 >= N) break;                           // warp-uniform
            if (lower && row_w + 31 < col0) continue;       // warp-uniform: chunk above the diagonal
            float v[32];
            load_acc<NACC, BNT>(tmem, warp, ch, v);
            if (row < M) apply_chunk(C + (long)row * ldc + col0, v, row, col0, N, lower, scale);
        }
    } else if (ok && row_w < M) {
        // C -= scale * acc through shared memory: the warp's 32 rows as
        // 32 x 32 boxes (4 KB each, 128-byte swizzle: 16-byte chunk q of
        // box row r sits at chunk q ^ (r & 7)), in the idle stage buffers
        float* slab = reinterpret_cast<float*>(base) + warp * 32 * BNT;
        int nbox = 0;
        uint32_t need = 0;  // boxes inside N and not wholly above the diagonal
        for (int ch = 0; ch < BNT / 32; ++ch) {
            const int col0 = bn * BNT + ch * 32;
            if (col0 >= N) break;
            nbox = ch + 1;
            if (!(lower && row_w + 31 < col0)) need |= 1u << ch;
        }
        if (lane == 0 && need) {
            tc::mbar_arrive_expect_tx(&cbar[warp], 4096u * __popc(need));
            for (int ch = 0; ch < nbox; ++ch)
                if (need >> ch & 1u)
                    tc::tma_load_2d(slab + ch * 1024, &mapC, cx0 + bn * BNT + ch * 32, cy0 + row_w, &cbar[warp]);
        }
        bool landed = !need || tc::mbar_wait(&cbar[warp], 0, abort_flag, WAIT_NS);
        landed = __all_sync(0xffffffffu, landed);
        if (landed) {
            for (int ch = 0; ch < nbox; ++ch) {
                if (!(need >> ch & 1u)) continue;  // warp-uniform
                float v[32];
                load_acc<NACC, BNT>(tmem, warp, ch, v);
                float4* rp = reinterpret_cast<float4*>(slab + ch * 1024 + lane * 32);
                const int col0 = bn * BNT + ch * 32;
                // rows >= M, columns >= N and (lower) entries above the
                // diagonal keep their value: the boxes may reach past the
                // update's block, and the stores write every box entry back
                const int lim = row < M ? (lower ? min(N - 1, row) : N - 1) : -1;  // last column to update
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
                    if (need >> ch & 1u) tc::tma_store_2d(&mapC, cx0 + bn * BNT + ch * 32, cy0 + row_w, slab + ch * 1024);
                tc::bulk_commit();
                tc::bulk_wait_all();
            }
            __syncwarp();
        } else {
            ok = false;
        }
    }
    if (!ok && threadIdx.x == 0) atomicOr(&st->flags, SPD_DEV_TIMEOUT);
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
// (plane stride rows*ld) with a box of (128 bytes of K) x box_rows x 1,
// 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const void* base, int kind, long rows, long cols, long ld, int box_rows) {
    auto enc = get_encode();
    if (!enc) return false;
    CUtensorMapDataType dt = kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : (kind == 2 || kind == 5) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                             : kind == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                         : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const int es = elem_bytes(kind);
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)slices_of(kind)};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(rows * ld * es)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
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

template <int KIND, int BNT, int ST, int NACC>
void set_smem() {
    cudaFuncSetAttribute(k_gemm_tc<KIND, BNT, ST, NACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_bytes<BNT, ST>());
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
        return true;
    }();
    (void)done;
}

// C[i][j] -= scale * sum_{z < S} P[z][i][j] (z in increasing order), only
// i >= j when lower.  Launched as a programmatic dependent of the split GEMM:
// everything before pdl_wait overlaps the GEMM's last CTAs.
__global__ void __launch_bounds__(256) k_reduce_parts(float* __restrict__ C, long ldc, int M, int N,
                                                      const float* __restrict__ P, int S, float scale, int lower) {
    pdl_wait();
    if ((N & 3) == 0) {
        const int n4 = N >> 2;
        const long total = (long)M * n4;
        for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
            const int i = (int)(e / n4), j = (int)(e - (long)i * n4) * 4;
            if (lower && i < j) continue;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int z = 0; z < S; ++z) {
                const float4 p = __ldcg(reinterpret_cast<const float4*>(P + ((long)z * M + i) * N + j));
                acc.x += p.x;
                acc.y += p.y;
                acc.z += p.z;
                acc.w += p.w;
            }
            float4* cp = reinterpret_cast<float4*>(C + (long)i * ldc + j);
            float4 c = *cp;
            c.x -= scale * acc.x;
            if (!lower || i >= j + 1) c.y -= scale * acc.y;
            if (!lower || i >= j + 2) c.z -= scale * acc.z;
            if (!lower || i >= j + 3) c.w -= scale * acc.w;
            *cp = c;
        }
    } else {
        const long total = (long)M * N;
        for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
            const int i = (int)(e / N), j = (int)(e - (long)i * N);
            if (lower && i < j) continue;
            float acc = 0.f;
            for (int z = 0; z < S; ++z) acc += __ldcg(P + ((long)z * M + i) * N + j);
            C[(long)i * ldc + j] -= scale * acc;
        }
    }
}

}  // namespace

struct TcGemm {
    CUtensorMap mapA, mapB, mapB128;  // box heights 128 (A), 256 and 128 (B)
    CUtensorMap mapC;                 // C in 32 x 32 boxes (when has_map_c)
    bool has_map_c;
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

spd_status tc_gemm_create(TcGemm** out, float* W, long ldw, void* Wh, long ldh, int kind, int n) {
    return tc_gemm_create_maps(out, Wh, n, ldh, Wh, n, ldh, n, W, n, n, ldw, kind);
}

namespace {

template <int BNT>
void launch_kind(TcGemm* g, cudaStream_t s, dim3 grid, int cx0, int cy0, int M, int N, int K, int a_row0,
                 int b_row0, int k0, int lower, float scale, int nseg, uint32_t segs, uint32_t accsel, int kslice,
                 float* Cpart, long ldp, DevStatus* st) {
    const CUtensorMap& mb = BNT == 128 ? g->mapB128 : g->mapB;
    const uint32_t idesc = idesc_for(g->kind, BNT);
    // without a tensor map of C the epilogue writes C (the block's origin) directly
    float* Cdirect = g->has_map_c ? nullptr : g->C + (long)cy0 * g->ldc + cx0;
#define SPD_GEMM_ARGS                                                                                            \
    g->mapA, mb, g->mapC, Cdirect, g->ldc, cx0, cy0, M, N, K, a_row0, b_row0, k0, lower, idesc, scale, nseg, \
        segs, accsel, kslice, Cpart, ldp, st
    switch (g->kind) {
        case 1: k_gemm_tc<1, BNT, 4, 1><<<grid, 128, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS); break;
        case 5: {  // float32 as bf16 slices: two accumulators; two CTAs per SM on 128-wide tiles
            constexpr int ST = BNT == 128 ? 3 : 4;
            k_gemm_tc<0, BNT, ST, 2><<<grid, 128, smem_bytes<BNT, ST>(), s>>>(SPD_GEMM_ARGS);
            break;
        }
        case 4: k_gemm_tc<2, BNT, 4, 1><<<grid, 128, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS); break;
        default: k_gemm_tc<0, BNT, 4, 1><<<grid, 128, smem_bytes<BNT, 4>(), s>>>(SPD_GEMM_ARGS);
    }
#undef SPD_GEMM_ARGS
}

}  // namespace

spd_status tc_gemm_launch(TcGemm* g, cudaStream_t s, int cy0, int cx0, int M, int N, int K, int a_row0, int b_row0,
                          int k0, int lower, DevStatus* st, int splits, const TcSplit* sb) {
    const int bk = g->kind == 1 ? 32 : g->kind == 4 ? 128 : 64;
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
    const int bnt = (N <= 128) ? 128 : 256;
    const int tiles = ((N + bnt - 1) / bnt) * ((M + BM - 1) / BM);
    // splits < 0: choose from the SM count -splits, filling the machine once
    // (two CTAs per SM for the 128-wide float32 tiles)
    if (splits < 0) {
        const int occ = (bnt == 128 && g->kind == 5) ? 2 : 1;
        splits = std::max(1, std::min(16, occ * (-splits) / std::max(tiles, 1)));
    }
    if (splits > nk) splits = nk;
    const bool split = splits > 1 && sb && sb->part && (size_t)splits * M * N <= sb->part_cap;
    const int kslice = split ? (nk + splits - 1) / splits : 0;
    if (split) splits = (nk + kslice - 1) / kslice;  // no empty share
    dim3 grid((N + bnt - 1) / bnt, (M + BM - 1) / BM, split ? splits : 1);
    const long ldp = N;
    float* part = split ? sb->part : nullptr;
    if (bnt == 128)
        launch_kind<128>(g, s, grid, cx0, cy0, M, N, K, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, kslice,
                         part, ldp, st);
    else
        launch_kind<256>(g, s, grid, cx0, cy0, M, N, K, a_row0, b_row0, k0, lower, scale, nseg, segs, accsel, kslice,
                         part, ldp, st);
    if (split) {
        cudaLaunchConfig_t cfg = {};
        const long work = (long)M * ((N & 3) == 0 ? N / 4 : N);
        cfg.gridDim = dim3((unsigned)std::max<long>(1, std::min<long>((work + 255) / 256, 4L * g->sms)));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        float* C = g->C + (long)cy0 * g->ldc + cx0;
        if (cudaLaunchKernelEx(&cfg, k_reduce_parts, C, g->ldc, M, N, (const float*)part, splits, scale, lower) !=
            cudaSuccess)
            return SPD_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? SPD_OK : SPD_ERR_CUDA;
}

spd_status tc_gemm_run(TcGemm* g, cudaStream_t s, int r0, int M, int c0, int N, int k0, int K, int lower,
                       DevStatus* st, int splits, const TcSplit* sb) {
    return tc_gemm_launch(g, s, r0, c0, M, N, K, r0, c0, k0, lower, st, splits, sb);
}

void tc_gemm_destroy(TcGemm* g) { delete g; }
