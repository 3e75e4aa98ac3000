// spd_gemm.cu -- the tensor-core trailing update exposed as a standalone
// C-ABI operation (operands rounded into tensor-core mirrors first).
#include "engine.cuh"
#include "gemm_tc.h"

namespace {

// out[r][k] = round(A[r][k]) for k < K, 0 for K <= k < Kp  (row-major, ldo;
// slice planes of plane_rows rows)
__global__ void k_to_mirror(const float* __restrict__ A, long lda, int rows, int K, int Kp, void* out, long ldo,
                            int kind, long plane_rows) {
    long total = (long)rows * Kp;
    Mirror m{out, ldo, kind, plane_rows * ldo};
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        long r = e / Kp, k = e - r * Kp;
        float v = (k < K) ? A[r * lda + k] : 0.f;
        mirror_store(m, r, k, v);
    }
}

int kind_of(int prec) {
    switch (prec) {
        case SPD_PREC_FP32: return 5;
        case SPD_PREC_TF32: return 1;
        case SPD_PREC_BF16: return 2;
        case SPD_PREC_FP16: return 3;
        case SPD_PREC_FP8: return 4;
        default: return 0;
    }
}

}  // namespace

extern "C" spd_status spd_gemm_update(spd_handle* h, int prec, int M, int N, int K, const float* A, int lda,
                                      const float* B, int ldb, float* C, int ldc, int flags) {
    if (!h) return SPD_ERR_ARG;
    if ((unsigned)flags & ~7u) return set_err(h, SPD_ERR_ARG, "spd_gemm_update: unknown flags 0x%x", flags);
    const int lower = flags & SPD_GEMM_LOWER;
    const bool stream_k = (flags & SPD_GEMM_STREAM_K) != 0;
    const bool narrow = (flags & SPD_GEMM_NARROW) != 0;
    if (narrow && (prec != SPD_PREC_FP32 || lower))
        return set_err(h, SPD_ERR_UNSUPPORTED, "spd_gemm_update: narrow tiles take FP32 operands and no LOWER");
    const int kind = kind_of(prec);
    if (!kind)
        return set_err(h, SPD_ERR_UNSUPPORTED, "spd_gemm_update: precision must be FP32, TF32, BF16, FP16 or FP8");
    if (M < 0 || N < 0 || K < 0 || (M > 0 && K > 0 && (!A || lda < K)) || (N > 0 && K > 0 && (!B || ldb < K)) ||
        (M > 0 && N > 0 && (!C || ldc < N)) || (lower && (M != N || A != B || lda != ldb)))
        return set_err(h, SPD_ERR_ARG, "spd_gemm_update: bad arguments");
    if (M == 0 || N == 0 || K == 0) return SPD_OK;
    const int es = kind == 5 ? 6 : kind == 1 ? 4 : kind == 4 ? 1 : 2;  // bytes per element over all slices
    const long Kp = round_up(K, 128);
    const long ldo = round_up(Kp, 64);
    const int bnt = N <= 32 ? 32 : 64;                 // narrow tile width
    const long nbrows = narrow ? round_up(N, bnt) : N;  // narrow: B rows padded with zeros to whole tiles
    WsPlan p;
    size_t oa = p.add<unsigned char>((size_t)M * ldo * es);
    size_t ob = lower ? oa : p.add<unsigned char>((size_t)nbrows * ldo * es);
    const size_t part_cap = (size_t)4 * std::max(h->sms, 1) * 128 * 128;  // stream-K partial slots
    size_t op = stream_k ? p.add<float>(part_cap) : 0;
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    void* Ah = ws_at<unsigned char>(h, oa);
    void* Bh = ws_at<unsigned char>(h, ob);
    cudaStream_t s = h->stream;
    if (narrow && nbrows > N) CUDA_TRY(h, cudaMemsetAsync(Bh, 0, (size_t)nbrows * ldo * es, s));
    ++h->launches, k_to_mirror<<<grid_for((long)M * Kp, 256, 8 * h->sms), 256, 0, s>>>(A, lda, M, K, (int)Kp, Ah, ldo,
                                                                                        kind, (long)M);
    if (!lower)
        ++h->launches, k_to_mirror<<<grid_for((long)N * Kp, 256, 8 * h->sms), 256, 0, s>>>(B, ldb, N, K, (int)Kp, Bh,
                                                                                            ldo, kind, nbrows);
    LAUNCH_CHECK(h);
    TcGemm* g = nullptr;
    st = narrow ? tc_gemm_create_narrow(&g, Ah, M, ldo, Bh, nbrows, ldo, Kp, C, M, N, ldc, bnt)
                : tc_gemm_create_maps(&g, Ah, M, ldo, Bh, N, ldo, Kp, C, M, N, ldc, kind);
    if (st != SPD_OK) return set_err(h, st, "spd_gemm_update: tensor map creation failed");
    ++h->launches;
    {
        const double celems = lower ? 0.5 * (double)M * (M + 1) : (double)M * N;  // (narrow: padding rows not counted)
        ProfScope ps(h, SPD_PHASE_TRAILING, 2.0 * celems * K,
                     8.0 * celems + (double)es * Kp * (lower ? M : (double)M + N));
        TcSplit sb{stream_k ? ws_at<float>(h, op) : nullptr, part_cap};
        st = tc_gemm_launch(g, s, 0, 0, M, N, (int)Kp, 0, 0, 0, lower, h->dst, stream_k ? 0 : 1, &sb);
    }
    tc_gemm_destroy(g);
    if (st != SPD_OK) return set_err(h, st, "spd_gemm_update: launch failed");
    return check_dev_status(h, nullptr, "spd_gemm_update");
}
