// gemm_tc.h -- tensor-core (tcgen05) trailing update of the factorisation:
//     W[r0+r][c0+c] -= sum_k Wh[r0+r][k0+k] * Wh[c0+c][k0+k]
// with W float32 (row-major, ldw) and Wh the operand mirror (tf32 / bf16 /
// fp16 / fp8 e4m3, row-major, ldh), float32 accumulation in tensor memory.
#pragma once
#include <cuda_runtime.h>
#include "spd.h"
#include "common.cuh"

struct TcGemm;

// Split-K scratch of one stream: room for the partial sums (part_cap floats).
struct TcSplit {
    float* part;
    size_t part_cap;
};

// Plan for one factor: tensor maps over Wh for the operand tiles.
// Returns SPD_ERR_UNSUPPORTED when the operand kind has no tensor-core path.
spd_status tc_gemm_create(TcGemm** out, float* W, long ldw, void* Wh, long ldh, int kind, int n);
// splits = -S with scratch sb lets the GEMM spread the tiles' K loops over
// the S SMs ("stream-K": equal contiguous ranges of (tile, K tile) units per
// CTA) when that is estimated faster than one CTA per tile; the pieces of
// shared tiles go to partial slots (2 slots x 128 x 256 floats per CTA: 4 S x
// 128 x 128 floats suffice) that a dependent kernel adds to C in K order.
// splits = 0 takes stream-K whenever it gives more CTAs than tiles (on all
// SMs).  Otherwise (splits = 1, or without room in sb) one CTA per tile.
spd_status tc_gemm_run(TcGemm* g, cudaStream_t s, int r0, int M, int c0, int N, int k0, int K, int lower,
                       DevStatus* st, int splits = 1, const TcSplit* sb = nullptr);
void tc_gemm_destroy(TcGemm* g);
// General form: separate operand arrays (rows x cols, ld elements each) and
// C (c_rows x c_cols, ldc floats, row-major).
spd_status tc_gemm_create_maps(TcGemm** out, const void* Ah, long a_rows, long a_ld, const void* Bh, long b_rows,
                               long b_ld, long cols, float* C, long c_rows, long c_cols, long ldc, int kind);
// Narrow form for skinny products (B with few rows: the right-hand sides of
// CG): float32 operands as three bf16 slices (kind 5 mirrors), tiles of
// 128 x bnt (bnt = 32 or 64) whose pipeline stages hold all three slices of
// both operand tiles; b_rows a multiple of bnt, c_cols and ldc multiples of
// 32 for the epilogue's 32 x 32 boxes of C.
spd_status tc_gemm_create_narrow(TcGemm** out, const void* Ah, long a_rows, long a_ld, const void* Bh, long b_rows,
                                 long b_ld, long cols, float* C, long c_rows, long c_cols, long ldc, int bnt);
// C[cy0 + i][cx0 + j] -= sum_k A[a_row0 + i][k0 + k] B[b_row0 + j][k0 + k]
// for i < M, j < N (cx0 a multiple of 4).
spd_status tc_gemm_launch(TcGemm* g, cudaStream_t s, int cy0, int cx0, int M, int N, int K, int a_row0, int b_row0,
                          int k0, int lower, DevStatus* st, int splits = 1, const TcSplit* sb = nullptr);
