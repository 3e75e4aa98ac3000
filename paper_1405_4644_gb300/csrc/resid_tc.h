// resid_tc.h -- the float64-accurate residual R = B - A X of Algorithm 1
// (lines 3, 7) and Algorithm 2 (line 2) on the bf16 tensor cores, by exact
// digit products (the splitting scheme of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication", 2012).
//
// Every row i of A is written as a_ij = 2^e_i sum_{p=1..10} D_p(i,j) 2^{-7p}
// with signed integer digits |D_p| <= 64 (truncating a_ij below
// 2^{e_i - 70}; e_i = ilogb(max_j |a_ij|) + 2), and every column c of X
// likewise with exponent f_c.  Digits are exact in bf16.  For each group
// t = p + q <= 11 (55 products) the tensor cores form sum_j D_p(i,j) E_q(j,c)
// exactly: each 64-wide chunk of j is accumulated in float32 (at most
// 10 x 64 x 64^2 < 2^22 in magnitude: exact integers) and added to integer
// sums.  The groups are combined in double-double with their scales
// 2^{e_i + f_c - 7t}, and b - (A X) is rounded once.  Per term the dropped
// products (t >= 12) and the truncation are below 2^-64.5 max_j|a_ij| max|x_c|.
#pragma once
#include <cuda.h>
#include <stdint.h>
#include "engine.cuh"

struct TcResidWs {
    CUtensorMap mapA, mapX;      // digit planes of A (rows) and of X (columns)
    uint16_t* Ad = nullptr;      // [10][n][ldp] bf16 digits of A's rows
    uint16_t* Xd = nullptr;      // [10][m][ldp] bf16 digits of X's columns
    unsigned long long* rowmax = nullptr;  // n: bits of max_j |a_ij|
    float* rowabs = nullptr;     // RS x n: partial sums of |a_ij| (float32)
    int* xe = nullptr;           // m: column exponents of X (INT_MIN: non-finite)
    unsigned long long* part = nullptr;  // (CB RB) x 10 x 16 x 128: 64-bit integer group sums
    long ldp = 0;
    int n = 0, m = 0, RS = 1, RB = 0, CB = 0, Nkc = 0, G = 0;
    long T = 0;                  // work items (column block, row block, K chunk)
};

// Workspace layout for an n x n matrix and m right-hand sides (6 offsets).
size_t tc_resid_plan(WsPlan& p, spd_handle* h, int n, int m, size_t* off);
// Bind the workspace and encode the tensor maps.  SPD_ERR_UNSUPPORTED when
// the driver has no tensor-map encoder.
spd_status tc_resid_bind(spd_handle* h, TcResidWs* w, int n, int m, const size_t* off);
// Row exponents, row sums of |A| and the digit planes of A (once per A).
spd_status tc_resid_prepare(spd_handle* h, TcResidWs* w, const double* A, long lda);
// R = B - A X (mode 0) or R = A X (mode 1) for the A of the last prepare;
// block partial norms into NP (256-row blocks, as k_resid_final).
// gate (device int, may be NULL): every kernel returns at once when it is 0
// (the refinement of a capturable solve is over)
spd_status tc_resid_run(spd_handle* h, const TcResidWs* w, const double* B, long ldb, const double* X, long ldx,
                        double* R, long ldr, double* NP, int mode, const int* gate = nullptr);
