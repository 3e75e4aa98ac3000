// spd_factor.cu -- Algorithm 1 line 1: the low-precision Cholesky
// factorisation A ~= R~^T R~ (Section 3.1, eq. (cholesky)), in one of two
// blocked schedules with 128x128 leaves (k_potrf_leaf32 / k_trsm_leaf32;
// k_potrf_leaf / k_trsm_leaf for FP64):
//
// - left-looking over 128-column block columns (potrf_left; the tensor-core
//   precisions by default): W[k:, k] -= L[k:, 0:k] L[k, 0:k]^T, leaf, panel
//   solve, with the bulk of the updates issued ahead, for two block columns
//   at a time, on the handle's second stream;
// - recursive (potrf_rec; FP64, the CUDA-core engine, SPD_FACTOR_RECURSIVE):
//     chol(A)   : chol(A11); L21 = A21 L11^{-T}; A22 -= L21 L21^T; chol(A22)
//     trsm(B,L) : trsm(B1, L11); B2 -= X1 L21^T; trsm(B2, L22)
//
// Every off-leaf update is a GEMM on the working matrix (tensor cores for
// TF32/BF16/FP16/FP8 and for FP32 as three bf16 slices; CUDA cores for
// FP64).  Split points are multiples of 128, so only the very last leaf can
// be ragged.
#include "engine.cuh"
#include "k_convert.cuh"
#include "k_leaf.cuh"
#include "k_leaf32.cuh"
#include "k_gemm_simt.cuh"
#include "k_trsv_sb.cuh"
#include "k_lanczos.cuh"
#include "gemm_tc.h"

namespace {

struct FCtx {
    spd_handle* h;
    spd_factor_t* F;
    Mirror mir;
    TcGemm* tc;               // tensor-core GEMM plan (nullptr: CUDA cores)
    TcSplit* bulk = nullptr;  // split-K scratch of the bulk updates (second stream)
};



// Launch with programmatic stream serialization: the kernel may be scheduled
// before the previous kernel in the stream finishes and waits for it itself
// (pdl_wait), which hides the launch gap on the factorisation's critical path.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename T>
spd_status leaf_potrf(FCtx& c, int k, int nb) {
    spd_factor_t* F = c.F;
    ProfScope ps(c.h, SPD_PHASE_LEAF, (double)nb * nb * nb / 3.0, (double)nb * nb * sizeof(T));
    if constexpr (sizeof(T) == 8) {
        ++(c.h)->launches, k_potrf_leaf<double><<<1, 256, potrf_leaf_smem<double>(), c.h->stream>>>(
            F->W64, F->ldw, k, nb, F->Dinv64, c.mir, c.h->dst);
    } else {
        ++(c.h)->launches;
        CUDA_TRY(c.h, launch_pdl(k_potrf_leaf32, dim3(1), dim3(256), potrf_leaf32_smem(), c.h->stream, F->W, F->ldw, k,
                                 nb, F->Dinv32, c.mir, c.h->dst));
    }
    LAUNCH_CHECK(c.h);
    return SPD_OK;
}

// b_ready: B (rows r0 .., block column c0) is final before the previous
// kernel in the stream, which is then the leaf of block c0
template <typename T>
spd_status leaf_trsm(FCtx& c, int r0, int m, int c0, int kb, bool b_ready = false) {
    spd_factor_t* F = c.F;
    ProfScope ps(c.h, SPD_PHASE_PANEL, (double)m * kb * kb, 2.0 * m * kb * sizeof(T));
    if constexpr (sizeof(T) == 8) {
        ++(c.h)->launches, k_trsm_leaf<double, 32><<<ceil_div(m, 32), 256, trsm_leaf_smem<double, 32>(), c.h->stream>>>(
            F->W64, F->ldw, r0, m, c0, kb, F->Dinv64, c.mir, c.h->dst);
    } else {
        ++(c.h)->launches;
        CUDA_TRY(c.h, launch_pdl(k_trsm_leaf32, dim3(ceil_div(m, 64)), dim3(256), trsm_leaf32_smem(), c.h->stream,
                                 F->W, F->ldw, r0, m, c0, (const float*)F->Dinv32, c.mir, (const DevStatus*)c.h->dst,
                                 b_ready ? 1 : 0));
    }
    LAUNCH_CHECK(c.h);
    return SPD_OK;
}

// crit: a rank-128 update on the factorisation's critical path (recorded
// as SPD_PHASE_TRAILING_LAST); otherwise a bulk update.  lower (r0 == c0):
// only entries with row >= column are updated.
template <typename T>
spd_status gemm(FCtx& c, int r0, int M, int c0, int N, int k0, int K, int lower, int splits = 1,
                cudaStream_t strm = nullptr, const TcSplit* sb = nullptr, bool crit = false) {
    if (M <= 0 || N <= 0 || K <= 0) return SPD_OK;
    spd_factor_t* F = c.F;
    cudaStream_t s = strm ? strm : c.h->stream;
    // algorithmic work: the lower part of an M x N block on the diagonal
    // (sum over its columns c < min(M, N) of M - c entries) or the full
    // block; C read+written once in T, each operand row read once in the
    // operand type (B's rows are A's first rows when lower)
    const double w = (double)std::min(M, N);
    const double celems = lower ? w * M - 0.5 * w * (w - 1.0) : (double)M * N;
    const double opsz = sizeof(T) == 8 ? 8.0
                        : c.mir.kind == 5 ? 6.0
                        : (c.mir.kind == 0 || c.mir.kind == 1 ? 4.0 : c.mir.kind == 4 ? 1.0 : 2.0);
    const int phase = crit ? SPD_PHASE_TRAILING_LAST
                           : (c.tc && c.mir.kind == 5) ? SPD_PHASE_TRAILING_X3 : SPD_PHASE_TRAILING;
    ProfScope ps(c.h, phase, 2.0 * celems * K,
                 2.0 * sizeof(T) * celems + opsz * (double)K * (lower ? M : (double)M + N), s);
    if constexpr (sizeof(T) == 8) {
        dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
        ++(c.h)->launches, k_gemm_nt_simt<double, double, 4, 4, 8><<<grid, 256, 0, s>>>(F->W64, F->ldw, F->W64, F->ldw, r0, M, c0, N,
                                                                     k0, K, lower, c.h->dst);
    } else {
        if (c.tc) {
            spd_status st = tc_gemm_run(c.tc, s, r0, M, c0, N, k0, K, lower, c.h->dst, splits, sb);
            if (st != SPD_OK) return set_err(c.h, st, "tensor-core trailing update failed");
            return SPD_OK;
        }
        dim3 grid(ceil_div(N, 128), ceil_div(M, 128));
        switch (c.mir.kind) {
            case 0:
            case 5:  // float32: plain products of the working matrix
            ++(c.h)->launches, k_gemm_nt_simt<float, float, 8, 8, 8><<<grid, 256, 0, s>>>(F->W, F->ldw, F->W, F->ldw, r0, M, c0,
                                                                           N, k0, K, lower, c.h->dst);
                break;
            case 1:
            ++(c.h)->launches, k_gemm_nt_simt<float, float, 8, 8, 8><<<grid, 256, 0, s>>>(
                    F->W, F->ldw, (const float*)F->Wh, F->ldh, r0, M, c0, N, k0, K, lower, c.h->dst);
                break;
            case 2:
            ++(c.h)->launches, k_gemm_nt_simt<float, __nv_bfloat16, 8, 8, 8><<<grid, 256, 0, s>>>(
                    F->W, F->ldw, (const __nv_bfloat16*)F->Wh, F->ldh, r0, M, c0, N, k0, K, lower, c.h->dst);
                break;
            case 3:
            ++(c.h)->launches, k_gemm_nt_simt<float, __half, 8, 8, 8><<<grid, 256, 0, s>>>(
                    F->W, F->ldw, (const __half*)F->Wh, F->ldh, r0, M, c0, N, k0, K, lower, c.h->dst);
                break;
            default:
                return set_err(c.h, SPD_ERR_UNSUPPORTED, "no CUDA-core path for this operand type");
        }
    }
    LAUNCH_CHECK(c.h);
    return SPD_OK;
}

inline int split_point(int nn) {
    int n1 = ((nn / 2 + SPD_LEAF - 1) / SPD_LEAF) * SPD_LEAF;
    if (n1 >= nn) n1 = nn - SPD_LEAF;
    return n1;
}

#define TRY(x)                            \
    do {                                  \
        spd_status s_ = (x);              \
        if (s_ != SPD_OK) return s_;      \
    } while (0)

template <typename T>
spd_status trsm_rec(FCtx& c, int r0, int m, int c0, int k) {
    if (m <= 0) return SPD_OK;
    if (k <= SPD_LEAF) return leaf_trsm<T>(c, r0, m, c0, k);
    int k1 = split_point(k);
    TRY(trsm_rec<T>(c, r0, m, c0, k1));
    TRY(gemm<T>(c, r0, m, c0 + k1, k - k1, c0, k1, 0));
    return trsm_rec<T>(c, r0, m, c0 + k1, k - k1);
}

template <typename T>
spd_status potrf_rec(FCtx& c, int n0, int nn) {
    if (nn <= SPD_LEAF) return leaf_potrf<T>(c, n0, nn);
    int n1 = split_point(nn);
    TRY(potrf_rec<T>(c, n0, n1));
    TRY(trsm_rec<T>(c, n0 + n1, nn - n1, n0, n1));
    TRY(gemm<T>(c, n0 + n1, nn - n1, n0 + n1, nn - n1, n0, n1, 1));
    return potrf_rec<T>(c, n0 + n1, nn - n1);
}

// Left-looking block-column schedule with a look-ahead (tensor-core
// factors).  Block columns are taken in pairs P = (j, j+1), j even.  Block
// column k needs every panel to its left applied:
//   bulk (second stream): W[j:, j:j+2] -= L[j:, 0:j-1] L[j:j+2, 0:j-1]^T
//        for the whole pair, as soon as panel j-2 is done; 256-wide tiles
//        (entries above the diagonal are left alone);
//   last (main stream, rank 128, on the critical path):
//        block j:   W[j:, j:j+2] -= L[j:, j-1] L[j:j+2, j-1]^T  (both columns)
//        block j+1: W[j+1:, j+1] -= L[j+1:, j] L[j+1, j]^T
// each followed by the block's leaf and the panel solve below it.  The bulk
// update of a pair, which holds nearly all of the tensor-core work, runs
// while the previous block's last update, leaf and panel run; the bulk
// update of pair P waits for panel j-2, the last update of block j for the
// bulk update of its pair (both write W[j:, j:j+2]).
template <typename T>
spd_status potrf_left(FCtx& c, int n, bool lookahead) {
    spd_handle* h = c.h;
    const int NB = ceil_div(n, SPD_LEAF);
    // without the look-ahead both parts run in order on the main stream
    cudaStream_t P = h->stream, U = lookahead ? h->aux : h->stream;
    // two events per block: panel done (main), bulk update of the pair
    // starting at this block done (second)
    const size_t need = 2 * (size_t)NB + 1;
    while (h->sync_ev.size() < need) {
        cudaEvent_t e = nullptr;
        CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->sync_ev.push_back(e);
    }
    cudaEvent_t* evPanel = h->sync_ev.data();
    cudaEvent_t* evBulk = h->sync_ev.data() + NB;
    cudaEvent_t evStart = h->sync_ev[2 * NB];
    CUDA_TRY(h, cudaEventRecord(evStart, P));  // the second stream starts after the conversion
    CUDA_TRY(h, cudaStreamWaitEvent(U, evStart, 0));
    spd_status st = SPD_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < NB && st == SPD_OK && e == cudaSuccess; ++k) {
        const int r0 = k * SPD_LEAF, nb = std::min(SPD_LEAF, n - r0), M = n - r0;
        const bool pair_start = (k % 2) == 0;
        if (pair_start && k >= 2) e = cudaStreamWaitEvent(P, evBulk[k], 0);
        if (e == cudaSuccess && k >= 1) {  // last: rank 128 with block column k-1
            if (pair_start)
                st = gemm<T>(c, r0, M, r0, std::min(2 * SPD_LEAF, M), r0 - SPD_LEAF, SPD_LEAF, 1, 1, P, nullptr, true);
            else
                st = gemm<T>(c, r0, M, r0, nb, r0 - SPD_LEAF, SPD_LEAF, 0, 1, P, nullptr, true);
        }
        if (e == cudaSuccess && st == SPD_OK) st = leaf_potrf<T>(c, r0, nb);
        if (e == cudaSuccess && st == SPD_OK && r0 + nb < n)
            st = leaf_trsm<T>(c, r0 + nb, n - r0 - nb, r0, nb, true);  // right after the leaf
        if (e != cudaSuccess || st != SPD_OK) break;
        e = cudaEventRecord(evPanel[k], P);
        // bulk update of the pair starting at block k+2 on the second stream:
        // panels 0..k
        if (e == cudaSuccess && pair_start && k + 2 < NB) {
            e = cudaStreamWaitEvent(U, evPanel[k], 0);
            const int r2 = (k + 2) * SPD_LEAF, M2 = n - r2;
            if (e == cudaSuccess)
                st = gemm<T>(c, r2, M2, r2, std::min(2 * SPD_LEAF, M2), 0, (k + 1) * SPD_LEAF, 1,
                             c.bulk ? -h->sms : 1, U, c.bulk);
            if (e == cudaSuccess) e = cudaEventRecord(evBulk[k + 2], U);
        }
    }
    // join, on every path: the main stream continues (and frees the split
    // scratch) only after everything queued on the second stream
    cudaEvent_t evEnd = h->sync_ev[2 * NB];
    cudaError_t e2 = cudaEventRecord(evEnd, U);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(P, evEnd, 0);
    if (e2 != cudaSuccess) cudaStreamSynchronize(U);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess && st == SPD_OK) st = set_err(h, SPD_ERR_CUDA, "look-ahead schedule: %s", cudaGetErrorString(e));
    return st;
}

void free_factor(spd_factor_t* F) {
    if (!F) return;
    // stream-ordered frees: no device-wide synchronisation, so factors on
    // other handles' streams keep running
    cudaStream_t s = F->h ? F->h->stream : nullptr;
    for (void* p : {(void*)F->W, (void*)F->W64, F->Wh, (void*)F->d, (void*)F->LinvT, (void*)F->Cpl, (void*)F->Dinv32,
                    (void*)F->Dinv64, (void*)F->Xsb})
        if (p) cudaFreeAsync(p, s);
    delete F;
}

int mirror_kind(int prec) {
    switch (prec) {
        case SPD_PREC_FP32: return 5;
        case SPD_PREC_TF32: return 1;
        case SPD_PREC_BF16: return 2;
        case SPD_PREC_FP16: return 3;
        case SPD_PREC_FP8: return 4;
        default: return 0;
    }
}
size_t mirror_elem(int kind) { return kind == 5 ? 6 : kind == 1 ? 4 : kind == 4 ? 1 : 2; }

// Extreme eigenvalues of the symmetric tridiagonal T (diagonal a[0..k-1],
// off-diagonal b[0..k-2]) by bisection on Sturm counts (the number of
// negative pivots of T - x I is the number of eigenvalues below x).
static int sturm_below(const double* a, const double* b, int k, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
        if (d == 0.0) d = -1e-300;  // x on an eigenvalue of a leading block: count it below
        cnt += d < 0.0;
    }
    return cnt;
}

static void tridiag_extremes(const double* a, const double* b, int k, double* lo_out, double* hi_out) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {  // Gershgorin interval
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    double l = lo, u = hi;  // smallest: the first x with one eigenvalue below
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(fabs(l), fabs(u)); ++it) {
        const double mid = 0.5 * (l + u);
        if (sturm_below(a, b, k, mid) >= 1) u = mid; else l = mid;
    }
    *lo_out = u;
    l = lo, u = hi;  // largest: the first x with all k below
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(fabs(l), fabs(u)); ++it) {
        const double mid = 0.5 * (l + u);
        if (sturm_below(a, b, k, mid) >= k) u = mid; else l = mid;
    }
    *hi_out = u;
}

// Lanczos lower bound on kappa_2 of the scaled matrix in W (float32 lower
// triangle, row-major): at most LZ_MAXK steps, checked every four from the
// eighth; stops as soon as the bound exceeds `stop_above` (or the Krylov
// space becomes invariant).  *bound = theta_max / theta_min of the last
// check (+inf when theta_min <= 0: the float32 products do not resolve
// lambda_min), 0 when the scratch could not be had (no bound).  From the
// twelfth step on it also stops when the bound is below half the threshold
// and grew by less than 10 % since the previous check: the decision then
// falls to the test after the FP16 factor, as it would without a bound.
spd_status lanczos_lower(spd_handle* h, const float* W, long ldw, int n, double stop_above, double* bound,
                         int* steps) {
    *bound = 0.0;
    *steps = 0;
    const int nb = ceil_div(n, LZ_T);
    const long ldq = round_up(n, 4);
    const size_t bytesP = sizeof(float) * (size_t)nb * nb * LZ_T;
    const size_t bytesQ = sizeof(float) * (size_t)(LZ_MAXK + 2) * ldq;  // Q_0..Q_K and y
    const size_t bytesD = sizeof(double) * ((LZ_MAXK + 1) * LZ_CHUNKS + LZ_CHUNKS + 2 * LZ_MAXK);
    if (over_cap(h, bytesP + bytesQ + bytesD)) return SPD_OK;
    cudaStream_t s = h->stream;
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, bytesP + bytesQ + bytesD, s) != cudaSuccess) {
        cudaGetLastError();
        return SPD_OK;  // no bound: the caller proceeds as without one
    }
    float* P = static_cast<float*>(mem);
    float* Q = reinterpret_cast<float*>(static_cast<char*>(mem) + bytesP);
    float* y = Q + (size_t)(LZ_MAXK + 1) * ldq;
    double* dpart = reinterpret_cast<double*>(static_cast<char*>(mem) + bytesP + bytesQ);
    double* npart = dpart + (LZ_MAXK + 1) * LZ_CHUNKS;
    double* alpha = npart + LZ_CHUNKS;
    double* beta = alpha + LZ_MAXK;
    ProfScope pl(h, SPD_PHASE_ESTIMATE, 0.0, 0.0);
    const long tiles = (long)nb * (nb + 1) / 2;
    ++h->launches, k_lz_start<<<ceil_div(n, 256), 256, 0, s>>>(y, n);
    ++h->launches, k_lz_orth<<<LZ_CHUNKS, 256, 0, s>>>(Q, ldq, y, n, -1, dpart, npart, alpha);
    ++h->launches, k_lz_normalize<<<LZ_CHUNKS, 256, 0, s>>>(y, Q, n, -1, npart, beta);
    spd_status st = SPD_OK;
    double ha[LZ_MAXK], hb[LZ_MAXK];
    double prev = 0.0;
    int j = 0;
    for (; j < LZ_MAXK; ++j) {
        ++h->launches, k_lz_symv_tiles<<<(unsigned)tiles, 256, 0, s>>>(W, ldw, n, nb, Q + (size_t)j * ldq, P);
        ++h->launches, k_lz_symv_reduce<<<nb, dim3(LZ_T, 8), 0, s>>>(P, n, nb, y);
        ++h->launches, k_lz_dots<<<dim3(LZ_CHUNKS, j + 1), 256, 0, s>>>(Q, ldq, y, n, dpart);
        ++h->launches, k_lz_orth<<<LZ_CHUNKS, 256, 0, s>>>(Q, ldq, y, n, j, dpart, npart, alpha);
        ++h->launches, k_lz_normalize<<<LZ_CHUNKS, 256, 0, s>>>(y, Q + (size_t)(j + 1) * ldq, n, j, npart, beta);
        const int k = j + 1;
        if (k < 8 || (k % 4 && k < LZ_MAXK)) continue;
        if (cudaGetLastError() != cudaSuccess) {
            st = set_err(h, SPD_ERR_CUDA, "condition bound: launch failed");
            break;
        }
        cudaError_t e = cudaMemcpyAsync(ha, alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb, beta, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = set_err(h, SPD_ERR_CUDA, "condition bound: %s", cudaGetErrorString(e));
            break;
        }
        // an invariant subspace ends the iteration: T_k's Ritz values are then
        // eigenvalues of As; stop at the first vanishing beta
        int kk = k;
        for (int i = 0; i < k - 1; ++i)
            if (!(hb[i] > 1e-7 * (fabs(ha[i]) + fabs(ha[i + 1])))) {
                kk = i + 1;
                break;
            }
        double lo = 0.0, hi = 0.0;
        tridiag_extremes(ha, hb, kk, &lo, &hi);
        *bound = lo > 0.0 ? hi / lo : INFINITY;
        *steps = kk;
        if (!(*bound <= stop_above) || kk < k || !(hb[k - 1] > 1e-7 * fabs(ha[k - 1]))) break;
        if (k >= 12 && *bound <= 0.5 * stop_above && *bound <= 1.1 * prev) break;  // settled well below
        prev = *bound;
    }
    // work of the symmetric products that ran: 2 n^2 flops, the lower
    // triangle read once (4 n^2 / 2 bytes) and the tile partials written and read
    const double ran = std::min(j + 1, LZ_MAXK);
    pl.r.flops = ran * 2.0 * n * (double)n;
    pl.r.bytes = ran * (2.0 * n * (double)n + 2.0 * bytesP);
    cudaFreeAsync(mem, s);
    return st;
}

// One factorisation attempt in a fixed precision.
// The AUTO pre-check of one attempt: when `lz` is given and n >= LZ_MIN_N,
// the Lanczos bound on the freshly scaled matrix runs before the factor, and
// a bound above lz->stop_above ends the attempt (SPD_ERR_NOT_SPD, lz->skip).
struct LzCheck {
    double stop_above;
    double bound;
    int steps;
    bool skip;
};
constexpr int LZ_MIN_N = 4096;

spd_status factor_once(spd_handle* h, int n, const double* A, int lda, int prec, unsigned flags,
                       spd_factor_t** out, spd_report* rep, double shift = 0.0, LzCheck* lz = nullptr) {
    spd_factor_t* F = new spd_factor_t();
    F->h = h;
    F->n = n;
    F->prec = prec;
    F->ldw = round_up(std::max(n, 1), 64);
    F->nblk128 = ceil_div(n, SPD_LEAF);
    const size_t nW = (size_t)n * F->ldw;
    // the float32 factor's mirror (three bf16 slices) is only needed by the
    // tensor-core engine
    const int kind = (prec == SPD_PREC_FP32 && (flags & SPD_FACTOR_CUDA_CORES)) ? 0 : mirror_kind(prec);
    auto fail = [&](spd_status s) {
        free_factor(F);
        return s;
    };
    {  // the factor's whole device request against the handle's cap
        const size_t nb = (size_t)std::max(F->nblk128, 1);
        size_t req = sizeof(double) * std::max(n, 1);
        if (prec == SPD_PREC_FP64) req += sizeof(double) * (std::max<size_t>(nW, 1) + 4096 * nb);
        else req += sizeof(float) * (std::max<size_t>(nW, 1) + (1 + 4 + 0.25) * 16384 * nb) +
                    (kind ? mirror_elem(kind) * std::max<size_t>(nW, 1) : 0) +
                    (nb >= 2 * SPD_SB_BLOCKS && !(flags & SPD_FACTOR_BLOCK_SWEEPS)
                         ? sizeof(float) * (size_t)ceil_div((long)nb, SPD_SB_BLOCKS) * SPD_SB_BLOCKS * 128 *
                               SPD_SB_BLOCKS * 128
                         : 0);
        if (over_cap(h, req))
            return fail(set_err(h, SPD_ERR_OOM, "factor of order %d needs %zu bytes, above the handle's memory cap "
                                "of %zu bytes", n, req, h->mem_cap));
    }
    cudaError_t e = cudaSuccess;
    cudaStream_t as = h->stream;  // stream-ordered allocations (see free_factor)
    e = cudaMallocAsync(&F->d, sizeof(double) * std::max(n, 1), as);
    if (e == cudaSuccess && prec == SPD_PREC_FP64) {
        e = cudaMallocAsync(&F->W64, sizeof(double) * std::max<size_t>(nW, 1), as);
        if (e == cudaSuccess) e = cudaMallocAsync(&F->Dinv64, sizeof(double) * 4096 * std::max(F->nblk128, 1), as);
    } else if (e == cudaSuccess) {
        e = cudaMallocAsync(&F->W, sizeof(float) * std::max<size_t>(nW, 1), as);
        if (e == cudaSuccess) e = cudaMallocAsync(&F->LinvT, sizeof(float) * 128 * 128 * std::max(F->nblk128, 1), as);
        if (e == cudaSuccess) e = cudaMallocAsync(&F->Cpl, sizeof(float) * 4 * 128 * 128 * std::max(F->nblk128, 1), as);
        if (e == cudaSuccess) e = cudaMallocAsync(&F->Dinv32, sizeof(float) * 4096 * std::max(F->nblk128, 1), as);
        if (e == cudaSuccess && kind) {
            F->ldh = F->ldw;
            e = cudaMallocAsync(&F->Wh, mirror_elem(kind) * std::max<size_t>(nW, 1), as);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(set_err(h, e == cudaErrorMemoryAllocation ? SPD_ERR_OOM : SPD_ERR_CUDA,
                            "factor allocation (n=%d): %s", n, cudaGetErrorString(e)));
    }
    cudaStream_t s = h->stream;
    if (n > 0) {
        ProfScope* pconv = new ProfScope(h, SPD_PHASE_CONVERT, 3.0 * n * (double)n / 2.0,
                                         8.0 * n * (double)n / 2.0 + (prec == SPD_PREC_FP64 ? 8.0 : 4.0) * n * (double)n / 2.0);
                                         ++(h)->launches, k_diag_scale<<<ceil_div(n, 256), 256, 0, s>>>(A, lda, n, (flags & SPD_SCALE_DIAG) ? 1 : 0, F->d, h->dst);
        const long nt = ceil_div(n, 64), ntiles = nt * (nt + 1) / 2;  // lower-triangle 64 x 64 tiles
        if (prec == SPD_PREC_FP64)
            ++(h)->launches, k_scale_convert<double><<<(unsigned)ntiles, 256, 0, s>>>(A, lda, n, F->d, F->W64,
                                                                                          F->ldw, h->dst);
        else
            ++(h)->launches, k_scale_convert<float><<<(unsigned)ntiles, 256, 0, s>>>(A, lda, n, F->d, F->W,
                                                                                         F->ldw, h->dst);
        if (shift > 0.0) {  // SPD_FACTOR_SHIFT: factor the scaled matrix plus shift I
            if (prec == SPD_PREC_FP64)
                ++(h)->launches, k_add_diag<double><<<ceil_div(n, 256), 256, 0, s>>>(F->W64, F->ldw, n, shift);
            else
                ++(h)->launches, k_add_diag<float><<<ceil_div(n, 256), 256, 0, s>>>(F->W, F->ldw, n, shift);
        }
        delete pconv;
        if (cudaGetLastError() != cudaSuccess) return fail(set_err(h, SPD_ERR_CUDA, "convert launch failed"));
        spd_status st = check_dev_status(h, rep, "spd_factor");
        if (st != SPD_OK) return fail(st);
        if (lz && n >= LZ_MIN_N && prec != SPD_PREC_FP64) {
            st = lanczos_lower(h, F->W, F->ldw, n, lz->stop_above, &lz->bound, &lz->steps);
            if (st != SPD_OK) return fail(st);
            if (!(lz->bound <= lz->stop_above)) {
                lz->skip = true;
                return fail(SPD_ERR_NOT_SPD);
            }
        }

        FCtx c{h, F, Mirror{F->Wh, F->ldh, kind, (long)n * F->ldh}, nullptr};
        TcGemm* tc = nullptr;
        if (kind && !(flags & SPD_FACTOR_CUDA_CORES)) {
            st = tc_gemm_create(&tc, F->W, F->ldw, F->Wh, F->ldh, kind, n);
            if (st == SPD_OK) c.tc = tc;
            else if (st != SPD_ERR_UNSUPPORTED) return fail(set_err(h, st, "tensor-core plan failed"));
        }
        if (prec == SPD_PREC_FP64) {
            st = potrf_rec<double>(c, 0, n);
        } else if (c.tc && !(flags & SPD_FACTOR_RECURSIVE)) {
            // stream-K partial slots of the bulk updates: 2 per CTA, at most
            // 2 sms CTAs of 128 x 128 or sms CTAs of 128 x 256
            TcSplit sb{nullptr, (size_t)4 * std::max(h->sms, 1) * 128 * 128};
            void* mem = nullptr;
            if (cudaMallocAsync(&mem, sizeof(float) * sb.part_cap, s) == cudaSuccess) {
                sb.part = static_cast<float*>(mem);
                c.bulk = &sb;
            } else {
                cudaGetLastError();  // the bulk updates then run unsplit
                mem = nullptr;
            }
            st = potrf_left<float>(c, n, !(flags & SPD_FACTOR_SERIAL));
            c.bulk = nullptr;
            if (mem) cudaFreeAsync(mem, s);
        } else {
            st = potrf_rec<float>(c, 0, n);
        }
        if (st == SPD_OK && prec != SPD_PREC_FP64) {
            // per-block inverses and sweep couplings: off the factorisation's
            // critical path, all blocks at once
            ProfScope pinv(h, SPD_PHASE_INVERSES, (double)F->nblk128 * 128.0 * 128.0 * 128.0 / 3.0,
                           (double)F->nblk128 * (8.0 * 16384.0 + 16384.0));
            ++h->launches, k_block_inverse<<<F->nblk128, 256, block_inverse_smem(), s>>>(F->W, F->ldw, n, F->Dinv32,
                                                                                        F->LinvT);
            if (cudaGetLastError() != cudaSuccess) st = set_err(h, SPD_ERR_CUDA, "block inverse launch failed");
        }
        if (st == SPD_OK && prec != SPD_PREC_FP64 && !(flags & SPD_FACTOR_BLOCK_SWEEPS) &&
            F->nblk128 >= 2 * SPD_SB_BLOCKS) {
            // inverses of the diagonal super-blocks for the super-block sweeps
            F->sbb = SPD_SB_BLOCKS;
            F->nsb = ceil_div(F->nblk128, F->sbb);
            const size_t S = (size_t)F->sbb * 128;
            if (cudaMallocAsync(&F->Xsb, sizeof(float) * S * S * F->nsb, s) != cudaSuccess) {
                cudaGetLastError();
                F->Xsb = nullptr;  // the 128-block sweeps serve instead
                F->sbb = F->nsb = 0;
            } else {
                static const bool attr = [] {
                    cudaFuncSetAttribute(k_sb_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sb_inverse_smem());
                    return true;
                }();
                (void)attr;
                ProfScope pinv(h, SPD_PHASE_INVERSES, (double)F->nsb * S * S * S / 3.0, 4.0 * F->nsb * S * S);
                ++h->launches, k_sb_inverse<<<dim3(F->sbb * SB_STRIPS, F->nsb), 256, sb_inverse_smem(), s>>>(
                    F->W, F->ldw, n, F->nblk128, F->LinvT, F->sbb, F->Xsb);
                if (cudaGetLastError() != cudaSuccess) st = set_err(h, SPD_ERR_CUDA, "super-block inverse launch failed");
            }
        }
        // the 128-block sweeps' couplings, only where they will run
        if (st == SPD_OK && prec != SPD_PREC_FP64 && !F->Xsb) st = factor_couplings(h, F);
        if (st == SPD_OK) st = check_dev_status(h, rep, "spd_factor");
        if (tc) tc_gemm_destroy(tc);
        if (st != SPD_OK) return fail(st);
    }
    *out = F;
    return SPD_OK;
}

// colsum[j] = d_j sum_i |A_ij| d_i  (one warp per column; A column-major)
__global__ void k_scaled_colsum(const double* __restrict__ A, long lda, int n, const double* __restrict__ d,
                                double* __restrict__ colsum) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= n) return;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += fabs(A[(long)j * lda + i]) * d[i];
    s = warp_sum(s);
    if (lane == 0) colsum[j] = s * d[j];
}

// Hager's 1-norm estimator of ||As^{-1}||_1 (As = D A D), applied through
// the factor F (the inverse is symmetric, so its transpose is itself).
spd_status hager_inv_norm1(spd_handle* h, const spd_factor_t* F, double* out) {
    const int n = F->n;
    float* dv = nullptr;
    CUDA_TRY(h, cudaMallocAsync(&dv, sizeof(float) * n, h->stream));
    std::vector<float> x(n, 1.0f / n), y(n), z(n), xi(n);
    double est = 0.0;
    spd_status st = SPD_OK;
    auto solve = [&](std::vector<float>& in, std::vector<float>& outv) -> spd_status {
        CUDA_TRY(h, cudaMemcpyAsync(dv, in.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
        spd_status s2 = factor_apply_scaled_f32(h, F, dv);
        if (s2 != SPD_OK) return s2;
        CUDA_TRY(h, cudaMemcpyAsync(outv.data(), dv, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return SPD_OK;
    };
    for (int k = 0; k < 5; ++k) {
        if ((st = solve(x, y)) != SPD_OK) break;
        double e1 = 0.0;
        for (int i = 0; i < n; ++i) e1 += fabs((double)y[i]);
        if (k > 0 && e1 <= est) break;
        est = e1;
        for (int i = 0; i < n; ++i) xi[i] = (y[i] >= 0.f) ? 1.f : -1.f;
        if ((st = solve(xi, z)) != SPD_OK) break;
        int jmax = 0;
        double zx = 0.0;
        for (int i = 0; i < n; ++i) {
            if (fabs(z[i]) > fabs(z[jmax])) jmax = i;
            zx += (double)z[i] * x[i];
        }
        if (k > 0 && fabs((double)z[jmax]) <= zx) break;
        std::fill(x.begin(), x.end(), 0.f);
        x[jmax] = 1.f;
    }
    cudaFreeAsync(dv, h->stream);
    *out = est;
    return st;
}

spd_status cond_estimate(spd_handle* h, const spd_factor_t* F, const double* A, int lda, double* kappa) {
    const int n = F->n;
    double* cs = nullptr;
    CUDA_TRY(h, cudaMallocAsync(&cs, sizeof(double) * n, h->stream));
    ++h->launches, k_scaled_colsum<<<ceil_div(n, 8), 256, 0, h->stream>>>(A, lda, n, F->d, cs);
    std::vector<double> hc(n);
    CUDA_TRY(h, cudaMemcpyAsync(hc.data(), cs, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    cudaFreeAsync(cs, h->stream);
    double anorm1 = 0.0;
    for (double v : hc) anorm1 = std::max(anorm1, v);
    double inv1 = 0.0;
    spd_status st = hager_inv_norm1(h, F, &inv1);
    *kappa = anorm1 * inv1;
    return st;
}

}  // namespace

static void setup_leaf_attrs() {
    static const bool done = [] {  // once per process, thread-safe
        cudaFuncSetAttribute(k_potrf_leaf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)potrf_leaf32_smem());
        cudaFuncSetAttribute(k_potrf_leaf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)potrf_leaf_smem<double>());
        cudaFuncSetAttribute(k_trsm_leaf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_leaf32_smem());
        cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_inverse_smem());
        cudaFuncSetAttribute(k_trsm_leaf<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)trsm_leaf_smem<double, 32>());
        return true;
    }();
    (void)done;
}

extern "C" spd_status spd_factor(spd_handle* h, int n, const double* A, int lda, int prec, unsigned flags,
                                 spd_factor_t** F, spd_report* rep) {
    if (!h) return SPD_ERR_ARG;
    if (!F || n < 0 || (n > 0 && (!A || lda < n)))
        return set_err(h, SPD_ERR_ARG, "spd_factor: bad arguments (n=%d lda=%d)", n, lda);
    if (prec < SPD_PREC_FP64 || prec > SPD_PREC_AUTO)
        return set_err(h, SPD_ERR_ARG, "spd_factor: unknown precision %d", prec);
    *F = nullptr;
    if (rep) memset(rep, 0, sizeof(*rep));
    setup_leaf_attrs();
    CUDA_TRY(h, cudaEventRecord(h->e0, h->stream));
    spd_status st;
    int used = prec;
    double kappa = 0.0, cond_lower = 0.0;
    if (prec == SPD_PREC_AUTO) {
        // FP16 tensor-core factor first; keep it when the estimated
        // kappa u_fp16 <= 1/4 (eq. (iterref) with margin), else FP32, and
        // FP64 if FP32 breaks down too.  kappa_1 / sqrt(n) stands in for the
        // 2-norm condition number (kappa_1 / n <= kappa_2 <= kappa_1 for a
        // symmetric matrix).
        // Before the FP16 factor (n >= LZ_MIN_N): a Lanczos lower bound on
        // kappa_2 of the scaled matrix; above 2^11 / 4 the same test can
        // only fail, so the FP16 attempt is skipped.
        used = SPD_PREC_FP16;
        LzCheck lz{0x1p11 * 0.25, 0.0, 0, false};
        st = factor_once(h, n, A, lda, SPD_PREC_FP16, flags, F, rep, 0.0, &lz);
        cond_lower = lz.bound;
        if (st == SPD_ERR_NOT_SPD && !lz.skip) kappa = -1.0;  // the FP16 factor broke down before any estimate
        if (st == SPD_OK && n > 0) {
            st = cond_estimate(h, *F, A, lda, &kappa);
            if (st != SPD_OK || !(kappa / sqrt((double)n) * 0x1p-11 <= 0.25)) {
                // too ill-conditioned for FP16, or the estimate itself failed:
                // no factor is handed out on either path
                spd_factor_destroy(*F);
                *F = nullptr;
                if (st == SPD_OK) st = SPD_ERR_NOT_SPD;
            }
        }
        if (st == SPD_ERR_NOT_SPD) {
            used = SPD_PREC_FP32;
            st = factor_once(h, n, A, lda, SPD_PREC_FP32, flags, F, rep);
        }
        if (st == SPD_ERR_NOT_SPD) {
            used = SPD_PREC_FP64;
            st = factor_once(h, n, A, lda, SPD_PREC_FP64, flags, F, rep);
        }
    } else {
        st = factor_once(h, n, A, lda, prec, flags, F, rep);
    }
    double sigma = 0.0;
    if (st == SPD_ERR_NOT_SPD && (flags & SPD_FACTOR_SHIFT) && prec != SPD_PREC_AUTO && prec != SPD_PREC_FP64) {
        // shifted retries: sigma = 2 u of the update operands (the updates'
        // rounding relative to the unit diagonal of the scaled matrix),
        // raised fourfold, at most 1
        const double u = prec == SPD_PREC_FP32 ? 0x1p-24 : prec == SPD_PREC_BF16 ? 0x1p-8
                         : prec == SPD_PREC_FP8 ? 0x1p-4 : 0x1p-11;
        for (sigma = 2.0 * u; st == SPD_ERR_NOT_SPD && sigma <= 1.0; sigma *= 4.0)
            st = factor_once(h, n, A, lda, prec, flags, F, rep, sigma);
        sigma /= 4.0;  // the sigma of the last attempt
        if (st != SPD_OK) sigma = 0.0;
    }
    CUDA_TRY(h, cudaEventRecord(h->e1, h->stream));
    CUDA_TRY(h, cudaEventSynchronize(h->e1));
    if (rep) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->e0, h->e1);
        rep->time_ms = ms;
        rep->status = st;
        rep->prec_used = used;
        rep->cond_est = kappa;
        rep->cond_lower = cond_lower;
        rep->shift = sigma;
        if (st == SPD_OK) rep->info = 0;  // a failed attempt before the kept factor leaves no trace
    }
    return st;
}

extern "C" spd_status spd_factor_destroy(spd_factor_t* F) {
    free_factor(F);
    return SPD_OK;
}

extern "C" spd_status spd_factor_info(const spd_factor_t* F, int* n, int* prec) {
    if (!F) return SPD_ERR_ARG;
    if (n) *n = F->n;
    if (prec) *prec = F->prec;
    return SPD_OK;
}

extern "C" spd_status spd_factor_copy(const spd_factor_t* F, void* L, int ldl, double* d) {
    if (!F || (L && ldl < F->n)) return SPD_ERR_ARG;
    spd_handle* h = F->h;
    const int n = F->n;
    if (n == 0) return SPD_OK;
    const size_t es = F->W64 ? sizeof(double) : sizeof(float);
    const void* src = F->W64 ? (const void*)F->W64 : (const void*)F->W;
    if (L)
        CUDA_TRY(h, cudaMemcpy2DAsync(L, es * ldl, src, es * F->ldw, es * n, n, cudaMemcpyDefault, h->stream));
    if (d) CUDA_TRY(h, cudaMemcpyAsync(d, F->d, sizeof(double) * n, cudaMemcpyDefault, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SPD_OK;
}
