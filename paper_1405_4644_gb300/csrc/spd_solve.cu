// spd_solve.cu -- handle management, the float64 residual, the
// low-precision triangular solves, Algorithm 1's refinement loop and
// Algorithm 2's CG with iterative refinement.
#include <mutex>

#include "engine.cuh"
#include "k_convert.cuh"
#include "k_solve.cuh"
#include "k_trsv32.cuh"
#include "k_trsv_sb.cuh"
#include "k_resid.cuh"
#include "k_cg.cuh"
#include "resid_tc.h"
#include "gemm_tc.h"

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
// SPD_RESID_AUTO: float64 fused multiply-adds for one right-hand side (8
// bytes per entry of A, against 20 for the digit planes and their one-time
// formation), the tensor-core residual from m = 2 on, where the FP64 rate
// bounds the float64 residual (2 m flops per 8 bytes).
static int resolve_resid(int resid, int m) {
    return resid == SPD_RESID_AUTO ? (m >= 2 ? SPD_RESID_TC : SPD_RESID_FP64) : resid;
}

extern "C" void spd_opts_default(spd_opts* o) {
    if (!o) return;
    o->tol = 1e-14;
    o->crit = SPD_CRIT_BERR;
    o->maxit = 50;
    o->maxit_inner = 2000;
    o->eta = 1e-4;
    o->band = -1;
    o->fallback = 1;
    o->resid = SPD_RESID_FP64;
    o->polish = 1;
    o->matvec_cores = SPD_MV_AUTO;
}

extern "C" spd_status spd_create(spd_handle** out, void* stream) {
    if (!out) return SPD_ERR_ARG;
    *out = nullptr;
    spd_handle* h = new spd_handle();
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->dst, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 4096);
    if (e == cudaSuccess) e = cudaEventCreate(&h->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->e1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // factors come from the device's stream-ordered pool: keep freed
        // blocks cached in the pool (like a caching allocator) instead of
        // returning them to the driver at every synchronisation
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (e == cudaSuccess) {
        DevStatus clear{0, INT_MAX, {0, 0}};
        e = cudaMemcpy(h->dst, &clear, sizeof(clear), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->dst) cudaFree(h->dst);
        if (h->pinned) cudaFreeHost(h->pinned);
        if (h->e0) cudaEventDestroy(h->e0);
        if (h->e1) cudaEventDestroy(h->e1);
        if (h->aux) cudaStreamDestroy(h->aux);
        delete h;
        return e == cudaErrorMemoryAllocation ? SPD_ERR_OOM : SPD_ERR_CUDA;
    }
    *out = h;
    return SPD_OK;
}

extern "C" spd_status spd_destroy(spd_handle* h) {
    if (!h) return SPD_OK;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    cudaFree(h->dst);
    cudaFreeHost(h->pinned);
    cudaEventDestroy(h->e0);
    cudaEventDestroy(h->e1);
    cudaFree(h->ready);
    cudaFree(h->stage);
    cudaFree(h->async_epoch_dev);
    cudaFree(h->sb_buf);
    if (h->aux) cudaStreamDestroy(h->aux);
    for (auto e : h->sync_ev) cudaEventDestroy(e);
    for (auto& r : h->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return SPD_OK;
}

extern "C" const char* spd_last_error_string(const spd_handle* h) { return h ? h->err : "null handle"; }

// ---------------------------------------------------------------------------
// internal building blocks
// ---------------------------------------------------------------------------
namespace {

struct ResidWs {
    double* P;      // max(S, Sdf) x m x n partial sums
    float* rowabs;  // max(S, Sdf) x n
    double* NP;     // G x m x 3
    int S;          // column splits of the float64 kernel
    double* xsc;    // 2 m column scales of the DF32 kernel
    int Sdf;        // column splits of the DF32 kernel
    const TcResidWs* tc = nullptr;  // prepared digit planes (SPD_RESID_TC)
};

// The tensor-core residual's workspace, planned beside a solver's and
// prepared (digit planes of A) once per call when opts.resid asks for it.
struct TcSetup {
    bool on = false;
    size_t off[6] = {0, 0, 0, 0, 0, 0};
    TcResidWs ws;
};

void tc_plan_if(WsPlan& p, spd_handle* h, int n, int m, int resid, TcSetup& t) {
    if (resid != SPD_RESID_TC) return;
    t.on = true;
    tc_resid_plan(p, h, n, m, t.off);
}

spd_status tc_bind_prepare(spd_handle* h, TcSetup& t, int n, int m, const double* A, long lda, ResidWs& rw) {
    if (!t.on) return SPD_OK;
    spd_status st = tc_resid_bind(h, &t.ws, n, m, t.off);
    if (st != SPD_OK) return st;
    ProfScope ps(h, SPD_PHASE_RESID_TC, 0.0, 36.0 * n * (double)n);  // A twice, 20 bytes of digits per entry
    st = tc_resid_prepare(h, &t.ws, A, lda);
    if (st != SPD_OK) return st;
    rw.tc = &t.ws;
    return SPD_OK;
}

// Column splits of the float64 residual: about four CTAs per SM, each split
// at least four column tiles long
int resid_splits(spd_handle* h, int n) {
    int rowblk = ceil_div(n, RESID_ROWS);
    int want = std::max(1, (4 * h->sms + rowblk - 1) / rowblk);
    int maxs = std::max(1, n / (4 * RESID_JT));
    return std::min(want, maxs);
}

// The DF32 kernel holds two CTAs per SM: pick the split count whose grid
// fills whole waves best (at least two waves when the size allows).
int resid_splits_df32(spd_handle* h, int n) {
    const int rowblk = ceil_div(n, RESID_ROWS);
    const int slots = 2 * h->sms;
    const int maxs = std::max(1, n / (2 * RESID_FOLD));
    int best = 1;
    double best_eff = -1.0;
    for (int s = 1; s <= maxs; ++s) {
        const long ctas = (long)rowblk * s;
        const long waves = (ctas + slots - 1) / slots;
        double eff = (double)ctas / ((double)waves * slots);
        if (ctas < 2L * slots && s < maxs) eff *= 0.5;  // too few CTAs to hide latency
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = s;
        }
        if (ctas >= 4L * slots) break;
    }
    return best;
}

size_t resid_plan(WsPlan& p, spd_handle* h, int n, int m, size_t* offs) {
    int S = resid_splits(h, n);
    int Smax = std::max(S, resid_splits_df32(h, n));
    int G = ceil_div(n, 256);
    offs[0] = p.add<double>((size_t)Smax * m * n);
    offs[1] = p.add<float>((size_t)Smax * n);
    offs[2] = p.add<double>((size_t)G * m * 3);
    offs[3] = p.add<double>((size_t)2 * m);
    return S;
}

ResidWs resid_ws(spd_handle* h, int n, const size_t* off, int S) {
    return ResidWs{ws_at<double>(h, off[0]), ws_at<float>(h, off[1]), ws_at<double>(h, off[2]), S,
                   ws_at<double>(h, off[3]), resid_splits_df32(h, n)};
}

// R = B - A X (mode 0) or R = A X (mode 1), float64; colnorms[3m]; if anorm
// is non-null also ||A||_inf.
// The DF32 variant of the partial-sum pass (same partial layout).
template <int MT>
void launch_df32(spd_handle* h, dim3 grid, const double* A, long lda, int n, const double* X, long ldx, int c0, int mc,
                 int jchunk, int m, const ResidWs& w, float* ra) {
    static const bool attr = [] {  // once per instantiation, thread-safe
        cudaFuncSetAttribute(k_resid_partial_df32<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)df32_smem<MT>());
        return true;
    }();
    (void)attr;
    ++(h)->launches, k_resid_partial_df32<MT><<<grid, RESID_ROWS, df32_smem<MT>(), h->stream>>>(
        A, lda, n, X, ldx, c0, mc, jchunk, m, w.xsc, w.P, ra, h->dst);
}

spd_status resid_partial_df32(spd_handle* h, const ResidWs& w, int n, int m, const double* A, long lda,
                              const double* X, long ldx, bool with_rowabs) {
    cudaStream_t s = h->stream;
    const int S = w.Sdf;
    const int jchunk = (int)round_up(ceil_div(n, S), RESID_JT);
    dim3 grid(ceil_div(n, RESID_ROWS), S);
    ++(h)->launches, k_xscale<<<m, 256, 0, s>>>(X, ldx, n, m, w.xsc);
    for (int c0 = 0; c0 < m; c0 += 16) {
        int mc = std::min(16, m - c0);
        float* ra = (with_rowabs && c0 == 0) ? w.rowabs : nullptr;
        if (mc == 1) launch_df32<1>(h, grid, A, lda, n, X, ldx, c0, mc, jchunk, m, w, ra);
        else if (mc == 2) launch_df32<2>(h, grid, A, lda, n, X, ldx, c0, mc, jchunk, m, w, ra);
        else if (mc <= 4) launch_df32<4>(h, grid, A, lda, n, X, ldx, c0, mc, jchunk, m, w, ra);
        else if (mc <= 8) launch_df32<8>(h, grid, A, lda, n, X, ldx, c0, mc, jchunk, m, w, ra);
        else launch_df32<16>(h, grid, A, lda, n, X, ldx, c0, mc, jchunk, m, w, ra);
        LAUNCH_CHECK(h);
    }
    return SPD_OK;
}

// SPD_RESID_DF32 in the refinement loops: float32-pair residuals while the
// largest backward error is above 2^-36 (16 times their own error bound
// 2^-40 |A||x|, so the correction they drive is as good as a float64 one)
// and, below that, while each sweep still shrinks it at least fourfold (the
// pairs' rounding has not been reached); float64 residuals from the first
// sweep that fails either test, or after a column met the rule on a pair
// residual.  Only a float64 residual may accept a column as converged.
constexpr double DF32_SWITCH = 1.4551915228366852e-11;  // 2^-36

struct ResidPolicy {
    bool df32;           // still on float32-pair residuals
    int last;            // the float64-accurate kind: SPD_RESID_FP64 or SPD_RESID_TC
    double prev = -1.0;  // largest backward error of the previous residual
    explicit ResidPolicy(const spd_opts& o)
        : df32(o.resid == SPD_RESID_DF32), last(o.resid == SPD_RESID_TC ? SPD_RESID_TC : SPD_RESID_FP64) {}
    int first() const { return df32 ? SPD_RESID_DF32 : last; }
    // kind of the next residual after one with summary sm; *restart = 1 when
    // the arithmetic changes
    int next(const IrSummary& sm, int* restart) {
        *restart = 0;
        if (df32) {
            const double b = sm.max_berr;
            const bool keep = sm.pending == 0 && b > 0.0 &&
                              (b > DF32_SWITCH || (prev > 0.0 && b <= 0.25 * prev));
            if (!keep) {
                df32 = false;
                *restart = 1;
            }
        }
        prev = sm.max_berr;
        return df32 ? SPD_RESID_DF32 : last;
    }
};

spd_status resid_run(spd_handle* h, const ResidWs& w, int n, int m, const double* A, long lda, const double* B,
                     long ldb, const double* X, long ldx, double* R, long ldr, double* colnorms, double* anorm,
                     int mode, int kind = SPD_RESID_FP64) {
    cudaStream_t s = h->stream;
    if (kind == SPD_RESID_TC) {
        if (!w.tc || w.tc->n != n || w.tc->m != m) return set_err(h, SPD_ERR_ARG, "tensor-core residual not prepared");
        // algorithmic work: 55 digit products of 2 n^2 m; bytes: the ten digit planes
        ProfScope ps(h, SPD_PHASE_RESID_TC, 110.0 * n * (double)n * m, 20.0 * n * (double)n + 24.0 * n * (double)m);
        spd_status st = tc_resid_run(h, w.tc, B, ldb, X, ldx, R, ldr, w.NP, mode, h->async_on ? h->async_gate : nullptr);
        if (st != SPD_OK) return st;
        const int G = ceil_div(n, 256);
        if (colnorms) {
            ++(h)->launches, k_colnorms<<<m, 256, 0, s>>>(w.NP, G, m, colnorms);
            LAUNCH_CHECK(h);
        }
        if (anorm) {
            ++(h)->launches, k_anorm<<<1, 1024, 0, s>>>(w.tc->rowabs, w.tc->RS, n, anorm);
            LAUNCH_CHECK(h);
        }
        return SPD_OK;
    }
    ProfScope ps(h, kind == SPD_RESID_DF32 ? SPD_PHASE_RESID_DF32 : SPD_PHASE_RESID, 2.0 * n * (double)n * m,
                 8.0 * n * (double)n + 24.0 * n * (double)m);
    const int* gate = h->async_on ? h->async_gate : nullptr;
    const int S = kind == SPD_RESID_DF32 ? w.Sdf : w.S;
    const int jchunk = (int)round_up(ceil_div(n, S), RESID_JT);
    dim3 grid(ceil_div(n, RESID_ROWS), S);
    if (kind == SPD_RESID_DF32) {
        spd_status st = resid_partial_df32(h, w, n, m, A, lda, X, ldx, anorm != nullptr);
        if (st != SPD_OK) return st;
    }
    for (int c0 = 0; c0 < m && kind != SPD_RESID_DF32; c0 += 16) {
        int mc = std::min(16, m - c0);
        float* ra = (anorm && c0 == 0) ? w.rowabs : nullptr;
        if (mc == 1)
            ++(h)->launches, k_resid_partial<1><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, w.P, ra, gate);
        else if (mc == 2)
            ++(h)->launches, k_resid_partial<2><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, w.P, ra, gate);
        else if (mc <= 4)
            ++(h)->launches, k_resid_partial<4><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, w.P, ra, gate);
        else if (mc <= 8)
            ++(h)->launches, k_resid_partial<8><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, w.P, ra, gate);
        else
            ++(h)->launches, k_resid_partial<16><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, w.P, ra, gate);
        LAUNCH_CHECK(h);
    }
    const int G = ceil_div(n, 256);
    ++(h)->launches, k_resid_final<<<dim3(G, m), 256, 0, s>>>(B, ldb, n, m, w.P, S, R, ldr, X, ldx, w.NP, mode, gate);
    LAUNCH_CHECK(h);
    if (colnorms) {
        ++(h)->launches, k_colnorms<<<m, 256, 0, s>>>(w.NP, G, m, colnorms);
        LAUNCH_CHECK(h);
    }
    if (anorm) {
        ++(h)->launches, k_anorm<<<1, 1024, 0, s>>>(w.rowabs, S, n, anorm);
        LAUNCH_CHECK(h);
    }
    return SPD_OK;
}

template <typename T>
void setup_solve_attrs() {
    static const bool done = [] {  // once per process, thread-safe
        constexpr int MC = solve_mc<T>();
        cudaFuncSetAttribute(k_trsv_fwd_step<T, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solve_smem_bytes<T>());
        cudaFuncSetAttribute(k_trsv_bwd_step<T, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solve_smem_bytes<T>());
        return true;
    }();
    (void)done;
}

// Y <- L^{-T} L^{-1} Y in place (n x m, ld n) with the factor's L and the
// inverses of its 32x32 diagonal sub-blocks.
template <typename T>
spd_status lp_sweeps(spd_handle* h, const T* W, long ldw, const T* Dinv, int n, int m, T* Y) {
    setup_solve_attrs<T>();
    ProfScope ps(h, SPD_PHASE_SOLVE, 2.0 * n * (double)n * m, (double)sizeof(T) * n * (double)n);
    constexpr int MC = solve_mc<T>();
    cudaStream_t s = h->stream;
    const int NB = ceil_div(n, 128);
    const size_t smem = solve_smem_bytes<T>();
    for (int c0 = 0; c0 < m; c0 += MC) {
        int mc = std::min(MC, m - c0);
        for (int J = -1; J <= NB - 2; ++J) {
            int grid = NB - 1 - J;
            ++(h)->launches, k_trsv_fwd_step<T, MC><<<grid, 256, smem, s>>>(W, ldw, n, Dinv, Y, c0, mc, J);
        }
        LAUNCH_CHECK(h);
        for (int J = NB; J >= 1; --J) {
            int grid = (J == NB) ? 1 : J;
            ++(h)->launches, k_trsv_bwd_step<T, MC><<<grid, 256, smem, s>>>(W, ldw, n, NB, Dinv, Y, c0, mc, J);
        }
        LAUNCH_CHECK(h);
    }
    return SPD_OK;
}

// Cooperative launches from every stream of the process run one after
// another: a cooperative grid needs all of its CTAs resident at once, and two
// such grids sharing the SMs could each hold part of the machine while
// waiting for the rest.  Ordinary kernels may overlap them (they always run
// to completion and release their SMs).
struct CoopGate {
    std::mutex mu;
    cudaEvent_t last = nullptr;
};
CoopGate& coop_gate() {
    static CoopGate g;
    return g;
}
cudaError_t coop_launch(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s) {
    // while s is being captured into a graph, the order against other
    // streams' cooperative launches cannot be recorded (an event from outside
    // the capture): the graph's launches are issued as they are, and the
    // caller must not replay it concurrently with other cooperative work
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusActive)
        return cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s);
    CoopGate& g = coop_gate();
    std::lock_guard<std::mutex> lock(g.mu);
    cudaError_t e = cudaSuccess;
    if (!g.last) e = cudaEventCreateWithFlags(&g.last, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.last, 0);  // a never-recorded event: no wait
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s);
    if (e == cudaSuccess) e = cudaEventRecord(g.last, s);
    return e;
}

template <int MC>
spd_status trsv32_pass(spd_handle* h, const spd_factor_t* F, float* Y, int n, int c0, int mc) {
    const size_t smem = trsv32_smem<MC>();
    auto fwd = k_trsv32<MC, true>;
    auto bwd = k_trsv32<MC, false>;
    struct Occ {
        int per_sm[2];
    };
    static const Occ occ = [&] {  // once per instantiation, thread-safe
        Occ o{{1, 1}};
        cudaFuncSetAttribute(fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd, 256, smem);
        o.per_sm[0] = std::max(1, per_sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd, 256, smem);
        o.per_sm[1] = std::max(1, per_sm);
        return o;
    }();
    const int NB = ceil_div(n, 128);
    // flags (NB ints) and, after them, the CTA slot table; both restart at
    // epoch 0 (all zero) whenever they are reallocated
    const size_t slot_off = (size_t)round_up((long)sizeof(int) * NB, 256);
    if (h->ready_n < NB) {
        if (h->ready) CUDA_TRY(h, cudaFree(h->ready));
        h->ready = nullptr;
        const size_t bytes = slot_off + sizeof(unsigned long long) * TV_SLOTS;
        CUDA_TRY(h, cudaMalloc(&h->ready, bytes));
        CUDA_TRY(h, cudaMemsetAsync(h->ready, 0, bytes, h->stream));
        h->ready_n = NB;
        h->epoch = 0;
    }
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->ready) +
                                                                      round_up((long)sizeof(int) * h->ready_n, 256));
    for (int dir = 0; dir < 2; ++dir) {
        // epochs: the host counter, or (capturable solves) an offset from
        // the device counter, which the solve advanced by async_total at its
        // start: 2^30 + base - total + 1 .. 2^30 + base, never a value of the
        // host counter (< 2^30) or of an earlier capturable solve
        const int ep = h->async_on ? (++h->async_rel - h->async_total) : ++h->epoch;
        TrsvArgs a{F->W, F->ldw, n, NB, F->LinvT, F->Cpl, Y, c0, mc, h->ready, ep, h->dst, slots, h->wait_ns,
                   h->async_on ? h->async_gate : nullptr, h->async_on ? h->async_epoch_dev : nullptr};
        void* args[] = {&a};
        const int grid = std::min({NB, occ.per_sm[dir] * h->sms, TV_SLOTS});
        ++h->launches;
        CUDA_TRY(h, coop_launch(dir == 0 ? (const void*)fwd : (const void*)bwd, dim3(grid), dim3(256), args, smem,
                                h->stream));
    }
    return SPD_OK;
}

}  // namespace

// The sweep couplings of a float32 factor (M_J, N_J of k_trsv32.cuh).
spd_status factor_couplings(spd_handle* h, spd_factor_t* F) {
    const int NB = F->nblk128;
    if (NB < 2) return SPD_OK;
    static const bool attr = [] {  // once per process, thread-safe
        cudaFuncSetAttribute(k_trsv_couplings, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)trsv_couplings_smem());
        return true;
    }();
    (void)attr;
    // distance 1 (NB - 1 per direction) and distance 2 (NB - 2 per direction)
    const int ncp = (NB - 1) + std::max(NB - 2, 0);
    ProfScope ps(h, SPD_PHASE_INVERSES, 2.0 * 2.0 * ncp * 128.0 * 128.0 * 128.0, 3.0 * 4.0 * 2.0 * ncp * 16384.0);
    ++h->launches, k_trsv_couplings<<<dim3(NB - 1, NB >= 3 ? 4 : 2), 256, trsv_couplings_smem(), h->stream>>>(
        F->W, F->ldw, F->n, NB, F->LinvT, F->Cpl);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

namespace {

// One forward and one backward super-block sweep of columns [c0, c0 + mc)
// (k_trsv_sb.cuh): the barrier words are cleared before each launch (a
// stream-ordered memset, so that a captured graph clears them on replay).
// The scratch (partial tiles, partial slots, barrier words) is sized once
// per handle; the first call on a handle must not be captured.
template <int MC>
spd_status trsv_sb_pass(spd_handle* h, const spd_factor_t* F, float* Y, int n, int c0, int mc) {
    const size_t smem = trsv_sb_smem<MC>();
    auto fwd = k_trsv_sb<MC, true>;
    auto bwd = k_trsv_sb<MC, false>;
    static const int per_sm = [&] {  // once per instantiation, thread-safe
        cudaFuncSetAttribute(fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fwd, 256, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bwd, 256, smem);
        return std::max(1, std::min(a, b));
    }();
    const size_t ntile = (size_t)F->sbb * (F->sbb + 1) / 2;
    // every SM streams the panel updates: one CTA per resident slot
    const int G = std::min(per_sm * h->sms, TV_SLOTS);
    const size_t pbytes = (size_t)round_up((long)(sizeof(float) * ntile * 128 * 16), 256);
    const size_t p2bytes = (size_t)round_up((long)(sizeof(float) * 2 * (size_t)G * 128 * 16), 256);
    const size_t zbytes = (size_t)round_up((long)(sizeof(float) * (size_t)n * 16), 256);
    const int nbar = 2 + F->nsb * F->sbb;  // barrier words, then the block-row tile counts
    const size_t bbytes = (size_t)round_up((long)(sizeof(int) * nbar), 256);
    const size_t need = pbytes + p2bytes + zbytes + bbytes;
    if (h->sb_bytes < need) {
        if (h->sb_buf) {
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            CUDA_TRY(h, cudaFree(h->sb_buf));
        }
        h->sb_buf = nullptr;
        h->sb_bytes = 0;
        CUDA_TRY(h, cudaMalloc(&h->sb_buf, need));
        h->sb_bytes = need;
    }
    char* base = static_cast<char*>(h->sb_buf);
    float* P = reinterpret_cast<float*>(base);
    float* P2 = reinterpret_cast<float*>(base + pbytes);
    float* Z = reinterpret_cast<float*>(base + pbytes + p2bytes);  // the forward sweep's result
    int* bar = reinterpret_cast<int*>(base + pbytes + p2bytes + zbytes);
    for (int dir = 0; dir < 2; ++dir) {
        // forward: Y (columns c0..) reduced, result to Z; backward: Z reduced, result to Y
        SbArgs a{F->W, F->ldw, n, F->nblk128, F->Xsb, F->sbb * 128, F->sbb, F->nsb,
                 dir == 0 ? Y : Z, dir == 0 ? c0 : 0, mc, dir == 0 ? Z : Y, dir == 0 ? 0 : c0, P, P2, bar,
                 h->wait_ns, h->dst, h->async_on ? h->async_gate : nullptr};
        void* args[] = {&a};
        CUDA_TRY(h, cudaMemsetAsync(bar, 0, sizeof(int) * nbar, h->stream));
        ++h->launches;
        CUDA_TRY(h, coop_launch(dir == 0 ? (const void*)fwd : (const void*)bwd, dim3(G), dim3(256), args, smem,
                                h->stream));
    }
    return SPD_OK;
}

// Y <- (L L^T)^{-1} Y for a float32 factor (n x m, ld n).
spd_status lp_sweeps32(spd_handle* h, const spd_factor_t* F, int n, int m, float* Y) {
    ProfScope ps(h, SPD_PHASE_SOLVE, 2.0 * n * (double)n * m, 4.0 * n * (double)n);
    for (int c0 = 0; c0 < m && F->Xsb; c0 += 16) {  // super-block sweeps
        const int mc = std::min(16, m - c0);
        spd_status st;
        if (mc == 1) st = trsv_sb_pass<1>(h, F, Y, n, c0, mc);
        else if (mc <= 2) st = trsv_sb_pass<2>(h, F, Y, n, c0, mc);
        else if (mc <= 4) st = trsv_sb_pass<4>(h, F, Y, n, c0, mc);
        else if (mc <= 8) st = trsv_sb_pass<8>(h, F, Y, n, c0, mc);
        else st = trsv_sb_pass<16>(h, F, Y, n, c0, mc);
        if (st != SPD_OK) return st;
    }
    for (int c0 = 0; c0 < m && !F->Xsb; c0 += 16) {
        const int mc = std::min(16, m - c0);
        spd_status st;
        if (mc == 1) st = trsv32_pass<1>(h, F, Y, n, c0, mc);
        else if (mc <= 2) st = trsv32_pass<2>(h, F, Y, n, c0, mc);
        else if (mc <= 4) st = trsv32_pass<4>(h, F, Y, n, c0, mc);
        else if (mc <= 8) st = trsv32_pass<8>(h, F, Y, n, c0, mc);
        else st = trsv32_pass<16>(h, F, Y, n, c0, mc);
        if (st != SPD_OK) return st;
    }
    return SPD_OK;
}

// X = d .* (L^{-T} L^{-1} (d .* R))  (mode 0)  or  X += ... on unfrozen
// columns (mode 1).  Y is scratch of n*m elements of the factor's type.
spd_status lp_apply(spd_handle* h, const spd_factor_t* F, int n, int m, const double* R, long ldr, void* Y,
                    double* X, long ldx, const int* frozen, int mode) {
    cudaStream_t s = h->stream;
    int g = grid_for((long)n * m, 256, 8 * h->sms);
    spd_status st;
    if (F->prec == SPD_PREC_FP64) {
        double* y = static_cast<double*>(Y);
        ++(h)->launches, k_scale_to<double><<<g, 256, 0, s>>>(R, ldr, F->d, n, m, y);
        LAUNCH_CHECK(h);
        st = lp_sweeps<double>(h, F->W64, F->ldw, F->Dinv64, n, m, y);
        if (st != SPD_OK) return st;
        ++(h)->launches, k_apply_correction<double><<<g, 256, 0, s>>>(X, ldx, F->d, y, n, m, frozen, mode);
    } else {
        float* y = static_cast<float*>(Y);
        ++(h)->launches, k_scale_to<float><<<g, 256, 0, s>>>(R, ldr, F->d, n, m, y);
        LAUNCH_CHECK(h);
        st = lp_sweeps32(h, F, n, m, y);
        if (st != SPD_OK) return st;
        ++(h)->launches, k_apply_correction<float><<<g, 256, 0, s>>>(X, ldx, F->d, y, n, m, frozen, mode);
    }
    LAUNCH_CHECK(h);
    return SPD_OK;
}

}  // namespace

spd_status factor_apply_scaled_f32(spd_handle* h, const spd_factor_t* F, float* y) {
    return lp_sweeps32(h, F, F->n, 1, y);
}

namespace {

__global__ void k_ircols_init(IrCol* cols, int m, int polish) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < m) {
        IrCol z;
        z.err = 0.0;
        z.prev = INFINITY;
        z.conv = 0;
        z.stall = 0;
        z.iters = 0;
        z.extra = polish;
        cols[c] = z;
    }
}

bool bad_args(int n, int m, const void* A, int lda, const void* B, int ldb, const void* X, int ldx) {
    if (n < 0 || m < 0) return true;
    if (n == 0 || m == 0) return false;
    if (!A || !B || !X) return true;
    if (lda < n || ldb < n || ldx < n) return true;
    if (m > SPD_MAXM) return true;
    return false;
}

}  // namespace

// ---------------------------------------------------------------------------
// public building blocks
// ---------------------------------------------------------------------------
namespace {
spd_status residual_entry(spd_handle* h, int kind, int n, int m, const double* A, int lda, const double* B, int ldb,
                          const double* X, int ldx, double* R, int ldr, double* colnorms) {
    if (!h) return SPD_ERR_ARG;
    if (bad_args(n, m, A, lda, B, ldb, X, ldx) || (n > 0 && m > 0 && (!R || ldr < n)))
        return set_err(h, SPD_ERR_ARG, "spd_residual: bad arguments");
    if (n == 0 || m == 0) return SPD_OK;
    WsPlan p;
    size_t off[4];
    int S = (int)resid_plan(p, h, n, m, off);
    TcSetup tcs;
    tc_plan_if(p, h, n, m, kind, tcs);
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    ResidWs rw = resid_ws(h, n, off, S);
    st = tc_bind_prepare(h, tcs, n, m, A, lda, rw);
    if (st != SPD_OK) return st;
    st = resid_run(h, rw, n, m, A, lda, B, ldb, X, ldx, R, ldr, colnorms, nullptr, 0, kind);
    if (st != SPD_OK) return st;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SPD_OK;
}
}  // namespace

extern "C" spd_status spd_residual(spd_handle* h, int n, int m, const double* A, int lda, const double* B, int ldb,
                                   const double* X, int ldx, double* R, int ldr, double* colnorms) {
    return residual_entry(h, SPD_RESID_FP64, n, m, A, lda, B, ldb, X, ldx, R, ldr, colnorms);
}

extern "C" spd_status spd_residual_df32(spd_handle* h, int n, int m, const double* A, int lda, const double* B,
                                        int ldb, const double* X, int ldx, double* R, int ldr, double* colnorms) {
    return residual_entry(h, SPD_RESID_DF32, n, m, A, lda, B, ldb, X, ldx, R, ldr, colnorms);
}

extern "C" spd_status spd_residual_tc(spd_handle* h, int n, int m, const double* A, int lda, const double* B,
                                      int ldb, const double* X, int ldx, double* R, int ldr, double* colnorms) {
    return residual_entry(h, SPD_RESID_TC, n, m, A, lda, B, ldb, X, ldx, R, ldr, colnorms);
}

extern "C" spd_status spd_factor_solve(spd_handle* h, const spd_factor_t* F, int n, int m, const double* R, int ldr,
                                       double* Z, int ldz) {
    if (!h) return SPD_ERR_ARG;
    if (!F || F->n != n || bad_args(n, m, F, n, R, ldr, Z, ldz))
        return set_err(h, SPD_ERR_ARG, "spd_factor_solve: bad arguments");
    if (n == 0 || m == 0) return SPD_OK;
    WsPlan p;
    size_t oy = p.add<double>((size_t)n * m);
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    st = lp_apply(h, F, n, m, R, ldr, ws_at<double>(h, oy), Z, ldz, nullptr, 0);
    if (st != SPD_OK) return st;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SPD_OK;
}

// ---------------------------------------------------------------------------
// CG with iterative refinement (Algorithm 2, nested low/high reading); also
// the float64 factor-preconditioned CG used as the refinement fallback.
// ---------------------------------------------------------------------------
namespace {

enum MatvecKind { MV_FP64 = 0, MV_FP32 = 1, MV_BF16 = 2, MV_BAND = 3, MV_TC = 4 };
constexpr int CG_GRAPH_STEPS = 8;  // inner steps per captured graph (= the host's check interval)

struct CgSetup {
    int matvec = MV_FP64;
    const void* At = nullptr;  // low-precision copy (dense row-major n x ldt, or band)
    long ldt = 0;
    int band = -1;
    int pc = SPD_PC_NONE;
    const spd_factor_t* F = nullptr;
    const spd_lowrank* LR = nullptr;
    const double* dinv = nullptr;
    // MV_TC: A~ and P^T as bf16 slice planes, the narrow GEMM's C and its
    // stream-K partial slots
    TcGemm* tg = nullptr;
    __nv_bfloat16* Pm = nullptr;
    float* Cf = nullptr;
    long ldo = 0, ldc = 0, plane_p = 0;
    int Kp = 0;
    TcSplit sk{nullptr, 0};
};

// Q = A~ P on the tensor cores (float32 operands as three bf16 slices each)
spd_status mv_tc(spd_handle* h, const CgSetup& cs, int n, int m, const float* Pf, double* Q) {
    ProfScope ps(h, SPD_PHASE_MATVEC, 2.0 * n * (double)n * m, 6.0 * n * (double)cs.Kp);
    cudaStream_t s = h->stream;
    const int gv = grid_for((long)n * m, 256, 8 * h->sms);
    ++h->launches, k_p_x3<<<gv, 256, 0, s>>>(Pf, n, m, cs.Pm, cs.ldo, cs.plane_p);
    CUDA_TRY(h, cudaMemsetAsync(cs.Cf, 0, sizeof(float) * n * cs.ldc, s));
    ++h->launches;
    const spd_status st = tc_gemm_launch(cs.tg, s, 0, 0, n, m, cs.Kp, 0, 0, 0, 0, h->dst, -h->sms, &cs.sk);
    if (st != SPD_OK) return set_err(h, st, "spd_cg: tensor-core product launch failed");
    ++h->launches, k_cf_to_q<<<gv, 256, 0, s>>>(cs.Cf, cs.ldc, n, m, Q);
    return SPD_OK;
}

template <typename T, int MC>
void mv_launch(spd_handle* h, const CgSetup& cs, int n, int m, const float* Pf, double* Q) {
    ProfScope ps(h, SPD_PHASE_MATVEC, 2.0 * n * (double)n * m, (double)sizeof(T) * n * (double)n);
    int grid = ceil_div(n, MV_ROWS);
    for (int c0 = 0; c0 < m; c0 += MC) {
        int mc = std::min(MC, m - c0);
        ++(h)->launches, k_matvec_lp<T, MC><<<grid, 256, 0, h->stream>>>(static_cast<const T*>(cs.At), cs.ldt, n, Pf, c0, mc, Q,
                                                        nullptr);
    }
}

template <typename T>
void mv_dispatch(spd_handle* h, const CgSetup& cs, int n, int m, const float* Pf, double* Q) {
    if (m == 1) mv_launch<T, 1>(h, cs, n, m, Pf, Q);
    else if (m <= 4) mv_launch<T, 4>(h, cs, n, m, Pf, Q);
    else if (m <= 8) mv_launch<T, 8>(h, cs, n, m, Pf, Q);
    else mv_launch<T, 16>(h, cs, n, m, Pf, Q);
}

struct CgWs {
    ResidWs rw;
    double *R, *colnorms, *anorm, *b2, *target, *E, *Rr, *Z, *P, *Q, *part, *Yz;
    float* Pf;
    IrCol* cols;
    IrSummary* sum;
    CgCol* cg;
    int *frozen, *active;
    int G2;
};

size_t cg_plan(WsPlan& p, spd_handle* h, int n, int m, size_t* o, int* S, int* G2) {
    *S = (int)resid_plan(p, h, n, m, o);
    // row chunks per column of the dot products: about 2 blocks per SM over
    // all m columns, at least 256 rows each
    *G2 = std::max(1, std::min(2 * h->sms, ceil_div(n, 256)) / std::max(m, 1));
    size_t nm = (size_t)n * m;
    o[4] = p.add<double>(nm);       // R
    o[5] = p.add<double>(3 * m);    // colnorms
    o[6] = p.add<double>(1);        // anorm
    o[7] = p.add<double>(m);        // b2
    o[8] = p.add<double>(m);        // target
    o[9] = p.add<double>(nm);       // E
    o[10] = p.add<double>(nm);       // Rr
    o[11] = p.add<double>(nm);      // Z
    o[12] = p.add<double>(nm);      // P
    o[13] = p.add<double>(nm);      // Q
    o[14] = p.add<double>((size_t)(*G2) * m * 2);  // part
    o[15] = p.add<double>(nm);      // Yz (factor preconditioner scratch)
    o[16] = p.add<float>(nm);       // Pf
    o[17] = p.add<IrCol>(m);
    o[18] = p.add<IrSummary>(1);
    o[19] = p.add<CgCol>(m);
    o[20] = p.add<int>(m);          // frozen
    o[21] = p.add<int>(1);          // active
    return p.bytes;
}

CgWs cg_bind(spd_handle* h, int n, const size_t* o, int S, int G2) {
    CgWs w;
    w.rw = resid_ws(h, n, o, S);
    w.R = ws_at<double>(h, o[4]);
    w.colnorms = ws_at<double>(h, o[5]);
    w.anorm = ws_at<double>(h, o[6]);
    w.b2 = ws_at<double>(h, o[7]);
    w.target = ws_at<double>(h, o[8]);
    w.E = ws_at<double>(h, o[9]);
    w.Rr = ws_at<double>(h, o[10]);
    w.Z = ws_at<double>(h, o[11]);
    w.P = ws_at<double>(h, o[12]);
    w.Q = ws_at<double>(h, o[13]);
    w.part = ws_at<double>(h, o[14]);
    w.Yz = ws_at<double>(h, o[15]);
    w.Pf = ws_at<float>(h, o[16]);
    w.cols = ws_at<IrCol>(h, o[17]);
    w.sum = ws_at<IrSummary>(h, o[18]);
    w.cg = ws_at<CgCol>(h, o[19]);
    w.frozen = ws_at<int>(h, o[20]);
    w.active = ws_at<int>(h, o[21]);
    w.G2 = G2;
    return w;
}

spd_status read_summary(spd_handle* h, const IrSummary* d, IrSummary* out) {
    IrSummary* hs = reinterpret_cast<IrSummary*>(static_cast<char*>(h->pinned) + 64);
    CUDA_TRY(h, cudaMemcpyAsync(hs, d, sizeof(IrSummary), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *out = *hs;
    return SPD_OK;
}

spd_status read_int(spd_handle* h, const int* d, int* out) {
    int* hs = reinterpret_cast<int*>(static_cast<char*>(h->pinned) + 128);
    CUDA_TRY(h, cudaMemcpyAsync(hs, d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *out = *hs;
    return SPD_OK;
}

// The nested CG-IR loop.  If reuse_state, the outer state (cols, R,
// colnorms, anorm, b2) already describes the current X.
spd_status cg_ir_core(spd_handle* h, CgWs& w, int n, int m, const double* A, long lda, const double* B, long ldb,
                      double* X, long ldx, const spd_opts& o, const CgSetup& cs, bool reuse_state, int* low,
                      int* high, IrSummary* last) {
    cudaStream_t s = h->stream;
    // a refinement that falls back here after float64 residuals stays on them
    ResidPolicy pol(o);
    if (reuse_state) pol.df32 = false;
    const int gv = grid_for((long)n * m, 256, 8 * h->sms);
    spd_status st;
    if (!reuse_state) {
        CUDA_TRY(h, cudaMemset2DAsync(X, sizeof(double) * ldx, 0, sizeof(double) * n, m, s));
        ++(h)->launches, k_ircols_init<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, 0);
        ++(h)->launches, k_col_nrm2<<<m, 256, 0, s>>>(B, ldb, n, w.b2);
        const int rk = pol.first();
        st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, w.anorm, 0, rk);
        if (st != SPD_OK) return st;
        ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 0, 0,
                                                      rk != SPD_RESID_DF32);
        LAUNCH_CHECK(h);
    }
    CUDA_TRY(h, cudaMemsetAsync(w.cg, 0, sizeof(CgCol) * m, s));
    const double* Zr = (cs.pc == SPD_PC_NONE) ? w.Rr : w.Z;
    // inner steps whose launches do not change from one step to the next
    // (every product; no preconditioner, Jacobi or the learned low-rank one;
    // not the factor preconditioner, whose sweeps number their epochs, nor
    // the float32-pair residual, which the host switches) replay as a CUDA
    // graph of CG_GRAPH_STEPS steps, captured once per call; not while
    // profiling (the phase records would be captured once)
    struct CgGraph {
        cudaGraphExec_t exec = nullptr;
        long kernels = 0;
        ~CgGraph() {
            if (exec) cudaGraphExecDestroy(exec);
        }
    } cg_graph;
    bool graph_ok = !h->prof_on && cs.pc != SPD_PC_FACTOR && o.resid != SPD_RESID_DF32;
    if (cs.pc == SPD_PC_LOWRANK) {
        st = lowrank_reserve(h, cs.LR, n, m);
        if (st != SPD_OK) return st;
    }
    int outer = 0;
    IrSummary sm{};
    for (;;) {
        st = read_summary(h, w.sum, &sm);
        if (st != SPD_OK) return st;
        if (sm.active == 0) break;
        if (outer >= o.maxit) {
            *last = sm;
            return set_err(h, SPD_ERR_NO_CONVERGENCE, "CG refinement: %d columns above tolerance after %d outer steps",
                           sm.active, outer);
        }
        ++(h)->launches, k_frozen_from_cols<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, w.frozen);
        ++(h)->launches, k_inner_target<<<ceil_div(m, 128), 128, 0, s>>>(w.b2, w.colnorms, w.anorm, m, o.crit, o.tol, n, w.target);
        const bool fac = (cs.pc == SPD_PC_FACTOR);
        const bool lowrank = (cs.pc == SPD_PC_LOWRANK);
        ++(h)->launches, k_cg_start<<<gv, 256, 0, s>>>(n, m, w.R, n, w.E, w.Rr, w.Z, w.P, w.Pf,
                                      cs.pc == SPD_PC_JACOBI ? cs.dinv : nullptr, (fac || lowrank) ? 0 : 1);
        LAUNCH_CHECK(h);
        if (fac || lowrank) {
            st = fac ? lp_apply(h, cs.F, n, m, w.Rr, n, w.Yz, w.Z, n, nullptr, 0)
                     : lowrank_apply_cg(h, cs.LR, n, m, w.Rr, n, w.Z, n);
            if (st != SPD_OK) return st;
            ++(h)->launches, k_copy_p<<<gv, 256, 0, s>>>(n, m, w.Z, w.P, w.Pf);
        }
        ++(h)->launches, k_dot2<<<dim3(w.G2, m), 256, 0, s>>>(w.Rr, Zr, w.Rr, w.Rr, n, m, w.part);
        ++(h)->launches, k_cg_init_cols<<<ceil_div(m, 4), 128, 0, s>>>(w.part, w.G2, m, w.cg, w.frozen, o.eta, w.target);
        LAUNCH_CHECK(h);
        // one inner step (products, dots, updates) at iteration t
        auto step = [&](int t) -> spd_status {
            const int par = t & 1;
            spd_status sst = SPD_OK;
            switch (cs.matvec) {
                case MV_FP32: mv_dispatch<float>(h, cs, n, m, w.Pf, w.Q); break;
                case MV_BF16: mv_dispatch<__nv_bfloat16>(h, cs, n, m, w.Pf, w.Q); break;
                case MV_TC:
                    sst = mv_tc(h, cs, n, m, w.Pf, w.Q);
                    if (sst != SPD_OK) return sst;
                    break;
                case MV_BAND: {  // (2b + 1) n float32 entries of the band per product
                    ProfScope ps(h, SPD_PHASE_MATVEC, 2.0 * (2.0 * cs.band + 1.0) * n * m,
                                 4.0 * (2.0 * cs.band + 1.0) * n, s);
                    ++(h)->launches, k_matvec_band<<<gv, 256, 0, s>>>(static_cast<const float*>(cs.At), n, cs.band,
                                                                       w.Pf, m, w.Q);
                    break;
                }
                default:
                    sst = resid_run(h, w.rw, n, m, A, lda, nullptr, 0, w.P, n, w.Q, n, nullptr, nullptr, 1, o.resid);
                    if (sst != SPD_OK) return sst;
            }
            LAUNCH_CHECK(h);
            ++(h)->launches, k_dot2<<<dim3(w.G2, m), 256, 0, s>>>(w.P, w.Q, nullptr, nullptr, n, m, w.part);
            if (lowrank) {
                // the Woodbury apply fused into the update and the next dots:
                // as many launches per step as Jacobi-PCG
                const LowrankView v = lowrank_view(cs.LR, n, m);
                ++(h)->launches, k_cg_update_wb<<<dim3(v.G, m), 256, 0, s>>>(w.part, w.G2, n, m, w.cg, par, w.E, w.Rr,
                                                                            w.P, w.Q, v.sdg, v.dh, v.Uh, v.wpart);
                ++(h)->launches, k_wb_apply_dot<<<dim3(v.G, m), 256, 0, s>>>(w.Rr, v.sdg, v.dh, v.Uh, v.Lc, v.wpart, v.G,
                                                                            n, m, w.Z, v.dpart);
                ++(h)->launches, k_cg_pupdate<<<gv, 256, 0, s>>>(v.dpart, v.G, n, m, w.cg, par, w.active, w.P, w.Pf, Zr);
                LAUNCH_CHECK(h);
                return SPD_OK;
            }
            ++(h)->launches, k_cg_update<<<gv, 256, 0, s>>>(w.part, w.G2, n, m, w.cg, par, w.E, w.Rr, w.P, w.Q,
                                           cs.pc == SPD_PC_JACOBI ? cs.dinv : nullptr, w.Z);
            LAUNCH_CHECK(h);
            if (fac) {
                sst = lp_apply(h, cs.F, n, m, w.Rr, n, w.Yz, w.Z, n, nullptr, 0);
                if (sst != SPD_OK) return sst;
            }
            ++(h)->launches, k_dot2<<<dim3(w.G2, m), 256, 0, s>>>(w.Rr, Zr, w.Rr, w.Rr, n, m, w.part);
            ++(h)->launches, k_cg_pupdate<<<gv, 256, 0, s>>>(w.part, w.G2, n, m, w.cg, par, w.active, w.P, w.Pf, Zr);
            LAUNCH_CHECK(h);
            return SPD_OK;
        };
        for (int t = 0; t < o.maxit_inner;) {
            if (graph_ok && (t & 1) == 0 && t + CG_GRAPH_STEPS <= o.maxit_inner) {
                if (!cg_graph.exec) {
                    // capture CG_GRAPH_STEPS steps (the launches are the same
                    // for every group starting at an even step); on any
                    // failure run the steps directly
                    const long l0 = h->launches;
                    cudaGraph_t graph = nullptr;
                    spd_status cst = SPD_OK;
                    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                        for (int k = 0; k < CG_GRAPH_STEPS && cst == SPD_OK; ++k) cst = step(t + k);
                        const cudaError_t e = cudaStreamEndCapture(s, &graph);
                        if (cst == SPD_OK && e == cudaSuccess &&
                            cudaGraphInstantiate(&cg_graph.exec, graph, 0) != cudaSuccess)
                            cg_graph.exec = nullptr;
                    }
                    if (graph) cudaGraphDestroy(graph);
                    cudaGetLastError();
                    cg_graph.kernels = h->launches - l0;
                    h->launches = l0;
                    if (!cg_graph.exec) {
                        graph_ok = false;
                        continue;
                    }
                }
                CUDA_TRY(h, cudaGraphLaunch(cg_graph.exec, s));
                h->launches += cg_graph.kernels;
                t += CG_GRAPH_STEPS;
            } else {
                st = step(t);
                if (st != SPD_OK) return st;
                ++t;
            }
            if (t % 8 == 0 || t == o.maxit_inner) {
                int act = 0;
                st = read_int(h, w.active, &act);
                if (st != SPD_OK) return st;
                if (act == 0) break;
            }
        }
        ++(h)->launches, k_add_cols<<<gv, 256, 0, s>>>(X, ldx, w.E, n, m, w.frozen);
        int restart = 0;
        const int rk = pol.next(sm, &restart);
        st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, nullptr, 0, rk);
        if (st != SPD_OK) return st;
        ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 1, 0,
                                                      rk != SPD_RESID_DF32, restart);
        LAUNCH_CHECK(h);
        ++outer;
    }
    *last = sm;
    // inner-step totals (max over columns)
    std::vector<CgCol> hc(m);
    CUDA_TRY(h, cudaMemcpy(hc.data(), w.cg, sizeof(CgCol) * m, cudaMemcpyDeviceToHost));
    int mx = 0;
    for (auto& c : hc) mx = std::max(mx, c.total);
    *low += mx;
    *high += outer;
    return SPD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Algorithm 1: refinement with a low-precision factor
// ---------------------------------------------------------------------------
extern "C" spd_status spd_solve_ir(spd_handle* h, const spd_factor_t* F, int n, int m, const double* A, int lda,
                                   const double* B, int ldb, double* X, int ldx, const spd_opts* opts_in,
                                   spd_report* rep) {
    if (!h) return SPD_ERR_ARG;
    spd_opts o;
    spd_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (rep) memset(rep, 0, sizeof(*rep));
    if (!F || F->n != n || bad_args(n, m, A, lda, B, ldb, X, ldx) || o.maxit < 0 || !(o.tol >= 0.0) ||
        o.crit < 0 || o.crit > 2 || o.resid < SPD_RESID_FP64 || o.resid > SPD_RESID_AUTO)
        return set_err(h, SPD_ERR_ARG, "spd_solve_ir: bad arguments");
    if (n == 0 || m == 0) return SPD_OK;
    cudaStream_t s = h->stream;
    WsPlan p;
    size_t o_[22];
    int S, G2;
    cg_plan(p, h, n, m, o_, &S, &G2);
    TcSetup tcs;
    o.resid = resolve_resid(o.resid, m);
    tc_plan_if(p, h, n, m, o.resid, tcs);
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    CgWs w = cg_bind(h, n, o_, S, G2);
    CUDA_TRY(h, cudaEventRecord(h->e0, s));
    st = tc_bind_prepare(h, tcs, n, m, A, lda, w.rw);
    if (st != SPD_OK) return st;

    ++(h)->launches, k_ircols_init<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, std::max(0, o.polish));
    ++(h)->launches, k_col_nrm2<<<m, 256, 0, s>>>(B, ldb, n, w.b2);
    LAUNCH_CHECK(h);
    st = lp_apply(h, F, n, m, B, ldb, w.Yz, X, ldx, nullptr, 0);  // line 2
    if (st != SPD_OK) return st;
    ResidPolicy pol(o);
    int rk = pol.first(), restart = 0;
    st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, w.anorm, 0, rk);  // line 3
    if (st != SPD_OK) return st;
    ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 0,
                                                  std::max(0, o.polish), rk != SPD_RESID_DF32);
    LAUNCH_CHECK(h);

    int sweeps = 0, low = 1, high = 1, fell = 0;
    IrSummary sm{};
    spd_status result = SPD_OK;
    for (;;) {
        st = read_summary(h, w.sum, &sm);
        if (st != SPD_OK) return st;
        if (sm.active == 0) break;
        if (sweeps >= o.maxit) {
            result = set_err(h, SPD_ERR_NO_CONVERGENCE, "refinement: %d columns above tolerance after %d sweeps",
                             sm.active, sweeps);
            break;
        }
        if (sm.stagnated && o.fallback) {
            // eq. (iterref) no longer holds in practice: continue with CG on A
            // in float64 preconditioned by the low-precision factor
            CgSetup cs;
            cs.matvec = MV_FP64;
            cs.pc = SPD_PC_FACTOR;
            cs.F = F;
            spd_opts fo = o;
            fo.maxit = std::max(1, o.maxit - sweeps);
            fo.eta = std::min(o.eta, 1e-6);
            int lo2 = 0, hi2 = 0;
            result = cg_ir_core(h, w, n, m, A, lda, B, ldb, X, ldx, fo, cs, true, &lo2, &hi2, &sm);
            low += lo2;
            high += hi2;
            fell = 1;
            break;
        }
        ++(h)->launches, k_frozen_from_cols<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, w.frozen);
        st = lp_apply(h, F, n, m, w.R, n, w.Yz, X, ldx, w.frozen, 1);  // lines 5-6
        if (st != SPD_OK) return st;
        rk = pol.next(sm, &restart);
        st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, nullptr, 0, rk);  // line 7
        if (st != SPD_OK) return st;
        ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 1,
                                                      std::max(0, o.polish), rk != SPD_RESID_DF32, restart);
        LAUNCH_CHECK(h);
        ++sweeps;
        ++low;
        ++high;
    }
    CUDA_TRY(h, cudaEventRecord(h->e1, s));
    CUDA_TRY(h, cudaEventSynchronize(h->e1));
    if (result != SPD_ERR_NO_CONVERGENCE && result != SPD_OK) return result;
    if (rep) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->e0, h->e1);
        rep->status = result;
        rep->iters_low = low;
        rep->iters_high = high;
        rep->prec_used = F->prec;
        rep->fell_back = fell;
        rep->berr = sm.max_berr;
        rep->rel_resid = sm.max_rel;
        rep->time_ms = ms;
    }
    return result;
}

// ---------------------------------------------------------------------------
// Algorithm 1, capturable: the loop's stop decision stays on the device
// ---------------------------------------------------------------------------
namespace {

__global__ void k_epoch_advance(int* e, int by) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *e += by;
}

// The report of a capturable solve, from the refinement state on the device.
__global__ void k_async_report(const IrSummary* __restrict__ sum, const IrCol* __restrict__ cols, int m,
                               const DevStatus* __restrict__ st, spd_report_dev* __restrict__ out) {
    __shared__ int s_sweeps;
    if (threadIdx.x == 0) s_sweeps = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) atomicMax(&s_sweeps, cols[c].iters);
    __syncthreads();
    if (threadIdx.x == 0) {
        out->status = st->flags ? (st->flags & SPD_DEV_TIMEOUT ? SPD_ERR_TIMEOUT : SPD_ERR_CUDA)
                                : (sum->active == 0 ? SPD_OK : SPD_ERR_NO_CONVERGENCE);
        out->active = sum->active;
        out->sweeps = s_sweeps;
        out->stagnated = sum->stagnated;
        out->dev_flags = st->flags;
        out->berr = sum->max_berr;
        out->rel_resid = sum->max_rel;
    }
}

// Clears h's capturable-solve state on every way out.
struct AsyncScope {
    spd_handle* h;
    ~AsyncScope() {
        h->async_on = false;
        h->async_gate = nullptr;
    }
};

}  // namespace

extern "C" spd_status spd_solve_ir_async(spd_handle* h, const spd_factor_t* F, int n, int m, const double* A, int lda,
                                         const double* B, int ldb, double* X, int ldx, const spd_opts* opts_in,
                                         spd_report_dev* rep) {
    if (!h) return SPD_ERR_ARG;
    spd_opts o;
    spd_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (!F || F->n != n || bad_args(n, m, A, lda, B, ldb, X, ldx) || !rep || o.maxit < 0 || !(o.tol >= 0.0) ||
        o.crit < 0 || o.crit > 2 || o.resid < SPD_RESID_FP64 || o.resid > SPD_RESID_AUTO || F->prec == SPD_PREC_FP64)
        return set_err(h, SPD_ERR_ARG, "spd_solve_ir_async: bad arguments");
    if (n == 0 || m == 0) return SPD_OK;
    o.resid = resolve_resid(o.resid, m);
    const int kind = o.resid == SPD_RESID_TC ? SPD_RESID_TC : SPD_RESID_FP64;  // no hybrid: no host decision
    cudaStream_t s = h->stream;
    WsPlan p;
    size_t o_[22];
    int S, G2;
    cg_plan(p, h, n, m, o_, &S, &G2);
    TcSetup tcs;
    tc_plan_if(p, h, n, m, kind, tcs);
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    if (!h->async_epoch_dev) {  // first capturable solve of this handle
        CUDA_TRY(h, cudaMalloc(&h->async_epoch_dev, 256));
        CUDA_TRY(h, cudaMemsetAsync(h->async_epoch_dev, 0, 256, s));
    }
    CgWs w = cg_bind(h, n, o_, S, G2);
    st = tc_bind_prepare(h, tcs, n, m, A, lda, w.rw);
    if (st != SPD_OK) return st;
    AsyncScope scope{h};
    h->async_on = true;
    h->async_gate = nullptr;  // line 2 and the first residual always run
    h->async_rel = 0;
    h->async_total = 2 * ceil_div(m, 16) * (1 + o.maxit);  // sweep launches of this solve
    ++h->launches, k_epoch_advance<<<1, 32, 0, s>>>(h->async_epoch_dev, h->async_total);
    ++(h)->launches, k_ircols_init<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, std::max(0, o.polish));
    ++(h)->launches, k_col_nrm2<<<m, 256, 0, s>>>(B, ldb, n, w.b2);
    LAUNCH_CHECK(h);
    st = lp_apply(h, F, n, m, B, ldb, w.Yz, X, ldx, nullptr, 0);  // line 2
    if (st != SPD_OK) return st;
    st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, w.anorm, 0, kind);  // line 3
    if (st != SPD_OK) return st;
    ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 0,
                                                  std::max(0, o.polish), 1);
    LAUNCH_CHECK(h);
    // maxit sweeps; the solves and residuals of each return at once when no
    // column is left (sum->active == 0); the frozen-column update and the
    // check leave a converged state as it is
    h->async_gate = &w.sum->active;
    for (int it = 0; it < o.maxit; ++it) {
        ++(h)->launches, k_frozen_from_cols<<<ceil_div(m, 128), 128, 0, s>>>(w.cols, m, w.frozen);
        st = lp_apply(h, F, n, m, w.R, n, w.Yz, X, ldx, w.frozen, 1);  // lines 5-6
        if (st != SPD_OK) return st;
        st = resid_run(h, w.rw, n, m, A, lda, B, ldb, X, ldx, w.R, n, w.colnorms, nullptr, 0, kind);  // line 7
        if (st != SPD_OK) return st;
        ++(h)->launches, k_ir_check<<<1, 256, 0, s>>>(w.colnorms, w.anorm, w.b2, m, o.crit, o.tol, w.cols, w.sum, 1,
                                                      std::max(0, o.polish), 1);
        LAUNCH_CHECK(h);
    }
    ++h->launches, k_async_report<<<1, 256, 0, s>>>(w.sum, w.cols, m, h->dst, rep);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 2
// ---------------------------------------------------------------------------
extern "C" spd_status spd_cg(spd_handle* h, int n, int m, const double* A, int lda, int matvec_prec, int pc,
                             const void* pc_data, const double* B, int ldb, double* X, int ldx,
                             const spd_opts* opts_in, spd_report* rep) {
    if (!h) return SPD_ERR_ARG;
    spd_opts o;
    spd_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (rep) memset(rep, 0, sizeof(*rep));
    if (bad_args(n, m, A, lda, B, ldb, X, ldx) || o.maxit < 0 || o.maxit_inner < 1 || !(o.tol >= 0.0) ||
        o.crit < 0 || o.crit > 2 || pc < SPD_PC_NONE || pc > SPD_PC_LOWRANK || o.resid < SPD_RESID_FP64 ||
        o.resid > SPD_RESID_AUTO ||
        ((pc == SPD_PC_FACTOR || pc == SPD_PC_LOWRANK) && !pc_data))
        return set_err(h, SPD_ERR_ARG, "spd_cg: bad arguments");
    if (matvec_prec != SPD_PREC_FP64 && matvec_prec != SPD_PREC_FP32 && matvec_prec != SPD_PREC_BF16)
        return set_err(h, SPD_ERR_UNSUPPORTED, "spd_cg: matrix-vector precision must be FP64, FP32 or BF16");
    if (o.band >= 0 && matvec_prec != SPD_PREC_FP32)
        return set_err(h, SPD_ERR_UNSUPPORTED, "spd_cg: the banded inner matrix is stored in FP32");
    if (pc == SPD_PC_FACTOR && static_cast<const spd_factor_t*>(pc_data)->n != n)
        return set_err(h, SPD_ERR_ARG, "spd_cg: factor order differs from n");
    if (pc == SPD_PC_LOWRANK && lowrank_order(static_cast<const spd_lowrank*>(pc_data)) != n)
        return set_err(h, SPD_ERR_ARG, "spd_cg: preconditioner order differs from n");
    if (n == 0 || m == 0) return SPD_OK;
    cudaStream_t s = h->stream;
    WsPlan p;
    size_t o_[22];
    int S, G2;
    cg_plan(p, h, n, m, o_, &S, &G2);
    CgSetup cs;
    cs.pc = pc;
    if (pc == SPD_PC_FACTOR) cs.F = static_cast<const spd_factor_t*>(pc_data);
    if (pc == SPD_PC_LOWRANK) cs.LR = static_cast<const spd_lowrank*>(pc_data);
    size_t o_at = 0, o_dinv = 0, o_pm = 0, o_cf = 0, o_sk = 0;
    long ldt = round_up(n, 64);
    // float32 products with several right-hand sides go to the tensor cores
    const bool tc_mv = o.band < 0 && matvec_prec == SPD_PREC_FP32 &&
                       (o.matvec_cores == SPD_MV_TENSOR || (o.matvec_cores == SPD_MV_AUTO && m >= 8));
    const int bnt = m <= 32 ? 32 : 64;
    if (o.band >= 0) {
        cs.matvec = MV_BAND;
        cs.band = o.band;
        o_at = p.add<float>((size_t)(2 * o.band + 1) * n);
    } else if (tc_mv) {
        cs.matvec = MV_TC;
        cs.Kp = (int)round_up(n, 128);
        cs.ldo = cs.Kp;
        const long prow = round_up(m, bnt);
        cs.plane_p = prow * cs.ldo;
        cs.ldc = round_up(m, 32);
        o_at = p.add<__nv_bfloat16>((size_t)3 * n * cs.ldo);
        o_pm = p.add<__nv_bfloat16>((size_t)3 * cs.plane_p);
        o_cf = p.add<float>((size_t)n * cs.ldc);
        cs.sk.part_cap = (size_t)2 * std::max(h->sms, 1) * 128 * bnt;
        o_sk = p.add<float>(cs.sk.part_cap);
    } else if (matvec_prec == SPD_PREC_FP32) {
        cs.matvec = MV_FP32;
        o_at = p.add<float>((size_t)n * ldt);
    } else if (matvec_prec == SPD_PREC_BF16) {
        cs.matvec = MV_BF16;
        o_at = p.add<__nv_bfloat16>((size_t)n * ldt);
    }
    if (pc == SPD_PC_JACOBI) o_dinv = p.add<double>(n);
    TcSetup tcs;
    o.resid = resolve_resid(o.resid, m);
    tc_plan_if(p, h, n, m, o.resid, tcs);
    spd_status st = ws_reserve(h, p.bytes);
    if (st != SPD_OK) return st;
    CgWs w = cg_bind(h, n, o_, S, G2);
    CUDA_TRY(h, cudaEventRecord(h->e0, s));
    st = tc_bind_prepare(h, tcs, n, m, A, lda, w.rw);
    if (st != SPD_OK) return st;
    const int gbig = grid_for((long)n * n, 256, 16 * h->sms);
    struct TgGuard {  // the narrow GEMM's maps live for this call
        TcGemm*& g;
        ~TgGuard() {
            if (g) tc_gemm_destroy(g);
        }
    } tg_guard{cs.tg};
    if (cs.matvec == MV_TC) {
        __nv_bfloat16* Am = ws_at<__nv_bfloat16>(h, o_at);
        cs.Pm = ws_at<__nv_bfloat16>(h, o_pm);
        cs.Cf = ws_at<float>(h, o_cf);
        cs.sk.part = ws_at<float>(h, o_sk);
        ++(h)->launches, k_convert_x3<<<gbig, 256, 0, s>>>(A, lda, n, cs.Kp, Am, cs.ldo, (long)n * cs.ldo, h->dst);
        CUDA_TRY(h, cudaMemsetAsync(cs.Pm, 0, sizeof(__nv_bfloat16) * 3 * cs.plane_p, s));
        st = tc_gemm_create_narrow(&cs.tg, Am, n, cs.ldo, cs.Pm, cs.plane_p / cs.ldo, cs.ldo, cs.Kp, cs.Cf, n,
                                   cs.ldc, cs.ldc, bnt);
        if (st != SPD_OK) return set_err(h, st, "spd_cg: tensor maps of the product failed");
        cs.At = Am;
    } else if (cs.matvec == MV_BAND) {
        float* Ab = ws_at<float>(h, o_at);
        ++(h)->launches, k_convert_band<<<grid_for((long)(2 * o.band + 1) * n, 256, 16 * h->sms), 256, 0, s>>>(A, lda, n, o.band, Ab,
                                                                                            h->dst);
        cs.At = Ab;
    } else if (cs.matvec == MV_FP32) {
        float* At = ws_at<float>(h, o_at);
        CUDA_TRY(h, cudaMemsetAsync(At, 0, sizeof(float) * n * ldt, s));
        ++(h)->launches, k_convert_full<float><<<gbig, 256, 0, s>>>(A, lda, n, At, ldt, h->dst);
        cs.At = At;
        cs.ldt = ldt;
    } else if (cs.matvec == MV_BF16) {
        __nv_bfloat16* At = ws_at<__nv_bfloat16>(h, o_at);
        CUDA_TRY(h, cudaMemsetAsync(At, 0, sizeof(__nv_bfloat16) * n * ldt, s));
        ++(h)->launches, k_convert_full<__nv_bfloat16><<<gbig, 256, 0, s>>>(A, lda, n, At, ldt, h->dst);
        cs.At = At;
        cs.ldt = ldt;
    }
    if (pc == SPD_PC_JACOBI) {
        double* dinv = ws_at<double>(h, o_dinv);
        ++(h)->launches, k_jacobi_dinv<<<ceil_div(n, 256), 256, 0, s>>>(A, lda, n, dinv);
        cs.dinv = dinv;
    }
    LAUNCH_CHECK(h);
    st = check_dev_status(h, rep, "spd_cg");
    if (st != SPD_OK) return st;
    int low = 0, high = 0;
    IrSummary sm{};
    spd_status result = cg_ir_core(h, w, n, m, A, lda, B, ldb, X, ldx, o, cs, false, &low, &high, &sm);
    CUDA_TRY(h, cudaEventRecord(h->e1, s));
    CUDA_TRY(h, cudaEventSynchronize(h->e1));
    if (result != SPD_ERR_NO_CONVERGENCE && result != SPD_OK) return result;
    if (rep) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->e0, h->e1);
        rep->status = result;
        rep->iters_low = low;
        rep->iters_high = high;
        rep->prec_used = matvec_prec;
        rep->berr = sm.max_berr;
        rep->rel_resid = sm.max_rel;
        rep->time_ms = ms;
    }
    return result;
}

// ---------------------------------------------------------------------------
// host-buffer convenience entry point
// ---------------------------------------------------------------------------
extern "C" spd_status spd_solve_ir_host(spd_handle* h, int n, int m, const double* A_host, int lda,
                                        const double* B_host, int ldb, double* X_host, int ldx, int prec,
                                        const spd_opts* opts, spd_report* rep) {
    if (!h) return SPD_ERR_ARG;
    if (bad_args(n, m, A_host, lda, B_host, ldb, X_host, ldx))
        return set_err(h, SPD_ERR_ARG, "spd_solve_ir_host: bad arguments");
    if (rep) memset(rep, 0, sizeof(*rep));
    if (n == 0 || m == 0) return SPD_OK;
    cudaStream_t s = h->stream;
    const size_t bytesA = (size_t)round_up((long)(sizeof(double) * (size_t)n * n), 256);
    const size_t bytesB = (size_t)round_up((long)(sizeof(double) * (size_t)n * m), 256);
    if (h->stage_bytes < bytesA + 2 * bytesB) {  // grow (the previous call ended synchronised)
        if (over_cap(h, bytesA + 2 * bytesB))
            return set_err(h, SPD_ERR_OOM, "spd_solve_ir_host: device copies of %zu bytes exceed the handle's "
                           "memory cap of %zu bytes", bytesA + 2 * bytesB, h->mem_cap);
        CUDA_TRY(h, cudaStreamSynchronize(s));
        cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        CUDA_TRY(h, cudaMalloc(&h->stage, bytesA + 2 * bytesB));
        h->stage_bytes = bytesA + 2 * bytesB;
    }
    double* dA = static_cast<double*>(h->stage);
    double* dB = reinterpret_cast<double*>(static_cast<char*>(h->stage) + bytesA);
    double* dX = reinterpret_cast<double*>(static_cast<char*>(h->stage) + bytesA + bytesB);
    auto release = [&]() { cudaStreamSynchronize(s); };
    cudaError_t e = cudaMemcpy2DAsync(dA, sizeof(double) * n, A_host, sizeof(double) * lda, sizeof(double) * n, n,
                                      cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dB, sizeof(double) * n, B_host, sizeof(double) * ldb, sizeof(double) * n, m,
                              cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        release();
        return set_err(h, SPD_ERR_CUDA, "spd_solve_ir_host: copy to device: %s", cudaGetErrorString(e));
    }
    spd_factor_t* F = nullptr;
    spd_report fr{};
    spd_status st = spd_factor(h, n, dA, n, prec, SPD_SCALE_DIAG, &F, &fr);
    if (st != SPD_OK) {
        if (rep) *rep = fr;
        release();
        return st;
    }
    st = spd_solve_ir(h, F, n, m, dA, n, dB, n, dX, n, opts, rep);
    if (st == SPD_OK || st == SPD_ERR_NO_CONVERGENCE) {
        e = cudaMemcpy2DAsync(X_host, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n, m,
                              cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = set_err(h, SPD_ERR_CUDA, "spd_solve_ir_host: copy back: %s", cudaGetErrorString(e));
    }
    if (rep) {
        rep->time_ms += fr.time_ms;
        rep->prec_used = fr.prec_used;
    }
    spd_factor_destroy(F);
    release();
    return st;
}

// ---------------------------------------------------------------------------
// phase timing
// ---------------------------------------------------------------------------
static void prof_clear(spd_handle* h) {
    for (auto& r : h->prof) {
        h->ev_pool.push_back(r.a);
        h->ev_pool.push_back(r.b);
    }
    h->prof.clear();
}

extern "C" spd_status spd_profile_enable(spd_handle* h, int on) {
    if (!h) return SPD_ERR_ARG;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    prof_clear(h);
    h->prof_on = on != 0;
    return SPD_OK;
}

extern "C" spd_status spd_profile_read(spd_handle* h, int phase, int* launches, double* ms, double* flops,
                                       double* bytes) {
    if (!h || phase < 0 || phase >= SPD_PHASE_COUNT) return SPD_ERR_ARG;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int cnt = 0;
    double t = 0.0, f = 0.0, b = 0.0;
    for (auto& r : h->prof) {
        if (r.phase != phase) continue;
        float e = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&e, r.a, r.b));
        ++cnt;
        t += e;
        f += r.flops;
        b += r.bytes;
    }
    if (launches) *launches = cnt;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
    return SPD_OK;
}

extern "C" spd_status spd_launch_count(const spd_handle* h, long long* count) {
    if (!h || !count) return SPD_ERR_ARG;
    *count = h->launches;
    return SPD_OK;
}
