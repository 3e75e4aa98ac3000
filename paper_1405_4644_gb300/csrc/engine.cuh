// engine.cuh -- host-side engine of libspd: handle, workspace, launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <climits>
#include <vector>
#include <algorithm>
#include "spd.h"
#include "common.cuh"

struct ProfRec {
    cudaEvent_t a, b;
    int phase;
    double flops, bytes;
};

struct spd_handle {
    cudaStream_t stream = nullptr;
    bool prof_on = false;
    long long launches = 0;             // kernels launched through this handle
    std::vector<ProfRec> prof;          // recorded launches
    std::vector<cudaEvent_t> ev_pool;   // free events
    int device = 0;
    int sms = 0;
    char err[512] = {0};
    DevStatus* dst = nullptr;   // device status word
    void* pinned = nullptr;     // 4 KB pinned host scratch
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void* ws = nullptr;         // grow-only device workspace
    size_t ws_bytes = 0;
    int* ready = nullptr;       // block flags of the persistent triangular sweeps
    int ready_n = 0;
    int epoch = 0;              // last flag value handed out
    cudaStream_t aux = nullptr; // second stream of the look-ahead factorisation
    std::vector<cudaEvent_t> sync_ev;  // timing-free events for stream joins
    void* stage = nullptr;      // grow-only device copies of spd_solve_ir_host's A, B, X
    size_t stage_bytes = 0;
    unsigned long long wait_ns = 1000000000ull;  // bound of a spin-wait on another CTA's flag
    // a capturable solve in progress (spd_solve_ir_async): its kernels return
    // at once while *async_gate == 0, and its sweeps take their flag epochs
    // from the device counter async_epoch_dev (advanced by the solve itself),
    // never from values fixed when the launches were issued
    bool async_on = false;
    const int* async_gate = nullptr;
    int* async_epoch_dev = nullptr;
    int async_rel = 0, async_total = 0;
    void* sb_buf = nullptr;     // super-block sweeps: partial tiles, then two barrier words
    size_t sb_bytes = 0;
    size_t mem_cap = 0;         // largest device request of one call (0 = no cap): spd_set_memory_cap
};

// SPD_ERR_OOM when one call's device request exceeds the handle's cap.
static inline bool over_cap(const spd_handle* h, size_t bytes) { return h->mem_cap && bytes > h->mem_cap; }

struct spd_factor_t {
    spd_handle* h = nullptr;
    int n = 0;
    long ldw = 0;
    int prec = SPD_PREC_FP32;
    float* W = nullptr;        // float32 factor (row-major lower)
    double* W64 = nullptr;     // float64 factor (SPD_PREC_FP64)
    void* Wh = nullptr;        // tensor-core operand mirror
    long ldh = 0;
    double* d = nullptr;       // scaling
    double* Dinv64 = nullptr;  // float64 factor: 32x32 diagonal sub-block inverses
    float* LinvT = nullptr;    // float32 factor: (L_JJ^{-1})^T of every 128x128 block
    float* Cpl = nullptr;      // float32 factor: sweep couplings M_J, N_J, P_J, Q_J (4 x nblk128 blocks)
    float* Dinv32 = nullptr;   // float32 factor: inverses of the 32x32 diagonal sub-blocks
    int nblk128 = 0;
    float* Xsb = nullptr;      // float32 factor: inverses of the diagonal super-blocks (sbb 128-blocks each)
    int sbb = 0, nsb = 0;      // 128-blocks per super-block, super-blocks (0: 128-block sweeps)
};

static spd_status set_err(spd_handle* h, spd_status s, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CUDA_TRY(h, call)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            if (e_ == cudaErrorMemoryAllocation) {                                               \
                cudaGetLastError();                                                              \
                return set_err(h, SPD_ERR_OOM, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                               __FILE__, __LINE__);                                              \
            }                                                                                    \
            return set_err(h, SPD_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                           __FILE__, __LINE__);                                                  \
        }                                                                                        \
    } while (0)

#define LAUNCH_CHECK(h) CUDA_TRY(h, cudaGetLastError())

static inline long round_up(long x, long a) { return (x + a - 1) / a * a; }
static inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Bump allocator over the handle's workspace.  size() first, then take().
struct WsPlan {
    size_t bytes = 0;
    template <typename T> size_t add(size_t count) {
        size_t off = bytes;
        bytes += round_up((long)(count * sizeof(T)), 256);
        return off;
    }
};

static inline spd_status ws_reserve(spd_handle* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return SPD_OK;
    if (over_cap(h, bytes))
        return set_err(h, SPD_ERR_OOM, "workspace of %zu bytes exceeds the handle's memory cap of %zu bytes", bytes,
                       h->mem_cap);
    if (h->ws) {
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        CUDA_TRY(h, cudaFree(h->ws));
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = (size_t)round_up((long)bytes, 1 << 20);
    CUDA_TRY(h, cudaMalloc(&h->ws, want));
    h->ws_bytes = want;
    return SPD_OK;
}

template <typename T> static inline T* ws_at(spd_handle* h, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(h->ws) + off);
}

static inline int grid_for(long work, int threads, int cap) {
    long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Read and clear the device status word; map to spd_status.
static inline spd_status check_dev_status(spd_handle* h, spd_report* rep, const char* what) {
    DevStatus* hs = static_cast<DevStatus*>(h->pinned);
    CUDA_TRY(h, cudaMemcpyAsync(hs, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    DevStatus s = *hs;
    if (s.flags == 0) return SPD_OK;
    DevStatus clear{0, INT_MAX, {0, 0}};
    CUDA_TRY(h, cudaMemcpyAsync(h->dst, &clear, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (rep) rep->info = (s.info == INT_MAX) ? 0 : s.info;
    if (s.flags & SPD_DEV_NONFINITE) return set_err(h, SPD_ERR_ARG, "%s: non-finite entry in the input", what);
    if (s.flags & SPD_DEV_BADDIAG)
        return set_err(h, SPD_ERR_NOT_SPD, "%s: non-positive diagonal entry at %d", what, s.info);
    if (s.flags & SPD_DEV_BREAKDOWN)
        return set_err(h, SPD_ERR_NOT_SPD, "%s: non-positive pivot at column %d", what, s.info);
    if (s.flags & SPD_DEV_TIMEOUT) return set_err(h, SPD_ERR_TIMEOUT, "%s: bounded device wait expired", what);
    return set_err(h, SPD_ERR_CUDA, "%s: device status 0x%x", what, s.flags);
}

// RAII phase marker: records an event pair around the launches in scope.
struct ProfScope {
    spd_handle* h;
    ProfRec r;
    bool on;
    static cudaEvent_t get_event(spd_handle* h) {
        if (!h->ev_pool.empty()) {
            cudaEvent_t e = h->ev_pool.back();
            h->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    cudaStream_t s;
    ProfScope(spd_handle* hh, int phase, double flops, double bytes, cudaStream_t st = nullptr)
        : h(hh), on(hh->prof_on), s(st ? st : hh->stream) {
        if (!on) return;
        r.a = get_event(h);
        r.b = get_event(h);
        r.phase = phase;
        r.flops = flops;
        r.bytes = bytes;
        cudaEventRecord(r.a, s);
    }
    ~ProfScope() {
        if (!on) return;
        cudaEventRecord(r.b, s);
        h->prof.push_back(r);
    }
};

// y <- (L L^T)^{-1} y for one float32 vector of the scaled system (no d
// scaling); defined with the triangular-solve kernels.
spd_status factor_apply_scaled_f32(spd_handle* h, const spd_factor_t* F, float* y);
spd_status factor_couplings(spd_handle* h, spd_factor_t* F);

// learned low-rank preconditioner hooks for the CG driver (spd_learned.cu)
struct spd_lowrank;
int lowrank_order(const spd_lowrank* P);
spd_status lowrank_apply_cg(spd_handle* h, const spd_lowrank* P, int n, int m, const double* R, long ldr, double* Z,
                            long ldz);
spd_status lowrank_reserve(spd_handle* h, const spd_lowrank* P, int n, int m);
// The arrays of a built low-rank preconditioner, for the CG kernels that fuse
// its Woodbury apply into the inner step (rank LOWRANK_RANK): G = 256-row
// chunks, wpart = G x m x rank partial projections, dpart = G x m x 2 dot
// partials (both inside the buffer lowrank_reserve sized for m columns).
constexpr int LOWRANK_RANK = 32;
struct LowrankView {
    const double *sdg, *dh, *Uh, *Lc;
    double *wpart, *dpart;
    int G;
};
LowrankView lowrank_view(const spd_lowrank* P, int n, int m);
