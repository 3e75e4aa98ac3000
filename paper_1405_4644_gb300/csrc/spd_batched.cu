// spd_batched.cu -- batched solves: a plan holds the device descriptor
// table, the schedule (systems by decreasing order), per-CTA scratch and one
// captured CUDA graph per (method, precision); an autotuner picks the CTA
// size on the first solve of each method by timing the candidates.
#include <numeric>
#include "engine.cuh"
#include "k_batched.cuh"

struct spd_batch {
    spd_handle* h = nullptr;
    int count = 0;
    int nmax = 0;
    BatchSys* sys = nullptr;   // device
    int* order = nullptr;      // device
    int* next = nullptr;       // device counter
    float* scratch = nullptr;  // device, ctas * BLD * BLD
    BatchRep* rep = nullptr;   // device
    int ctas = 0;
    int threads[2] = {0, 0};   // tuned CTA size per method (0 = not tuned)
    float tune_ms[2][2] = {{0, 0}, {0, 0}};
    cudaGraphExec_t graph[2][8] = {};  // [method][prec]
    int graph_nt[2][8] = {};
    double graph_tol[2][8] = {};
    int graph_maxit[2][8] = {};
    int graph_polish[2][8] = {};
};

namespace {

template <int NT>
void launch_batch(spd_batch* b, int method, const BatchArgs& a, cudaStream_t s) {
    const size_t smem = batch_smem_bytes();
    if (method == 0) k_batch_chol_ir<NT><<<b->ctas, NT, smem, s>>>(a);
    else k_batch_pcg<NT><<<b->ctas, NT, smem, s>>>(a);
}

void set_batch_attrs() {
    static const bool done = [] {  // once per process, thread-safe
        const int smem = (int)batch_smem_bytes();
        cudaFuncSetAttribute(k_batch_chol_ir<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_batch_chol_ir<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_batch_pcg<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_batch_pcg<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        return true;
    }();
    (void)done;
}

spd_status run_once(spd_batch* b, int method, int nt, const BatchArgs& a) {
    spd_handle* h = b->h;
    CUDA_TRY(h, cudaMemsetAsync(b->next, 0, sizeof(int), h->stream));
    ++h->launches;
    if (nt == 512) launch_batch<512>(b, method, a, h->stream);
    else launch_batch<256>(b, method, a, h->stream);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

}  // namespace

extern "C" spd_status spd_batch_create(spd_handle* h, int count, const int* n, const double* const* A,
                                       const int* lda, const double* const* B, double* const* X, spd_batch** out) {
    if (!h) return SPD_ERR_ARG;
    if (!out || count < 0 || (count > 0 && (!n || !A || !lda || !B || !X)))
        return set_err(h, SPD_ERR_ARG, "spd_batch_create: bad arguments");
    std::vector<BatchSys> hs(count);
    int nmax = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || n[i] > BMAX || lda[i] < n[i] || !A[i] || !B[i] || !X[i])
            return set_err(h, SPD_ERR_ARG, "spd_batch_create: system %d: n must be in [1, %d] with lda >= n", i, BMAX);
        hs[i] = BatchSys{A[i], B[i], X[i], n[i], lda[i]};
        nmax = std::max(nmax, n[i]);
    }
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
    spd_batch* b = new spd_batch();
    b->h = h;
    b->count = count;
    b->nmax = nmax;
    b->ctas = std::max(1, std::min(h->sms, count));
    set_batch_attrs();
    cudaError_t e = cudaMalloc(&b->sys, sizeof(BatchSys) * std::max(count, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->order, sizeof(int) * std::max(count, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->next, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->rep, sizeof(BatchRep) * std::max(count, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->scratch, sizeof(float) * (size_t)b->ctas * BLD * BLD);
    if (e == cudaSuccess && count > 0)
        e = cudaMemcpy(b->sys, hs.data(), sizeof(BatchSys) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && count > 0) e = cudaMemcpy(b->order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->sys);
        cudaFree(b->order);
        cudaFree(b->next);
        cudaFree(b->rep);
        cudaFree(b->scratch);
        delete b;
        return set_err(h, e == cudaErrorMemoryAllocation ? SPD_ERR_OOM : SPD_ERR_CUDA, "spd_batch_create: %s",
                       cudaGetErrorString(e));
    }
    *out = b;
    return SPD_OK;
}

extern "C" spd_status spd_batch_destroy(spd_batch* b) {
    if (!b) return SPD_OK;
    cudaStreamSynchronize(b->h->stream);
    for (auto& row : b->graph)
        for (auto& g : row)
            if (g) cudaGraphExecDestroy(g);
    cudaFree(b->sys);
    cudaFree(b->order);
    cudaFree(b->next);
    cudaFree(b->rep);
    cudaFree(b->scratch);
    delete b;
    return SPD_OK;
}

namespace {

// The graph of (method, prec, opts): tune the CTA size on first use, then
// capture (or reuse) counter reset + one persistent launch.
spd_status batch_graph(spd_batch* b, int method, int prec, const spd_opts* opts_in, cudaGraphExec_t* out) {
    spd_handle* h = b->h;
    spd_opts o;
    spd_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (method != SPD_BATCH_CHOL_IR && method != SPD_BATCH_PCG_JACOBI)
        return set_err(h, SPD_ERR_ARG, "spd_batch: unknown method %d", method);
    if (method == SPD_BATCH_CHOL_IR && prec != SPD_PREC_FP32 && prec != SPD_PREC_BF16 && prec != SPD_PREC_FP16)
        return set_err(h, SPD_ERR_UNSUPPORTED, "spd_batch: Cholesky-IR precision must be FP32, BF16 or FP16");
    const int mi = method == SPD_BATCH_CHOL_IR ? 0 : 1;
    const int pi = method == SPD_BATCH_CHOL_IR ? prec : 0;
    BatchArgs a{b->sys, b->order, b->count, b->next, b->scratch, b->rep, prec, o.tol,
                method == SPD_BATCH_CHOL_IR ? o.maxit : std::max(o.maxit_inner, 1), std::max(0, o.polish)};
    cudaStream_t s = h->stream;
    spd_status st;
    // autotune the CTA size on the first solve of this method
    if (!b->threads[mi]) {
        const int cand[2] = {256, 512};
        float best = 1e30f;
        for (int c = 0; c < 2; ++c) {
            if ((st = run_once(b, method, cand[c], a)) != SPD_OK) return st;  // warm
            CUDA_TRY(h, cudaEventRecord(h->e0, s));
            if ((st = run_once(b, method, cand[c], a)) != SPD_OK) return st;
            CUDA_TRY(h, cudaEventRecord(h->e1, s));
            CUDA_TRY(h, cudaEventSynchronize(h->e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->e0, h->e1);
            b->tune_ms[mi][c] = ms;
            if (ms < best) {
                best = ms;
                b->threads[mi] = cand[c];
            }
        }
    }
    const int nt = b->threads[mi];
    cudaGraphExec_t& gx = b->graph[mi][pi];
    if (gx && (b->graph_nt[mi][pi] != nt || b->graph_tol[mi][pi] != o.tol || b->graph_maxit[mi][pi] != a.maxit ||
               b->graph_polish[mi][pi] != a.polish)) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
    }
    if (!gx) {  // capture: counter reset + one persistent launch
        cudaStream_t cs;
        CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->next, 0, sizeof(int), cs);
            if (nt == 512) launch_batch<512>(b, method, a, cs);
            else launch_batch<256>(b, method, a, cs);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&gx, g, 0);
            cudaGraphDestroy(g);
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            gx = nullptr;
            return set_err(h, SPD_ERR_CUDA, "spd_batch: graph capture failed: %s", cudaGetErrorString(e));
        }
        b->graph_nt[mi][pi] = nt;
        b->graph_tol[mi][pi] = o.tol;
        b->graph_maxit[mi][pi] = a.maxit;
        b->graph_polish[mi][pi] = a.polish;
    }
    *out = gx;
    return SPD_OK;
}

// Per-system results of the last launch (the handle's stream is drained first).
spd_status batch_results(spd_batch* b, int method, int prec, float ms, spd_report* summary, int* status,
                         double* berr, int* iters) {
    spd_handle* h = b->h;
    std::vector<BatchRep> hr(b->count);
    CUDA_TRY(h, cudaMemcpyAsync(hr.data(), b->rep, sizeof(BatchRep) * b->count, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int bad = 0, maxit = 0, notspd = 0;
    double maxb = 0.0;
    for (int i = 0; i < b->count; ++i) {
        if (status) status[i] = hr[i].status;
        if (berr) berr[i] = hr[i].berr;
        if (iters) iters[i] = hr[i].iters;
        if (hr[i].status != SPD_OK) ++bad;
        if (hr[i].status == SPD_ERR_NOT_SPD) ++notspd;
        maxit = std::max(maxit, hr[i].iters);
        maxb = std::max(maxb, hr[i].berr);
    }
    spd_status result = SPD_OK;
    if (notspd) result = set_err(h, SPD_ERR_NOT_SPD, "spd_batch: %d systems broke down", notspd);
    else if (bad) result = set_err(h, SPD_ERR_NO_CONVERGENCE, "spd_batch: %d systems did not converge", bad);
    if (summary) {
        memset(summary, 0, sizeof(*summary));
        summary->status = result;
        summary->info = bad;
        summary->iters_low = maxit;
        summary->iters_high = maxit;
        summary->prec_used = method == SPD_BATCH_CHOL_IR ? prec : SPD_PREC_FP64;
        summary->berr = maxb;
        summary->time_ms = ms;
    }
    return result;
}

}  // namespace

extern "C" spd_status spd_batch_solve(spd_batch* b, int method, int prec, const spd_opts* opts_in, spd_report* summary,
                                      int* status, double* berr, int* iters) {
    if (!b) return SPD_ERR_ARG;
    spd_handle* h = b->h;
    if (summary) memset(summary, 0, sizeof(*summary));
    if (b->count == 0) return SPD_OK;
    cudaGraphExec_t gx = nullptr;
    spd_status st = batch_graph(b, method, prec, opts_in, &gx);
    if (st != SPD_OK) return st;
    cudaStream_t s = h->stream;
    CUDA_TRY(h, cudaEventRecord(h->e0, s));
    {
        ProfScope ps(h, SPD_PHASE_BATCH, 0.0, 0.0);
        ++h->launches;
        CUDA_TRY(h, cudaGraphLaunch(gx, s));
    }
    CUDA_TRY(h, cudaEventRecord(h->e1, s));
    CUDA_TRY(h, cudaEventSynchronize(h->e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    return batch_results(b, method, prec, ms, summary, status, berr, iters);
}

extern "C" spd_status spd_batch_graph(spd_batch* b, int method, int prec, const spd_opts* opts, void** graph_exec) {
    if (!b || !graph_exec) return SPD_ERR_ARG;
    *graph_exec = nullptr;
    if (b->count == 0) return set_err(b->h, SPD_ERR_ARG, "spd_batch_graph: empty plan");
    cudaGraphExec_t gx = nullptr;
    spd_status st = batch_graph(b, method, prec, opts, &gx);
    if (st == SPD_OK) *graph_exec = gx;
    return st;
}

extern "C" spd_status spd_batch_results(spd_batch* b, int method, int prec, spd_report* summary, int* status,
                                        double* berr, int* iters) {
    if (!b) return SPD_ERR_ARG;
    if (b->count == 0) return SPD_OK;
    return batch_results(b, method, prec, 0.f, summary, status, berr, iters);
}

extern "C" spd_status spd_graph_launch(void* graph_exec, void* stream) {
    if (!graph_exec) return SPD_ERR_ARG;
    return cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SPD_OK
               : SPD_ERR_CUDA;
}

extern "C" spd_status spd_batch_info(const spd_batch* b, int method, int* threads_per_cta, int* ctas,
                                     float* tune_ms) {
    if (!b || (method != SPD_BATCH_CHOL_IR && method != SPD_BATCH_PCG_JACOBI)) return SPD_ERR_ARG;
    const int mi = method == SPD_BATCH_CHOL_IR ? 0 : 1;
    if (threads_per_cta) *threads_per_cta = b->threads[mi];
    if (ctas) *ctas = b->ctas;
    if (tune_ms) {
        tune_ms[0] = b->tune_ms[mi][0];
        tune_ms[1] = b->tune_ms[mi][1];
    }
    return SPD_OK;
}
