// spd_noalloc.cu -- the float64 residual R = B - A X for callers that cannot
// allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator's own hooks, in a process whose memory
// budget is fixed up front (an embedded solver service, a plugin given a
// pre-sized arena), or in a real-time loop that must never stall on the
// allocator.  spd_residual keeps its partial sums in the handle's workspace,
// which it grows with cudaMalloc on demand; this entry point instead uses a
// fixed scratch array that is part of the library image, so it allocates
// nothing at all -- not even a handle.
//
// The scratch is one file-scope __device__ array (SPD_NOALLOC_SCRATCH_BYTES).
// Every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it for the life of the process; make that first
// call before any stream capture.  The cache assumes the device's context
// lives as long as the process: a program that calls cudaDeviceReset on a
// device must not call this entry point on that device afterwards.  All calls
// share the array and it keeps the last call's partial sums: calls whose work
// overlaps on the GPU (two streams, or two host threads) race on it and must
// be serialised by the caller.  Nothing in the array has to start at zero:
// each call writes every partial sum before it reads it.  The call returns
// after `stream` has drained.
#include <mutex>
#include "engine.cuh"
#include "k_resid.cuh"

#define SPD_NOALLOC_SCRATCH_BYTES (16u << 20)
#define SPD_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_resid_scratch[SPD_NOALLOC_SCRATCH_BYTES / sizeof(double)];

namespace {

std::mutex g_mu;
double* g_scratch_ptr[SPD_NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= SPD_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_resid_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" spd_status spd_residual_static(void* stream, int n, int m, const double* A, int lda, const double* B,
                                          int ldb, const double* X, int ldx, double* R, int ldr, double* colnorms) {
    if (n < 0 || m < 0) return SPD_ERR_ARG;
    if (n == 0 || m == 0) return SPD_OK;
    if (!A || !B || !X || !R || lda < n || ldb < n || ldx < n || ldr < n) return SPD_ERR_ARG;
    // launch errors are read back below; clear one left by unrelated earlier
    // work so that it is not reported as this call's
    (void)cudaGetLastError();
    const size_t cap = SPD_NOALLOC_SCRATCH_BYTES / sizeof(double);
    const int G = ceil_div(n, 256);
    const size_t np = (size_t)G * m * 3;        // block partial norms
    const size_t per_split = (size_t)n * m;     // one column split of partial sums
    if (np + per_split > cap) return SPD_ERR_SCRATCH;  // too large for the fixed scratch
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPD_ERR_CUDA;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return SPD_ERR_CUDA;
    // as many column splits as fit, up to the same target as the handle path
    const int rowblk = ceil_div(n, RESID_ROWS);
    int S = std::max(1, (4 * sms + rowblk - 1) / rowblk);
    S = std::min(S, std::max(1, n / (4 * RESID_JT)));
    S = std::min<long>(S, (long)((cap - np) / per_split));
    double* P = scratch;
    double* NP = scratch + (size_t)S * per_split;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int jchunk = (int)round_up(ceil_div(n, S), RESID_JT);
    dim3 grid(rowblk, S);
    for (int c0 = 0; c0 < m; c0 += 16) {
        const int mc = std::min(16, m - c0);
        if (mc == 1)
            k_resid_partial<1><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, P, nullptr);
        else if (mc == 2)
            k_resid_partial<2><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, P, nullptr);
        else if (mc <= 4)
            k_resid_partial<4><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, P, nullptr);
        else if (mc <= 8)
            k_resid_partial<8><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, P, nullptr);
        else
            k_resid_partial<16><<<grid, RESID_ROWS, 0, s>>>(A, lda, n, X, ldx, c0, mc, jchunk, m, P, nullptr);
    }
    k_resid_final<<<dim3(G, m), 256, 0, s>>>(B, ldb, n, m, P, S, R, ldr, X, ldx, NP, 0);
    if (colnorms) k_colnorms<<<m, 256, 0, s>>>(NP, G, m, colnorms);
    if (cudaGetLastError() != cudaSuccess) return SPD_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? SPD_OK : SPD_ERR_CUDA;
}
