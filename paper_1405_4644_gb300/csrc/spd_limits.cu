// spd_limits.cu -- the handle's resource limits (the bound of its device-side
// waits, a cap on its device requests) and a probe that makes one bounded
// wait run out, for callers that check their failure handling: no fault,
// trap or unbounded wait is involved.
#include "engine.cuh"

namespace {

// One thread waits for *flag to become nonzero, polling with a bound of
// limit_ns (%globaltimer); nothing sets the flag, so the wait gives up and
// raises SPD_DEV_TIMEOUT, the same path a sweep takes when a neighbour's
// block flag does not arrive in time.
__global__ void k_wait_probe(const volatile int* flag, unsigned long long limit_ns, DevStatus* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*flag != 0) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) break;
        __nanosleep(1000);
    }
    dev_raise(st, SPD_DEV_TIMEOUT);
}

}  // namespace

extern "C" spd_status spd_set_wait_limit(spd_handle* h, double seconds) {
    if (!h) return SPD_ERR_ARG;
    if (!(seconds > 0.0) || seconds > 60.0)
        return set_err(h, SPD_ERR_ARG, "spd_set_wait_limit: %g s is outside (0, 60]", seconds);
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return SPD_OK;
}

extern "C" spd_status spd_set_memory_cap(spd_handle* h, size_t bytes) {
    if (!h) return SPD_ERR_ARG;
    h->mem_cap = bytes;
    return SPD_OK;
}

extern "C" spd_status spd_wait_probe(spd_handle* h) {
    if (!h) return SPD_ERR_ARG;
    spd_status st = ws_reserve(h, 256);
    if (st != SPD_OK) return st;
    int* flag = ws_at<int>(h, 0);
    CUDA_TRY(h, cudaMemsetAsync(flag, 0, sizeof(int), h->stream));
    ++h->launches, k_wait_probe<<<1, 32, 0, h->stream>>>(flag, h->wait_ns, h->dst);
    LAUNCH_CHECK(h);
    return check_dev_status(h, nullptr, "spd_wait_probe");
}
