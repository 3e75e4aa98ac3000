// spd_learned.cu -- host side of the learned diagonal-plus-low-rank PCG
// preconditioner: network parameters and Adam state, the probe loss and its
// gradient, preconditioner build/apply, and the PCG solve with the
// Cholesky-IR fallback.
#include <random>
#include <string>
#include "engine.cuh"
#include "k_learned.cuh"

struct spd_mlp {
    spd_handle* h = nullptr;
    int F = LR_FEAT, H = 256, O = 1 + LR_RANK;
    int bf16 = 1;
    long count = 0;           // number of parameters
    float* p = nullptr;       // parameters (float32 master copy)
    float* g = nullptr;       // gradient of the last loss_grad call
    float* m1 = nullptr;      // Adam moments
    float* m2 = nullptr;
    long step = 0;
    // activations of the last forward pass (grown on demand)
    int cap_n = 0;
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Ob = nullptr, *dO = nullptr, *dH = nullptr,
          *dH2 = nullptr;
};

struct spd_lowrank {
    spd_handle* h = nullptr;
    int n = 0;
    double *dh = nullptr, *Uh = nullptr, *Lc = nullptr, *sdg = nullptr, *w = nullptr;
    int wcap = 0;
};

namespace {

// parameter offsets
struct Lay {
    long W1, b1, W2, b2, W3, b3, total;
};
Lay layout(const spd_mlp* m) {
    Lay L;
    L.W1 = 0;
    L.b1 = L.W1 + (long)m->H * m->F;
    L.W2 = L.b1 + m->H;
    L.b2 = L.W2 + (long)m->H * m->H;
    L.W3 = L.b2 + m->H;
    L.b3 = L.W3 + (long)m->O * m->H;
    L.total = L.b3 + m->O;
    return L;
}

void gemm(spd_handle* h, int M, int N, int K, const float* A, long sam, long sak, const float* B, long sbk, long sbn,
          float* C, long ldc, float alpha, float beta, int bf16) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    ++h->launches, k_gemm_strided<<<grid, 256, 0, h->stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta,
                                                               bf16);
}

spd_status ensure_acts(spd_mlp* m, int n) {
    if (n <= m->cap_n) return SPD_OK;
    spd_handle* h = m->h;
    float** bufs[] = {&m->Z1, &m->H1, &m->Z2, &m->H2, &m->dH, &m->dH2};
    for (float** b : bufs) {
        cudaFree(*b);
        *b = nullptr;
        CUDA_TRY(h, cudaMalloc(b, sizeof(float) * (size_t)n * m->H));
    }
    cudaFree(m->Ob);
    cudaFree(m->dO);
    CUDA_TRY(h, cudaMalloc(&m->Ob, sizeof(float) * (size_t)n * m->O));
    CUDA_TRY(h, cudaMalloc(&m->dO, sizeof(float) * (size_t)n * m->O));
    m->cap_n = n;
    return SPD_OK;
}

// forward pass: F (n x 16) -> O (n x 33)
void forward(spd_mlp* m, int n, const float* F) {
    spd_handle* h = m->h;
    const Lay L = layout(m);
    const int H = m->H;
    const int g = grid_for((long)n * H, 256, 8 * h->sms);
    gemm(h, n, H, m->F, F, m->F, 1, m->p + L.W1, 1, m->F, m->Z1, H, 1.f, 0.f, m->bf16);
    ++h->launches, k_bias_act<<<g, 256, 0, h->stream>>>(m->Z1, m->p + L.b1, m->H1, n, H, 1, m->bf16);
    gemm(h, n, H, H, m->H1, H, 1, m->p + L.W2, 1, H, m->Z2, H, 1.f, 0.f, m->bf16);
    ++h->launches, k_bias_act<<<g, 256, 0, h->stream>>>(m->Z2, m->p + L.b2, m->H2, n, H, 1, m->bf16);
    gemm(h, n, m->O, H, m->H2, H, 1, m->p + L.W3, 1, H, m->Ob, m->O, 1.f, 0.f, m->bf16);
    ++h->launches, k_bias_act<<<grid_for((long)n * m->O, 256, 8 * h->sms), 256, 0, h->stream>>>(
        m->Ob, m->p + L.b3, m->Ob, n, m->O, 0, 0);
}

// backward pass from dO (n x 33) into m->g
void backward(spd_mlp* m, int n, const float* F) {
    spd_handle* h = m->h;
    const Lay L = layout(m);
    const int H = m->H, O = m->O;
    cudaStream_t s = h->stream;
    // layer 3
    gemm(h, O, H, n, m->dO, 1, O, m->H2, H, 1, m->g + L.W3, H, 1.f, 0.f, 0);
    ++h->launches, k_colsum<<<(O + 127) / 128, 128, 0, s>>>(m->dO, n, O, m->g + L.b3);
    gemm(h, n, H, O, m->dO, O, 1, m->p + L.W3, H, 1, m->dH2, H, 1.f, 0.f, 0);
    ++h->launches, k_act_back<<<grid_for((long)n * H, 256, 8 * h->sms), 256, 0, s>>>(m->Z2, m->dH2, (long)n * H);
    // layer 2
    gemm(h, H, H, n, m->dH2, 1, H, m->H1, H, 1, m->g + L.W2, H, 1.f, 0.f, 0);
    ++h->launches, k_colsum<<<(H + 127) / 128, 128, 0, s>>>(m->dH2, n, H, m->g + L.b2);
    gemm(h, n, H, H, m->dH2, H, 1, m->p + L.W2, H, 1, m->dH, H, 1.f, 0.f, 0);
    ++h->launches, k_act_back<<<grid_for((long)n * H, 256, 8 * h->sms), 256, 0, s>>>(m->Z1, m->dH, (long)n * H);
    // layer 1
    gemm(h, H, m->F, n, m->dH, 1, H, F, m->F, 1, m->g + L.W1, m->F, 1.f, 0.f, 0);
    ++h->launches, k_colsum<<<(H + 127) / 128, 128, 0, s>>>(m->dH, n, H, m->g + L.b1);
}

__global__ void k_sdiag(const double* __restrict__ A, long lda, int n, double* __restrict__ s) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) s[i] = 1.0 / sqrt(A[(long)i * lda + i]);
}

// Q = A P in float64 (A column-major symmetric, P n x p with ld n)
__global__ void __launch_bounds__(256) k_gemv64(const double* __restrict__ A, long lda, int n, const double* __restrict__ P,
                                                int p, double* __restrict__ Q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc[8];
    for (int c0 = 0; c0 < p; c0 += 8) {
        const int pc = min(8, p - c0);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.0;
        for (int j = 0; j < n; ++j) {
            const double a = A[(long)j * lda + i];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < pc) acc[c] = fma(a, P[(long)(c0 + c) * n + j], acc[c]);
        }
        for (int c = 0; c < pc; ++c) Q[(long)(c0 + c) * n + i] = acc[c];
    }
}

// PV[c][k] = sum_i Uh_ik V_ic  (one CTA per column, fixed order)
__global__ void __launch_bounds__(256) k_proj(const double* __restrict__ Uh, const double* __restrict__ V, int n,
                                              double* __restrict__ PV) {
    __shared__ double red[8][LR_RANK];
    const int c = blockIdx.x;
    double acc[LR_RANK];
#pragma unroll
    for (int k = 0; k < LR_RANK; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double v = V[(long)c * n + i];
#pragma unroll
        for (int k = 0; k < LR_RANK; ++k) acc[k] = fma(Uh[(long)i * LR_RANK + k], v, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < LR_RANK; ++k) {
        double v = warp_sum(acc[k]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < LR_RANK) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        PV[c * LR_RANK + threadIdx.x] = s;
    }
}

// loss pieces per column: E = Q - Z; returns per-column ||E||^2 and ||Z||^2
// (one CTA per column, fixed order); G = E (scaled later by k_scale_cols)
__global__ void __launch_bounds__(256) k_probe_err(const double* __restrict__ Q, const double* __restrict__ Z, int n,
                                                   double* __restrict__ E, double* __restrict__ sums) {
    __shared__ double red[2][8];
    const int c = blockIdx.x;
    double se = 0.0, sz = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double z = Z[(long)c * n + i];
        const double e = Q[(long)c * n + i] - z;
        E[(long)c * n + i] = e;
        se += e * e;
        sz += z * z;
    }
    se = warp_sum(se);
    sz = warp_sum(sz);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = se;
        red[1][threadIdx.x >> 5] = sz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        sums[2 * c] = a;
        sums[2 * c + 1] = b;
    }
}

// G_c = coef_c * G_c ; optional supervised term on column 0:
// G_0 += 2 w (Y_0 - T_0) / ||T_0||^2 (tnorm2 given)
__global__ void k_scale_cols(double* __restrict__ G, const double* __restrict__ coef, int n, int p,
                             const double* __restrict__ Y, const double* __restrict__ T, double wsup, double tnorm2) {
    long total = (long)n * p;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        double g = coef[c] * G[e];
        if (T && c == 0) g += 2.0 * wsup * (Y[e] - T[e]) / tnorm2;
        G[e] = g;
    }
}

__global__ void k_unscale(const double* __restrict__ V, const double* __restrict__ s, int n, int p, double* __restrict__ Vh) {
    long total = (long)n * p;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x)
        Vh[e] = V[e] / s[e % n];
}

// row chunks of the Woodbury projection (256 rows each)
int wb_chunks(int n) { return std::max(1, ceil_div(n, 256)); }

spd_status lowrank_alloc(spd_handle* h, spd_lowrank* P, int n) {
    P->h = h;
    P->n = n;
    CUDA_TRY(h, cudaMalloc(&P->dh, sizeof(double) * n));
    CUDA_TRY(h, cudaMalloc(&P->Uh, sizeof(double) * (size_t)n * LR_RANK));
    CUDA_TRY(h, cudaMalloc(&P->Lc, sizeof(double) * 2 * LR_RANK * LR_RANK));  // Lc, then the core's inverse
    CUDA_TRY(h, cudaMalloc(&P->sdg, sizeof(double) * n));
    return SPD_OK;
}

void lowrank_free(spd_lowrank* P) {
    if (!P) return;
    cudaFree(P->dh);
    cudaFree(P->Uh);
    cudaFree(P->Lc);
    cudaFree(P->sdg);
    cudaFree(P->w);
}

// dh, Uh, Lc from the network output currently in m->Ob; returns SPD_ERR_NOT_SPD
// if the 32x32 core is not positive definite.
spd_status build_core(spd_mlp* m, spd_lowrank* P, int n, int* dbad) {
    spd_handle* h = m->h;
    ++h->launches, k_out_to_dU<<<grid_for(n, 256, 4 * h->sms), 256, 0, h->stream>>>(m->Ob, n, P->dh, P->Uh);
    CUDA_TRY(h, cudaMemsetAsync(dbad, 0, sizeof(int), h->stream));
    // the Gram term over 128-row chunks on many SMs, then one CTA for the
    // 32 x 32 core (one float64 division per row, not per row and entry)
    const int G = ceil_div(n, CORE_ROWS);
    double* part = nullptr;
    CUDA_TRY(h, cudaMallocAsync(&part, sizeof(double) * (size_t)G * LR_RANK * LR_RANK, h->stream));
    ++h->launches, k_core_gram<<<G, 1024, 0, h->stream>>>(P->dh, P->Uh, n, part);
    ++h->launches, k_core_chol<<<1, 1024, 0, h->stream>>>(part, G, P->Lc, dbad);
    cudaFreeAsync(part, h->stream);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

}  // namespace

// Woodbury apply used by spd_cg (declared in engine.cuh).
spd_status lowrank_apply_internal(spd_handle* h, const spd_lowrank* P, int n, int m, const double* R, long ldr,
                                  double* Z, long ldz, double* wbuf) {
    ProfScope ps(h, SPD_PHASE_VECTOR, 4.0 * LR_RANK * n * (double)m, 8.0 * (LR_RANK + 4) * n * (double)m);
    const int G = wb_chunks(n);
    ++h->launches, k_wb_proj<<<dim3(G, m), 256, 0, h->stream>>>(R, ldr, P->sdg, P->dh, P->Uh, n, m, wbuf);
    dim3 g(grid_for(n, 256, 2 * h->sms), m);
    ++h->launches, k_wb_apply<<<g, 256, 0, h->stream>>>(R, ldr, P->sdg, P->dh, P->Uh, P->Lc, wbuf, G, n, m, Z, ldz);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

int lowrank_order(const spd_lowrank* P) { return P ? P->n : -1; }

LowrankView lowrank_view(const spd_lowrank* P, int n, int m) {
    static_assert(LR_RANK == LOWRANK_RANK, "one rank for the kernels and the view");
    const int G = wb_chunks(n);
    return LowrankView{P->sdg, P->dh, P->Uh, P->Lc, P->w, P->w + (long)G * LR_RANK * m, G};
}

// The projection buffer of the Woodbury apply for m columns (grown on
// demand; spd_cg sizes it before its inner steps, which may be captured).
spd_status lowrank_reserve(spd_handle* h, const spd_lowrank* Pc, int n, int m) {
    spd_lowrank* P = const_cast<spd_lowrank*>(Pc);
    const int need = wb_chunks(n) * (LR_RANK + 2) * m;  // partial projections, then dot partials
    if (P->wcap < need) {
        cudaFree(P->w);
        P->w = nullptr;
        CUDA_TRY(h, cudaMalloc(&P->w, sizeof(double) * need));
        P->wcap = need;
    }
    return SPD_OK;
}

// Woodbury apply for the CG loop.
spd_status lowrank_apply_cg(spd_handle* h, const spd_lowrank* Pc, int n, int m, const double* R, long ldr, double* Z,
                            long ldz) {
    const spd_status st = lowrank_reserve(h, Pc, n, m);
    if (st != SPD_OK) return st;
    return lowrank_apply_internal(h, Pc, n, m, R, ldr, Z, ldz, Pc->w);
}

extern "C" spd_status spd_mlp_create(spd_handle* h, int hidden, unsigned long long seed, int bf16, spd_mlp** out) {
    if (!h) return SPD_ERR_ARG;
    if (!out || hidden < 8 || hidden > 4096) return set_err(h, SPD_ERR_ARG, "spd_mlp_create: bad arguments");
    spd_mlp* m = new spd_mlp();
    m->h = h;
    m->H = hidden;
    m->bf16 = bf16 ? 1 : 0;
    const Lay L = layout(m);
    m->count = L.total;
    std::vector<float> p(L.total, 0.f);
    std::mt19937_64 rng(seed);
    auto unif = [&](float lim) { return (float)((rng() >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * lim; };
    for (long i = 0; i < (long)m->H * m->F; ++i) p[L.W1 + i] = unif(1.f / sqrtf((float)m->F));
    for (long i = 0; i < (long)m->H * m->H; ++i) p[L.W2 + i] = unif(1.f / sqrtf((float)m->H));
    for (long i = 0; i < (long)m->O * m->H; ++i) p[L.W3 + i] = unif(0.1f / sqrtf((float)m->H));
    p[L.b3] = 0.5413f;  // softplus^{-1}(1): the diagonal starts at ~1 (scaled matrix)
    cudaError_t e = cudaMalloc(&m->p, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->m1, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->m2, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMemcpy(m->p, p.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMemset(m->g, 0, sizeof(float) * L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(m->p);
        cudaFree(m->g);
        cudaFree(m->m1);
        cudaFree(m->m2);
        delete m;
        return set_err(h, SPD_ERR_OOM, "spd_mlp_create: %s", cudaGetErrorString(e));
    }
    *out = m;
    return SPD_OK;
}

extern "C" spd_status spd_mlp_destroy(spd_mlp* m) {
    if (!m) return SPD_OK;
    cudaStreamSynchronize(m->h->stream);
    float* bufs[] = {m->p, m->g, m->m1, m->m2, m->Z1, m->H1, m->Z2, m->H2, m->Ob, m->dO, m->dH, m->dH2};
    for (float* b : bufs) cudaFree(b);
    delete m;
    return SPD_OK;
}

extern "C" spd_status spd_mlp_params(spd_mlp* m, float* out, const float* in, float* grad_out, long* count) {
    if (!m) return SPD_ERR_ARG;
    spd_handle* h = m->h;
    if (count) *count = m->count;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (in) CUDA_TRY(h, cudaMemcpy(m->p, in, sizeof(float) * m->count, cudaMemcpyDefault));
    if (out) CUDA_TRY(h, cudaMemcpy(out, m->p, sizeof(float) * m->count, cudaMemcpyDefault));
    if (grad_out) CUDA_TRY(h, cudaMemcpy(grad_out, m->g, sizeof(float) * m->count, cudaMemcpyDefault));
    return SPD_OK;
}

// ---------------------------------------------------------------------------
// checkpoint: <path>.json (manifest) + <path>.bin (float32 parameters, little
// endian, in layout order W1 b1 W2 b2 W3 b3) + <path>.adam.bin (the two Adam
// moments, 2 count float32), so that training can resume where it stopped
// ---------------------------------------------------------------------------
namespace {

bool write_file(const std::string& path, const void* data, size_t bytes) {
    FILE* f = fopen(path.c_str(), "wb");
    if (!f) return false;
    const bool ok = fwrite(data, 1, bytes, f) == bytes;
    return fclose(f) == 0 && ok;
}

bool read_file(const std::string& path, void* data, size_t bytes) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return false;
    const bool ok = fread(data, 1, bytes, f) == bytes && fgetc(f) == EOF;
    fclose(f);
    return ok;
}

// value of "key": <integer> in the manifest text (false if absent)
bool json_long(const std::string& text, const char* key, long* out) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t pos = text.find(k);
    if (pos == std::string::npos) return false;
    return sscanf(text.c_str() + pos + k.size(), " %ld", out) == 1;
}

}  // namespace

extern "C" spd_status spd_learned_save(spd_mlp* m, const char* path) {
    if (!m || !path || !*path) return SPD_ERR_ARG;
    spd_handle* h = m->h;
    std::vector<float> p(m->count), mom(2 * m->count);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaMemcpy(p.data(), m->p, sizeof(float) * m->count, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(mom.data(), m->m1, sizeof(float) * m->count, cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(mom.data() + m->count, m->m2, sizeof(float) * m->count, cudaMemcpyDeviceToHost));
    char js[512];
    snprintf(js, sizeof(js),
             "{\"format\": \"spd-mlp\", \"version\": 1, \"features\": %d, \"hidden\": %d, \"outputs\": %d, "
             "\"bf16\": %d, \"count\": %ld, \"adam_step\": %ld, \"dtype\": \"float32\", "
             "\"layout\": \"W1 b1 W2 b2 W3 b3\"}\n",
             m->F, m->H, m->O, m->bf16, m->count, m->step);
    const std::string base(path);
    if (!write_file(base + ".bin", p.data(), sizeof(float) * p.size()) ||
        !write_file(base + ".adam.bin", mom.data(), sizeof(float) * mom.size()) ||
        !write_file(base + ".json", js, strlen(js)))
        return set_err(h, SPD_ERR_ARG, "spd_learned_save: cannot write %s.{json,bin,adam.bin}", path);
    return SPD_OK;
}

extern "C" spd_status spd_learned_load(spd_handle* h, const char* path, spd_mlp** out) {
    if (!h) return SPD_ERR_ARG;
    if (!path || !*path || !out) return set_err(h, SPD_ERR_ARG, "spd_learned_load: bad arguments");
    *out = nullptr;
    const std::string base(path);
    std::string text;
    {
        FILE* f = fopen((base + ".json").c_str(), "rb");
        if (!f) return set_err(h, SPD_ERR_ARG, "spd_learned_load: cannot open %s.json", path);
        char buf[1024];
        const size_t k = fread(buf, 1, sizeof(buf) - 1, f);
        fclose(f);
        text.assign(buf, k);
    }
    long F = 0, H = 0, O = 0, bf16 = 0, count = 0, step = 0;
    if (text.find("\"spd-mlp\"") == std::string::npos || !json_long(text, "features", &F) ||
        !json_long(text, "hidden", &H) || !json_long(text, "outputs", &O) || !json_long(text, "bf16", &bf16) ||
        !json_long(text, "count", &count) || !json_long(text, "adam_step", &step))
        return set_err(h, SPD_ERR_ARG, "spd_learned_load: %s.json is not an spd-mlp manifest", path);
    if (F != LR_FEAT || O != 1 + LR_RANK)
        return set_err(h, SPD_ERR_ARG, "spd_learned_load: %ld features / %ld outputs, this library has %d / %d", F,
                       O, LR_FEAT, 1 + LR_RANK);
    spd_mlp* m = nullptr;
    spd_status st = spd_mlp_create(h, (int)H, 0, (int)bf16, &m);
    if (st != SPD_OK) return st;
    if (m->count != count) {
        spd_mlp_destroy(m);
        return set_err(h, SPD_ERR_ARG, "spd_learned_load: manifest count %ld, layout of hidden %ld has %ld", count, H,
                       m->count);
    }
    std::vector<float> p(count), mom(2 * count);
    if (!read_file(base + ".bin", p.data(), sizeof(float) * count)) {
        spd_mlp_destroy(m);
        return set_err(h, SPD_ERR_ARG, "spd_learned_load: %s.bin does not hold %ld float32 values", path, count);
    }
    const bool adam = read_file(base + ".adam.bin", mom.data(), sizeof(float) * mom.size());
    cudaError_t e = cudaMemcpy(m->p, p.data(), sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && adam) e = cudaMemcpy(m->m1, mom.data(), sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && adam)
        e = cudaMemcpy(m->m2, mom.data() + count, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        spd_mlp_destroy(m);
        return set_err(h, SPD_ERR_CUDA, "spd_learned_load: %s", cudaGetErrorString(e));
    }
    m->step = adam ? step : 0;
    *out = m;
    return SPD_OK;
}

extern "C" spd_status spd_learned_features(spd_handle* h, int n, const double* A, int lda, const double* coords,
                                           double ell, double nugget, float* F) {
    if (!h) return SPD_ERR_ARG;
    if (n < 1 || !A || lda < n || !coords || !F || !(ell > 0) || !(nugget > 0))
        return set_err(h, SPD_ERR_ARG, "spd_learned_features: bad arguments");
    double* sd = nullptr;
    CUDA_TRY(h, cudaMallocAsync(&sd, sizeof(double) * n, h->stream));
    {
        ProfScope ps(h, SPD_PHASE_CONVERT, 3.0 * n * (double)n, 8.0 * n * (double)n);
        ++h->launches, k_sdiag<<<ceil_div(n, 256), 256, 0, h->stream>>>(A, lda, n, sd);
        ++h->launches, k_features<<<ceil_div(n, 8), 256, 0, h->stream>>>(A, lda, n, coords, ell, nugget, F, sd);
    }
    LAUNCH_CHECK(h);
    CUDA_TRY(h, cudaFreeAsync(sd, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SPD_OK;
}

extern "C" spd_status spd_mlp_loss_grad(spd_mlp* m, int n, const double* A, int lda, const float* F, int p,
                                        const double* Zp, const double* T, double wsup, double* loss) {
    if (!m) return SPD_ERR_ARG;
    spd_handle* h = m->h;
    if (n < 1 || !A || lda < n || !F || p < 1 || p > 64 || !Zp)
        return set_err(h, SPD_ERR_ARG, "spd_mlp_loss_grad: bad arguments");
    spd_status st = ensure_acts(m, n);
    if (st != SPD_OK) return st;
    cudaStream_t s = h->stream;
    const size_t np = (size_t)n * p;
    WsPlan pl;
    size_t o_sd = pl.add<double>(n), o_Y = pl.add<double>(np), o_Q = pl.add<double>(np), o_E = pl.add<double>(np),
           o_G = pl.add<double>(np), o_Wv = pl.add<double>(np), o_Yh = pl.add<double>(np), o_Wh = pl.add<double>(np),
           o_PY = pl.add<double>(LR_RANK * p), o_PW = pl.add<double>(LR_RANK * p),
           o_w = pl.add<double>((size_t)wb_chunks(n) * LR_RANK * p),
           o_sums = pl.add<double>(2 * p + 2), o_coef = pl.add<double>(p), o_dh = pl.add<double>(n),
           o_Uh = pl.add<double>((size_t)n * LR_RANK), o_Lc = pl.add<double>(2 * LR_RANK * LR_RANK),
           o_bad = pl.add<int>(1);
    if ((st = ws_reserve(h, pl.bytes)) != SPD_OK) return st;
    double *sd = ws_at<double>(h, o_sd), *Y = ws_at<double>(h, o_Y), *Q = ws_at<double>(h, o_Q),
           *E = ws_at<double>(h, o_E), *G = ws_at<double>(h, o_G), *Wv = ws_at<double>(h, o_Wv),
           *Yh = ws_at<double>(h, o_Yh), *Wh = ws_at<double>(h, o_Wh), *PY = ws_at<double>(h, o_PY),
           *PW = ws_at<double>(h, o_PW), *wb = ws_at<double>(h, o_w), *sums = ws_at<double>(h, o_sums),
           *coef = ws_at<double>(h, o_coef);
    spd_lowrank P;
    P.h = h;
    P.n = n;
    P.dh = ws_at<double>(h, o_dh);
    P.Uh = ws_at<double>(h, o_Uh);
    P.Lc = ws_at<double>(h, o_Lc);
    P.sdg = sd;
    int* dbad = ws_at<int>(h, o_bad);
    const int gv = grid_for((long)np, 256, 8 * h->sms);

    ++h->launches, k_sdiag<<<ceil_div(n, 256), 256, 0, s>>>(A, lda, n, sd);
    forward(m, n, F);
    if ((st = build_core(m, &P, n, dbad)) != SPD_OK) return st;
    if ((st = lowrank_apply_internal(h, &P, n, p, Zp, n, Y, n, wb)) != SPD_OK) return st;  // Y = M Z
    ++h->launches, k_gemv64<<<ceil_div(n, 256), 256, 0, s>>>(A, lda, n, Y, p, Q);          // Q = A Y
    ++h->launches, k_probe_err<<<p, 256, 0, s>>>(Q, Zp, n, E, sums);                        // E = A M Z - Z
    ++h->launches, k_gemv64<<<ceil_div(n, 256), 256, 0, s>>>(A, lda, n, E, p, G);          // G = A E
    // host: loss and per-column coefficients 2 / (p ||z_c||^2); supervised target norm
    std::vector<double> hs(2 * p + 2);
    double tn2 = 1.0;
    CUDA_TRY(h, cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 2 * p, cudaMemcpyDeviceToHost, s));
    if (T) {
        ++h->launches, k_probe_err<<<1, 256, 0, s>>>(T, T, n, Q, sums + 2 * p);  // sums[2p+1] = ||T_0||^2
        CUDA_TRY(h, cudaMemcpyAsync(hs.data() + 2 * p, sums + 2 * p, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    double L = 0.0;
    std::vector<double> cf(p);
    for (int c = 0; c < p; ++c) {
        L += hs[2 * c] / hs[2 * c + 1] / p;
        cf[c] = 2.0 / (p * hs[2 * c + 1]);
    }
    if (T) tn2 = hs[2 * p + 1];
    CUDA_TRY(h, cudaMemcpyAsync(coef, cf.data(), sizeof(double) * p, cudaMemcpyHostToDevice, s));
    ++h->launches, k_scale_cols<<<gv, 256, 0, s>>>(G, coef, n, p, Y, T, wsup, tn2);         // dL/dY
    if (T) {  // supervised term value: ||Y_0 - T_0||^2 / ||T_0||^2
        ++h->launches, k_probe_err<<<1, 256, 0, s>>>(Y, T, n, E, sums + 2 * p);
        CUDA_TRY(h, cudaMemcpyAsync(hs.data() + 2 * p, sums + 2 * p, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, cudaStreamSynchronize(s));
        // ||Y_0 - T_0|| computed as ||T_0 - Y_0||: k_probe_err(Q=Y, Z=T) gives sum (Y-T)^2
        L += wsup * hs[2 * p] / tn2;
    }
    if ((st = lowrank_apply_internal(h, &P, n, p, G, n, Wv, n, wb)) != SPD_OK) return st;  // W = M G
    ++h->launches, k_unscale<<<gv, 256, 0, s>>>(Y, sd, n, p, Yh);
    ++h->launches, k_unscale<<<gv, 256, 0, s>>>(Wv, sd, n, p, Wh);
    ++h->launches, k_proj<<<p, 256, 0, s>>>(P.Uh, Yh, n, PY);
    ++h->launches, k_proj<<<p, 256, 0, s>>>(P.Uh, Wh, n, PW);
    ++h->launches, k_loss_grad_out<<<grid_for(n, 256, 4 * h->sms), 256, 0, s>>>(Yh, Wh, n, p, P.Uh, PY, PW, m->Ob, m->dO);
    backward(m, n, F);
    LAUNCH_CHECK(h);
    int hbad = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    if (loss) *loss = L;
    if (hbad) return set_err(h, SPD_ERR_NOT_SPD, "spd_mlp_loss_grad: low-rank core not positive definite");
    return SPD_OK;
}

extern "C" spd_status spd_mlp_adam(spd_mlp* m, double lr) {
    if (!m) return SPD_ERR_ARG;
    spd_handle* h = m->h;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    ++h->launches, k_adam<<<grid_for(m->count, 256, 4 * h->sms), 256, 0, h->stream>>>(m->p, m->g, m->m1, m->m2, m->count,
                                                                                   (float)lr, b1, b2, 1e-8f, c1, c2);
    LAUNCH_CHECK(h);
    return SPD_OK;
}

extern "C" spd_status spd_lowrank_build(spd_mlp* m, int n, const double* A, int lda, const float* F, spd_lowrank** out) {
    if (!m || !out) return SPD_ERR_ARG;
    spd_handle* h = m->h;
    if (n < 1 || !A || lda < n || !F) return set_err(h, SPD_ERR_ARG, "spd_lowrank_build: bad arguments");
    spd_status st = ensure_acts(m, n);
    if (st != SPD_OK) return st;
    spd_lowrank* P = new spd_lowrank();
    if ((st = lowrank_alloc(h, P, n)) != SPD_OK) {
        lowrank_free(P);
        delete P;
        return st;
    }
    int* dbad = nullptr;
    CUDA_TRY(h, cudaMallocAsync(&dbad, sizeof(int), h->stream));
    ++h->launches, k_sdiag<<<ceil_div(n, 256), 256, 0, h->stream>>>(A, lda, n, P->sdg);
    forward(m, n, F);
    st = build_core(m, P, n, dbad);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(dbad, h->stream);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (st == SPD_OK && hbad) st = set_err(h, SPD_ERR_NOT_SPD, "spd_lowrank_build: low-rank core not positive definite");
    if (st != SPD_OK) {
        lowrank_free(P);
        delete P;
        return st;
    }
    *out = P;
    return SPD_OK;
}

extern "C" spd_status spd_lowrank_apply(spd_lowrank* P, int m, const double* R, int ldr, double* Z, int ldz) {
    if (!P) return SPD_ERR_ARG;
    spd_handle* h = P->h;
    if (m < 0 || (m > 0 && (!R || !Z || ldr < P->n || ldz < P->n)))
        return set_err(h, SPD_ERR_ARG, "spd_lowrank_apply: bad arguments");
    if (m == 0) return SPD_OK;
    if (P->wcap < m) {
        cudaFree(P->w);
        P->w = nullptr;
        CUDA_TRY(h, cudaMalloc(&P->w, sizeof(double) * LR_RANK * m));
        P->wcap = m;
    }
    spd_status st = lowrank_apply_internal(h, P, P->n, m, R, ldr, Z, ldz, P->w);
    if (st != SPD_OK) return st;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SPD_OK;
}

extern "C" spd_status spd_lowrank_destroy(spd_lowrank* P) {
    if (!P) return SPD_OK;
    cudaStreamSynchronize(P->h->stream);
    lowrank_free(P);
    delete P;
    return SPD_OK;
}

// PCG with the learned preconditioner; Cholesky-IR in float32 when PCG
// does not reach the tolerance within opts->maxit_inner steps.
extern "C" spd_status spd_solve_learned(spd_handle* h, const spd_lowrank* P, int n, int m, const double* A, int lda,
                                        const double* B, int ldb, double* X, int ldx, const spd_opts* opts_in,
                                        spd_report* rep) {
    if (!h) return SPD_ERR_ARG;
    if (!P || P->n != n) return set_err(h, SPD_ERR_ARG, "spd_solve_learned: preconditioner order differs from n");
    spd_opts o;
    spd_opts_default(&o);
    if (opts_in) o = *opts_in;
    spd_opts po = o;
    po.eta = std::min(o.eta, 1e-12);  // float64 products: one outer step normally suffices
    po.maxit = std::min(o.maxit, 3);
    spd_report r1{};
    spd_status st = spd_cg(h, n, m, A, lda, SPD_PREC_FP64, SPD_PC_LOWRANK, P, B, ldb, X, ldx, &po, &r1);
    if (st == SPD_OK) {
        if (rep) *rep = r1;
        return SPD_OK;
    }
    if (st != SPD_ERR_NO_CONVERGENCE) return st;
    // fallback: float32 Cholesky + refinement, which also judges the result
    spd_factor_t* F = nullptr;
    spd_report fr{};
    st = spd_factor(h, n, A, lda, SPD_PREC_FP32, SPD_SCALE_DIAG, &F, &fr);
    if (st != SPD_OK) return st;
    spd_report r2{};
    st = spd_solve_ir(h, F, n, m, A, lda, B, ldb, X, ldx, &o, &r2);
    spd_factor_destroy(F);
    if (rep) {
        *rep = r2;
        rep->iters_low += r1.iters_low;
        rep->iters_high += r1.iters_high;
        rep->fell_back = 1;
        rep->time_ms += r1.time_ms + fr.time_ms;
    }
    return st;
}
