// k_batched.cuh -- many independent SPD systems of uneven order (n <= 512)
// solved in one persistent launch: Algorithm 1 (low-precision Cholesky +
// float64 refinement) or Jacobi-preconditioned CG, one system per CTA at a
// time.  CTAs take systems from a shared counter over a list sorted by
// decreasing n, so the long systems start first.  Every system is processed
// by exactly one CTA with a fixed sequence of operations, so its result
// does not depend on the schedule.
//
// Per-CTA scratch in global memory (L2-resident): the scaled working
// matrix W (column-major lower, ld 512, float32).  Shared memory holds the
// 32x32 diagonal-block inverses, the current panel, and the vectors.
#pragma once
#include "common.cuh"

#define BMAX 512           // largest system order
#define BLD 512            // leading dimension of the per-CTA working matrix
#define BPANEL 32

struct BatchSys {
    const double* A;  // n x n, column-major, lda
    const double* B;  // n
    double* X;        // n
    int n, lda;
};

struct BatchRep {
    int status;   // SPD_OK, SPD_ERR_NOT_SPD, SPD_ERR_NO_CONVERGENCE
    int info;     // failing column (1-based) on breakdown
    int iters;    // refinement sweeps / CG steps
    int pad;
    double berr;  // final normwise backward error
};

struct BatchArgs {
    const BatchSys* sys;
    const int* order;    // system indices, decreasing n
    int count;
    int* next;           // work counter (zeroed before the launch)
    float* scratch;      // per CTA: BLD * BLD floats
    BatchRep* rep;
    int prec;            // SPD_PREC_FP32 / BF16 / FP16: rounding of the update operands
    double tol;
    int maxit;
    int polish;
};

// The panel's rows transposed: PnT[l * BLDP + i] = L[i][k0 + l] (rounded to the
// update type), rows contiguous so that four rows are one 16-byte load.
#define BLDP 516
constexpr size_t batch_smem_bytes() {
    return (size_t)(BMAX / 32) * 32 * 33 * sizeof(float)  // Inv
           + (size_t)BMAX * 33 * sizeof(float)            // panel (PnT: 32 x BLDP floats fit in it)
           + (size_t)4 * BMAX * sizeof(double)            // x, r, d, rowabs
           + (size_t)2 * BMAX * sizeof(float);            // y, z
}

__device__ __forceinline__ float round_op(float v, int prec) {
    if (prec == 3) return __bfloat162float(__float2bfloat16_rn(v));  // SPD_PREC_BF16
    if (prec == 4) return __half2float(__float2half_rn(v));          // SPD_PREC_FP16
    return v;
}

template <int NT>
__device__ double block_max(double v, double* red) {
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < NT / 32; ++w) r = fmax(r, red[w]);
    __syncthreads();
    return r;
}
template <int NT>
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < NT / 32; ++w) r += red[w];  // fixed order
    __syncthreads();
    return r;
}

// y <- (L L^T)^{-1} y in place (float32, shared memory) with the factor in W
// and the diagonal-block inverses in Inv.
template <int NT>
__device__ void batch_lsolve(const float* W, const float* Inv, float* y, int n) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = (n + 31) / 32;
    for (int kb = 0; kb < nb; ++kb) {  // forward
        const int k0 = kb * 32;
        if (warp == 0) {
            const float* I = Inv + kb * 32 * 33;
            float s = 0.f;
            for (int l = 0; l <= lane; ++l) s += I[lane * 33 + l] * ((k0 + l < n) ? y[k0 + l] : 0.f);
            __syncwarp();
            if (k0 + lane < n) y[k0 + lane] = s;
        }
        __syncthreads();
        for (int i = k0 + 32 + tid; i < n; i += NT) {
            float s = 0.f;
#pragma unroll 8
            for (int c = 0; c < 32; ++c) s += W[i + (long)(k0 + c) * BLD] * y[k0 + c];
            y[i] -= s;
        }
        __syncthreads();
    }
    for (int kb = nb - 1; kb >= 0; --kb) {  // backward
        const int k0 = kb * 32;
        if (warp == 0) {
            const float* I = Inv + kb * 32 * 33;
            float s = 0.f;
            for (int l = lane; l < 32; ++l) s += I[l * 33 + lane] * ((k0 + l < n) ? y[k0 + l] : 0.f);
            __syncwarp();
            if (k0 + lane < n) y[k0 + lane] = s;
        }
        __syncthreads();
        // y_i -= sum_c L[k0+c][i] z[k0+c]: one warp per row i, lane c reading
        // L[k0+c][i] (32 contiguous floats of W's column i), a fixed shuffle sum
        for (int i = warp; i < k0; i += NT / 32) {
            const float v = (k0 + lane < n) ? W[(long)i * BLD + k0 + lane] * y[k0 + lane] : 0.f;
            const float s = warp_sum(v);
            if (lane == 0) y[i] -= s;
        }
        __syncthreads();
    }
}

// r = b - A x (float64) for one system; returns berr = ||r||_inf / (anorm ||x||_inf).
template <int NT>
__device__ double batch_residual(const BatchSys& S, const double* x, double* r, const double* anorm_p,
                                 double* rowabs, bool want_anorm, double* red, double* anorm_out) {
    const int n = S.n;
    double rmax = 0.0, amax = 0.0, xmax = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        // four interleaved accumulators (column j into j % 4), eight loads in
        // flight, added in a fixed order
        double q[4] = {0.0, 0.0, 0.0, 0.0}, a = 0.0;
        const double* Ai = S.A + i;
        int j = 0;
        for (; j + 8 <= n; j += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = Ai[(long)(j + u) * S.lda];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                q[u & 3] = fma(v[u], x[j + u], q[u & 3]);
                if (want_anorm) a += fabs(v[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {  // the last n % 8 columns (j is a multiple of 8 here)
            if (j + u < n) {
                const double v = Ai[(long)(j + u) * S.lda];
                q[u & 3] = fma(v, x[j + u], q[u & 3]);
                if (want_anorm) a += fabs(v);
            }
        }
        const double s = S.B[i] - ((q[0] + q[1]) + (q[2] + q[3]));
        r[i] = s;
        rmax = fmax(rmax, fabs(s));
        xmax = fmax(xmax, fabs(x[i]));
        if (want_anorm) amax = fmax(amax, a);
    }
    rmax = block_max<NT>(rmax, red);
    xmax = block_max<NT>(xmax, red);
    double an;
    if (want_anorm) {
        an = block_max<NT>(amax, red);
        *anorm_out = an;
    } else {
        an = *anorm_p;
    }
    return (an > 0.0 && xmax > 0.0) ? rmax / (an * xmax) : rmax;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_batch_chol_ir(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Inv = reinterpret_cast<float*>(smem_raw);          // [16][32][33]
    float* Pn = Inv + (BMAX / 32) * 32 * 33;                   // [512][33]
    double* xs = reinterpret_cast<double*>(Pn + BMAX * 33);    // [512]
    double* rs = xs + BMAX;
    double* ds = rs + BMAX;
    double* ra = ds + BMAX;
    float* ys = reinterpret_cast<float*>(ra + BMAX);           // [512]
    __shared__ int s_idx, s_bad;
    __shared__ double red[NT / 32];
    __shared__ double s_anorm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* W = a.scratch + (long)blockIdx.x * BLD * BLD;

    for (;;) {
        if (tid == 0) s_idx = atomicAdd(a.next, 1);
        __syncthreads();
        if (s_idx >= a.count) break;
        const int sid = a.order[s_idx];
        const BatchSys S = a.sys[sid];
        const int n = S.n;
        // scaling and conversion (A0): W[i][j] = d_i A_ij d_j, j <= i
        for (int i = tid; i < n; i += NT) {
            const double v = S.A[i + (long)i * S.lda];
            ds[i] = (v > 0.0) ? 1.0 / sqrt(v) : 1.0;
        }
        if (tid == 0) s_bad = 0;
        __syncthreads();
        // (every entry of the n x n block, four per thread at a time; only
        // the lower triangle is kept)
        for (int e0 = tid; e0 < n * n; e0 += 4 * NT) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * NT, j = e / n, i = e - j * n;
                v[u] = (e < n * n && i >= j) ? S.A[i + (long)j * S.lda] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * NT, j = e / n, i = e - j * n;
                if (e < n * n && i >= j) W[i + (long)j * BLD] = (float)(ds[i] * v[u] * ds[j]);
            }
        }
        __syncthreads();
        // factor (A1-A3) by 32-column panels
        const int nb = (n + 31) / 32;
        for (int kb = 0; kb < nb && !s_bad; ++kb) {
            const int k0 = kb * 32;
            if (warp == 0) {
                float av[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int r = k0 + lane, cc = k0 + c;
                    av[c] = (r < n && cc < n) ? ((c <= lane) ? W[r + (long)cc * BLD] : 0.f) : (lane == c ? 1.f : 0.f);
                }
                int badj = -1;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float piv = __shfl_sync(0xffffffffu, av[j], j);
                    if (!(piv > 0.f)) {
                        if (badj < 0) badj = j;
                        piv = 1.f;
                    }
                    const float dj = sqrtf(piv), inv = 1.f / dj;
                    av[j] = (lane == j) ? dj : (lane > j ? av[j] * inv : av[j]);
#pragma unroll
                    for (int l = 0; l < 32; ++l) {
                        if (l > j) {
                            const float t = __shfl_sync(0xffffffffu, av[j], l);
                            av[l] = (lane >= l) ? fmaf(-av[j], t, av[l]) : av[l];
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (k0 + lane < n && k0 + c < n && c <= lane) W[k0 + lane + (long)(k0 + c) * BLD] = av[c];
                if (badj >= 0 && k0 + badj < n && lane == 0) {
                    s_bad = 1;
                    a.rep[sid].info = k0 + badj + 1;
                }
                __syncwarp();
                // inverse of the 32x32 diagonal block: lane = column
                float* I = Inv + kb * 32 * 33;
                float xv[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    float s = (i == lane) ? 1.f : 0.f;
                    const float lii = __shfl_sync(0xffffffffu, av[i], i);
#pragma unroll
                    for (int l = 0; l < 32; ++l)
                        if (l < i) s = fmaf(-__shfl_sync(0xffffffffu, av[l], i), xv[l], s);
                    xv[i] = s / lii;
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) I[i * 33 + lane] = xv[i];
            }
            __syncthreads();
            if (s_bad) break;
            const int R = n - k0 - 32;
            if (R <= 0) break;
            const float* I = Inv + kb * 32 * 33;
            // panel: rows below, X = B I^T
            for (int i = tid; i < R; i += NT) {
                float b[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) b[c] = W[(k0 + 32 + i) + (long)(k0 + c) * BLD];
#pragma unroll 4
                for (int c = 0; c < 32; ++c) {
                    float s = 0.f;
#pragma unroll
                    for (int l = 0; l < 32; ++l)
                        if (l <= c) s = fmaf(b[l], I[c * 33 + l], s);
                    W[(k0 + 32 + i) + (long)(k0 + c) * BLD] = s;
                    Pn[c * BLDP + i] = round_op(s, a.prec);
                }
            }
            for (int e = tid; e < 32 * 4; e += NT) Pn[(e >> 2) * BLDP + R + (e & 3)] = 0.f;  // rows R.. of the last group
            __syncthreads();
            // trailing update of the lower part, 4x4 register blocks: consecutive
            // threads take consecutive row groups bi of one column group bj, so
            // that the panel reads are 16-byte broadcasts or contiguous and the
            // updates of W are contiguous rows of a column
            const int Rb = (R + 3) / 4;
            for (int e = tid; e < Rb * Rb; e += NT) {
                const int bj = e / Rb, bi = e - bj * Rb;
                if (bj > bi) continue;
                float acc[4][4] = {};
#pragma unroll 8
                for (int l = 0; l < 32; ++l) {
                    const float4 pi = *reinterpret_cast<const float4*>(Pn + l * BLDP + 4 * bi);
                    const float4 pj = *reinterpret_cast<const float4*>(Pn + l * BLDP + 4 * bj);
                    const float ip[4] = {pi.x, pi.y, pi.z, pi.w}, jq[4] = {pj.x, pj.y, pj.z, pj.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(ip[p], jq[q], acc[p][q]);
                }
                const bool full = (bi > bj) && (4 * bi + 3 < R);  // four rows inside, below the diagonal block
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * bj + q;
                    if (j >= R) break;
                    float* w = W + (k0 + 32 + 4 * bi) + (long)(k0 + 32 + j) * BLD;
                    if (full) {
                        float4 v = *reinterpret_cast<float4*>(w);
                        v.x -= acc[0][q];
                        v.y -= acc[1][q];
                        v.z -= acc[2][q];
                        v.w -= acc[3][q];
                        *reinterpret_cast<float4*>(w) = v;
                    } else {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const int i = 4 * bi + p;
                            if (i < R && j <= i) w[p] -= acc[p][q];
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (s_bad) {
            if (tid == 0) {
                a.rep[sid].status = SPD_ERR_NOT_SPD;
                a.rep[sid].iters = 0;
                a.rep[sid].berr = INFINITY;
            }
            __syncthreads();
            continue;
        }
        // refinement (Algorithm 1, lines 2-7)
        for (int i = tid; i < n; i += NT) ys[i] = (float)(ds[i] * S.B[i]);
        __syncthreads();
        batch_lsolve<NT>(W, Inv, ys, n);
        for (int i = tid; i < n; i += NT) xs[i] = ds[i] * (double)ys[i];
        __syncthreads();
        double berr = batch_residual<NT>(S, xs, rs, &s_anorm, ra, true, red, &s_anorm);
        int it = 0, extra = a.polish;
        bool conv = false;
        for (;;) {
            if (berr <= a.tol) {
                if (extra <= 0) {
                    conv = true;
                    break;
                }
                --extra;
            } else {
                extra = a.polish;
            }
            if (it >= a.maxit) break;
            for (int i = tid; i < n; i += NT) ys[i] = (float)(ds[i] * rs[i]);
            __syncthreads();
            batch_lsolve<NT>(W, Inv, ys, n);
            for (int i = tid; i < n; i += NT) xs[i] += ds[i] * (double)ys[i];
            __syncthreads();
            berr = batch_residual<NT>(S, xs, rs, &s_anorm, ra, false, red, nullptr);
            ++it;
        }
        for (int i = tid; i < n; i += NT) S.X[i] = xs[i];
        if (tid == 0) {
            a.rep[sid].status = conv ? SPD_OK : SPD_ERR_NO_CONVERGENCE;
            a.rep[sid].iters = it;
            a.rep[sid].berr = berr;
        }
        __syncthreads();
    }
}

// Jacobi-preconditioned CG in float64 per system (x0 = 0), restarted from
// the true residual when the recursive one claims convergence but the true
// backward error does not meet the tolerance.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_batch_pcg(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* xs = reinterpret_cast<double*>(smem_raw);
    double* rs = xs + BMAX;
    double* ps = rs + BMAX;
    double* zs = ps + BMAX;
    double* qs = zs + BMAX;
    double* dinv = qs + BMAX;
    __shared__ int s_idx;
    __shared__ double red[NT / 32];
    __shared__ double s_anorm;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(a.next, 1);
        __syncthreads();
        if (s_idx >= a.count) break;
        const int sid = a.order[s_idx];
        const BatchSys S = a.sys[sid];
        const int n = S.n;
        for (int i = tid; i < n; i += NT) {
            dinv[i] = 1.0 / S.A[i + (long)i * S.lda];
            xs[i] = 0.0;
        }
        __syncthreads();
        double berr = batch_residual<NT>(S, xs, rs, &s_anorm, nullptr, true, red, &s_anorm);
        int it = 0;
        bool conv = false;
        for (int restart = 0; restart < 4 && !conv; ++restart) {
            double rho = 0.0;
            for (int i = tid; i < n; i += NT) {
                zs[i] = dinv[i] * rs[i];
                ps[i] = zs[i];
                rho += rs[i] * zs[i];
            }
            rho = block_sum<NT>(rho, red);
            for (; it < a.maxit; ++it) {
                double xmax = 0.0, rmax = 0.0;
                for (int i = tid; i < n; i += NT) {
                    xmax = fmax(xmax, fabs(xs[i]));
                    rmax = fmax(rmax, fabs(rs[i]));
                }
                xmax = block_max<NT>(xmax, red);
                rmax = block_max<NT>(rmax, red);
                if (xmax > 0.0 && rmax <= 0.5 * a.tol * s_anorm * xmax) break;
                double pq = 0.0;
                for (int i = tid; i < n; i += NT) {
                    double s = 0.0;
                    for (int j = 0; j < n; ++j) s = fma(S.A[i + (long)j * S.lda], ps[j], s);
                    qs[i] = s;
                    pq += ps[i] * s;
                }
                pq = block_sum<NT>(pq, red);
                const double alpha = rho / pq;
                double rz = 0.0;
                for (int i = tid; i < n; i += NT) {
                    xs[i] = fma(alpha, ps[i], xs[i]);
                    rs[i] = fma(-alpha, qs[i], rs[i]);
                    zs[i] = dinv[i] * rs[i];
                    rz += rs[i] * zs[i];
                }
                rz = block_sum<NT>(rz, red);
                const double beta = rz / rho;
                rho = rz;
                for (int i = tid; i < n; i += NT) ps[i] = fma(beta, ps[i], zs[i]);
                __syncthreads();
            }
            berr = batch_residual<NT>(S, xs, rs, &s_anorm, nullptr, false, red, nullptr);
            conv = berr <= a.tol;
            if (it >= a.maxit) break;
        }
        for (int i = tid; i < n; i += NT) S.X[i] = xs[i];
        if (tid == 0) {
            a.rep[sid].status = conv ? SPD_OK : SPD_ERR_NO_CONVERGENCE;
            a.rep[sid].iters = it;
            a.rep[sid].berr = berr;
            a.rep[sid].info = 0;
        }
        __syncthreads();
    }
}
