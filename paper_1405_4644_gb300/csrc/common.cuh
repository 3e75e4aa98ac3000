// common.cuh -- shared device helpers for libspd (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#define SPD_LEAF 128   // order of the diagonal blocks factored by one CTA
#define SPD_SUB 32     // order of the warp-level sub-blocks inside a leaf
#define SPD_MAXM 4096  // largest right-hand-side count per call
#define SPD_FP8_SCALE 256.0f  // operand scale of the e4m3 mirror (products carry 2^16)
#define SPD_SB_BLOCKS 8       // 128-blocks per diagonal super-block of the super-block sweeps

// Device-side error word: bit flags raised by kernels, read by the host.
enum : int {
    SPD_DEV_NONFINITE = 1,   // NaN/Inf met in an input
    SPD_DEV_BREAKDOWN = 2,   // non-positive pivot
    SPD_DEV_TIMEOUT = 4,     // a bounded wait gave up
    SPD_DEV_BADDIAG = 8,     // non-positive diagonal entry (scaling impossible)
    SPD_DEV_INTERNAL = 16    // a kernel met launch arguments it cannot serve
};

struct DevStatus {
    int flags;      // OR of SPD_DEV_*
    int info;       // smallest 1-based failing column (INT32_MAX = none)
    int pad[2];
};

__device__ __forceinline__ void dev_raise(DevStatus* st, int flag) { atomicOr(&st->flags, flag); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Round-to-nearest-even conversions of a float32 value into the tensor-core
// operand types.  tf32 is kept in a 32-bit container with the low 13
// fraction bits cleared.
__device__ __forceinline__ float round_tf32(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;  // Inf/NaN unchanged
    uint32_t lsb = (u >> 13) & 1u;
    u = (u + 0x0fffu + lsb) & 0xffffe000u;
    return __uint_as_float(u);
}

template <typename OpT> struct OpConv;
template <> struct OpConv<float> {  // tf32 operands
    static __device__ __forceinline__ float cvt(float x) { return round_tf32(x); }
};
template <> struct OpConv<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 cvt(float x) { return __float2bfloat16_rn(x); }
};
template <> struct OpConv<__half> {
    static __device__ __forceinline__ __half cvt(float x) { return __float2half_rn(x); }
};
template <> struct OpConv<__nv_fp8_e4m3> {
    static __device__ __forceinline__ __nv_fp8_e4m3 cvt(float x) { return __nv_fp8_e4m3(x); }
};

// Description of the tensor-core operand mirror of the factor: the
// finalised entries of L are also written here, rounded to the operand type,
// so that trailing updates read them without a conversion pass.
struct Mirror {
    void* ptr;     // n x ld elements of the operand type (nullptr = no mirror)
    long ld;       // leading dimension in elements (row-major)
    int kind;      // 0 none, 1 tf32 (float), 2 bf16, 3 fp16, 4 fp8 e4m3 (x SPD_FP8_SCALE),
                   // 5 float32 as three bf16 slices (planes of `plane` elements)
    long plane;    // kind 5: elements per slice plane (n * ld)
};

// x ~ s0 + s1 + s2 with bf16 slices: s0 = bf16(x), s1 = bf16(x - s0),
// s2 = bf16(x - s0 - s1); the remainders are exact in float32, so the three
// slices carry x's 24 significant bits up to a last rounding below 2^-24 |x|
__device__ __forceinline__ void split_bf16x3(float x, __nv_bfloat16& s0, __nv_bfloat16& s1, __nv_bfloat16& s2) {
    s0 = __float2bfloat16_rn(x);
    const float r1 = __fsub_rn(x, __bfloat162float(s0));
    s1 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(s1));
    s2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ void mirror_store(const Mirror& m, long r, long c, float v) {
    switch (m.kind) {
        case 1: ((float*)m.ptr)[r * m.ld + c] = round_tf32(v); break;
        case 2: ((__nv_bfloat16*)m.ptr)[r * m.ld + c] = __float2bfloat16_rn(v); break;
        case 3: ((__half*)m.ptr)[r * m.ld + c] = __float2half_rn(v); break;
        case 4:  // fixed power-of-two scale: |entries| <= 1 after diagonal scaling
            ((__nv_fp8_e4m3*)m.ptr)[r * m.ld + c] = __nv_fp8_e4m3(v * SPD_FP8_SCALE);
            break;
        case 5: {
            __nv_bfloat16 s0, s1, s2;
            split_bf16x3(v, s0, s1, s2);
            __nv_bfloat16* p = (__nv_bfloat16*)m.ptr + r * m.ld + c;
            p[0] = s0;
            p[m.plane] = s1;
            p[2 * m.plane] = s2;
            break;
        }
        default: break;
    }
}
__device__ __forceinline__ void mirror_store(const Mirror&, long, long, double) {}

// Four consecutive entries (c a multiple of 4) in one packed store per plane.
__device__ __forceinline__ uint2 pack_bf16x4(float a, float b, float c, float d) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}
__device__ __forceinline__ void mirror_store4(const Mirror& m, long r, long c, float4 v) {
    const long o = r * m.ld + c;
    switch (m.kind) {
        case 1:
            *reinterpret_cast<float4*>((float*)m.ptr + o) =
                make_float4(round_tf32(v.x), round_tf32(v.y), round_tf32(v.z), round_tf32(v.w));
            break;
        case 2: *reinterpret_cast<uint2*>((__nv_bfloat16*)m.ptr + o) = pack_bf16x4(v.x, v.y, v.z, v.w); break;
        case 3: {
            __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
            *reinterpret_cast<uint2*>((__half*)m.ptr + o) =
                make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
            break;
        }
        case 5: {
            __nv_bfloat16 s[4][3];
            split_bf16x3(v.x, s[0][0], s[0][1], s[0][2]);
            split_bf16x3(v.y, s[1][0], s[1][1], s[1][2]);
            split_bf16x3(v.z, s[2][0], s[2][1], s[2][2]);
            split_bf16x3(v.w, s[3][0], s[3][1], s[3][2]);
            __nv_bfloat16* p = (__nv_bfloat16*)m.ptr + o;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                __nv_bfloat162 lo, hi;
                lo.x = s[0][q];
                lo.y = s[1][q];
                hi.x = s[2][q];
                hi.y = s[3][q];
                *reinterpret_cast<uint2*>(p + q * m.plane) =
                    make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
            }
            break;
        }
        default:
            mirror_store(m, r, c, v.x);
            mirror_store(m, r, c + 1, v.y);
            mirror_store(m, r, c + 2, v.z);
            mirror_store(m, r, c + 3, v.w);
    }
}

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

// Bounded spin-wait on a device flag (volatile load).  Returns false after
// `limit` polls without seeing `want`.
__device__ __forceinline__ bool spin_until_geq(const volatile int* flag, int want, long limit) {
    for (long it = 0; it < limit; ++it) {
        if (*flag >= want) return true;
        __nanosleep(64);
    }
    return false;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization waits here until the previous kernel in its stream has
// completed and its writes are visible; the previous kernel may let it be
// scheduled earlier with pdl_trigger().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
