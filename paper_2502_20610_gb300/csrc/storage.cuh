// Field storage formats of libfdtd (FP32, FP16, BF16).
//
// A field component c is held in memory as q = fl_S(v / s_c), where s_c is a
// power of two chosen at create time, so v = s_c * q exactly (scaling by a
// power of two neither rounds nor changes which values are representable,
// away from overflow and the subnormal range).  Every curl and every
// accumulation runs in FP32 on decoded values; a new value is rounded once,
// to nearest even, when it is stored.  The systolic kernel keeps fields in
// registers as FP32 numbers that are already rounded this way (rnd), so both
// schedules hold the same values at every step and stay bit-identical.
//
// Two values are rounded together where the kernels allow it (rnd2, enc2):
// one packed conversion instruction rounds both, each to nearest even exactly
// as the scalar conversion does, so the results are the same bits.
//
// When all six scales are equal (s), the update is linear and homogeneous in
// the fields, so the kernels step the stored values q = v / s directly (the
// "uniform" formats): no scaling on load or store, and point-source
// amplitudes are multiplied by 1/s (exact) instead.  Both schedules pick the
// same format, so they stay bit-identical; the host converts with s at the
// boundary either way.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdtd.h"

// Kernel format codes: the storage codes of fdtd.h, plus the uniform-scale
// variants of the 16-bit formats.
enum { FMT_F16U = 3, FMT_BF16U = 4 };

struct StoreF32 {
    using T = float;
    static constexpr int code = FDTD_STORAGE_F32;
    static constexpr bool narrow = false;
    __device__ __forceinline__ static float src_amp(float a, float) { return a; }
    __device__ __forceinline__ static float dec(T q, float) { return q; }
    __device__ __forceinline__ static T enc(float v, float) { return v; }
    __device__ __forceinline__ static float rnd(float v, float, float) { return v; }
    __device__ __forceinline__ static void rnd2(float &, float &, float, float) {}
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

// Packed round trips of the 16-bit formats: q = fl16(a'), fl16(b') by one
// cvt.rn.{f16,bf16}x2.f32, then both decoded.
__device__ __forceinline__ unsigned pack_f16(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ unsigned pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ float2 unpack_f16(unsigned u)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ float2 unpack_bf16(unsigned u)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}

struct StoreF16 {
    using T = unsigned short;  // IEEE binary16 bits
    static constexpr int code = FDTD_STORAGE_F16;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float src_amp(float a, float) { return a; }
    __device__ __forceinline__ static float dec(T q, float s) { return __fmul_rn(__half2float(__ushort_as_half(q)), s); }
    __device__ __forceinline__ static T enc(float v, float inv_s) { return __half_as_ushort(__float2half_rn(__fmul_rn(v, inv_s))); }
    __device__ __forceinline__ static float rnd(float v, float s, float inv_s) { return dec(enc(v, inv_s), s); }
    __device__ __forceinline__ static unsigned enc2(float a, float b, float inv_s)
    {
        return pack_f16(__fmul_rn(a, inv_s), __fmul_rn(b, inv_s));
    }
    __device__ __forceinline__ static void rnd2(float &a, float &b, float s, float inv_s)
    {
        const float2 f = unpack_f16(enc2(a, b, inv_s));
        a = __fmul_rn(f.x, s);
        b = __fmul_rn(f.y, s);
    }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

struct StoreBF16 {
    using T = unsigned short;  // bfloat16 bits
    static constexpr int code = FDTD_STORAGE_BF16;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float src_amp(float a, float) { return a; }
    __device__ __forceinline__ static float dec(T q, float s)
    {
        return __fmul_rn(__bfloat162float(__ushort_as_bfloat16(q)), s);
    }
    __device__ __forceinline__ static T enc(float v, float inv_s)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(__fmul_rn(v, inv_s)));
    }
    __device__ __forceinline__ static float rnd(float v, float s, float inv_s) { return dec(enc(v, inv_s), s); }
    __device__ __forceinline__ static unsigned enc2(float a, float b, float inv_s)
    {
        return pack_bf16(__fmul_rn(a, inv_s), __fmul_rn(b, inv_s));
    }
    __device__ __forceinline__ static void rnd2(float &a, float &b, float s, float inv_s)
    {
        const float2 f = unpack_bf16(enc2(a, b, inv_s));
        a = __fmul_rn(f.x, s);
        b = __fmul_rn(f.y, s);
    }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

// Uniform scale: registers hold q = v / s; loads and stores only convert.
struct StoreF16U {
    using T = unsigned short;
    static constexpr int code = FMT_F16U;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float src_amp(float a, float inv_s) { return __fmul_rn(a, inv_s); }
    __device__ __forceinline__ static float dec(T q, float) { return __half2float(__ushort_as_half(q)); }
    __device__ __forceinline__ static T enc(float v, float) { return __half_as_ushort(__float2half_rn(v)); }
    __device__ __forceinline__ static float rnd(float v, float, float) { return __half2float(__float2half_rn(v)); }
    __device__ __forceinline__ static unsigned enc2(float a, float b, float) { return pack_f16(a, b); }
    __device__ __forceinline__ static void rnd2(float &a, float &b, float, float)
    {
        const float2 f = unpack_f16(pack_f16(a, b));
        a = f.x;
        b = f.y;
    }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

struct StoreBF16U {
    using T = unsigned short;
    static constexpr int code = FMT_BF16U;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float src_amp(float a, float inv_s) { return __fmul_rn(a, inv_s); }
    __device__ __forceinline__ static float dec(T q, float) { return __bfloat162float(__ushort_as_bfloat16(q)); }
    __device__ __forceinline__ static T enc(float v, float) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
    __device__ __forceinline__ static float rnd(float v, float, float)
    {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
    __device__ __forceinline__ static unsigned enc2(float a, float b, float) { return pack_bf16(a, b); }
    __device__ __forceinline__ static void rnd2(float &a, float &b, float, float)
    {
        const float2 f = unpack_bf16(pack_bf16(a, b));
        a = f.x;
        b = f.y;
    }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

// Per-component scales as kernels receive them: v = s[c] * q, q = v * is[c];
// src = 1/s for the uniform formats (source amplitudes in stored units).
struct Scales {
    float s[6], is[6];
    float src;
};

// Bytes of one stored field value (storage or kernel format code).
inline int storage_bytes(int code) { return code == FDTD_STORAGE_F32 ? 4 : 2; }

// Dispatch on a kernel format code: DISPATCH_FORMAT(fmt, S, expr) evaluates
// `expr` with S bound to the traits of `fmt` and returns its value.
#define DISPATCH_FORMAT(fmt, S, ...)                                           \
    do {                                                                       \
        switch (fmt) {                                                         \
        case FDTD_STORAGE_F16: { using S = StoreF16; return __VA_ARGS__; }     \
        case FDTD_STORAGE_BF16: { using S = StoreBF16; return __VA_ARGS__; }   \
        case FMT_F16U: { using S = StoreF16U; return __VA_ARGS__; }            \
        case FMT_BF16U: { using S = StoreBF16U; return __VA_ARGS__; }          \
        default: { using S = StoreF32; return __VA_ARGS__; }                   \
        }                                                                      \
    } while (0)
