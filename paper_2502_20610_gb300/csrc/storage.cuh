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
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdtd.h"

struct StoreF32 {
    using T = float;
    static constexpr int code = FDTD_STORAGE_F32;
    static constexpr bool narrow = false;
    __device__ __forceinline__ static float dec(T q, float) { return q; }
    __device__ __forceinline__ static T enc(float v, float) { return v; }
    __device__ __forceinline__ static float rnd(float v, float, float) { return v; }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

struct StoreF16 {
    using T = unsigned short;  // IEEE binary16 bits
    static constexpr int code = FDTD_STORAGE_F16;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float dec(T q, float s) { return __fmul_rn(__half2float(__ushort_as_half(q)), s); }
    __device__ __forceinline__ static T enc(float v, float inv_s) { return __half_as_ushort(__float2half_rn(__fmul_rn(v, inv_s))); }
    __device__ __forceinline__ static float rnd(float v, float s, float inv_s) { return dec(enc(v, inv_s), s); }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

struct StoreBF16 {
    using T = unsigned short;  // bfloat16 bits
    static constexpr int code = FDTD_STORAGE_BF16;
    static constexpr bool narrow = true;
    __device__ __forceinline__ static float dec(T q, float s)
    {
        return __fmul_rn(__bfloat162float(__ushort_as_bfloat16(q)), s);
    }
    __device__ __forceinline__ static T enc(float v, float inv_s)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(__fmul_rn(v, inv_s)));
    }
    __device__ __forceinline__ static float rnd(float v, float s, float inv_s) { return dec(enc(v, inv_s), s); }
    __device__ __forceinline__ static T ld_cg(const T *p) { return __ldcg(p); }
};

// Per-component scales as kernels receive them: v = s[c] * q, q = v * is[c].
struct Scales {
    float s[6], is[6];
};

// Bytes of one stored field value.
inline int storage_bytes(int code) { return code == FDTD_STORAGE_F32 ? 4 : 2; }
