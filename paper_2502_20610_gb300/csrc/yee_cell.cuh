// One Yee cell component update, shared by every schedule so that the naive
// and the systolic kernels perform the identical sequence of FP32 roundings.
//
// Sec. 2, Eq. 1: Ex += (dt/dy)(Hz[j] - Hz[j-1]) - (dt/dz)(Hy[k] - Hy[k-1]),
// here with dx = dy = dz = 1 and the per-cell coefficient ce = dt/eps.  The
// H rows are the forward-difference (adjoint) form with coefficient -dt.
//
// Every operation is an explicit round-to-nearest intrinsic, so the result
// does not depend on the compiler's FMA contraction choices:
//     c = (a1 - a0) - (b1 - b0);   out = fma(coef, c, v)
#pragma once

__device__ __forceinline__ float yee_comp(float v, float a1, float a0, float b1, float b0,
                                          float coef)
{
    const float d1 = __fsub_rn(a1, a0);
    const float d2 = __fsub_rn(b1, b0);
    return __fmaf_rn(coef, __fsub_rn(d1, d2), v);
}

// H half-step of one cell (coef = -dt):
//   Hx -= dt((Ez[j+1]-Ez) - (Ey[k+1]-Ey))
//   Hy -= dt((Ex[k+1]-Ex) - (Ez[i+1]-Ez))
//   Hz -= dt((Ey[i+1]-Ey) - (Ex[j+1]-Ex))
__device__ __forceinline__ float h_x(float hx, float ez_jp, float ez, float ey_kp, float ey, float ndt)
{ return yee_comp(hx, ez_jp, ez, ey_kp, ey, ndt); }
__device__ __forceinline__ float h_y(float hy, float ex_kp, float ex, float ez_ip, float ez, float ndt)
{ return yee_comp(hy, ex_kp, ex, ez_ip, ez, ndt); }
__device__ __forceinline__ float h_z(float hz, float ey_ip, float ey, float ex_jp, float ex, float ndt)
{ return yee_comp(hz, ey_ip, ey, ex_jp, ex, ndt); }

// E half-step of one cell (coef = ce = dt/eps), Eq. 1 and its permutations:
//   Ex += ce((Hz-Hz[j-1]) - (Hy-Hy[k-1]))
//   Ey += ce((Hx-Hx[k-1]) - (Hz-Hz[i-1]))
//   Ez += ce((Hy-Hy[i-1]) - (Hx-Hx[j-1]))
__device__ __forceinline__ float e_x(float ex, float hz, float hz_jm, float hy, float hy_km, float ce)
{ return yee_comp(ex, hz, hz_jm, hy, hy_km, ce); }
__device__ __forceinline__ float e_y(float ey, float hx, float hx_km, float hz, float hz_im, float ce)
{ return yee_comp(ey, hx, hx_km, hz, hz_im, ce); }
__device__ __forceinline__ float e_z(float ez, float hy, float hy_im, float hx, float hx_jm, float ce)
{ return yee_comp(ez, hy, hy_im, hx, hx_jm, ce); }

// Point source: added after the E update with one FP32 rounding.
__device__ __forceinline__ float add_source(float e, float amp) { return __fadd_rn(e, amp); }

// Conducting cells (the lossy form E <- ca E + cb curl H): the old value is
// first scaled by ca with one rounding; lossless kernels skip the multiply
// (ca = 1 would leave E unchanged anyway).
template <bool LOSSY>
__device__ __forceinline__ float decay(float ca, float e) { return LOSSY ? __fmul_rn(ca, e) : e; }
