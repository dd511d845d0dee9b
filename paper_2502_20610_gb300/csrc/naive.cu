// Naive schedule: one streaming kernel per half-step over the whole grid
// (the "very straightforward" implementation of Sec. 2 whose cost model is
// 6 memory operations and 6 flops per component).  Every launch boundary is
// a grid-wide synchronisation.  It is the in-library baseline, and the
// systolic kernel must reproduce its results bit for bit.
//
// Layout: 256-thread CTAs of 32 (x) x 8 (y) threads; each thread marches up
// a column of NAIVE_KZ cells in z and carries the z-neighbour in registers,
// so x rows are read coalesced and the z-neighbour plane is read once.
#include "internal.h"
#include "yee_cell.cuh"

namespace {

constexpr int NAIVE_BX = 32, NAIVE_BY = 8, NAIVE_KZ = 8;

__global__ void __launch_bounds__(NAIVE_BX *NAIVE_BY)
naive_h_kernel(float *__restrict__ ex_, float *__restrict__ ey_, float *__restrict__ ez_,
               float *__restrict__ hx_, float *__restrict__ hy_, float *__restrict__ hz_,
               int nx, int ny, int nz, int pitch, float ndt)
{
    const int i = blockIdx.x * NAIVE_BX + threadIdx.x;
    const int j = blockIdx.y * NAIVE_BY + threadIdx.y;
    const int k0 = blockIdx.z * NAIVE_KZ;
    if (i >= nx || j >= ny || k0 >= nz) return;
    const int k1 = min(k0 + NAIVE_KZ, nz);
    const long long sxy = (long long)pitch * ny;
    const bool ip = i + 1 < nx, jp = j + 1 < ny;
    const float *Ex = ex_, *Ey = ey_, *Ez = ez_;
    long long p = i + (long long)pitch * (j + (long long)ny * k0);
    float exc = __ldg(Ex + p), eyc = __ldg(Ey + p);
    for (int k = k0; k < k1; ++k, p += sxy) {
        const bool kp = k + 1 < nz;
        const float exn = kp ? __ldg(Ex + p + sxy) : 0.f;
        const float eyn = kp ? __ldg(Ey + p + sxy) : 0.f;
        const float ez = __ldg(Ez + p);
        const float ez_ip = ip ? __ldg(Ez + p + 1) : 0.f;
        const float ey_ip = ip ? __ldg(Ey + p + 1) : 0.f;
        const float ez_jp = jp ? __ldg(Ez + p + pitch) : 0.f;
        const float ex_jp = jp ? __ldg(Ex + p + pitch) : 0.f;
        hx_[p] = h_x(hx_[p], ez_jp, ez, eyn, eyc, ndt);
        hy_[p] = h_y(hy_[p], exn, exc, ez_ip, ez, ndt);
        hz_[p] = h_z(hz_[p], ey_ip, eyc, ex_jp, exc, ndt);
        exc = exn;
        eyc = eyn;
    }
}

__global__ void __launch_bounds__(NAIVE_BX *NAIVE_BY)
naive_e_kernel(float *__restrict__ ex_, float *__restrict__ ey_, float *__restrict__ ez_,
               float *__restrict__ hx_, float *__restrict__ hy_, float *__restrict__ hz_,
               const float *__restrict__ ce_, int nx, int ny, int nz, int pitch, long long step,
               const SrcSet src)
{
    const int i = blockIdx.x * NAIVE_BX + threadIdx.x;
    const int j = blockIdx.y * NAIVE_BY + threadIdx.y;
    const int k0 = blockIdx.z * NAIVE_KZ;
    if (i >= nx || j >= ny || k0 >= nz) return;
    const int k1 = min(k0 + NAIVE_KZ, nz);
    const long long sxy = (long long)pitch * ny;
    const float *Hx = hx_, *Hy = hy_, *Hz = hz_;
    long long p = i + (long long)pitch * (j + (long long)ny * k0);
    float hxm = k0 > 0 ? __ldg(Hx + p - sxy) : 0.f;
    float hym = k0 > 0 ? __ldg(Hy + p - sxy) : 0.f;
    for (int k = k0; k < k1; ++k, p += sxy) {
        const float hx = __ldg(Hx + p), hy = __ldg(Hy + p), hz = __ldg(Hz + p);
        const float ce = __ldg(ce_ + p);
        float ex = ex_[p], ey = ey_[p], ez = ez_[p];
        // PEC: tangential E on the low planes is never updated
        if (j > 0 && k > 0) ex = e_x(ex, hz, __ldg(Hz + p - pitch), hy, hym, ce);
        if (i > 0 && k > 0) ey = e_y(ey, hx, hxm, hz, __ldg(Hz + p - 1), ce);
        if (i > 0 && j > 0) ez = e_z(ez, hy, __ldg(Hy + p - 1), hx, __ldg(Hx + p - pitch), ce);
        for (int q = 0; q < src.n; ++q) {
            const SrcDesc &s = src.s[q];
            if (s.idx == p && step < s.n_amp) {
                const float a = s.amp[step];
                if (s.comp == 0) ex = add_source(ex, a);
                else if (s.comp == 1) ey = add_source(ey, a);
                else ez = add_source(ez, a);
            }
        }
        ex_[p] = ex;
        ey_[p] = ey;
        ez_[p] = ez;
        hxm = hx;
        hym = hy;
    }
}

dim3 naive_grid(int nx, int ny, int nz)
{
    return dim3((nx + NAIVE_BX - 1) / NAIVE_BX, (ny + NAIVE_BY - 1) / NAIVE_BY,
                (nz + NAIVE_KZ - 1) / NAIVE_KZ);
}

} // namespace

cudaError_t launch_naive_h(float *const f[6], int nx, int ny, int nz, int pitch, float neg_dt,
                           cudaStream_t st)
{
    naive_h_kernel<<<naive_grid(nx, ny, nz), dim3(NAIVE_BX, NAIVE_BY), 0, st>>>(
        f[0], f[1], f[2], f[3], f[4], f[5], nx, ny, nz, pitch, neg_dt);
    return cudaGetLastError();
}

cudaError_t launch_naive_e(float *const f[6], const float *ce, int nx, int ny, int nz, int pitch,
                           long long step, const SrcSet &src, cudaStream_t st)
{
    naive_e_kernel<<<naive_grid(nx, ny, nz), dim3(NAIVE_BX, NAIVE_BY), 0, st>>>(
        f[0], f[1], f[2], f[3], f[4], f[5], ce, nx, ny, nz, pitch, step, src);
    return cudaGetLastError();
}
