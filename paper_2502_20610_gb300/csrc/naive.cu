// Naive schedule: one streaming kernel per half-step over the whole grid
// (the "very straightforward" implementation of Sec. 2 whose cost model is
// 6 memory operations and 6 flops per component).  Every launch boundary is
// a grid-wide synchronisation.  It is the in-library baseline, and the
// systolic kernel must reproduce its results bit for bit.
//
// Layout: 256-thread CTAs of 32 (x) x 8 (y) threads; each thread marches up
// a column of NAIVE_KZ cells in z and carries the z-neighbour in registers,
// so x rows are read coalesced and the z-neighbour plane is read once.
// Fields are stored as FP32, FP16 or BF16 (storage.cuh); arithmetic is FP32.
#include "internal.h"
#include "storage.cuh"
#include "yee_cell.cuh"

namespace {

constexpr int NAIVE_BX = 32, NAIVE_BY = 8, NAIVE_KZ = 8;
constexpr int NAIVE_BLOCK_CELLS = 1024;

template <class S>
__global__ void __launch_bounds__(NAIVE_BX *NAIVE_BY)
naive_h_kernel(typename S::T *__restrict__ ex_, typename S::T *__restrict__ ey_, typename S::T *__restrict__ ez_,
               typename S::T *__restrict__ hx_, typename S::T *__restrict__ hy_, typename S::T *__restrict__ hz_,
               int nx, int ny, int nz, int pitch, float ndt, const Scales sc)
{
    using T = typename S::T;
    const int i = blockIdx.x * NAIVE_BX + threadIdx.x;
    const int j = blockIdx.y * NAIVE_BY + threadIdx.y;
    const int k0 = blockIdx.z * NAIVE_KZ;
    if (i >= nx || j >= ny || k0 >= nz) return;
    const int k1 = min(k0 + NAIVE_KZ, nz);
    const long long sxy = (long long)pitch * ny;
    const bool ip = i + 1 < nx, jp = j + 1 < ny;
    const T *Ex = ex_, *Ey = ey_, *Ez = ez_;
    const float s0 = sc.s[0], s1 = sc.s[1], s2 = sc.s[2];
    long long p = i + (long long)pitch * (j + (long long)ny * k0);
    float exc = S::dec(__ldg(Ex + p), s0), eyc = S::dec(__ldg(Ey + p), s1);
    for (int k = k0; k < k1; ++k, p += sxy) {
        const bool kp = k + 1 < nz;
        const float exn = kp ? S::dec(__ldg(Ex + p + sxy), s0) : 0.f;
        const float eyn = kp ? S::dec(__ldg(Ey + p + sxy), s1) : 0.f;
        const float ez = S::dec(__ldg(Ez + p), s2);
        const float ez_ip = ip ? S::dec(__ldg(Ez + p + 1), s2) : 0.f;
        const float ey_ip = ip ? S::dec(__ldg(Ey + p + 1), s1) : 0.f;
        const float ez_jp = jp ? S::dec(__ldg(Ez + p + pitch), s2) : 0.f;
        const float ex_jp = jp ? S::dec(__ldg(Ex + p + pitch), s0) : 0.f;
        hx_[p] = S::enc(h_x(S::dec(hx_[p], sc.s[3]), ez_jp, ez, eyn, eyc, ndt), sc.is[3]);
        hy_[p] = S::enc(h_y(S::dec(hy_[p], sc.s[4]), exn, exc, ez_ip, ez, ndt), sc.is[4]);
        hz_[p] = S::enc(h_z(S::dec(hz_[p], sc.s[5]), ey_ip, eyc, ex_jp, exc, ndt), sc.is[5]);
        exc = exn;
        eyc = eyn;
    }
}

template <class S, bool LOSSY>
__global__ void __launch_bounds__(NAIVE_BX *NAIVE_BY)
naive_e_kernel(typename S::T *__restrict__ ex_, typename S::T *__restrict__ ey_, typename S::T *__restrict__ ez_,
               typename S::T *__restrict__ hx_, typename S::T *__restrict__ hy_, typename S::T *__restrict__ hz_,
               const float *__restrict__ ce_, const float *__restrict__ ca_, int nx, int ny, int nz, int pitch,
               long long step, const SrcSet src, const Scales sc)
{
    using T = typename S::T;
    const int i = blockIdx.x * NAIVE_BX + threadIdx.x;
    const int j = blockIdx.y * NAIVE_BY + threadIdx.y;
    const int k0 = blockIdx.z * NAIVE_KZ;
    if (i >= nx || j >= ny || k0 >= nz) return;
    const int k1 = min(k0 + NAIVE_KZ, nz);
    const long long sxy = (long long)pitch * ny;
    const T *Hx = hx_, *Hy = hy_, *Hz = hz_;
    const float s3 = sc.s[3], s4 = sc.s[4], s5 = sc.s[5];
    long long p = i + (long long)pitch * (j + (long long)ny * k0);
    float hxm = k0 > 0 ? S::dec(__ldg(Hx + p - sxy), s3) : 0.f;
    float hym = k0 > 0 ? S::dec(__ldg(Hy + p - sxy), s4) : 0.f;
    for (int k = k0; k < k1; ++k, p += sxy) {
        const float hx = S::dec(__ldg(Hx + p), s3), hy = S::dec(__ldg(Hy + p), s4);
        const float hz = S::dec(__ldg(Hz + p), s5);
        const float ce = __ldg(ce_ + p);
        const float ca = LOSSY ? __ldg(ca_ + p) : 1.f;
        float ex = S::dec(ex_[p], sc.s[0]), ey = S::dec(ey_[p], sc.s[1]), ez = S::dec(ez_[p], sc.s[2]);
        // PEC: tangential E on the low planes is never updated.  Lossy cells:
        // E <- ca E + cb curl H, with cb in place of dt/eps
        if (j > 0 && k > 0) ex = e_x(decay<LOSSY>(ca, ex), hz, S::dec(__ldg(Hz + p - pitch), s5), hy, hym, ce);
        if (i > 0 && k > 0) ey = e_y(decay<LOSSY>(ca, ey), hx, hxm, hz, S::dec(__ldg(Hz + p - 1), s5), ce);
        if (i > 0 && j > 0)
            ez = e_z(decay<LOSSY>(ca, ez), hy, S::dec(__ldg(Hy + p - 1), s4), hx, S::dec(__ldg(Hx + p - pitch), s3), ce);
        for (int q = 0; q < src.n; ++q) {
            const SrcDesc &s = src.s[q];
            if (s.idx == p && step < s.n_amp) {
                const float a = S::src_amp(s.amp[step], sc.src);
                if (s.comp == 0) ex = add_source(ex, a);
                else if (s.comp == 1) ey = add_source(ey, a);
                else ez = add_source(ez, a);
            }
        }
        ex_[p] = S::enc(ex, sc.is[0]);
        ey_[p] = S::enc(ey, sc.is[1]);
        ez_[p] = S::enc(ez, sc.is[2]);
        hxm = hx;
        hym = hy;
    }
}

// Small domains (at most NAIVE_BLOCK_CELLS cells, the largest thread block):
// one CTA, one thread per cell, runs all the steps of a call with block
// barriers between the half-steps instead of kernel boundaries, the regime
// of Fig. 1 in which the update needs no global synchronisation.  The data
// change inside the launch, so loads are plain (coherent) loads; the block
// barrier orders each half-step's stores before the next one's loads.
template <class S, bool LOSSY>
__global__ void __launch_bounds__(NAIVE_BLOCK_CELLS)
naive_block_kernel(typename S::T *__restrict__ ex_, typename S::T *__restrict__ ey_, typename S::T *__restrict__ ez_,
                   typename S::T *__restrict__ hx_, typename S::T *__restrict__ hy_, typename S::T *__restrict__ hz_,
                   const float *__restrict__ ce_, const float *__restrict__ ca_, int nx, int ny, int nz, int pitch, float ndt, long long step0,
                   int nsteps, const SrcSet src, const Scales sc)
{
    const int q = threadIdx.x;
    const bool own = q < nx * ny * nz;
    const int i = own ? q % nx : 0, j = own ? (q / nx) % ny : 0, k = own ? q / (nx * ny) : 0;
    const long long sxy = (long long)pitch * ny;
    const long long p = i + (long long)pitch * (j + (long long)ny * k);
    const bool ip = i + 1 < nx, jp = j + 1 < ny, kp = k + 1 < nz;
    const float ce = own ? ce_[p] : 0.f;
    const float ca = LOSSY && own ? ca_[p] : 1.f;
    for (int s = 0; s < nsteps; ++s) {
        if (own) {
            const float exc = S::dec(ex_[p], sc.s[0]), eyc = S::dec(ey_[p], sc.s[1]), ezc = S::dec(ez_[p], sc.s[2]);
            const float exn = kp ? S::dec(ex_[p + sxy], sc.s[0]) : 0.f;
            const float eyn = kp ? S::dec(ey_[p + sxy], sc.s[1]) : 0.f;
            const float ez_ip = ip ? S::dec(ez_[p + 1], sc.s[2]) : 0.f;
            const float ey_ip = ip ? S::dec(ey_[p + 1], sc.s[1]) : 0.f;
            const float ez_jp = jp ? S::dec(ez_[p + pitch], sc.s[2]) : 0.f;
            const float ex_jp = jp ? S::dec(ex_[p + pitch], sc.s[0]) : 0.f;
            hx_[p] = S::enc(h_x(S::dec(hx_[p], sc.s[3]), ez_jp, ezc, eyn, eyc, ndt), sc.is[3]);
            hy_[p] = S::enc(h_y(S::dec(hy_[p], sc.s[4]), exn, exc, ez_ip, ezc, ndt), sc.is[4]);
            hz_[p] = S::enc(h_z(S::dec(hz_[p], sc.s[5]), ey_ip, eyc, ex_jp, exc, ndt), sc.is[5]);
        }
        __syncthreads();
        if (own) {
            const float hx = S::dec(hx_[p], sc.s[3]), hy = S::dec(hy_[p], sc.s[4]), hz = S::dec(hz_[p], sc.s[5]);
            float ex = S::dec(ex_[p], sc.s[0]), ey = S::dec(ey_[p], sc.s[1]), ez = S::dec(ez_[p], sc.s[2]);
            if (j > 0 && k > 0)
                ex = e_x(decay<LOSSY>(ca, ex), hz, S::dec(hz_[p - pitch], sc.s[5]), hy, S::dec(hy_[p - sxy], sc.s[4]), ce);
            if (i > 0 && k > 0)
                ey = e_y(decay<LOSSY>(ca, ey), hx, S::dec(hx_[p - sxy], sc.s[3]), hz, S::dec(hz_[p - 1], sc.s[5]), ce);
            if (i > 0 && j > 0)
                ez = e_z(decay<LOSSY>(ca, ez), hy, S::dec(hy_[p - 1], sc.s[4]), hx, S::dec(hx_[p - pitch], sc.s[3]), ce);
            const long long step = step0 + s;
            for (int qq = 0; qq < src.n; ++qq) {
                const SrcDesc &d = src.s[qq];
                if (d.idx == p && step < d.n_amp) {
                    const float a = S::src_amp(d.amp[step], sc.src);
                    if (d.comp == 0) ex = add_source(ex, a);
                    else if (d.comp == 1) ey = add_source(ey, a);
                    else ez = add_source(ez, a);
                }
            }
            ex_[p] = S::enc(ex, sc.is[0]);
            ey_[p] = S::enc(ey, sc.is[1]);
            ez_[p] = S::enc(ez, sc.is[2]);
        }
        __syncthreads();
    }
}

dim3 naive_grid(int nx, int ny, int nz)
{
    return dim3((nx + NAIVE_BX - 1) / NAIVE_BX, (ny + NAIVE_BY - 1) / NAIVE_BY,
                (nz + NAIVE_KZ - 1) / NAIVE_KZ);
}

template <class S>
cudaError_t launch_h(void *const f[6], int nx, int ny, int nz, int pitch, float neg_dt, const Scales &sc,
                     cudaStream_t st)
{
    using T = typename S::T;
    naive_h_kernel<S><<<naive_grid(nx, ny, nz), dim3(NAIVE_BX, NAIVE_BY), 0, st>>>(
        (T *)f[0], (T *)f[1], (T *)f[2], (T *)f[3], (T *)f[4], (T *)f[5], nx, ny, nz, pitch, neg_dt, sc);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_e(void *const f[6], const float *ce, const float *ca, int nx, int ny, int nz, int pitch,
                     long long step, const SrcSet &src, const Scales &sc, cudaStream_t st)
{
    using T = typename S::T;
    if (ca)
        naive_e_kernel<S, true><<<naive_grid(nx, ny, nz), dim3(NAIVE_BX, NAIVE_BY), 0, st>>>(
            (T *)f[0], (T *)f[1], (T *)f[2], (T *)f[3], (T *)f[4], (T *)f[5], ce, ca, nx, ny, nz, pitch, step, src,
            sc);
    else
        naive_e_kernel<S, false><<<naive_grid(nx, ny, nz), dim3(NAIVE_BX, NAIVE_BY), 0, st>>>(
            (T *)f[0], (T *)f[1], (T *)f[2], (T *)f[3], (T *)f[4], (T *)f[5], ce, ca, nx, ny, nz, pitch, step, src,
            sc);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_block(void *const f[6], const float *ce, const float *ca, int nx, int ny, int nz, int pitch,
                         float neg_dt, long long step0, int nsteps, const SrcSet &src, const Scales &sc,
                         cudaStream_t st)
{
    using T = typename S::T;
    const int threads = (nx * ny * nz + 31) / 32 * 32;
    if (ca)
        naive_block_kernel<S, true><<<1, threads, 0, st>>>((T *)f[0], (T *)f[1], (T *)f[2], (T *)f[3], (T *)f[4],
                                                            (T *)f[5], ce, ca, nx, ny, nz, pitch, neg_dt, step0,
                                                            nsteps, src, sc);
    else
        naive_block_kernel<S, false><<<1, threads, 0, st>>>((T *)f[0], (T *)f[1], (T *)f[2], (T *)f[3], (T *)f[4],
                                                             (T *)f[5], ce, ca, nx, ny, nz, pitch, neg_dt, step0,
                                                             nsteps, src, sc);
    return cudaGetLastError();
}

} // namespace

int naive_block_max_cells() { return NAIVE_BLOCK_CELLS; }

cudaError_t launch_naive_block(void *const f[6], int fmt, const float *ce, const float *ca, int nx, int ny, int nz,
                               int pitch, float neg_dt, long long step0, int nsteps, const SrcSet &src,
                               const Scales &sc, cudaStream_t st)
{
    DISPATCH_FORMAT(fmt, S, launch_block<S>(f, ce, ca, nx, ny, nz, pitch, neg_dt, step0, nsteps, src, sc, st));
}

cudaError_t launch_naive_h(void *const f[6], int fmt, int nx, int ny, int nz, int pitch, float neg_dt,
                           const Scales &sc, cudaStream_t st)
{
    DISPATCH_FORMAT(fmt, S, launch_h<S>(f, nx, ny, nz, pitch, neg_dt, sc, st));
}

cudaError_t launch_naive_e(void *const f[6], int fmt, const float *ce, const float *ca, int nx, int ny, int nz,
                           int pitch, long long step, const SrcSet &src, const Scales &sc, cudaStream_t st)
{
    DISPATCH_FORMAT(fmt, S, launch_e<S>(f, ce, ca, nx, ny, nz, pitch, step, src, sc, st));
}
