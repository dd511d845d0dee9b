// Adjoint (reverse-time) kernels for dL/deps of the Yee map.
//
// The forward step, with c = dt/eps per cell and M = 0 on the PEC-fixed
// tangential E of the low walls,
//     H^{n+1/2} = H^{n-1/2} - dt curl_f E^n,
//     E^{n+1}   = E^n + M c curl_b H^{n+1/2} + s^n,
// is linear; its transpose, with curl_f^T = curl_b (fields beyond the high
// walls and H before the low walls read 0), steps the adjoint state back:
//     lambda_H^n = lambda_H^{n+1} + curl_f(M c lambda_E^{n+1})     (adj_h)
//     lambda_E^n = lambda_E^{n+1} - dt curl_b lambda_H^n + dg_n/dE^n (adj_e)
// and the gradient over a box of cells accumulates, in FP64,
//     dL/deps_p -= (1/eps_p) sum_a lambda_{E,a}^{n+1}(p) (E^{n+1} - E^n)_a(p)
// (the source scales with 1/eps as well, so E^{n+1} - E^n is the whole
// derivative of E^{n+1} with respect to c, times c).
// The objective L = sum over the last W steps of O_n^2, O_n = sum_{i,j}
// m(i,j) Ez^n(i,j,k0) (overlap of Ez on a plane with a mode profile), gives
// dg_n/dEz^n(i,j,k0) = 2 O_n m(i,j).
#include "adjoint.h"
#include "internal.h"

namespace {

struct Geo {
    int nx, ny, nz, pitch;
    long long fs;  // floats between components
};

__device__ __forceinline__ long long at(const Geo &g, int i, int j, int k)
{
    return i + (long long)g.pitch * (j + (long long)g.ny * k);
}

// M c lambda_E component a at (i,j,k); 0 beyond the high walls
__device__ __forceinline__ float w_of(const Geo &g, const float *lam, const float *ce, int a, int i, int j, int k)
{
    if (i >= g.nx || j >= g.ny || k >= g.nz) return 0.f;
    const bool fixed = a == 0 ? (j == 0 || k == 0) : a == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
    if (fixed) return 0.f;
    const long long p = at(g, i, j, k);
    return __fmul_rn(ce[p], lam[a * g.fs + p]);
}

// lambda_H += curl_f(M c lambda_E); gradient of the box cells from
// lambda_E^{n+1} and the box's E history (3 components, box cells x fastest)
__global__ void __launch_bounds__(256) adj_h_kernel(Geo g, float *__restrict__ lam, const float *__restrict__ ce,
                                                    int3 lo, int3 hi, const float *__restrict__ e_next,
                                                    const float *__restrict__ e_now, long long box_cells,
                                                    float dt, double *__restrict__ grad)
{
    const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long p = at(g, i, j, k);
    const float *le = lam;
    float *lh = lam + 3 * g.fs;
    if (i >= lo.x && i < hi.x && j >= lo.y && j < hi.y && k >= lo.z && k < hi.z) {
        const long long b = (i - lo.x) + (long long)(hi.x - lo.x) * ((j - lo.y) + (long long)(hi.y - lo.y) * (k - lo.z));
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += (double)le[a * g.fs + p] * ((double)e_next[a * box_cells + b] - (double)e_now[a * box_cells + b]);
        const double inv_eps = (double)ce[p] / (double)dt;  // 1/eps of the coefficient in use
        grad[b] -= inv_eps * s;
    }
    const float wx = w_of(g, le, ce, 0, i, j, k), wy = w_of(g, le, ce, 1, i, j, k), wz = w_of(g, le, ce, 2, i, j, k);
    const float cx = __fsub_rn(__fsub_rn(w_of(g, le, ce, 2, i, j + 1, k), wz), __fsub_rn(w_of(g, le, ce, 1, i, j, k + 1), wy));
    const float cy = __fsub_rn(__fsub_rn(w_of(g, le, ce, 0, i, j, k + 1), wx), __fsub_rn(w_of(g, le, ce, 2, i + 1, j, k), wz));
    const float cz = __fsub_rn(__fsub_rn(w_of(g, le, ce, 1, i + 1, j, k), wy), __fsub_rn(w_of(g, le, ce, 0, i, j + 1, k), wx));
    lh[p] = __fadd_rn(lh[p], cx);
    lh[g.fs + p] = __fadd_rn(lh[g.fs + p], cy);
    lh[2 * g.fs + p] = __fadd_rn(lh[2 * g.fs + p], cz);
}

// lambda_E -= dt curl_b lambda_H (every component); plus the objective's
// source 2 O m(i,j) on Ez of the plane k0 when `amp2` != 0
__global__ void __launch_bounds__(256) adj_e_kernel(Geo g, float *__restrict__ lam, float ndt, int k0,
                                                    const float *__restrict__ mode, double amp2)
{
    const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long p = at(g, i, j, k);
    float *le = lam;
    const float *lh = lam + 3 * g.fs;
    const float hx = lh[p], hy = lh[g.fs + p], hz = lh[2 * g.fs + p];
    const float hx_jm = j > 0 ? lh[p - g.pitch] : 0.f, hx_km = k > 0 ? lh[p - (long long)g.pitch * g.ny] : 0.f;
    const float hy_im = i > 0 ? lh[g.fs + p - 1] : 0.f, hy_km = k > 0 ? lh[g.fs + p - (long long)g.pitch * g.ny] : 0.f;
    const float hz_im = i > 0 ? lh[2 * g.fs + p - 1] : 0.f, hz_jm = j > 0 ? lh[2 * g.fs + p - g.pitch] : 0.f;
    const float cx = __fsub_rn(__fsub_rn(hz, hz_jm), __fsub_rn(hy, hy_km));
    const float cy = __fsub_rn(__fsub_rn(hx, hx_km), __fsub_rn(hz, hz_im));
    const float cz = __fsub_rn(__fsub_rn(hy, hy_im), __fsub_rn(hx, hx_jm));
    le[p] = __fmaf_rn(ndt, cx, le[p]);
    le[g.fs + p] = __fmaf_rn(ndt, cy, le[g.fs + p]);
    float ez = __fmaf_rn(ndt, cz, le[2 * g.fs + p]);
    if (amp2 != 0.0 && k == k0) ez = __fadd_rn(ez, (float)(amp2 * (double)mode[i + (long long)g.nx * j]));
    le[2 * g.fs + p] = ez;
}

// out = sum_{i,j} m(i,j) Ez(i,j,k0): one block, fixed summation order, so
// the objective (and the adjoint sources built from it) are reproducible
__global__ void __launch_bounds__(1024) overlap_kernel(Geo g, const float *__restrict__ ez, int k0,
                                                       const float *__restrict__ mode, double *__restrict__ out)
{
    __shared__ double part[1024];
    double s = 0.0;
    const long long n = (long long)g.nx * g.ny;
    for (long long q = threadIdx.x; q < n; q += 1024) {
        const int i = (int)(q % g.nx), j = (int)(q / g.nx);
        s += (double)mode[q] * (double)ez[at(g, i, j, k0)];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// the E components of the box cells into dst [3][box cells] (x fastest)
__global__ void __launch_bounds__(256) box_copy_kernel(Geo g, const float *__restrict__ f, int3 lo, int3 hi,
                                                       float *__restrict__ dst, long long box_cells)
{
    const long long q = blockIdx.x * 256ll + threadIdx.x;
    if (q >= box_cells) return;
    const int bx = hi.x - lo.x, by = hi.y - lo.y;
    const int i = lo.x + (int)(q % bx), j = lo.y + (int)((q / bx) % by), k = lo.z + (int)(q / ((long long)bx * by));
    const long long p = at(g, i, j, k);
    for (int a = 0; a < 3; ++a) dst[a * box_cells + q] = f[a * g.fs + p];
}

dim3 cells_grid(const Geo &g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }

Geo geo(const AdjGeo &a)
{
    Geo g;
    g.nx = a.nx; g.ny = a.ny; g.nz = a.nz; g.pitch = a.pitch; g.fs = a.fstride;
    return g;
}

} // namespace

cudaError_t adjoint_h(const AdjGeo &a, float *lam, const float *ce, const int lo[3], const int hi[3],
                      const float *e_next, const float *e_now, float dt, double *grad, cudaStream_t st)
{
    const Geo g = geo(a);
    const long long bc = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    adj_h_kernel<<<cells_grid(g), 256, 0, st>>>(g, lam, ce, make_int3(lo[0], lo[1], lo[2]),
                                                make_int3(hi[0], hi[1], hi[2]), e_next, e_now, bc, dt, grad);
    return cudaGetLastError();
}

cudaError_t adjoint_e(const AdjGeo &a, float *lam, float dt, int k0, const float *mode, double amp2, cudaStream_t st)
{
    const Geo g = geo(a);
    adj_e_kernel<<<cells_grid(g), 256, 0, st>>>(g, lam, -dt, k0, mode, amp2);
    return cudaGetLastError();
}

cudaError_t adjoint_overlap(const AdjGeo &a, const float *ez, int k0, const float *mode, double *out, cudaStream_t st)
{
    const Geo g = geo(a);
    overlap_kernel<<<1, 1024, 0, st>>>(g, ez, k0, mode, out);
    return cudaGetLastError();
}

cudaError_t adjoint_box_copy(const AdjGeo &a, const float *f, const int lo[3], const int hi[3], float *dst,
                             cudaStream_t st)
{
    const Geo g = geo(a);
    const long long bc = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    if (bc <= 0) return cudaSuccess;
    box_copy_kernel<<<(unsigned)((bc + 255) / 256), 256, 0, st>>>(g, f, make_int3(lo[0], lo[1], lo[2]),
                                                                   make_int3(hi[0], hi[1], hi[2]), dst, bc);
    return cudaGetLastError();
}
