// Adjoint (reverse-time) kernels for dL/deps of the Yee map.
//
// The forward step, with c = dt/eps per cell and M = 0 on the PEC-fixed
// tangential E of the low walls,
//     H^{n+1/2} = H^{n-1/2} - dt curl_f E^n,
//     E^{n+1}   = E^n + M c curl_b H^{n+1/2} + s^n,
// is linear; its transpose, with curl_f^T = curl_b (fields beyond the high
// walls and H before the low walls read 0), steps the adjoint state back:
//     lambda_H^n = lambda_H^{n+1} + curl_f(M c lambda_E^{n+1})
//     lambda_E^n = lambda_E^{n+1} - dt curl_b lambda_H^n + dg_n/dE^n.
// In the variables  Et = M c lambda_E,  Ht = -dt lambda_H  this is the
// forward step itself:
//     Ht^n = Ht^{n+1} - dt curl_f Et^{n+1}
//     Et^n = Et^{n+1} + M c curl_b Ht^n + M c dg_n/dE^n,
// so the adjoint sweep runs on the simulation's own update kernels (the
// systolic schedule included), with the objective's source added by
// plane_source_kernel.  The gradient over a box of cells,
//     dL/deps_p = -(1/eps_p) sum_n sum_a lambda_{E,a}^{n+1}(p) (E^{n+1} - E^n)_a(p)
//               = -(1/dt) sum_n sum_a Et_a^{n+1}(p) (E^{n+1} - E^n)_a(p)
// (c = dt/eps; the source scales with 1/eps as well, so E^{n+1} - E^n is the
// whole derivative of E^{n+1} with respect to c, times c), is accumulated in
// FP64 from the box's histories of E and Et (gradient_kernel).
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

// Et_z(i,j,k0) += M c(i,j,k0) amp2 m(i,j): the objective's source in the
// transformed variables (Ez is PEC-fixed where i = 0 or j = 0), one rounding
__global__ void __launch_bounds__(256) plane_source_kernel(Geo g, float *__restrict__ ez,
                                                           const float *__restrict__ ce, int k0,
                                                           const float *__restrict__ mode, double amp2)
{
    const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32;
    if (i >= g.nx || j >= g.ny || i == 0 || j == 0) return;
    const long long p = at(g, i, j, k0);
    ez[p] = __fadd_rn(ez[p], (float)((double)ce[p] * amp2 * (double)mode[i + (long long)g.nx * j]));
}

// grad[b] -= (1/dt) sum_a Et_a^{q+1}(b) (E^{q+1} - E^q)_a(b) for the steps q
// of one segment [s0, s0 + len), from q = s0 + len - 1 down to s0: e_hist
// plane r holds E^{s0 + r} (r = 0..len), et_hist plane r holds Et^{s0 + len - r}
// (r = 0..len - 1), both [r][3][box cells].  One thread per box cell,
// subtracting step by step in that order, so the sum is the same for every
// segment length; the loads of GU steps are issued before their sums.  A
// step's term is formed in FP32 from the FP32 states (a few units of 2^-24)
// and the sum over the steps is FP64.
constexpr int GU = 8;
__global__ void __launch_bounds__(128) gradient_kernel(const float *__restrict__ et_hist,
                                                       const float *__restrict__ e_hist, long long bc, int len,
                                                       double inv_dt, double *__restrict__ grad)
{
    const long long b = blockIdx.x * 128ll + threadIdx.x;
    if (b >= bc) return;
    const long long ps = 3 * bc;  // floats per plane
    double g = grad[b];
    float hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) hi[a] = e_hist[(long long)len * ps + a * bc + b];
    for (int r0 = 0; r0 < len; r0 += GU) {
        float et[GU][3], lo[GU][3];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            if (r0 + u < len) {
                const float *e_lo = e_hist + (long long)(len - 1 - r0 - u) * ps + b;
                const float *e_t = et_hist + (long long)(r0 + u) * ps + b;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[u][a] = e_lo[a * bc];
                    et[u][a] = e_t[a * bc];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            if (r0 + u < len) {
                // one step's term in FP32 (FP64 is a small fraction of the
                // FP32 rate on this part), accumulated in FP64
                float s = __fmul_rn(et[u][0], __fsub_rn(hi[0], lo[u][0]));
                s = __fmaf_rn(et[u][1], __fsub_rn(hi[1], lo[u][1]), s);
                s = __fmaf_rn(et[u][2], __fsub_rn(hi[2], lo[u][2]), s);
#pragma unroll
                for (int a = 0; a < 3; ++a) hi[a] = lo[u][a];
                g = fma(-(double)s, inv_dt, g);
            }
        }
    }
    grad[b] = g;
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

// out[w] = sum_{i,j} m(i,j) Ez_w(i,j) for the planes w of `planes` ([w][3]
// [nx*ny], Ez = component 2): one block per plane, fixed summation order
__global__ void __launch_bounds__(1024) overlaps_kernel(const float *__restrict__ planes, long long plane_cells,
                                                        const float *__restrict__ mode, double *__restrict__ out)
{
    __shared__ double part[1024];
    const float *ez = planes + (3 * blockIdx.x + 2) * plane_cells;
    double s = 0.0;
    for (long long q = threadIdx.x; q < plane_cells; q += 1024) s += (double)mode[q] * (double)ez[q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = part[0];
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

Geo geo(const AdjGeo &a)
{
    Geo g;
    g.nx = a.nx; g.ny = a.ny; g.nz = a.nz; g.pitch = a.pitch; g.fs = a.fstride;
    return g;
}

} // namespace

cudaError_t adjoint_plane_source(const AdjGeo &a, float *ez, const float *ce, int k0, const float *mode, double amp2,
                                 cudaStream_t st)
{
    const Geo g = geo(a);
    plane_source_kernel<<<dim3((g.nx + 31) / 32, (g.ny + 7) / 8), 256, 0, st>>>(g, ez, ce, k0, mode, amp2);
    return cudaGetLastError();
}

cudaError_t adjoint_gradient(const float *et_hist, const float *e_hist, long long box_cells, int len, double dt,
                             double *grad, cudaStream_t st)
{
    if (box_cells <= 0 || len <= 0) return cudaSuccess;
    gradient_kernel<<<(unsigned)((box_cells + 127) / 128), 128, 0, st>>>(et_hist, e_hist, box_cells, len, 1.0 / dt,
                                                                         grad);
    return cudaGetLastError();
}

cudaError_t adjoint_overlap(const AdjGeo &a, const float *ez, int k0, const float *mode, double *out, cudaStream_t st)
{
    const Geo g = geo(a);
    overlap_kernel<<<1, 1024, 0, st>>>(g, ez, k0, mode, out);
    return cudaGetLastError();
}

cudaError_t adjoint_overlaps(const float *planes, long long plane_cells, int n, const float *mode, double *out,
                             cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    overlaps_kernel<<<n, 1024, 0, st>>>(planes, plane_cells, mode, out);
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
