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

// One whole transposed step in one kernel (the two kernels above, fused):
//   lambda_H^n = lambda_H^{n+1} + curl_f(M c lambda_E^{n+1})
//   lambda_E^n = lambda_E^{n+1} - dt curl_b lambda_H^n (+ the objective's source)
// and the gradient of the box cells from lambda_E^{n+1}.  A block of 32 x 8
// threads marches z-columns (i0-1 .. i0+30) x (j0-1 .. j0+6) through a chunk
// of FZ planes: every thread computes the new lambda_H of its column, the
// columns of the low x and y halo only so that the other 31 x 7 can take
// curl_b from shared memory; the k-1 neighbour of lambda_H is the thread's
// own previous value (below the chunk, recomputed).  The
// adjoint state is read from `old` and written to `nw` (two buffers: another
// block's halo may still read a column's old values after its owner has
// updated it).  The FP32 operations are those of the two-kernel form, in the
// same order.
// (4 planes per block and 4 resident blocks per SM measured fastest: 8
// planes or an unbounded register count left the kernel latency-bound at
// fewer resident warps)
constexpr int FX = 32, FY = 8, FZ = 4;
__global__ void __launch_bounds__(FX * FY, 4) adj_step_kernel(Geo g, const float *__restrict__ old,
                                                           float *__restrict__ nw,
                                                           const float *__restrict__ ce, int3 lo, int3 hi,
                                                           const float *__restrict__ e_next,
                                                           const float *__restrict__ e_now, long long box_cells,
                                                           float dt, double *__restrict__ grad, int k0,
                                                           const float *__restrict__ mode, double amp2)
{
    // w = M c lambda_E of this block's columns at the current plane, and the
    // new lambda_H, exchanged with the x+1 / y+1 and x-1 / y-1 neighbours
    __shared__ float sw[3][FY][FX], sh[3][FY][FX];
    const int tx = threadIdx.x % FX, ty = threadIdx.x / FX;
    const int i = blockIdx.x * (FX - 1) - 1 + tx, j = blockIdx.y * (FY - 1) - 1 + ty;
    const bool col = i >= 0 && i < g.nx && j >= 0 && j < g.ny;  // a column of the domain
    const bool own = col && tx > 0 && ty > 0;                    // this block updates it
    const float ndt = -dt;
    const float *const le_old = old, *const lh = old + 3 * g.fs;
    float *const le_new = nw, *const lh_new = nw + 3 * g.fs;
    // everything a plane needs from global memory, loaded one plane ahead
    // (the loads of plane k+1 are in flight while plane k is computed):
    // lambda_E, w and old lambda_H of this column, and for the block's last
    // column / row the w of the x+1 / y+1 neighbour column
    struct Plane {
        float le[3], w[3], lh[3], wip[2], wjp[2];  // wip: Wy, Wz at x+1; wjp: Wx, Wz at y+1
    };
    auto load_plane = [&](int k, Plane &q) {
#pragma unroll
        for (int a = 0; a < 3; ++a) q.le[a] = q.w[a] = q.lh[a] = 0.f;
        q.wip[0] = q.wip[1] = q.wjp[0] = q.wjp[1] = 0.f;
        if (col && k < g.nz) {
            const long long p = at(g, i, j, k);
            const float c = ce[p];
            q.le[0] = le_old[p];
            q.le[1] = le_old[g.fs + p];
            q.le[2] = le_old[2 * g.fs + p];
            q.lh[0] = lh[p];
            q.lh[1] = lh[g.fs + p];
            q.lh[2] = lh[2 * g.fs + p];
            q.w[0] = (j == 0 || k == 0) ? 0.f : __fmul_rn(c, q.le[0]);
            q.w[1] = (i == 0 || k == 0) ? 0.f : __fmul_rn(c, q.le[1]);
            q.w[2] = (i == 0 || j == 0) ? 0.f : __fmul_rn(c, q.le[2]);
            if (tx == FX - 1) {
                q.wip[0] = w_of(g, le_old, ce, 1, i + 1, j, k);
                q.wip[1] = w_of(g, le_old, ce, 2, i + 1, j, k);
            }
            if (ty == FY - 1) {
                q.wjp[0] = w_of(g, le_old, ce, 0, i, j + 1, k);
                q.wjp[1] = w_of(g, le_old, ce, 2, i, j + 1, k);
            }
        }
    };
    const int kz0 = blockIdx.z * FZ, kz1 = min(g.nz, kz0 + FZ);
    Plane cur, nxt;
    load_plane(max(0, kz0 - 1), cur);
    float (&le_c)[3] = cur.le, (&w_c)[3] = cur.w, (&w_n)[3] = nxt.w;
    float pz_x = 0.f, pz_y = 0.f;  // new lambda_H at (i, j, k-1): Hx, Hy
    for (int k = max(0, kz0 - 1); k < kz1; ++k) {
        load_plane(k + 1, nxt);
#pragma unroll
        for (int a = 0; a < 3; ++a) sw[a][ty][tx] = w_c[a];
        __syncthreads();
        float nhx = 0.f, nhy = 0.f, nhz = 0.f;
        long long p = 0;
        if (col) {
            p = at(g, i, j, k);
            // x+1 and y+1 neighbours: from shared memory, or (the block's
            // last column / row) computed from global memory
            const float wy_ip = tx < FX - 1 ? sw[1][ty][tx + 1] : cur.wip[0];
            const float wz_ip = tx < FX - 1 ? sw[2][ty][tx + 1] : cur.wip[1];
            const float wx_jp = ty < FY - 1 ? sw[0][ty + 1][tx] : cur.wjp[0];
            const float wz_jp = ty < FY - 1 ? sw[2][ty + 1][tx] : cur.wjp[1];
            const float cx = __fsub_rn(__fsub_rn(wz_jp, w_c[2]), __fsub_rn(w_n[1], w_c[1]));
            const float cy = __fsub_rn(__fsub_rn(w_n[0], w_c[0]), __fsub_rn(wz_ip, w_c[2]));
            const float cz = __fsub_rn(__fsub_rn(wy_ip, w_c[1]), __fsub_rn(wx_jp, w_c[0]));
            nhx = __fadd_rn(cur.lh[0], cx);
            nhy = __fadd_rn(cur.lh[1], cy);
            nhz = __fadd_rn(cur.lh[2], cz);
        }
        sh[0][ty][tx] = nhx;
        sh[1][ty][tx] = nhy;
        sh[2][ty][tx] = nhz;
        __syncthreads();
        if (k >= kz0 && own) {
            // gradient of a box cell from lambda_E^{n+1} (old) and E^{n+1} - E^n
            if (i >= lo.x && i < hi.x && j >= lo.y && j < hi.y && k >= lo.z && k < hi.z) {
                const long long b = (i - lo.x) +
                                    (long long)(hi.x - lo.x) * ((j - lo.y) + (long long)(hi.y - lo.y) * (k - lo.z));
                double s = 0.0;
                for (int a = 0; a < 3; ++a)
                    s += (double)le_c[a] * ((double)e_next[a * box_cells + b] - (double)e_now[a * box_cells + b]);
                const double inv_eps = (double)ce[p] / (double)dt;
                grad[b] -= inv_eps * s;
            }
            // curl_b of the new lambda_H: x-1 and y-1 neighbours from shared
            // memory, k-1 from this thread's previous value (0 before a wall)
            const float hx_jm = j > 0 ? sh[0][ty - 1][tx] : 0.f, hx_km = k > 0 ? pz_x : 0.f;
            const float hy_im = i > 0 ? sh[1][ty][tx - 1] : 0.f, hy_km = k > 0 ? pz_y : 0.f;
            const float hz_im = i > 0 ? sh[2][ty][tx - 1] : 0.f, hz_jm = j > 0 ? sh[2][ty - 1][tx] : 0.f;
            const float ex_c = __fsub_rn(__fsub_rn(nhz, hz_jm), __fsub_rn(nhy, hy_km));
            const float ey_c = __fsub_rn(__fsub_rn(nhx, hx_km), __fsub_rn(nhz, hz_im));
            const float ez_c = __fsub_rn(__fsub_rn(nhy, hy_im), __fsub_rn(nhx, hx_jm));
            le_new[p] = __fmaf_rn(ndt, ex_c, le_c[0]);
            le_new[g.fs + p] = __fmaf_rn(ndt, ey_c, le_c[1]);
            float ez = __fmaf_rn(ndt, ez_c, le_c[2]);
            if (amp2 != 0.0 && k == k0) ez = __fadd_rn(ez, (float)(amp2 * (double)mode[i + (long long)g.nx * j]));
            le_new[2 * g.fs + p] = ez;
            lh_new[p] = nhx;
            lh_new[g.fs + p] = nhy;
            lh_new[2 * g.fs + p] = nhz;
        }
        pz_x = nhx;
        pz_y = nhy;
        cur = nxt;
    }
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

cudaError_t adjoint_step(const AdjGeo &a, const float *lam_old, float *lam_new, const float *ce, const int lo[3],
                         const int hi[3], const float *e_next, const float *e_now, float dt, double *grad, int k0,
                         const float *mode, double amp2, cudaStream_t st)
{
    const Geo g = geo(a);
    const long long bc = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    const dim3 grid((g.nx + FX - 1) / (FX - 1), (g.ny + FY - 1) / (FY - 1), (g.nz + FZ - 1) / FZ);
    adj_step_kernel<<<grid, FX * FY, 0, st>>>(g, lam_old, lam_new, ce, make_int3(lo[0], lo[1], lo[2]),
                                              make_int3(hi[0], hi[1], hi[2]), e_next, e_now, bc, dt, grad, k0,
                                              mode, amp2);
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
