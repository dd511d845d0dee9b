// fdtd_systolic_step_noalloc: the systolic scheme for callers that cannot
// allocate device memory.  The kernel's scratch (per-tile progress flags, the
// tile hand-out order and the control words) lives in one file-scope device
// array of fixed size instead of a caller workspace; the caller passes only
// its own field and coefficient buffers.  Declared in include/fdtd.h.
#include "fdtd.h"
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

namespace {

constexpr size_t NOALLOC_CTRL_BYTES = 256;          // 64 control words
constexpr int NOALLOC_VARIANT = 0;                  // 31 x 15 x 15 tiles
constexpr int NOALLOC_MAX_STEPS_PER_LAUNCH = 1024;

// Shared by every call on a device and kept until the process exits:
//   [0, 256)            control words (ticket, error word, error info)
//   [256, 256 + 4G)     progress flag per tile
//   [256 + 4G, ...)     tile hand-out order
static __device__ __align__(256) unsigned char g_noalloc_scratch[FDTD_NOALLOC_SCRATCH_BYTES];

constexpr long long NOALLOC_MAX_TILES = (long long)(FDTD_NOALLOC_SCRATCH_BYTES - NOALLOC_CTRL_BYTES) / 8;

constexpr int MAX_DEVICES = 64;
struct DeviceState {
    bool ready;
    unsigned char *scratch;  // device address of g_noalloc_scratch on this device
    int max_ctas;
};
DeviceState g_dev[MAX_DEVICES];
std::mutex g_mu;

fdtd_status cuda_fail(cudaError_t e, const char *what)
{
    std::fprintf(stderr, "libfdtd: fdtd_systolic_step_noalloc: %s: %s\n", what, cudaGetErrorString(e));
    return FDTD_ERR_CUDA;
}

// Once per device, with that device current: the device address of the
// scratch array (the symbol itself is only a host-side stand-in), the kernel's
// shared-memory opt-in, and the number of co-resident CTAs.
fdtd_status setup_device(int dev, DeviceState *&out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        e = systolic_configure(NOALLOC_VARIANT, FDTD_STORAGE_F32, false);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        const int per_sm = systolic_max_ctas_per_sm(NOALLOC_VARIANT, FDTD_STORAGE_F32, false);
        if (per_sm < 1) return FDTD_ERR_UNSUPPORTED;
        d.scratch = (unsigned char *)p;
        d.max_ctas = sms * per_sm;
        d.ready = true;
    }
    out = &d;
    return FDTD_OK;
}

long long tiles_for(const fdtd_grid &g, int T)
{
    const SysShape sh = systolic_shape(NOALLOC_VARIANT);
    auto cd = [](long long a, long long b) { return (a + b - 1) / b; };
    return cd((long long)g.nx + T - 1, sh.tx) * cd((long long)g.ny + T - 1, sh.ty) *
           cd((long long)g.nz + T - 1, sh.tz);
}

} // namespace

extern "C" fdtd_status fdtd_systolic_step_noalloc(const fdtd_grid *grid, float *d_fields, const float *d_coef,
                                                  double dt, int64_t n_steps, void *stream)
{
    if (!grid || !d_fields || !d_coef || n_steps < 0 || !(dt > 0.0) || !std::isfinite(dt))
        return FDTD_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return FDTD_ERR_INVALID_ARG;
    // the same extent limit as fdtd_create
    if (grid->nx > (1 << 20) || grid->ny > (1 << 20) || grid->nz > (1 << 20)) return FDTD_ERR_INVALID_ARG;
    if (n_steps == 0) return FDTD_OK;
    const fdtd_grid g = *grid;
    // largest steps-per-launch whose tile grid fits the scratch array
    int T = (int)std::min<int64_t>(n_steps, NOALLOC_MAX_STEPS_PER_LAUNCH);
    while (T > 1 && tiles_for(g, T) > NOALLOC_MAX_TILES) T = (T + 1) / 2;
    if (tiles_for(g, T) > NOALLOC_MAX_TILES) {
        std::fprintf(stderr,
                     "libfdtd: fdtd_systolic_step_noalloc: a %d x %d x %d grid needs %lld tiles, the "
                     "fixed scratch holds %lld\n",
                     g.nx, g.ny, g.nz, tiles_for(g, T), NOALLOC_MAX_TILES);
        return FDTD_ERR_UNSUPPORTED;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return FDTD_ERR_UNSUPPORTED;
    DeviceState *ds = nullptr;
    fdtd_status st = setup_device(dev, ds);
    if (st != FDTD_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> tiles;
    std::vector<long long> count_le;
    int gx = 0, gy = 0, gz = 0;
    systolic_tile_order(g, NOALLOC_VARIANT, T, tiles, count_le, gx, gy, gz);
    const long long G = (long long)gx * gy * gz;
    int *ctrl = (int *)ds->scratch;
    unsigned *progress = (unsigned *)(ds->scratch + NOALLOC_CTRL_BYTES);
    int *order = (int *)(ds->scratch + NOALLOC_CTRL_BYTES + sizeof(unsigned) * (size_t)G);
    // the array keeps the previous call's contents: clear flags and control words
    if ((e = cudaMemsetAsync(ds->scratch, 0, NOALLOC_CTRL_BYTES + sizeof(unsigned) * (size_t)G, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if (!tiles.empty() &&
        (e = cudaMemcpyAsync(order, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");

    const size_t n = (size_t)g.nx * g.ny * g.nz;
    SysLaunch p;
    for (int k = 0; k < 6; ++k) p.f[k] = d_fields + (size_t)k * n;
    p.ce = d_coef;
    p.ca = nullptr;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.pitch = g.nx;  // the caller's dense arrays
    p.fbase = d_fields;
    p.fstride = (long long)n;
    for (int c = 0; c < 6; ++c) p.sc.s[c] = p.sc.is[c] = 1.f;  // FP32 storage
    p.sc.src = 1.f;
    p.xf = p.yf = nullptr;  // the shared-memory kernel keeps its faces in the field arrays
    p.fxs = p.fys = 0;
    p.nzb = p.nzblk = 0;
    p.cap = nullptr;
    p.cap_bc = 0;
    p.gx = gx;
    p.gy = gy;
    p.gz = gz;
    p.tiles = order;
    p.progress = progress;
    p.ctrl = ctrl;
    p.neg_dt = -(float)dt;
    p.timeout_ns = 2000000000ll;
    p.dbg_kind = 0;
    p.dbg_ticket = p.dbg_param = p.dbg_param2 = 0;
    p.src.n = 0;
    unsigned epoch = 1;
    long long step = 0;
    while (n_steps > 0) {
        const int Tl = (int)std::min<int64_t>(n_steps, T);
        if (epoch + (unsigned)Tl + 1u > (1u << 30)) {  // keep flag values far from wrap-around
            if ((e = cudaMemsetAsync(progress, 0, sizeof(unsigned) * (size_t)G, s)) != cudaSuccess)
                return cuda_fail(e, "cudaMemsetAsync");
            epoch = 1;
        }
        if ((e = cudaMemsetAsync(ctrl, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        p.T = Tl;
        p.epoch = epoch;
        p.step0 = step;
        p.ntiles = (int)count_le[(size_t)Tl];
        const int grid_ctas = (int)std::max<long long>(1, std::min<long long>(p.ntiles, ds->max_ctas));
        if ((e = launch_systolic(p, grid_ctas, s, NOALLOC_VARIANT, FDTD_STORAGE_F32)) != cudaSuccess) return cuda_fail(e, "launch");
        epoch += (unsigned)Tl + 1u;
        step += Tl;
        n_steps -= Tl;
    }
    int host_ctrl[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(host_ctrl, ctrl, sizeof(host_ctrl), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return host_ctrl[1] != DEV_OK ? FDTD_ERR_TIMEOUT : FDTD_OK;
}
