// Internal declarations shared by the host API and the kernels of libfdtd.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <algorithm>
#include <vector>

#include "fdtd.h"
#include "storage.cuh"

#define FDTD_MAX_SOURCES 16

// Device error word values (ctrl[1]); anything non-zero stops every CTA.
enum : int { DEV_OK = 0, DEV_ERR_TIMEOUT = 1 };

// A point source as the kernels see it: E component `comp` of cell
// (i,j,k) receives amp[n] after the E half-step of absolute step n < n_amp.
struct SrcDesc {
    int comp, i, j, k;
    long long idx;           // i + pitch*(j + ny*k)
    long long n_amp;
    const float *amp;
};

struct SrcSet {
    int n;
    SrcDesc s[FDTD_MAX_SOURCES];
};

// Naive scheme: one H launch and one E launch per step.
// Arrays are nx*ny*nz cells with rows of `pitch` elements (pitch >= nx) in
// kernel format `fmt` (FDTD_STORAGE_* or FMT_*U of storage.cuh); dt/eps is
// always FP32.
cudaError_t launch_naive_h(void *const f[6], int fmt, int nx, int ny, int nz, int pitch, float neg_dt,
                           const Scales &sc, cudaStream_t st);
// ca: per-cell E decay of conducting cells (absorber), or null when lossless;
// ce then holds cb.
cudaError_t launch_naive_e(void *const f[6], int fmt, const float *ce, const float *ca, int nx, int ny, int nz,
                           int pitch, long long step, const SrcSet &src, const Scales &sc, cudaStream_t st);

// Naive scheme on a domain of at most naive_block_max_cells() cells: one
// CTA, one thread per cell, `nsteps` steps in one launch (block barriers
// between the half-steps).
int naive_block_max_cells();
cudaError_t launch_naive_block(void *const f[6], int fmt, const float *ce, const float *ca, int nx, int ny, int nz,
                               int pitch, float neg_dt, long long step0, int nsteps, const SrcSet &src,
                               const Scales &sc, cudaStream_t st);

// FP32 <-> storage conversion of one component (convert.cu): `dense` holds
// nx*ny*nz values, `pitched` rows of `pitch` elements.
cudaError_t launch_to_storage(void *pitched, const float *dense, int storage, int nx, int ny, int nz, int pitch,
                              float inv_scale, cudaStream_t st);
cudaError_t launch_from_storage(float *dense, const void *pitched, int storage, int nx, int ny, int nz,
                                int pitch, float scale, cudaStream_t st);

// Systolic scheme: the subdomain ("tile") geometry is a compile-time ring of
// 32 x RY x RZ shared-memory slots per CTA of which 31 x (RY-1) x (RZ-1)
// cells are updated per step.  Shape 0 is the paper's 31 x 15 x 15 updated /
// 32 x 16 x 16 stored tile (one CTA per SM); shape 1 is 31 x 7 x 15 (two CTAs
// per SM, so one hides the other's waits and barriers).
struct SysShape { int tx, ty, tz; };
constexpr int SYS_NSHAPES = 4;  // 2, 3: register-resident kernel, 31 x 15 x 12 / x 8 (systolic_reg.cu)
SysShape systolic_shape(int variant);
SysShape systolic_reg_shape(int k);
// cl: CTAs per thread-block cluster along x (1, or 2 for x pairs of the
// 31 x 15 x 12 lossless tile)
cudaError_t systolic_reg_configure(int k, int fmt, bool lossy, int cl);
int systolic_reg_max_ctas_per_sm(int k, int fmt, bool lossy);
int systolic_reg_max_pairs(int k, int fmt);  // co-resident x-pair clusters, 0 if unsupported

struct SysLaunch {
    float *f[6];             // field arrays (elements of the storage format; FP32 for the
                             // shared-memory kernel)
    const float *ce;         // dt/eps, or cb in conducting cells
    const float *ca;         // E decay per cell (absorber), null when lossless
    int nx, ny, nz;
    int pitch;               // elements between consecutive x rows (>= nx)
    float *fbase;            // f[c] == fbase + c*fstride elements for c in 0..5 when the
    long long fstride;       // arrays sit at a uniform stride (else fstride == 0)
    Scales sc;               // storage scales (16-bit formats)
    // top x and y faces of the register kernel, in z-blocks: component c of
    // column (x, y), rows of z-block kb (of nzblk) at
    //   x faces: xf + c*fxs + ((kb*nx + x)*ny + y)*BZ + r,
    //   y faces: yf + c*fys + ((kb*ny + y)*nx + x)*BZ + r,
    // BZ = the tile's z rows rounded up to 16 bytes, nzb = nzblk*BZ (the
    // field arrays never carry these faces)
    float *xf, *yf;
    long long fxs, fys;
    int nzb, nzblk;
    int gx, gy, gz;          // tile grid over skewed space sigma = p + t
    int T;                   // steps of this launch
    unsigned epoch;          // progress values of this launch are epoch + k
    long long step0;         // absolute step at launch start
    const int *tiles;        // ticket -> linear tile id, topological order
    int ntiles;
    unsigned *progress;      // per linear tile id
    int *ctrl;               // [0] ticket counter, [1] error word, [2..] error info
    float neg_dt;
    long long timeout_ns;
    int dbg_kind;
    long long dbg_ticket, dbg_param, dbg_param2;
    SrcSet src;
    // register kernel, optional: the E of the cells of box [cap_lo, cap_hi)
    // after every step t of the launch into cap + 3*cap_bc*t (component a at
    // + a*cap_bc, box cells x fastest), for the adjoint's recompute; null = off
    float *cap;
    int cap_lo[3], cap_hi[3];
    long long cap_bc;
    // bulk-tensor (TMA) maps of the register kernel's shell staging:
    // [shell][0] the six fields, [shell][1] the FP32 coefficients cb (dt/eps)
    // and, when lossy, ca, each with the array index as a 4th dimension;
    // shells = lower z, y, x
    CUtensorMap tm[3][2];
};

// Encode the shell maps of the register kernel with `nr` z rows per column
// and z-blocks of `bz` elements: the lower z shell of the six fields (storage
// format `storage`, at fbase + c*fstride elements, rows of `pitch`
// elements), their lower y and x shells from the face buffers yf and xf
// (z-block extent nzb, see SysLaunch), and the lower z, y and x shells of the
// FP32 coefficients ce (and ca, at any 16-byte multiple after ce).  One map
// covers all arrays of a kind (4th dimension), so one bulk copy fetches a
// shell of all of them.  Returns false on failure.
bool encode_shell_maps(CUtensorMap tm[3][2], void *fbase, long long fstride, const float *ce, const float *ca,
                       int storage, int nx, int ny, int nz, int pitch, int nr, int bz, void *xf, long long fxs,
                       void *yf, long long fys, int nzb);
int systolic_reg_rows(int k);
// z-block length of the face buffers for a tile of nz_tile rows and fields of
// eb bytes: nz_tile rounded up to a whole number of 16-byte chunks
inline int face_block(int nz_tile, int eb) { return (nz_tile * eb + 15) / 16 * 16 / eb; }

size_t systolic_smem_bytes(int variant);
// `fmt` is a kernel format code as for the naive scheme; the shared-memory
// variants (0, 1) take FP32 only.
// Lossy (absorber) launches need the register kernel (variant >= 2).
cudaError_t systolic_configure(int variant, int fmt, bool lossy, int cl = 1);
int systolic_max_ctas_per_sm(int variant, int fmt, bool lossy);
// `grid` CTAs; with cl = 2 a multiple of 2 (one cluster per x pair of tiles)
cudaError_t launch_systolic(const SysLaunch &p, int grid, cudaStream_t st, int variant, int fmt, int cl = 1);
cudaError_t launch_systolic_reg(const SysLaunch &p, int grid, cudaStream_t st, int k, int fmt, int cl);

// Tile order for one systolic launch of up to T steps (fdtd_api.cu), single
// tiles (clusters of one).
void systolic_tile_order(const fdtd_grid &g, int variant, int T, std::vector<int> &tiles,
                         std::vector<long long> &count_le, int &gx, int &gy, int &gz);
