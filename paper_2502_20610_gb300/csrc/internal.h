// Internal declarations shared by the host API and the kernels of libfdtd.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <vector>

#include "fdtd.h"

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
// Arrays are nx*ny*nz cells with rows of `pitch` floats (pitch >= nx).
cudaError_t launch_naive_h(float *const f[6], int nx, int ny, int nz, int pitch, float neg_dt,
                           cudaStream_t st);
cudaError_t launch_naive_e(float *const f[6], const float *ce, int nx, int ny, int nz, int pitch,
                           long long step, const SrcSet &src, cudaStream_t st);

// Systolic scheme: the subdomain ("tile") geometry is a compile-time ring of
// 32 x RY x RZ shared-memory slots per CTA of which 31 x (RY-1) x (RZ-1)
// cells are updated per step.  Shape 0 is the paper's 31 x 15 x 15 updated /
// 32 x 16 x 16 stored tile (one CTA per SM); shape 1 is 31 x 7 x 15 (two CTAs
// per SM, so one hides the other's waits and barriers).
struct SysShape { int tx, ty, tz; };
constexpr int SYS_NSHAPES = 4;  // 2, 3: register-resident kernel, 31 x 15 x 12 / x 8 (systolic_reg.cu)
SysShape systolic_shape(int variant);
SysShape systolic_reg_shape(int k);
cudaError_t systolic_reg_configure(int k);
int systolic_reg_max_ctas_per_sm(int k);

struct SysLaunch {
    float *f[6];
    const float *ce;
    int nx, ny, nz;
    int pitch;               // floats between consecutive x rows (>= nx)
    float *fbase;            // f[c] == fbase + c*fstride for c in 0..5 and ce == fbase + 6*fstride,
    long long fstride;       // when the arrays sit at a uniform stride (else fstride == 0)
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
    // bulk-tensor (TMA) maps of the 6 fields and dt/eps, for the register
    // kernel's shell staging: [shape][array], shapes = lower z, y, x shell
    CUtensorMap tm[3][7];
};

// Encode the 21 shell maps of the register kernel with `nr` z rows per
// column; fbase/fstride/pitch as in SysLaunch.  Returns false on failure.
bool encode_shell_maps(CUtensorMap tm[3][7], float *fbase, long long fstride, int nx, int ny, int nz,
                       int pitch, int nr);
int systolic_reg_rows(int k);

size_t systolic_smem_bytes(int variant);
cudaError_t systolic_configure(int variant);
int systolic_max_ctas_per_sm(int variant);
cudaError_t launch_systolic(const SysLaunch &p, int grid, cudaStream_t st, int variant);
cudaError_t launch_systolic_reg(const SysLaunch &p, int grid, cudaStream_t st, int k);

// Tile order for one systolic launch of up to T steps (fdtd_api.cu).
void systolic_tile_order(const fdtd_grid &g, int variant, int T, std::vector<int> &tiles,
                         std::vector<long long> &count_le, int &gx, int &gy, int &gz);
