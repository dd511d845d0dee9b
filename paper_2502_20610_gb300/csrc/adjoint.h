// Adjoint kernels of adjoint.cu (FP32 fields and adjoint state in the
// workspace layout: component c at base + c*fstride, rows of `pitch`).
#pragma once

#include <cuda_runtime.h>

struct AdjGeo {
    int nx, ny, nz, pitch;
    long long fstride;
};

// lambda (6 components, E then H): lambda_H += curl_f(M c lambda_E), and the
// gradient of the box [lo, hi) from lambda_E and the box's E at steps n+1
// (e_next) and n (e_now), [3][box cells], FP64 into grad [box cells].
cudaError_t adjoint_h(const AdjGeo &g, float *lam, const float *ce, const int lo[3], const int hi[3],
                      const float *e_next, const float *e_now, float dt, double *grad, cudaStream_t st);
// lambda_E -= dt curl_b lambda_H, plus amp2 * mode(i,j) on Ez of plane k0.
cudaError_t adjoint_e(const AdjGeo &g, float *lam, float dt, int k0, const float *mode, double amp2, cudaStream_t st);
// Both of the above in one kernel (same FP32 results): the adjoint state
// (6 components, E then H) from lam_old into lam_new.
cudaError_t adjoint_step(const AdjGeo &g, const float *lam_old, float *lam_new, const float *ce, const int lo[3],
                         const int hi[3], const float *e_next, const float *e_now, float dt, double *grad, int k0,
                         const float *mode, double amp2, cudaStream_t st);
// out[w] = sum m(i,j) Ez_w(i,j) for n captured planes [w][3][plane cells]
// (component 2 = Ez), each in the same fixed order as adjoint_overlap
cudaError_t adjoint_overlaps(const float *planes, long long plane_cells, int n, const float *mode, double *out,
                             cudaStream_t st);
// *out = sum m(i,j) Ez(i,j,k0), in a fixed order (reproducible)
cudaError_t adjoint_overlap(const AdjGeo &g, const float *ez, int k0, const float *mode, double *out, cudaStream_t st);
cudaError_t adjoint_box_copy(const AdjGeo &g, const float *f, const int lo[3], const int hi[3], float *dst,
                             cudaStream_t st);
