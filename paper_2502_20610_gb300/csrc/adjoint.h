// Adjoint kernels of adjoint.cu (FP32 fields and adjoint state in the
// workspace layout: component c at base + c*fstride, rows of `pitch`).
#pragma once

#include <cuda_runtime.h>

struct AdjGeo {
    int nx, ny, nz, pitch;
    long long fstride;
};

// The objective's source in the adjoint's transformed variables
// (Et = M c lambda_E): ez(i,j,k0) += M c(i,j,k0) amp2 mode(i,j), where ez is
// the Ez component of a state in the workspace layout.
cudaError_t adjoint_plane_source(const AdjGeo &g, float *ez, const float *ce, int k0, const float *mode, double amp2,
                                 cudaStream_t st);
// grad[b] -= (1/dt) sum_a Et_a^{q+1}(b) (E^{q+1} - E^q)_a(b) over the steps q
// of a segment of `len` steps, last step first: e_hist planes 0..len hold the
// box's E from the segment's first step on, et_hist planes 0..len-1 its Et
// from the segment's last step back ([plane][3][box cells], x fastest).
cudaError_t adjoint_gradient(const float *et_hist, const float *e_hist, long long box_cells, int len, double dt,
                             double *grad, cudaStream_t st);
// out[w] = sum m(i,j) Ez_w(i,j) for n captured planes [w][3][plane cells]
// (component 2 = Ez), each in the same fixed order as adjoint_overlap
cudaError_t adjoint_overlaps(const float *planes, long long plane_cells, int n, const float *mode, double *out,
                             cudaStream_t st);
// *out = sum m(i,j) Ez(i,j,k0), in a fixed order (reproducible)
cudaError_t adjoint_overlap(const AdjGeo &g, const float *ez, int k0, const float *mode, double *out, cudaStream_t st);
cudaError_t adjoint_box_copy(const AdjGeo &g, const float *f, const int lo[3], const int hi[3], float *dst,
                             cudaStream_t st);
