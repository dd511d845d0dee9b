// Learned-boundary network: sizes, parameter layout and the internal entry
// points of mlp.cu.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

namespace mlpnet {
constexpr int NI = 324, NH = 64, NO = 6;  // 3x3x3 stencil x 6 fields x 2 steps -> 64 -> 64 -> 6
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;
constexpr float R_MIN = 1e-30f;  // smaller stencil RMS counts as a zero stencil
} // namespace mlpnet

// Scratch of the forward / gradient / training calls for minibatches of
// `batch` samples over a set of n samples (the training permutation).
size_t mlp_scratch_bytes(int batch, long long n);
cudaError_t mlp_forward(const float *params, const float *X, long long n, float *Y, void *scratch, int batch,
                        cudaStream_t st);
cudaError_t mlp_grad(const float *params, const float *X, const float *T, int n, float *grad, double *loss_host,
                     void *scratch, int batch, cudaStream_t st);
cudaError_t mlp_train(float *params, const float *X, const float *T, long long n, int batch, int epochs, double lr,
                      unsigned long long seed, void *scratch, cudaStream_t st, double *last_epoch_loss);
// ce, ca (nullable): the reference's E coefficients, for the box's own Yee
// step of each recorded cell.
cudaError_t mlp_record(const float *prev, const float *cur, const float *nxt, long long fstride, int pitch, int ny,
                       const int lo[3], const int hi[3], const int *cells, int n, const float *ce, const float *ca,
                       float neg_dt, float *X, float *Y, cudaStream_t st);

// Layer update of a simulation step (FP32 fields at f + c*fstride, rows of
// `pitch`): corrections r f for `ncells` layer cells (x,y,z triplets) from
// the current and previous band snapshots (each followed by its x slab,
// below) into out [ncells][6]; scatter adds them to the cells after the Yee
// step.
size_t learned_layer_smem();
cudaError_t learned_layer_configure();
cudaError_t learned_layer_predict(const float *params, const float *cur, const float *prev, long long fstride,
                                  int pitch, int nx, int ny, int nz, const int *cells, int ncells, float *out,
                                  int grid, cudaStream_t st);
cudaError_t learned_layer_scatter(float *f, long long fstride, int pitch, int ny, const int *cells, int ncells,
                                  const float *vals, cudaStream_t st);
cudaError_t learned_copy_cells(float *dst, const float *src, long long fstride, int pitch, int ny, const int *cells,
                               int ncells, cudaStream_t st);
// A band snapshot (6 * fstride floats) is followed by its x slab: the planes
// x = 0, 1, nx-2, nx-1 of the six components, y fastest, which the layer
// update reads for the cells on the two x faces.  learned_fill_xslab copies
// them from the fields f into the slab of `snap`.
size_t learned_xslab_bytes(int ny, int nz);
cudaError_t learned_fill_xslab(float *snap, const float *f, long long fstride, int pitch, int nx, int ny, int nz,
                               cudaStream_t st);
