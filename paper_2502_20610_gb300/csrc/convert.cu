// FP32 <-> storage-format conversion of one field component, used by
// fdtd_write_fields / fdtd_read_fields when fields are stored as FP16 or
// BF16: q = fl_S(v / s) on the way in (round to nearest even), v = s * q on
// the way out (exact).  Dense arrays hold nx*ny*nz values; the device arrays
// have rows of `pitch` elements.
#include "internal.h"
#include "storage.cuh"

namespace {

template <class S>
__global__ void to_storage_kernel(typename S::T *__restrict__ dst, const float *__restrict__ src, int nx,
                                  long long rows, int pitch, float inv_s)
{
    const long long n = (long long)nx * rows;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / nx, x = q - r * nx;
        dst[x + r * pitch] = S::enc(src[q], inv_s);
    }
}

template <class S>
__global__ void from_storage_kernel(float *__restrict__ dst, const typename S::T *__restrict__ src, int nx,
                                    long long rows, int pitch, float s)
{
    const long long n = (long long)nx * rows;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / nx, x = q - r * nx;
        dst[q] = S::dec(src[x + r * pitch], s);
    }
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

} // namespace

cudaError_t launch_to_storage(void *pitched, const float *dense, int storage, int nx, int ny, int nz, int pitch,
                              float inv_scale, cudaStream_t st)
{
    const long long rows = (long long)ny * nz, n = (long long)nx * rows;
    if (n == 0) return cudaSuccess;
    if (storage == FDTD_STORAGE_F16)
        to_storage_kernel<StoreF16><<<blocks_for(n), 256, 0, st>>>((unsigned short *)pitched, dense, nx, rows, pitch,
                                                                    inv_scale);
    else if (storage == FDTD_STORAGE_BF16)
        to_storage_kernel<StoreBF16><<<blocks_for(n), 256, 0, st>>>((unsigned short *)pitched, dense, nx, rows,
                                                                     pitch, inv_scale);
    else
        to_storage_kernel<StoreF32><<<blocks_for(n), 256, 0, st>>>((float *)pitched, dense, nx, rows, pitch,
                                                                    inv_scale);
    return cudaGetLastError();
}

cudaError_t launch_from_storage(float *dense, const void *pitched, int storage, int nx, int ny, int nz,
                                int pitch, float scale, cudaStream_t st)
{
    const long long rows = (long long)ny * nz, n = (long long)nx * rows;
    if (n == 0) return cudaSuccess;
    if (storage == FDTD_STORAGE_F16)
        from_storage_kernel<StoreF16><<<blocks_for(n), 256, 0, st>>>(dense, (const unsigned short *)pitched, nx,
                                                                      rows, pitch, scale);
    else if (storage == FDTD_STORAGE_BF16)
        from_storage_kernel<StoreBF16><<<blocks_for(n), 256, 0, st>>>(dense, (const unsigned short *)pitched, nx,
                                                                       rows, pitch, scale);
    else
        from_storage_kernel<StoreF32><<<blocks_for(n), 256, 0, st>>>(dense, (const float *)pitched, nx, rows,
                                                                      pitch, scale);
    return cudaGetLastError();
}
