// Learned absorbing boundary: the network's kernels.
//
// The network (2 hidden layers of 64, FP32, tanh) maps the 3x3x3 stencil of
// the six fields at steps n and n-1 around a cell of the wall layer (324
// inputs) to a correction of that cell's Yee step.  Every cell of the
// domain takes the Yee step with the domain's PEC walls (Yee_D); a layer
// cell then adds the correction, scale-equivariantly: with
// r = sqrt(mean(x^2)) the network sees x / r and
//     S^{n+1}(centre) = Yee_D(S^n)(centre) + r * f(x / r),
// so a wave of any amplitude meets the same boundary operator (the update is
// linear in the fields), and f = 0 is the plain PEC box.  Only the values
// the box's own walls get wrong are corrected: on a cell of a low face the
// two E components tangential to it (PEC holds them), on a cell of a high
// face the two tangential H components (PEC reads E beyond it as 0).  Every
// other value of the box's Yee step is exact, so its correction is zero
// (tangent_mask).  A stencil with r < R_MIN (1e-30, where 1/r would
// leave the FP32 range) counts as zero: the cell keeps its value.  Parameters, in this order: W1 [64][324], b1 [64],
// W2 [64][64], b2 [64], W3 [6][64], b3 [6] (row = output unit).
//
// Training runs on the GPU with these kernels: a tiled FP32 GEMM with
// bias / tanh / tanh-derivative epilogues for the forward and backward
// passes, column sums for the bias gradients, and Adam.  The layer update of
// a simulation step is one fused persistent kernel: it gathers the stencils
// of 64 layer cells into shared memory and runs the three layers on them
// with the weights resident in shared memory, the two large contractions on
// the tensor cores (mma.sync TF32, three-term split for FP32 accuracy).
#include "internal.h"
#include "mlp.h"
#include "yee_cell.cuh"

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

namespace {

using namespace mlpnet;

// ------------------------------------------------------------------ GEMM

// C[m][n] = epi(sum_k A(m,k) B(k,n)) with
//   A(m,k) = A[ra(m)*sam + k*sak], ra(m) = arows ? arows[m] : m,
//   B(k,n) = B[rb(k)*sbk + n*sbn], rb(k) = brows ? brows[k] : k.
struct GemmArgs {
    int M, N, K;
    const float *A;
    long long sam, sak;
    const int *arows;
    const float *B;
    long long sbk, sbn;
    const int *brows;
    float *C;
    long long ldc;
    const float *bias;  // [N]
    const float *aux;   // [M][ldaux]: the layer's activation (EPI_DTANH)
    long long ldaux;
};

enum { EPI_NONE = 0, EPI_BIAS_TANH = 1, EPI_BIAS = 2, EPI_DTANH = 3 };

constexpr int GT = 64, GK = 16;

template <int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs g)
{
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tm = tid >> 4, tn = tid & 15;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < g.K; k0 += GK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int mm = e >> 4, kk = e & 15;
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < g.M && k < g.K) {
                const long long r = g.arows ? g.arows[m] : m;
                v = g.A[r * g.sam + (long long)k * g.sak];
            }
            As[kk][mm] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int kk = e >> 6, nn = e & 63;
            const int k = k0 + kk, n = n0 + nn;
            float v = 0.f;
            if (k < g.K && n < g.N) {
                const long long r = g.brows ? g.brows[k] : k;
                v = g.B[r * g.sbk + (long long)n * g.sbn];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tm * 4 + i, n = n0 + tn * 4 + j;
            if (m >= g.M || n >= g.N) continue;
            float v = acc[i][j];
            if (EPI == EPI_BIAS_TANH) v = tanhf(__fadd_rn(v, g.bias[n]));
            if (EPI == EPI_BIAS) v = __fadd_rn(v, g.bias[n]);
            if (EPI == EPI_DTANH) {
                const float h = g.aux[(long long)m * g.ldaux + n];
                v = __fmul_rn(v, __fsub_rn(1.f, __fmul_rn(h, h)));
            }
            g.C[(long long)m * g.ldc + n] = v;
        }
}

template <int EPI>
cudaError_t gemm(const GemmArgs &g, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT);
    gemm_kernel<EPI><<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
}

GemmArgs ga(int M, int N, int K, const float *A, long long sam, long long sak, const int *arows, const float *B,
            long long sbk, long long sbn, const int *brows, float *C, long long ldc, const float *bias = nullptr,
            const float *aux = nullptr, long long ldaux = 0)
{
    GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sam = sam; g.sak = sak; g.arows = arows;
    g.B = B; g.sbk = sbk; g.sbn = sbn; g.brows = brows;
    g.C = C; g.ldc = ldc; g.bias = bias; g.aux = aux; g.ldaux = ldaux;
    return g;
}

// out[n] = sum_m A[m][n] (A is M x N row-major), one block per column
__global__ void __launch_bounds__(256) colsum_kernel(const float *__restrict__ A, int M, int N,
                                                     float *__restrict__ out)
{
    __shared__ float part[256];
    const int n = blockIdx.x;
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += 256) s = __fadd_rn(s, A[(long long)m * N + n]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] = __fadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = part[0];
}

// dY = 2 (Y - T[rows]) / (B * 6); loss += sum (Y - T)^2 (FP64)
__global__ void __launch_bounds__(256) dy_kernel(const float *__restrict__ Y, const float *__restrict__ T,
                                                 const int *__restrict__ rows, int B, float *__restrict__ dY,
                                                 double *__restrict__ loss)
{
    __shared__ double part[256];
    const int e = blockIdx.x * 256 + threadIdx.x;
    double s = 0.0;
    if (e < B * NO) {
        const int b = e / NO, o = e - b * NO;
        const long long r = rows ? rows[b] : b;
        const float d = __fsub_rn(Y[e], T[r * NO + o]);
        dY[e] = __fmul_rn(d, 2.f / (float)(B * NO));
        s = (double)d * (double)d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0]);
}

// Adam (Kingma & Ba): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v, int n, float lr,
                                                   float c1, float c2)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------- forward / backward pass

struct Scratch {
    float *H1, *H2, *Y, *dY, *dZ2, *dZ1, *grad, *m, *v;
    double *loss;
    int *rows;  // the training permutation (n entries)
};

size_t scratch_bytes(int batch, long long n)
{
    const size_t b = (size_t)batch;
    return sizeof(float) * (b * NH * 4 + b * NO * 2 + 3 * (size_t)NPARAM) + sizeof(double) * 2 +
           sizeof(int) * (size_t)n + 12 * 256;
}

Scratch carve(void *base, int batch, long long n)
{
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    const size_t b = (size_t)batch;
    Scratch s;
    s.loss = (double *)take(sizeof(double) * 2);
    s.H1 = (float *)take(sizeof(float) * b * NH);
    s.H2 = (float *)take(sizeof(float) * b * NH);
    s.dZ2 = (float *)take(sizeof(float) * b * NH);
    s.dZ1 = (float *)take(sizeof(float) * b * NH);
    s.Y = (float *)take(sizeof(float) * b * NO);
    s.dY = (float *)take(sizeof(float) * b * NO);
    s.grad = (float *)take(sizeof(float) * NPARAM);
    s.m = (float *)take(sizeof(float) * NPARAM);
    s.v = (float *)take(sizeof(float) * NPARAM);
    s.rows = (int *)take(sizeof(int) * (size_t)n);
    return s;
}

#define CKE(x)                                                                 \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess) return e_;                                      \
    } while (0)

// H1, H2, Y of B samples X[rows[b]] (rows may be null).
cudaError_t forward(const float *P, const float *X, const int *rows, int B, const Scratch &s, float *Y,
                    cudaStream_t st)
{
    CKE(gemm<EPI_BIAS_TANH>(ga(B, NH, NI, X, NI, 1, rows, P + OFF_W1, 1, NI, nullptr, s.H1, NH, P + OFF_B1), st));
    CKE(gemm<EPI_BIAS_TANH>(ga(B, NH, NH, s.H1, NH, 1, nullptr, P + OFF_W2, 1, NH, nullptr, s.H2, NH, P + OFF_B2),
                            st));
    CKE(gemm<EPI_BIAS>(ga(B, NO, NH, s.H2, NH, 1, nullptr, P + OFF_W3, 1, NH, nullptr, Y, NO, P + OFF_B3), st));
    return cudaSuccess;
}

// Gradient of the mean squared error of B samples into s.grad; adds the
// sum of squared errors to *s.loss.
cudaError_t backward(const float *P, const float *X, const float *T, const int *rows, int B, const Scratch &s,
                     cudaStream_t st)
{
    CKE(forward(P, X, rows, B, s, s.Y, st));
    dy_kernel<<<(B * NO + 255) / 256, 256, 0, st>>>(s.Y, T, rows, B, s.dY, s.loss);
    CKE(cudaGetLastError());
    float *G = s.grad;
    // layer 3: dW3 = dY^T H2, db3 = sum dY, dZ2 = (dY W3) * (1 - H2^2)
    CKE(gemm<EPI_NONE>(ga(NO, NH, B, s.dY, 1, NO, nullptr, s.H2, NH, 1, nullptr, G + OFF_W3, NH), st));
    colsum_kernel<<<NO, 256, 0, st>>>(s.dY, B, NO, G + OFF_B3);
    CKE(gemm<EPI_DTANH>(ga(B, NH, NO, s.dY, NO, 1, nullptr, P + OFF_W3, NH, 1, nullptr, s.dZ2, NH, nullptr, s.H2, NH),
                        st));
    // layer 2
    CKE(gemm<EPI_NONE>(ga(NH, NH, B, s.dZ2, 1, NH, nullptr, s.H1, NH, 1, nullptr, G + OFF_W2, NH), st));
    colsum_kernel<<<NH, 256, 0, st>>>(s.dZ2, B, NH, G + OFF_B2);
    CKE(gemm<EPI_DTANH>(ga(B, NH, NH, s.dZ2, NH, 1, nullptr, P + OFF_W2, NH, 1, nullptr, s.dZ1, NH, nullptr, s.H1, NH),
                        st));
    // layer 1
    CKE(gemm<EPI_NONE>(ga(NH, NI, B, s.dZ1, 1, NH, nullptr, X, NI, 1, rows, G + OFF_W1, NI), st));
    colsum_kernel<<<NH, 256, 0, st>>>(s.dZ1, B, NH, G + OFF_B1);
    return cudaGetLastError();
}

// Components of cell (x,y,z) that the correction applies to (bit c = Ex..Hz):
// tangential E on the low faces, tangential H on the high faces it lies on.
__device__ __forceinline__ unsigned tangent_mask(int x, int y, int z, int nx, int ny, int nz)
{
    unsigned m = 0;
    if (x == 0) m |= 0x6;         // Ey, Ez
    if (y == 0) m |= 0x5;         // Ex, Ez
    if (z == 0) m |= 0x3;         // Ex, Ey
    if (x == nx - 1) m |= 0x30;   // Hy, Hz
    if (y == ny - 1) m |= 0x28;   // Hx, Hz
    if (z == nz - 1) m |= 0x18;   // Hx, Hy
    return m;
}

// ---------------------------------------------------- sample recording

// Yee step of the centre of a stencil of S^n (v: [c][dz][dy][dx], 0 outside
// the box) in the box standing alone with PEC walls: tangential E on the
// box's low faces stays, E and H beyond it read 0.  Same operations as the
// naive kernels (yee_cell.cuh).
__device__ void yee_centre(const float *v, float ndt, float cb, float ca, bool lossy, bool lo_x, bool lo_y, bool lo_z,
                           float out[6])
{
    auto V = [&](int c, int dx, int dy, int dz) { return v[c * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; };
    // H^{n+1/2} at offset o from the E^n and H^{n-1/2} of the stencil
    auto Hx = [&](int dx, int dy, int dz) {
        return h_x(V(3, dx, dy, dz), V(2, dx, dy + 1, dz), V(2, dx, dy, dz), V(1, dx, dy, dz + 1), V(1, dx, dy, dz), ndt);
    };
    auto Hy = [&](int dx, int dy, int dz) {
        return h_y(V(4, dx, dy, dz), V(0, dx, dy, dz + 1), V(0, dx, dy, dz), V(2, dx + 1, dy, dz), V(2, dx, dy, dz), ndt);
    };
    auto Hz = [&](int dx, int dy, int dz) {
        return h_z(V(5, dx, dy, dz), V(1, dx + 1, dy, dz), V(1, dx, dy, dz), V(0, dx, dy + 1, dz), V(0, dx, dy, dz), ndt);
    };
    const float hx = Hx(0, 0, 0), hy = Hy(0, 0, 0), hz = Hz(0, 0, 0);
    const float ex = V(0, 0, 0, 0), ey = V(1, 0, 0, 0), ez = V(2, 0, 0, 0);
    const float dex = lossy ? __fmul_rn(ca, ex) : ex, dey = lossy ? __fmul_rn(ca, ey) : ey,
                dez = lossy ? __fmul_rn(ca, ez) : ez;
    out[0] = (lo_y || lo_z) ? ex : e_x(dex, hz, Hz(0, -1, 0), hy, Hy(0, 0, -1), cb);
    out[1] = (lo_x || lo_z) ? ey : e_y(dey, hx, Hx(0, 0, -1), hz, Hz(-1, 0, 0), cb);
    out[2] = (lo_x || lo_y) ? ez : e_z(dez, hy, Hy(-1, 0, 0), hx, Hx(0, -1, 0), cb);
    out[3] = hx;
    out[4] = hy;
    out[5] = hz;
}

// Training pairs from a reference run: for cells (x,y,z) of the layer region
// (inside the box [lo, hi) of the reference grid), the normalised stencil of
// (S^n, S^{n-1}) -- cells outside the box read 0, as they would at a wall --
// and the normalised correction (S^{n+1} - Yee_box(S^n))(centre) / r that
// takes the box's own Yee step to the reference's next state.
__global__ void __launch_bounds__(256) record_kernel(const float *__restrict__ prev, const float *__restrict__ cur,
                                                     const float *__restrict__ nxt, long long fstride, int pitch,
                                                     int ny, int3 lo, int3 hi, const int *__restrict__ cells, int n,
                                                     const float *__restrict__ ce, const float *__restrict__ ca,
                                                     float ndt, float *__restrict__ X, float *__restrict__ Y)
{
    const int q = blockIdx.x * 256 + threadIdx.x;
    if (q >= n) return;
    const int x = cells[3 * q], y = cells[3 * q + 1], z = cells[3 * q + 2];
    float *xo = X + (long long)q * NI;
    double ss = 0.0;
    for (int s = 0; s < 2; ++s) {
        const float *F = s == 0 ? cur : prev;
        for (int c = 0; c < 6; ++c)
            for (int d = 0; d < 27; ++d) {
                const int xx = x + d % 3 - 1, yy = y + (d / 3) % 3 - 1, zz = z + d / 9 - 1;
                float v = 0.f;
                if (xx >= lo.x && xx < hi.x && yy >= lo.y && yy < hi.y && zz >= lo.z && zz < hi.z)
                    v = F[c * fstride + xx + (long long)pitch * (yy + (long long)ny * zz)];
                xo[(s * 6 + c) * 27 + d] = v;
                ss += (double)v * v;
            }
    }
    const long long p = x + (long long)pitch * (y + (long long)ny * z);
    float yee[6];
    yee_centre(xo, ndt, ce[p], ca ? ca[p] : 1.f, ca != nullptr, x == lo.x, y == lo.y, z == lo.z, yee);
    // r below R_MIN counts as a zero stencil (its reciprocal would overflow
    // FP32): the pair is recorded as zeros
    const double r = sqrt(ss / NI);
    const double ir = r >= (double)R_MIN ? 1.0 / r : 0.0;
    for (int k = 0; k < NI; ++k) xo[k] = (float)(xo[k] * ir);
    const unsigned m = tangent_mask(x - lo.x, y - lo.y, z - lo.z, hi.x - lo.x, hi.y - lo.y, hi.z - lo.z);
    for (int c = 0; c < 6; ++c)
        Y[(long long)q * NO + c] = (m >> c) & 1u ? (float)(((double)nxt[c * fstride + p] - (double)yee[c]) * ir) : 0.f;
}

// -------------------------------------------------- layer update (fused)

// Tensor-core contraction of the fused layer kernel: mma.sync m16n8k8 with
// TF32 operands and FP32 accumulation, each operand split in two TF32 terms
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) and the product taken as
// lo*hi + hi*lo + hi*hi ("3xTF32"): ~22 significant bits per operand, the
// dropped lo*lo term below FP32 rounding of the sum, so the layer keeps
// FP32 accuracy.
__device__ __forceinline__ unsigned tf32_rna(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(__fsub_rn(x, __uint_as_float(hi)));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9},"
                 " {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared tiles [k][64] (k = input feature or unit, 64 = cells or units) are
// stored with the column index XOR-swizzled by (k mod 4) * 8, so the
// fragment loads of a warp (rows k .. k+3, eight consecutive columns each)
// hit 32 different banks.
__device__ __forceinline__ int swz(int k, int c) { return c ^ ((k & 3) << 3); }

// D[64 x 64] of this CTA's eight warps (warp w: rows 16*(w%4).., columns
// 32*(w/4).., four m16n8 tiles) = sum_k A[k][row] B[k][col] over K (a
// multiple of 8; A, B swizzled [k][64] tiles in shared memory).
template <int K>
__device__ __forceinline__ void warp_gemm_3xtf32(const float *A, const float *B, float (&acc)[4][4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int m0 = 16 * (w & 3), n0 = 32 * (w >> 2);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
#pragma unroll 2
    for (int k0 = 0; k0 < K; k0 += 8) {
        const int ka = k0 + q, kb = k0 + q + 4;
        unsigned ah[4], al[4];
        split_tf32(A[ka * 64 + swz(ka, m0 + g)], ah[0], al[0]);
        split_tf32(A[ka * 64 + swz(ka, m0 + g + 8)], ah[1], al[1]);
        split_tf32(A[kb * 64 + swz(kb, m0 + g)], ah[2], al[2]);
        split_tf32(A[kb * 64 + swz(kb, m0 + g + 8)], ah[3], al[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 8 * j + g;
            unsigned bh0, bl0, bh1, bl1;
            split_tf32(B[ka * 64 + swz(ka, n)], bh0, bl0);
            split_tf32(B[kb * 64 + swz(kb, n)], bh1, bl1);
            mma_tf32(acc[j], al[0], al[1], al[2], al[3], bh0, bh1);
            mma_tf32(acc[j], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
            mma_tf32(acc[j], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
        }
    }
}

// Shared memory of the fused layer kernel, in floats; the float4-read arrays
// come first, each a multiple of 64 floats, so they stay 16-byte aligned.
constexpr int LC = 64;  // layer cells per tile
constexpr int NIP = 328;  // NI padded to a multiple of 8 (zero rows)
static_assert((NIP - NI) * LC == 256, "one padding float per thread of the layer kernel");
constexpr int SM_W1T = NIP * NH, SM_W2T = NH * NH, SM_W3T = NH * NO, SM_XT = NIP * LC, SM_H = NH * LC;
constexpr size_t LAYER_SMEM =
    sizeof(float) * (SM_W1T + SM_W2T + SM_XT + 2 * SM_H + SM_W3T + 2 * NH + NO + 2 * LC + 4 * LC);

// Asynchronous 4-byte copy, global -> shared (cp.async, cached in L1).  With
// valid == false nothing is read and the shared word is zero-filled; src is
// then still an address inside the field array.
__device__ __forceinline__ void cp_async_4(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Each band snapshot (six components at c * fstride, rows of `pitch`) is
// followed by its x slab: the planes x = 0, 1 (side 0) and x = nx-2, nx-1
// (side 1) of every component, y fastest, [comp][side][xd][z][y], so that
// the stencils of the cells on the two x faces (a full row apart from each
// other in the snapshot) are read with consecutive y across the lanes.
__device__ __host__ __forceinline__ long long xslab_floats(int ny, int nz) { return 24LL * ny * nz; }

// Stage the unnormalised stencils of `tile` into Xt ([k][cell], swizzled)
// with asynchronous copies: thread -> cell q = tid % 64 and three of the
// twelve (level, component) pairs, (tid / 64) * 3 + 0..2, each a 27-cell
// stencil; neighbour offsets are unrolled, validity is per axis, neighbours
// outside the domain and cells past the list are zero.  Cells on an x face
// read the x slab, the others the snapshot itself (same values).
__device__ __forceinline__ void stage_stencils(float *Xt, const float *__restrict__ cur,
                                               const float *__restrict__ prev, long long fstride, int pitch,
                                               int nx, int ny, int nz, const int *__restrict__ cells, int ncells,
                                               int tile)
{
    const int tid = threadIdx.x, q = tid & (LC - 1), p0 = (tid >> 6) * 3;
    const int cell = tile * LC + q;
    if (cell < ncells) {
        const int x = cells[3 * cell], y = cells[3 * cell + 1], z = cells[3 * cell + 2];
        const bool vx[3] = {x > 0, true, x + 1 < nx}, vy[3] = {y > 0, true, y + 1 < ny},
                   vz[3] = {z > 0, true, z + 1 < nz};
        const long long nyz = (long long)ny * nz;
        // address of (x', y', z') of component c: level base + c * cs + o0 + x' sx + y' sy + z' sz
        long long sx = 1, sy = pitch, sz = (long long)pitch * ny, cs = fstride, o0 = 0;
        if (x == 0 || x == nx - 1) {
            const int side = x == 0 ? 0 : 1, base = side ? nx - 2 : 0;
            sx = nyz, sy = 1, sz = ny, cs = 4 * nyz;
            o0 = 6 * fstride + (2 * side - base) * nyz;
        }
        const long long centre = o0 + x * sx + y * sy + z * sz;
        const long long ox[3] = {-sx, 0, sx}, oy[3] = {-sy, 0, sy}, oz[3] = {-sz, 0, sz};
#pragma unroll 1
        for (int pq = 0; pq < 3; ++pq) {
            const int pr = p0 + pq, lev = pr / 6, comp = pr - lev * 6;
            const float *src = (lev == 0 ? cur : prev) + comp * cs + centre;
#pragma unroll
            for (int d = 0; d < 27; ++d) {
                const int dx = d % 3, dy = (d / 3) % 3, dz = d / 9;
                const int k = pr * 27 + d;
                const bool ok = vx[dx] && vy[dy] && vz[dz];
                const float *a = ok ? src + (ox[dx] + oy[dy] + oz[dz]) : src;
                cp_async_4(&Xt[k * LC + swz(k, q)], a, ok);
            }
        }
    } else {
#pragma unroll
        for (int pq = 0; pq < 3; ++pq)
#pragma unroll
            for (int d = 0; d < 27; ++d) {
                const int k = (p0 + pq) * 27 + d;
                Xt[k * LC + swz(k, q)] = 0.f;
            }
    }
}

__global__ void __launch_bounds__(256, 1) layer_kernel(const float *__restrict__ P, const float *__restrict__ cur,
                                                       const float *__restrict__ prev, long long fstride, int pitch,
                                                       int nx, int ny, int nz, const int *__restrict__ cells,
                                                       int ncells, float *__restrict__ out)
{
    extern __shared__ __align__(16) float sm[];
    float *W1t = sm;                  // [k][unit]
    float *W2t = W1t + SM_W1T;        // [k][unit]
    float *Xt = W2t + SM_W2T;         // [k][cell]: the unnormalised stencil
    float *H1t = Xt + SM_XT;          // [unit][cell]
    float *H2t = H1t + SM_H;
    float *W3t = H2t + SM_H;          // [k][out]
    float *b1 = W3t + SM_W3T, *b2 = b1 + NH, *b3 = b2 + NH;
    float *rr = b3 + NO;              // r per cell
    float *ir = rr + LC;              // 1/r per cell (0 if r = 0)
    float *part = ir + LC;            // [4][cell] partial sums of x^2
    const int tid = threadIdx.x;
    const int ntiles = (ncells + LC - 1) / LC;
    // the first tile's stencils are in flight while the weights are loaded
    if ((int)blockIdx.x < ntiles)
        stage_stencils(Xt, cur, prev, fstride, pitch, nx, ny, nz, cells, ncells, blockIdx.x);
    for (int e = tid; e < NH * NI; e += 256) {
        const int u = e / NI, k = e - u * NI;
        W1t[k * NH + swz(k, u)] = P[OFF_W1 + e];
    }
    for (int e = tid; e < (NIP - NI) * NH; e += 256) W1t[NI * NH + e] = 0.f;  // padding rows
    for (int e = tid; e < NH * NH; e += 256) {
        const int u = e / NH, k = e - u * NH;
        W2t[k * NH + swz(k, u)] = P[OFF_W2 + e];
    }
    for (int e = tid; e < NO * NH; e += 256) {
        const int o = e / NH, k = e - o * NH;
        W3t[k * NO + o] = P[OFF_W3 + e];
    }
    if (tid < NH) {
        b1[tid] = P[OFF_B1 + tid];
        b2[tid] = P[OFF_B2 + tid];
    }
    if (tid < NO) b3[tid] = P[OFF_B3 + tid];
    Xt[NI * LC + tid] = 0.f;  // padding rows of the stencil (256 zeros), never staged over
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();  // this tile's stencils have landed; the previous tile is done with H / rr
        {
            // sum of squares of the thread's own 81 staged values, in staging order
            const int q = tid & (LC - 1), p0 = (tid >> 6) * 3;
            float ss = 0.f;
#pragma unroll
            for (int pq = 0; pq < 3; ++pq)
#pragma unroll
                for (int d = 0; d < 27; ++d) {
                    const int k = (p0 + pq) * 27 + d;
                    const float v = Xt[k * LC + swz(k, q)];
                    ss = __fmaf_rn(v, v, ss);
                }
            part[(tid >> 6) * LC + q] = ss;
        }
        __syncthreads();
        if (tid < LC) {
            const float ss = part[tid] + part[LC + tid] + part[2 * LC + tid] + part[3 * LC + tid];
            const float r = sqrtf(ss / NI);
            const bool live = r >= R_MIN;  // smaller r: the cell keeps its value
            rr[tid] = live ? r : 0.f;
            ir[tid] = live ? 1.f / r : 0.f;
        }
        __syncthreads();
        // layers 1 and 2 on the tensor cores (3xTF32): H1 = tanh((W1 x) / r +
        // b1), H2 = tanh(W2 H1 + b2); warp w holds cells 16*(w%4) + g (+8) and
        // units 32*(w/4) + 8j + 2q (+1) of its accumulator fragments
        {
            const int lane = tid & 31, w = tid >> 5, g = lane >> 2, q = lane & 3;
            const int m0 = 16 * (w & 3), n0 = 32 * (w >> 2);
            float acc[4][4];
            warp_gemm_3xtf32<NIP>(Xt, W1t, acc);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int cell = m0 + g + 8 * (e >> 1), unit = n0 + 8 * j + 2 * q + (e & 1);
                    H1t[unit * LC + swz(unit, cell)] = tanhf(__fmaf_rn(acc[j][e], ir[cell], b1[unit]));
                }
            __syncthreads();  // every warp is past layer 1's reads of Xt
            // the next tile's stencils fly while layers 2 and 3 run
            const int next = tile + gridDim.x;
            if (next < ntiles) stage_stencils(Xt, cur, prev, fstride, pitch, nx, ny, nz, cells, ncells, next);
            warp_gemm_3xtf32<NH>(H1t, W2t, acc);
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int cell = m0 + g + 8 * (e >> 1), unit = n0 + 8 * j + 2 * q + (e & 1);
                    H2t[unit * LC + swz(unit, cell)] = tanhf(__fadd_rn(acc[j][e], b2[unit]));
                }
        }
        __syncthreads();
        // layer 3: the correction r f added to the Yee step later
        for (int e = tid; e < LC * NO; e += 256) {
            const int q = e / NO, o = e - q * NO;
            const int cell = tile * LC + q;
            if (cell >= ncells) continue;
            float f = b3[o];
            for (int k = 0; k < NH; ++k) f = __fmaf_rn(H2t[k * LC + swz(k, q)], W3t[k * NO + o], f);
            const unsigned m = tangent_mask(cells[3 * cell], cells[3 * cell + 1], cells[3 * cell + 2], nx, ny, nz);
            out[(long long)cell * NO + o] = (m >> o) & 1u ? __fmul_rn(rr[q], f) : 0.f;
        }
    }
    cp_async_wait_all();  // nothing left in flight at exit
}

__global__ void __launch_bounds__(256) scatter_kernel(float *__restrict__ f, long long fstride, int pitch, int ny,
                                                      const int *__restrict__ cells, int ncells,
                                                      const float *__restrict__ vals)
{
    const int q = blockIdx.x * 256 + threadIdx.x;
    if (q >= ncells) return;
    const long long p = cells[3 * q] + (long long)pitch * (cells[3 * q + 1] + (long long)ny * cells[3 * q + 2]);
    for (int c = 0; c < NO; ++c) f[c * fstride + p] = __fadd_rn(f[c * fstride + p], vals[(long long)q * NO + c]);
}

__global__ void __launch_bounds__(256) copy_cells_kernel(float *__restrict__ dst, const float *__restrict__ src,
                                                         long long fstride, int pitch, int ny,
                                                         const int *__restrict__ cells, int ncells)
{
    const int q = blockIdx.x * 256 + threadIdx.x;
    if (q >= ncells) return;
    const long long p = cells[3 * q] + (long long)pitch * (cells[3 * q + 1] + (long long)ny * cells[3 * q + 2]);
    for (int c = 0; c < NO; ++c) dst[c * fstride + p] = src[c * fstride + p];
}

// The x slab of a band snapshot (layout above): element e of the slab is
// (comp, side, xd, z, y) in that order, y fastest; planes outside the grid
// (nx < 2) are zero and never read.
__global__ void __launch_bounds__(256) fill_xslab_kernel(float *__restrict__ snap, const float *__restrict__ f,
                                                         long long fstride, int pitch, int nx, int ny, int nz)
{
    const long long n = xslab_floats(ny, nz);
    float *slab = snap + 6 * fstride;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int y = (int)(e % ny);
        long long r = e / ny;
        const int z = (int)(r % nz);
        r /= nz;
        const int xd = (int)(r & 1), side = (int)((r >> 1) & 1), comp = (int)(r >> 2);
        const int x = side ? nx - 2 + xd : xd;
        slab[e] = (x >= 0 && x < nx) ? f[comp * fstride + x + (long long)pitch * (y + (long long)ny * z)] : 0.f;
    }
}

} // namespace

// ------------------------------------------------------------ internal API

size_t mlp_scratch_bytes(int batch, long long n) { return scratch_bytes(batch, n); }

cudaError_t mlp_forward(const float *params, const float *X, long long n, float *Y, void *scratch, int batch,
                        cudaStream_t st)
{
    Scratch s = carve(scratch, batch, 0);
    for (long long b0 = 0; b0 < n; b0 += batch) {
        const int B = (int)std::min<long long>(batch, n - b0);
        CKE(forward(params, X + b0 * NI, nullptr, B, s, Y + b0 * NO, st));
    }
    return cudaSuccess;
}

cudaError_t mlp_grad(const float *params, const float *X, const float *T, int n, float *grad, double *loss_host,
                     void *scratch, int batch, cudaStream_t st)
{
    if (n > batch) return cudaErrorInvalidValue;
    Scratch s = carve(scratch, batch, 0);
    CKE(cudaMemsetAsync(s.loss, 0, sizeof(double), st));
    CKE(backward(params, X, T, nullptr, n, s, st));
    CKE(cudaMemcpyAsync(grad, s.grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st));
    double l = 0.0;
    CKE(cudaMemcpyAsync(&l, s.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    CKE(cudaStreamSynchronize(st));
    if (loss_host) *loss_host = l / ((double)n * NO);
    return cudaSuccess;
}

cudaError_t mlp_train(float *params, const float *X, const float *T, long long n, int batch, int epochs, double lr,
                      unsigned long long seed, void *scratch, cudaStream_t st, double *last_epoch_loss)
{
    Scratch s = carve(scratch, batch, n);
    CKE(cudaMemsetAsync(s.m, 0, sizeof(float) * NPARAM, st));
    CKE(cudaMemsetAsync(s.v, 0, sizeof(float) * NPARAM, st));
    std::mt19937_64 rng(seed);
    std::vector<int> perm((size_t)n);
    for (long long i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
    const long long nb = n / batch;  // whole batches only
    long long t = 0;
    double epoch_loss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CKE(cudaMemsetAsync(s.loss, 0, sizeof(double), st));
        CKE(cudaMemcpyAsync(s.rows, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
        for (long long b = 0; b < nb; ++b) {
            CKE(backward(params, X, T, s.rows + b * batch, batch, s, st));
            ++t;
            const float c1 = (float)(1.0 - std::pow(0.9, (double)t)), c2 = (float)(1.0 - std::pow(0.999, (double)t));
            adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(params, s.grad, s.m, s.v, NPARAM, (float)lr, c1, c2);
            CKE(cudaGetLastError());
        }
        double l = 0.0;
        CKE(cudaMemcpyAsync(&l, s.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        CKE(cudaStreamSynchronize(st));
        epoch_loss = nb > 0 ? l / ((double)nb * batch * NO) : 0.0;
    }
    if (last_epoch_loss) *last_epoch_loss = epoch_loss;
    return cudaSuccess;
}

cudaError_t mlp_record(const float *prev, const float *cur, const float *nxt, long long fstride, int pitch, int ny,
                       const int lo[3], const int hi[3], const int *cells, int n, const float *ce, const float *ca,
                       float neg_dt, float *X, float *Y, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    record_kernel<<<(n + 255) / 256, 256, 0, st>>>(prev, cur, nxt, fstride, pitch, ny, make_int3(lo[0], lo[1], lo[2]),
                                                    make_int3(hi[0], hi[1], hi[2]), cells, n, ce, ca, neg_dt, X, Y);
    return cudaGetLastError();
}

size_t learned_layer_smem() { return LAYER_SMEM; }

cudaError_t learned_layer_configure()
{
    return cudaFuncSetAttribute(layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LAYER_SMEM);
}

cudaError_t learned_layer_predict(const float *params, const float *cur, const float *prev, long long fstride,
                                  int pitch, int nx, int ny, int nz, const int *cells, int ncells, float *out,
                                  int grid, cudaStream_t st)
{
    if (ncells <= 0) return cudaSuccess;
    const int tiles = (ncells + LC - 1) / LC;
    layer_kernel<<<std::min(grid, tiles), 256, LAYER_SMEM, st>>>(params, cur, prev, fstride, pitch, nx, ny, nz, cells,
                                                                 ncells, out);
    return cudaGetLastError();
}

cudaError_t learned_layer_scatter(float *f, long long fstride, int pitch, int ny, const int *cells, int ncells,
                                  const float *vals, cudaStream_t st)
{
    if (ncells <= 0) return cudaSuccess;
    scatter_kernel<<<(ncells + 255) / 256, 256, 0, st>>>(f, fstride, pitch, ny, cells, ncells, vals);
    return cudaGetLastError();
}

cudaError_t learned_copy_cells(float *dst, const float *src, long long fstride, int pitch, int ny, const int *cells,
                               int ncells, cudaStream_t st)
{
    if (ncells <= 0) return cudaSuccess;
    copy_cells_kernel<<<(ncells + 255) / 256, 256, 0, st>>>(dst, src, fstride, pitch, ny, cells, ncells);
    return cudaGetLastError();
}

size_t learned_xslab_bytes(int ny, int nz) { return sizeof(float) * (size_t)xslab_floats(ny, nz); }

cudaError_t learned_fill_xslab(float *snap, const float *f, long long fstride, int pitch, int nx, int ny, int nz,
                               cudaStream_t st)
{
    const long long n = xslab_floats(ny, nz);
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    fill_xslab_kernel<<<blocks, 256, 0, st>>>(snap, f, fstride, pitch, nx, ny, nz);
    return cudaGetLastError();
}
