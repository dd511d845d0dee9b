// Systolic schedule, register-resident form (Sec. 3, Fig. 7; Sec. 4).
//
// Same method as systolic.cu: each CTA owns a tile, a box [A, A+n) of
// skewed space sigma = p + t, scans it down the x-y-z-t diagonal, takes its
// lower shell (level t) from the upwind tiles through global memory and
// leaves its top faces there for the downwind ones, with per-tile progress
// flags and no grid-wide synchronisation.  What differs is where the tile
// lives: in registers instead of shared memory.
//
//   x: lane = physical x mod 32 (a ring, as in shared memory);
//   y: warp = physical y mod 16 (a ring);
//   z: register row r in [-1, NZ) = skewed z, sigma_z = A_z + r.
//
// Because rows are indexed by skewed z, the value a row needs from the
// previous level sits one row below it in the same thread (sigma - 1 is the
// same physical cell one step earlier): the diagonal scan is an implicit
// register shift, H[r] <- f(H[r-1], E[r-1], E[r], ...), applied top-down in
// place.  Row -1 holds the lower z shell.  x neighbours come by warp
// shuffle, y neighbours through a small shared-memory exchange, so one cell
// update costs 4 shared-memory loads/stores, 4 shuffles and 24 FP32
// operations instead of ~27 shared-memory accesses.
//
// The slot that leaves the tile at the top in x (one lane per warp) and in y
// (one warp) is refilled each step with the lower x / y shell, and row -1
// with the lower z shell.  All three shells of level t are fetched into a
// shared staging buffer by bulk tensor copies (TMA): the z shell (with its x
// and y edges) from the field arrays, the y and x shells from two face
// buffers, one copy per shell for the six fields (the field index is a
// dimension of the copy) and one per shell for the coefficients.  Each
// thread waits on the buffer's mbarrier itself.
//
// Face buffers: the top y and x faces of a tile do not go to the field
// arrays but to a y-face and an x-face buffer indexed by physical (x, y) and
// by skewed z modulo a period of whole tile z-extents, in z-blocks: rows
// 1..NZ of a column sit at consecutive addresses (rounded up to 16 bytes), at
// a place that stays fixed for the whole life of the tile.  So the lane
// leaving the box in x and the warp leaving it in y store their whole columns
// with 16-byte stores, and the x lane and the y-shell warp refill theirs
// with 16-byte shared loads.  The period is at least the grid's z extent, so
// a wrapped position is next written only by a tile downwind of every reader
// of the value there; rows outside the domain are neither stored nor kept
// from a refill.
//
// The warp whose y slot is outside the box sits out both half-steps, so it
// carries the tile's bookkeeping: after the second barrier it publishes the
// tile's own level t-1, then polls the upwind tiles' progress once for level
// t+1 and, if they have published it, fetches those shells into the second
// staging buffer.  Only when that poll failed (or on a tile's first
// step) does warp 0 wait for the upwind tiles at the start of the step, and
// thread 0 fetch the shells then.
//
// Top faces: the z face goes to the field arrays at the end of each step;
// the y face goes to the y-face buffer one step late, from the warp whose y
// slot leaves, while it sits out the H half-step; the x face goes to the
// x-face buffer at the end of each step.  A tile therefore publishes level
// t-1 after the second barrier of step t.  Two block barriers per step: after
// the E rows are exchanged for the H half-step, and after the H rows are
// exchanged for the E half-step.
//
// Tile: 31 x 15 x NZ updated cells.  A step whose box lies inside the domain
// and clear of the low walls (most steps of a large grid) runs both
// half-steps with no per-cell masks.  Every arithmetic step is yee_cell.cuh,
// so the result equals the naive schedule bit for bit.
//
// Storage: fields live in global memory as FP32, FP16 or BF16 (S, see
// storage.cuh); registers hold FP32 values already rounded to the storage
// format, so each new H value is rounded where it is computed and each new
// E value once its point source (if any) has been added, exactly where the
// naive schedule rounds on store.  dt/eps stays FP32.
#include "internal.h"
#include "storage.cuh"
#include "sys_common.cuh"
#include "yee_cell.cuh"

#include <type_traits>

namespace {

using namespace sysc;

template <int NZ_, class S_, bool LOSSY_, int TY_, int CL_ = 1>
struct RegTile {
    using S = S_;
    static constexpr bool LOSSY = LOSSY_;  // conducting cells: E <- ca E + cb curl H
    // CTAs per thread-block cluster along x: 2 = pairs of x-adjacent tiles,
    // the upwind one sending its top x face through distributed shared memory
    static constexpr int CL = CL_;
    static_assert(CL_ == 1 || (CL_ == 2 && !LOSSY_), "clusters of one, or x pairs of lossless tiles");
    using T = typename S_::T;
    static constexpr int NZ = NZ_;        // updated z rows (registers 0..NZ-1)
    static constexpr int NR = NZ_ + 1;    // plus the shell row -1
    static constexpr int RY = 16, NT = 32 * RY;
    // TY = RY - 1: one y slot outside the box, the y shell (its warp also
    // holds the previous step's top y row until its refill); TY = RY - 2:
    // the previous top row has a slot (and warp) of its own
    static constexpr int TX = 31, TY = TY_, TZ = NZ_;
    static_assert(TY_ == RY - 1 || TY_ == RY - 2, "one or two y slots outside the box");
    static_assert(NR <= 16 && TY <= 16, "cooperative entries: row < 16, warp offset < 16");
    static_assert(NZ % 4 == 0, "rows move in groups of four (16-byte accesses) and pairs (packed rounding)");
    // shared memory, in floats
    // y-neighbour exchange, one component.  VX (16-bit storage): [warp][lane]
    // [row], rows moved in 16-byte groups of four; a lane's rows start XR
    // floats after the previous lane's, XR / 4 odd, so the 8 lanes of a
    // quarter warp hit disjoint banks.  FP32: [warp][row][lane], one row per
    // access (measured faster there: 176 vs 169 GCUPS at 256^3, while 16-bit
    // storage gains 156 -> 164 from the vector form)
    static constexpr bool VX = S_::narrow;
    static constexpr int XR = (NZ_ / 4) % 2 ? NZ_ : NZ_ + 4;
    static constexpr int XE_F = VX ? RY * 32 * XR : RY * NZ_ * 32;
    // lower-shell staging, filled per step by bulk tensor copies (TMA) of
    // boxes whose x start is rounded down to 16 bytes (XA elements): SW =
    // 32 + XA elements cover the 32-wide x window.  One copy per shell
    // fetches all six fields ([field][...] in shared memory), one more the
    // FP32 coefficients (C-suffixed sizes, [cb, ca][...]); sizes below are
    // per array, in elements, and every shell's region starts on a 128-byte
    // boundary.
    static constexpr int EB = (int)sizeof(T);
    static constexpr int XA = 16 / EB, SW = 32 + XA;
    static constexpr int ZB = RY * SW;        // z shell box {SW,16,1}: [y][x]
    // The top x and y faces go to two face buffers in z-blocks: rows 1..NZ of
    // one (x, y) column of a tile sit at BZ consecutive elements (NZ rounded
    // up to 16 bytes), so shells and faces move with 16-byte accesses.
    static constexpr int BZ = (NZ_ * EB + 15) / 16 * 16 / EB;
    static_assert(BZ % (16 / EB) == 0 && NZ_ % 4 == 0, "z-blocks of whole 16-byte chunks, 4 rows per access");
    static constexpr int YB = 32 * BZ;        // y shell box {BZ,32,1} from the y-face buffer: [x][z]
    static constexpr int XB = 16 * BZ;        // x shell box {BZ,16,1} from the x-face buffer: [y][z]
    static constexpr int XAC = 4, SWC = 36;
    static constexpr int ZBC = RY * SWC, YBC = NR * SWC, XBC = NR * 16 * XAC;
    static constexpr int NCOEF = LOSSY ? 2 : 1;   // FP32 coefficient arrays: cb (dt/eps), ca
    static constexpr size_t r128(size_t b) { return (b + 127) / 128 * 128; }
    // byte offsets of the shells within one staging buffer
    static constexpr size_t OFF_Y = r128(6 * (size_t)ZB * EB);
    static constexpr size_t OFF_X = OFF_Y + r128(6 * (size_t)YB * EB);
    static constexpr size_t OFF_ZC = OFF_X + r128(6 * (size_t)XB * EB);
    static constexpr size_t OFF_YC = OFF_ZC + r128(NCOEF * 4 * (size_t)ZBC);
    static constexpr size_t OFF_XC = OFF_YC + r128(NCOEF * 4 * (size_t)YBC);
    static constexpr unsigned TMA_BYTES =
        6u * EB * (ZB + YB + XB) + NCOEF * 4u * (ZBC + YBC + XBC);
    static constexpr int CR = 16;                 // coefficient ring rows (>= NR, power of 2)
    static constexpr int CE_F = RY * CR * 32;
    static_assert(CR >= NR, "coefficient ring holds the whole column");
    // staging buffers: two (the next step's shells are fetched during this
    // step) unless the lossy form's second coefficient set leaves no room
    static constexpr int NBUF = LOSSY_ ? 1 : 2;
    static constexpr size_t STG_B = OFF_XC + r128(NCOEF * 4 * (size_t)XBC);  // one buffer, bytes
    // x pairs: the downwind tile's receive ring of x faces, NSLOT slots of
    // [field][box row y][z-block] (rows 1..NZ of the x shell of one step)
    static constexpr int NSLOT = 6;
    static constexpr int RXS = 6 * 16 * BZ;  // elements per slot
    static constexpr size_t RX_B = CL_ == 2 ? NSLOT * (size_t)RXS * EB : 0;
    static constexpr size_t smem_bytes()
    {
        return NBUF * STG_B + sizeof(float) * (4 * (size_t)XE_F + NCOEF * (size_t)CE_F) + RX_B;
    }
};

__device__ __forceinline__ float shfl_from(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Four consecutive rows of one field as one 16-byte (FP32) or 8-byte (16-bit)
// access: p must be aligned to it.
template <class S>
__device__ __forceinline__ void ld4(const typename S::T *p, float s, float &a, float &b, float &c, float &d)
{
    if constexpr (sizeof(typename S::T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a = v.x; b = v.y; c = v.z; d = v.w;
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        a = S::dec((typename S::T)(v.x & 0xffffu), s); b = S::dec((typename S::T)(v.x >> 16), s);
        c = S::dec((typename S::T)(v.y & 0xffffu), s); d = S::dec((typename S::T)(v.y >> 16), s);
    }
}

template <class S>
__device__ __forceinline__ void st4(typename S::T *p, float is, float a, float b, float c, float d)
{
    if constexpr (sizeof(typename S::T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    } else {
        uint2 v;
        v.x = S::enc2(a, b, is);
        v.y = S::enc2(c, d, is);
        *reinterpret_cast<uint2 *>(p) = v;
    }
}

// Rows 1..NZ of one field of a column: loaded from a z-block, and stored into
// one.  A store writes only the rows whose physical z (z0 + i - 1) lies in
// the domain: with whole 16-byte chunks when all of them do, else row by row
// (face-buffer positions of rows outside the domain belong to other cells).
template <class S, int NR>
__device__ __forceinline__ void ld_rows(const typename S::T *p, float s, float (&v)[NR])
{
#pragma unroll
    for (int q = 0; q < (NR - 1) / 4; ++q) ld4<S>(p + 4 * q, s, v[4 * q + 1], v[4 * q + 2], v[4 * q + 3], v[4 * q + 4]);
}

template <class S, int NR>
__device__ __forceinline__ void st_rows(typename S::T *p, float is, const float (&v)[NR], int z0, int nz)
{
    if (z0 >= 0 && z0 + NR - 1 <= nz) {
#pragma unroll
        for (int q = 0; q < (NR - 1) / 4; ++q)
            st4<S>(p + 4 * q, is, v[4 * q + 1], v[4 * q + 2], v[4 * q + 3], v[4 * q + 4]);
    } else {
#pragma unroll
        for (int i = 1; i < NR; ++i)
            if ((unsigned)(z0 + i - 1) < (unsigned)nz) p[i - 1] = S::enc(v[i], is);
    }
}

// Bulk tensor copy of one box of a 4D map (TMA: x, y, z, array) starting at
// array 0 into shared memory, completing on an mbarrier; elements outside
// the tensor are written as zero.
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *map, int x, int y, int z,
                                        unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(0),
                 "r"(smem_u32(bar))
                 : "memory");
}

// The same for a 5D map (face buffers: z-block rows, y or x, x or y, block,
// field), starting at field 0.
__device__ __forceinline__ void tma_box5(void *dst, const CUtensorMap *map, int r, int a, int b, int kb,
                                         unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(r), "r"(a), "r"(b), "r"(kb), "r"(0),
                 "r"(smem_u32(bar))
                 : "memory");
}

// Thread-block cluster primitives (x pairs).
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the shared::cluster address of local shared address `a` in CTA `rank`
__device__ __forceinline__ unsigned mapa(unsigned a, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// every thread of every CTA of the cluster (orders all prior memory accesses,
// distributed shared memory included, before all later ones)
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_remote_u32(unsigned a, unsigned v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void arrive_remote(unsigned bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Four rows of one field into another CTA's shared memory (16 bytes FP32,
// 8 bytes 16-bit, packed as st4 does).
template <class S>
__device__ __forceinline__ void st4_remote(unsigned a, float is, float x, float y, float z, float w)
{
    if constexpr (sizeof(typename S::T) == 4) {
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w)
                     : "memory");
    } else {
        asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(S::enc2(x, y, is)),
                     "r"(S::enc2(z, w, is))
                     : "memory");
    }
}
template <class S, int NR>
__device__ __forceinline__ void st_rows_remote(unsigned a, float is, const float (&v)[NR])
{
#pragma unroll
    for (int q = 0; q < (NR - 1) / 4; ++q)
        st4_remote<S>(a + 4 * q * (unsigned)sizeof(typename S::T), is, v[4 * q + 1], v[4 * q + 2], v[4 * q + 3],
                      v[4 * q + 4]);
}

// Bounded wait (acquire at cluster scope) for phase `parity` of a local
// mbarrier that a partner CTA of the cluster completes.  Returns false (error
// word set) past the launch's timeout.
__device__ bool wait_cluster_bar(const SysLaunch &P, unsigned long long *bar, unsigned parity, int ticket)
{
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        unsigned done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;"
                     " selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (ld_volatile(P.ctrl + 1) != DEV_OK) return false;
        const unsigned long long now = globaltimer();
        if (it == 0) {
            t0 = now;
        } else if (now - t0 > (unsigned long long)P.timeout_ns) {
            if (atomicCAS(P.ctrl + 1, DEV_OK, DEV_ERR_TIMEOUT) == DEV_OK) {
                P.ctrl[2] = ticket;
                P.ctrl[3] = -2;
            }
            return false;
        }
    }
}

// Bounded wait for phase `parity` of the staging barrier.  Returns false if
// the wait ran past the launch's timeout (the error word is then set).
__device__ bool wait_stage(const SysLaunch &P, unsigned long long *bar, unsigned parity, int ticket)
{
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        unsigned done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
                     " selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        const unsigned long long now = globaltimer();
        if (it == 0) {
            t0 = now;
        } else if (now - t0 > (unsigned long long)P.timeout_ns) {
            if (atomicCAS(P.ctrl + 1, DEV_OK, DEV_ERR_TIMEOUT) == DEV_OK) {
                P.ctrl[2] = ticket;
                P.ctrl[3] = -1;
            }
            return false;
        }
    }
}

template <class R>
__global__ void __launch_bounds__(R::NT, 1) systolic_reg_kernel(const __grid_constant__ SysLaunch P)
{
    using S = typename R::S;
    using T = typename R::T;
    constexpr int NZ = R::NZ, NR = R::NR, TX = R::TX, TY = R::TY, TZ = R::TZ;
    constexpr int SW = R::SW, XA = R::XA, SWC = R::SWC;
    extern __shared__ __align__(1024) float4 smem4[];
    // staging buffers first (the dynamic shared memory base is 1024-byte
    // aligned), each: the lower z, y and x shells of the 6 fields, then those
    // of dt/eps (and ca); the pointers below are buffer 0's, buffer b is
    // R::STG_B bytes further
    char *const stg0 = reinterpret_cast<char *>(smem4);
    // y exchange (layout: RegTile::VX): E^t (level t-1) rows i = 0..NZ-1, and
    // the new H rows r = 1..NZ at row r-1
    float *const XEx = reinterpret_cast<float *>(stg0 + R::NBUF * R::STG_B);
    float *const XEz = XEx + R::XE_F;
    float *const XHx = XEz + R::XE_F;
    float *const XHz = XHx + R::XE_F;
    // element (warp, row, lane) of one exchanged component
    auto xe_at = [](int wq, int row, int ln) {
        return R::VX ? (wq * 32 + ln) * R::XR + row : (wq * NZ + row) * 32 + ln;
    };
    // dt/eps of each column, indexed by physical z mod CR: a cell's coefficient
    // stays in place while the skewed register rows move past it
    float *const CEs = XHz + R::XE_F;      // [warp][physical z mod CR][lane]
    float *const CAs = CEs + R::CE_F;      // the same for ca (lossy only)
    // x pairs: the receive ring of x faces (downwind CTA), after the rings
    T *const RX = reinterpret_cast<T *>(CEs + R::NCOEF * R::CE_F);  // [slot][field][box row][BZ]
    __shared__ int s_ticket, s_abort;
    // x pairs: a slot of the receive ring is full (the upwind CTA arrives
    // once its x lanes have written it) / free again (the downwind CTA arrives)
    __shared__ alignas(8) unsigned long long s_rxf[R::NSLOT], s_rxe[R::NSLOT];
    __shared__ alignas(8) unsigned long long s_bar[2];  // staging barriers, one per buffer: one phase per fill
    // state of the next step's shells, decided during this one: 0 = the
    // upwind tiles have not published them yet, 1 = published and fetched
    // into the other buffer, 2 = published, not yet fetched (one buffer)
    __shared__ int s_pref;
    __shared__ unsigned s_niss[2];                      // fills issued into each buffer
    __shared__ unsigned s_seen[3];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float ndt = P.neg_dt;
    const long long sxy = (long long)P.pitch * P.ny;
    // field pointers and scales are read from the kernel parameters where
    // used (they stay in the constant bank instead of taking registers)
#define F0 reinterpret_cast<T *>(P.f[0])
#define F1 reinterpret_cast<T *>(P.f[1])
#define F2 reinterpret_cast<T *>(P.f[2])
#define F3 reinterpret_cast<T *>(P.f[3])
#define F4 reinterpret_cast<T *>(P.f[4])
#define F5 reinterpret_cast<T *>(P.f[5])
#define CE P.ce
#define CA P.ca
#define SC(c) P.sc.s[c]
#define IS(c) P.sc.is[c]
#define RND(v, c) S::rnd(v, SC(c), IS(c))
#define RND2(a, b, c) S::rnd2(a, b, SC(c), IS(c))
#define STORE6(g, i)                                                                          \
    do {                                                                                      \
        F0[g] = S::enc(ex[i], IS(0)); F1[g] = S::enc(ey[i], IS(1)); F2[g] = S::enc(ez[i], IS(2)); \
        F3[g] = S::enc(hx[i], IS(3)); F4[g] = S::enc(hy[i], IS(4)); F5[g] = S::enc(hz[i], IS(5)); \
    } while (0)

    // Face buffers: rows 1..NZ of component f of column (x, y) of a tile in
    // z-block kb are at
    //   x faces: XF + f*fxs + ((kb*nx + x)*ny + y)*BZ + (row - 1),
    //   y faces: YF + f*fys + ((kb*ny + y)*nx + x)*BZ + (row - 1),
    // kb = K mod (number of z-blocks): block kb holds skewed z (sigma_z = z +
    // t) modulo the blocks' period, so a tile's faces and lower x / y shells
    // keep one aligned place for its whole life, and a face (or shell) of one
    // tile step is one contiguous run per field.  A tile's top x face is
    // stored by the lane leaving the box in x, its top y face by the warp
    // leaving it in y, straight from registers.
    T *const XF = reinterpret_cast<T *>(P.xf);
    T *const YF = reinterpret_cast<T *>(P.yf);
    constexpr int BZ = R::BZ;
#define FACE_STORE(dst, fs, z0)                                                             \
    do {                                                                                    \
        st_rows<S>((dst), IS(0), ex, (z0), P.nz); st_rows<S>((dst) + (fs), IS(1), ey, (z0), P.nz);         \
        st_rows<S>((dst) + 2 * (fs), IS(2), ez, (z0), P.nz); st_rows<S>((dst) + 3 * (fs), IS(3), hx, (z0), P.nz); \
        st_rows<S>((dst) + 4 * (fs), IS(4), hy, (z0), P.nz); st_rows<S>((dst) + 5 * (fs), IS(5), hz, (z0), P.nz); \
    } while (0)

    constexpr int CR = R::CR;
    if (tid == 0) {
        s_niss[0] = s_niss[1] = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar[1])) : "memory");
        if constexpr (R::CL == 2) {
#pragma unroll
            for (int k = 0; k < R::NSLOT; ++k) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_rxf[k])) : "memory");
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_rxe[k])) : "memory");
            }
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // x pairs: rank 0 holds the upwind tile (I even), rank 1 the downwind one;
    // every CTA of the cluster must be running before distributed shared
    // memory is touched
    const unsigned rank = R::CL == 2 ? cluster_rank() : 0u;
    if constexpr (R::CL == 2) cluster_sync_all();
    const unsigned rx_remote = R::CL == 2 ? mapa(smem_u32(RX), 1u) : 0u;        // rank 0 -> rank 1's ring
    const unsigned rxf_remote = R::CL == 2 ? mapa(smem_u32(&s_rxf[0]), 1u) : 0u;
    const unsigned rxe_remote = R::CL == 2 ? mapa(smem_u32(&s_rxe[0]), 0u) : 0u;  // rank 1 -> rank 0
    // messages (x faces) sent / received over this CTA's life: message m
    // uses slot m % NSLOT, its (m / NSLOT)-th use of that slot
    int msg_base = 0;
    // slot to signal after the next block barrier (the y-shell warp does it):
    // rank 0, the slot its x lanes have just filled; rank 1, the slot its x
    // lane has just read
    int sig_slot = -1;
    // fills waited for on each buffer (every thread waits on every fill, so
    // every thread keeps the same counts)
    unsigned n_wait0 = 0, n_wait1 = 0;
    // lower shells of level t into buffer b: six bulk tensor copies issued by
    // one thread (x start rounded down to 16 bytes; zero fill off the domain),
    // counted in s_niss for the final drain
    auto issue_shells = [&](int t, int b, int Ax, int Ay, int Az, int kb) {
        const int bx = Ax - t, by = Ay - t, bz = Az - t;
        const int x0 = (bx - 1) & ~(XA - 1), x0c = (bx - 1) & ~(R::XAC - 1);
        char *sb = stg0 + (size_t)b * R::STG_B;
        unsigned long long *bar = &s_bar[b];
        // order this thread's view of the upwind tiles' global stores (generic
        // proxy, acquired through their progress flags) before the bulk copies
        // that read them
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"(R::TMA_BYTES) : "memory");
        tma_box(sb, &P.tm[0][0], x0, by - 1, bz - 1, bar);              // z shell: field arrays
        tma_box5(sb + R::OFF_Y, &P.tm[1][0], 0, bx, by - 1, kb, bar);        // y shell: y-face buffer
        tma_box5(sb + R::OFF_X, &P.tm[2][0], 0, by - 1, bx - 1, kb, bar);    // x shell: x-face buffer
        tma_box(sb + R::OFF_ZC, &P.tm[0][1], x0c, by - 1, bz - 1, bar);
        tma_box(sb + R::OFF_YC, &P.tm[1][1], x0c, by - 1, bz - 1, bar);
        tma_box(sb + R::OFF_XC, &P.tm[2][1], x0c, by, bz - 1, bar);
        ++s_niss[b];
    };
    // the tile column of this thread: registers row i <-> r = i-1
    float ex[NR], ey[NR], ez[NR], hx[NR], hy[NR], hz[NR];

    for (;;) {
        if constexpr (R::CL == 2) {
            // the pair takes one ticket: both CTAs have finished their previous
            // tiles (barrier), rank 0 takes the ticket and reads the error
            // word for both, both read them after the second barrier, so the
            // two always stop together
            cluster_sync_all();
            if (rank == 0 && tid == 0) {
                const int tk = atomicAdd(P.ctrl, 1);
                const int ab = ld_volatile(P.ctrl + 1) != DEV_OK;
                s_ticket = tk;
                s_abort = ab;
                st_remote_u32(mapa(smem_u32(&s_ticket), 1u), (unsigned)tk);
                st_remote_u32(mapa(smem_u32(&s_abort), 1u), (unsigned)ab);
            }
            if (tid == 0) s_pref = 0;
            if (tid < 3) s_seen[tid] = 0u;
            cluster_sync_all();
        } else {
            if (tid == 0) {
                s_ticket = atomicAdd(P.ctrl, 1);
                s_abort = ld_volatile(P.ctrl + 1) != DEV_OK;
                s_pref = 0;
            }
            if (tid < 3) s_seen[tid] = 0u;
            __syncthreads();
        }
        const int ticket = s_ticket;
        const bool stop = s_abort || ticket >= P.ntiles;
        __syncthreads();
        if (stop) break;
        bool abort = false;
        int nmsg = 0;
        do {  // one tile (`break` leaves it early: an abort, or a pair member without a tile)
        int I, J, K;
        int m_lo = 1, m_hi = 0;  // x pairs: steps whose x face goes through the ring
        if constexpr (R::CL == 2) {
            const int gxp = (P.gx + 1) / 2, pr = P.tiles[ticket];
            const int pp = pr % gxp;
            J = (pr / gxp) % P.gy;
            K = pr / (gxp * P.gy);
            I = 2 * pp + (int)rank;
            if (2 * pp + 1 < P.gx) {
                const Interval i0 = tile_interval<TX, TY, TZ>(P, 2 * pp, J, K);
                const Interval i1 = tile_interval<TX, TY, TZ>(P, 2 * pp + 1, J, K);
                if (i0.s <= i0.e && i1.s <= i1.e) {
                    m_lo = i1.s;
                    m_hi = min(i0.e, i1.e);
                }
            }
            nmsg = max(0, m_hi - m_lo + 1);
            if (I >= P.gx) break;  // the last pair of an odd tile row has one tile
        } else {
            const int tl = P.tiles[ticket];
            I = tl % P.gx;
            J = (tl / P.gx) % P.gy;
            K = tl / (P.gx * P.gy);
        }
        const int tile = I + P.gx * (J + P.gy * K);
        const int Ax = I * TX, Ay = J * TY, Az = K * TZ;
        const int kb = K % P.nzblk;  // this tile's z-block in the face buffers
        T *const XFk = XF + (long long)kb * P.nx * P.ny * BZ;
        T *const YFk = YF + (long long)kb * P.nx * P.ny * BZ;
        const Interval iv = tile_interval<TX, TY, TZ>(P, I, J, K);
        Upwind U;
        upwind_of<TX, TY, TZ>(P, I, J, K, U);

        if (iv.s > 0) {
            if (w == 0) {
                const bool ok = wait_level(P, U, s_seen, iv.s - 1, ticket);
                if (tid == 0) s_abort = !ok;
            }
            __syncthreads();
            if (s_abort) { abort = true; break; }
        }
        if (iv.s > iv.e) {  // enters the domain only after this launch: relay only
            if (tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.s);
            __syncthreads();
            continue;
        }

        // initial load: level start-1, rows sigma_z = Az + r at physical Az + r - start + 1
        {
            const int bx = Ax - iv.s, by = Ay - iv.s;
            const int px = bx + ((lane - bx) & 31), py = by + ((w - by) & (R::RY - 1));
            const bool cin = (unsigned)px < (unsigned)P.nx && (unsigned)py < (unsigned)P.ny;
            // rows 1..NZ of the lower x shell column and of the lower y shell
            // row at level start-1: written by the upwind tiles into the face
            // buffers during this launch (start >= 1; the x-face buffer holds
            // the corner column), else the launch's initial state in the
            // field arrays (start = 0); row 0 is the lower z shell
            const bool xshell = px == bx && iv.s > 0;
            const bool yshell = py == by && iv.s > 0 && !xshell;
            const long long col = px + (long long)P.pitch * py;
            const T *const fq = xshell ? XFk + ((long long)px * P.ny + py) * BZ
                                       : YFk + ((long long)py * P.nx + px) * BZ;
            const long long fqs = xshell ? P.fxs : P.fys;
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const int pz = Az + i - 1 - iv.s + 1;
                float c = 0.f, a = 0.f;
                if (cin && (unsigned)pz < (unsigned)P.nz) {
                    const long long g = col + sxy * pz;
                    if (i > 0 && (xshell || yshell)) {  // the upwind tiles' top x / y face of level start-1
                        const T *q = fq + (i - 1);
                        ex[i] = S::dec(S::ld_cg(q), SC(0)); ey[i] = S::dec(S::ld_cg(q + fqs), SC(1));
                        ez[i] = S::dec(S::ld_cg(q + 2 * fqs), SC(2)); hx[i] = S::dec(S::ld_cg(q + 3 * fqs), SC(3));
                        hy[i] = S::dec(S::ld_cg(q + 4 * fqs), SC(4)); hz[i] = S::dec(S::ld_cg(q + 5 * fqs), SC(5));
                    } else {
                        ex[i] = S::dec(S::ld_cg(F0 + g), SC(0)); ey[i] = S::dec(S::ld_cg(F1 + g), SC(1));
                        ez[i] = S::dec(S::ld_cg(F2 + g), SC(2)); hx[i] = S::dec(S::ld_cg(F3 + g), SC(3));
                        hy[i] = S::dec(S::ld_cg(F4 + g), SC(4)); hz[i] = S::dec(S::ld_cg(F5 + g), SC(5));
                    }
                    c = __ldg(CE + g);
                    if (R::LOSSY) a = __ldg(CA + g);
                } else {
                    ex[i] = ey[i] = ez[i] = hx[i] = hy[i] = hz[i] = 0.f;
                }
                CEs[(w * CR + (pz & (CR - 1))) * 32 + lane] = c;
                if (R::LOSSY) CAs[(w * CR + (pz & (CR - 1))) * 32 + lane] = a;
            }
        }
        if (iv.s > 0 && tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.s);

        // may a point source lie in the box during this tile's steps?  (per
        // axis, the box holds coordinate c at steps A - c .. A - c + n - 1)
        bool tile_src = false;
        for (int q = 0; q < P.src.n; ++q) {
            const SrcDesc &s = P.src.s[q];
            const int lo = max(max(iv.s, Ax - s.i), max(Ay - s.j, Az - s.k));
            const int hi = min(min(iv.e, Ax - s.i + TX - 1), min(Ay - s.j + TY - 1, Az - s.k + TZ - 1));
            tile_src |= lo <= hi;
        }
        for (int t = iv.s; t <= iv.e; ++t) {
            const int bx = Ax - t, by = Ay - t, bz = Az - t;  // box low corner at step t
            const int cur = R::NBUF == 2 ? (t & 1) : 0;
            char *const sb = stg0 + (size_t)cur * R::STG_B;
            const T *const ZST = reinterpret_cast<const T *>(sb);
            const T *const YST = reinterpret_cast<const T *>(sb + R::OFF_Y);
            const T *const XST = reinterpret_cast<const T *>(sb + R::OFF_X);
            const float *const ZSC = reinterpret_cast<const float *>(sb + R::OFF_ZC), *const ZSA = ZSC + R::ZBC;
            const float *const YSC = reinterpret_cast<const float *>(sb + R::OFF_YC), *const YSA = YSC + R::YBC;
            const float *const XSC = reinterpret_cast<const float *>(sb + R::OFF_XC), *const XSA = XSC + R::XBC;
            const int dx = (lane - bx) & 31, dy = (w - by) & (R::RY - 1);
            const int px = bx + dx, py = by + dy;
            const bool xbox = dx < TX, ybox = dy < TY;
            const bool colin = xbox && ybox && (unsigned)px < (unsigned)P.nx && (unsigned)py < (unsigned)P.ny;
            const int ey_w = (by - 1) & (R::RY - 1);  // warp holding the y shell this step
            const int yf_w = (by + TY) & (R::RY - 1);  // warp holding the top y row of step t-1
            const long long col = px + (long long)P.pitch * py;
            // rows i with physical z = bz + i - 1 inside the domain
            const int i_lo = max(1, 1 - bz), i_hi = min(NR, P.nz - bz + 1);
            // the box is clear of the low walls: every box cell is updated
            // with no mask.  (The x-shell lane and the y-shell warp compute
            // values that their refills overwrite.)  Cells beyond the high
            // walls need none either: their dt/eps (and c_a) is 0 (the
            // coefficient shells are zero-filled off the domain), so their E
            // stays 0, and their H, whose curl reads only such E, stays 0 too.
            const bool inner = bx >= 1 && by >= 1 && bz >= 1;
            // every row of the box's z range lies in the domain (rows refilled
            // from the face buffers need no clearing)
            const bool zin = bz >= 0 && bz + TZ <= P.nz;
            // physical x of this lane's column after the refills (the x-shell
            // lane moves to bx - 1)
            const int xw = (bx - 1) + ((lane - bx + 1) & 31);

            // A. publish E^t (old) rows for the warp below's H half-step
            if constexpr (R::VX) {
                float *const qx = XEx + xe_at(w, 0, lane), *const qz = XEz + xe_at(w, 0, lane);
#pragma unroll
                for (int i = 0; i < NZ; i += 4) {
                    *reinterpret_cast<float4 *>(qx + i) = make_float4(ex[i], ex[i + 1], ex[i + 2], ex[i + 3]);
                    *reinterpret_cast<float4 *>(qz + i) = make_float4(ez[i], ez[i + 1], ez[i + 2], ez[i + 3]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < NZ; ++i) {
                    XEx[xe_at(w, i, lane)] = ex[i];
                    XEz[xe_at(w, i, lane)] = ez[i];
                }
            }
            __syncthreads();  // B1
            if (s_abort) { abort = true; break; }
            // x pairs: this step's x face travels through ring slot `slot`
            const bool msg = R::CL == 2 && t >= m_lo && t <= m_hi;
            const bool rx_msg = msg && rank == 1, tx_msg = msg && rank == 0;
            const int mi = msg_base + (t - m_lo);
            const int slot = mi % R::NSLOT;
            if constexpr (R::CL == 2) {
                // every lane is past last step's ring accesses: rank 0's x
                // lanes have written the slot (the release covers their stores),
                // rank 1's x lane has read it; the y-shell warp, idle in the H
                // half-step, tells the partner
                if (sig_slot >= 0) {
                    if (w == ((by - 1) & (R::RY - 1)) && lane == 0)
                        arrive_remote((rank == 0 ? rxf_remote : rxe_remote) + 8u * (unsigned)sig_slot);
                    sig_slot = -1;
                }
            }
            // unless the previous step found this step's shells published,
            // wait here for the upwind tiles' level t; fetch the shells now
            // unless they were fetched during the previous step
            const int pst = s_pref;
            if (pst == 0) {
                if (w == 0) {
                    const bool ok = wait_level(P, U, s_seen, t, ticket);
                    if (tid == 0) s_abort = !ok;
                }
                __syncthreads();
                if (s_abort) { abort = true; break; }
            }
            if (pst != 1 && tid == 0) issue_shells(t, cur, Ax, Ay, Az, kb);

            // B. the warp whose y slot leaves the tile this step is idle during
            //    the H half-step: it stores last step's top y face, which its
            //    registers still hold, into the y-face buffer
            if (w == yf_w && t > iv.s) {
                const int pbx = bx + 1, pby = by + 1, pbz = bz + 1;  // box corner of step t-1
                const int pdx = (lane - pbx) & 31;
                const int qx = pbx + pdx, qy = pby + TY - 1;
                if (pdx < TX && (unsigned)qx < (unsigned)P.nx && (unsigned)qy < (unsigned)P.ny)
                    FACE_STORE(YFk + ((long long)qy * P.nx + qx) * BZ, P.fys, pbz);
            }
            // x start of the staged z shell (rounded down to 16 bytes)
            const int x0 = (bx - 1) & ~(XA - 1), x0c = (bx - 1) & ~(R::XAC - 1);

            // C. H half-step, top-down in place: H[i] <- H[i-1] - dt curl_f(E[i-1], E[i], ...)
            if (ybox) {
                const int wn = (w + 1) & (R::RY - 1);
                const int src = (lane + 1) & 31;
                // rows in pairs (i, i-1), both computed from the old values
                // before either is written, so 16-bit storage rounds two new
                // values with one packed conversion
                const float *const qx = XEx + xe_at(wn, 0, lane), *const qz = XEz + xe_at(wn, 0, lane);
                auto h_pass = [&](auto masked) {
                    float4 gx, gz;  // VX: the y+1 neighbour's E rows 4q .. 4q+3
#pragma unroll
                    for (int i = NR - 1; i >= 2; i -= 2) {
                        if (R::VX && i % 4 == 0) {  // rows i-4 .. i-1
                            gx = *reinterpret_cast<const float4 *>(qx + i - 4);
                            gz = *reinterpret_cast<const float4 *>(qz + i - 4);
                        }
                        float nh[2][3];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int r = i - k;
                            const float ez_xp = shfl_from(ez[r - 1], src);
                            const float ey_xp = shfl_from(ey[r - 1], src);
                            const int m = (r - 1) & 3;
                            const float ez_yp = !R::VX ? qz[(r - 1) * 32]
                                                : m == 0 ? gz.x : m == 1 ? gz.y : m == 2 ? gz.z : gz.w;
                            const float ex_yp = !R::VX ? qx[(r - 1) * 32]
                                                : m == 0 ? gx.x : m == 1 ? gx.y : m == 2 ? gx.z : gx.w;
                            nh[k][0] = h_x(hx[r - 1], ez_yp, ez[r - 1], ey[r], ey[r - 1], ndt);
                            nh[k][1] = h_y(hy[r - 1], ex[r], ex[r - 1], ez_xp, ez[r - 1], ndt);
                            nh[k][2] = h_z(hz[r - 1], ey_xp, ey[r - 1], ex_yp, ex[r - 1], ndt);
                        }
                        RND2(nh[0][0], nh[1][0], 3);
                        RND2(nh[0][1], nh[1][1], 4);
                        RND2(nh[0][2], nh[1][2], 5);
                        const bool u0 = !decltype(masked)::value || (colin && i >= i_lo && i < i_hi);
                        const bool u1 = !decltype(masked)::value || (colin && i - 1 >= i_lo && i - 1 < i_hi);
                        const float a0 = u0 ? nh[0][0] : hx[i - 1], b0 = u0 ? nh[0][1] : hy[i - 1],
                                    c0 = u0 ? nh[0][2] : hz[i - 1];
                        const float a1 = u1 ? nh[1][0] : hx[i - 2], b1 = u1 ? nh[1][1] : hy[i - 2],
                                    c1 = u1 ? nh[1][2] : hz[i - 2];
                        hx[i] = a0; hy[i] = b0; hz[i] = c0;
                        hx[i - 1] = a1; hy[i - 1] = b1; hz[i - 1] = c1;
                    }
                };
                if (inner)
                    h_pass(std::false_type());
                else
                    h_pass(std::true_type());
            }
            // every thread waits on the staging barrier itself: its completion
            // makes the copied shells visible to that thread, so no block
            // barrier is needed here (a timeout is noticed after B2)
            {
                unsigned &nw = cur ? n_wait1 : n_wait0;
                if (!wait_stage(P, &s_bar[cur], nw & 1u, ticket)) s_abort = 1;
                ++nw;
            }

            // D. refills from the staged shells, then publish new H rows for the
            //    warp above's E half-step
            const int xec = (bx - 1) - x0c;  // x offset of the coefficient shell column in its chunk
            // rows of a refilled column whose physical z lies outside the
            // domain: the face buffers hold other cells' values there
#define CLEAR_OUT_ROWS(a, b, c)                                                          \
    do {                                                                                 \
        if (!zin) {                                                                      \
            _Pragma("unroll") for (int i_ = 1; i_ < NR; ++i_) if (i_ < i_lo || i_ >= i_hi) \
                a[i_] = b[i_] = c[i_] = 0.f;                                               \
        }                                                                                \
    } while (0)
            if (w == ey_w) {  // the y shell warp takes its whole column set (level t)
                // row 0 from the lower z shell (its row y = by - 1); rows
                // 1..NZ from the y-face shell (x = bx .. bx+30) or, in the
                // corner lane (x = bx - 1), from the x-face shell's row by - 1
                const int xl = xw - x0, xlc = xw - x0c;
                ex[0] = S::dec(ZST[0 * R::ZB + xl], SC(0));
                ey[0] = S::dec(ZST[1 * R::ZB + xl], SC(1));
                ez[0] = S::dec(ZST[2 * R::ZB + xl], SC(2));
                hx[0] = S::dec(ZST[3 * R::ZB + xl], SC(3));
                hy[0] = S::dec(ZST[4 * R::ZB + xl], SC(4));
                hz[0] = S::dec(ZST[5 * R::ZB + xl], SC(5));
                const bool corner = xw == bx - 1;
                const T *src = corner ? XST : YST + (xw - bx) * BZ;
                const int fst = corner ? R::XB : R::YB;
                ld_rows<S>(src, SC(0), ex);
                ld_rows<S>(src + fst, SC(1), ey);
                ld_rows<S>(src + 2 * fst, SC(2), ez);
                ld_rows<S>(src + 3 * fst, SC(3), hx);
                ld_rows<S>(src + 4 * fst, SC(4), hy);
                ld_rows<S>(src + 5 * fst, SC(5), hz);
                CLEAR_OUT_ROWS(ex, ey, ez);
                CLEAR_OUT_ROWS(hx, hy, hz);
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    CEs[(w * CR + ((bz - 1 + i) & (CR - 1))) * 32 + lane] = YSC[i * SWC + xlc];
                    if (R::LOSSY) CAs[(w * CR + ((bz - 1 + i) & (CR - 1))) * 32 + lane] = YSA[i * SWC + xlc];
                }
            } else if (!ybox) {  // the previous top y row (two outside slots): kept
            } else {  // every lane's row -1 takes the lower z shell's H and coefficient
                const int o = (dy + 1) * SW + (xw - x0), oc = (dy + 1) * SWC + (xw - x0c);
                hx[0] = S::dec(ZST[3 * R::ZB + o], SC(3));
                hy[0] = S::dec(ZST[4 * R::ZB + o], SC(4));
                hz[0] = S::dec(ZST[5 * R::ZB + o], SC(5));
                CEs[(w * CR + ((bz - 1) & (CR - 1))) * 32 + lane] = ZSC[oc];
                if (R::LOSSY) CAs[(w * CR + ((bz - 1) & (CR - 1))) * 32 + lane] = ZSA[oc];
                if (!xbox) {  // the lane leaving the tile in x: rows 1..NZ of H from the x-face shell
                    // (x pairs: from the ring, once the upwind CTA's lanes have arrived)
                    const T *xs = XST + (dy + 1) * BZ;
                    int xst = R::XB;
                    if (R::CL == 2 && rx_msg) {
                        if (!wait_cluster_bar(P, &s_rxf[slot], (unsigned)(mi / R::NSLOT) & 1u, ticket)) s_abort = 1;
                        xs = RX + slot * R::RXS + dy * BZ;
                        xst = 16 * BZ;
                    }
                    ld_rows<S>(xs + 3 * xst, SC(3), hx);
                    ld_rows<S>(xs + 4 * xst, SC(4), hy);
                    ld_rows<S>(xs + 5 * xst, SC(5), hz);
                    CLEAR_OUT_ROWS(hx, hy, hz);
                    const float *xsc = XSC + dy * R::XAC + xec;
                    const float *xsa = XSA + dy * R::XAC + xec;
#pragma unroll
                    for (int i = 1; i < NR; ++i) {
                        CEs[(w * CR + ((bz - 1 + i) & (CR - 1))) * 32 + lane] = xsc[i * 16 * R::XAC];
                        if (R::LOSSY) CAs[(w * CR + ((bz - 1 + i) & (CR - 1))) * 32 + lane] = xsa[i * 16 * R::XAC];
                    }
                }
            }
            if constexpr (R::VX) {
                float *const qx = XHx + xe_at(w, 0, lane), *const qz = XHz + xe_at(w, 0, lane);
#pragma unroll
                for (int i = 1; i < NR; i += 4) {
                    *reinterpret_cast<float4 *>(qx + i - 1) = make_float4(hx[i], hx[i + 1], hx[i + 2], hx[i + 3]);
                    *reinterpret_cast<float4 *>(qz + i - 1) = make_float4(hz[i], hz[i + 1], hz[i + 2], hz[i + 3]);
                }
            } else {
#pragma unroll
                for (int i = 1; i < NR; ++i) {
                    XHx[xe_at(w, i - 1, lane)] = hx[i];
                    XHz[xe_at(w, i - 1, lane)] = hz[i];
                }
            }
            __syncthreads();  // B2
            if (s_abort) { abort = true; break; }
            // the warps outside the box in y sit out the E half-step: the one
            // holding the previous top y row (the y shell's when the box leaves
            // one y slot) publishes level t-1; the y shell's then checks (one
            // poll) whether the upwind tiles have published level t+1 and
            // fetches those shells into the other buffer if so (two buffers).
            // (The release first: the poll after it is cheaper than before it.)
            if (w == yf_w && lane == 0 && t > iv.s) publish(P, tile, ticket, P.epoch + (unsigned)t);  // level t-1 done
            if (w == ey_w) {
                const bool nxt = t + 1 <= iv.e && level_ready(P, U, s_seen, t + 1);
                __syncwarp();  // orders lanes 1, 2's acquires before lane 0's copies
                if (lane == 0) {
                    if (R::NBUF == 2 && nxt) issue_shells(t + 1, cur ^ 1, Ax, Ay, Az, kb);
                    s_pref = nxt ? (R::NBUF == 2 ? 1 : 2) : 0;
                }
            }

            // does this thread own a point source this step?  (16-bit storage:
            // its E rows are rounded after the source is added, not before)
            const long long step = P.step0 + t;
            bool srcthr = false;
            if (S::narrow && tile_src) {
                for (int q = 0; q < P.src.n; ++q) {
                    const SrcDesc &s = P.src.s[q];
                    srcthr |= step < s.n_amp && s.i >= bx && s.i < bx + TX && s.j >= by && s.j < by + TY &&
                              s.k >= bz && s.k < bz + TZ && lane == (s.i & 31) && w == (s.j & (R::RY - 1));
                }
            }

            if (ybox) {
                // F. E half-step, top-down in place: E[i] <- E[i-1] + ce curl_b(H[i], H[i-1], ...)
                const int wm = (w - 1) & (R::RY - 1);
                const int src = (lane - 1) & 31;
                const bool ux = py > 0, uy = px > 0, uz = px > 0 && py > 0;
                const float *const qx = XHx + xe_at(wm, 0, lane), *const qz = XHz + xe_at(wm, 0, lane);
                auto e_pass = [&](auto round, auto masked) {
                    float4 gx, gz;  // VX: the y-1 neighbour's new H rows 4q .. 4q+3
#pragma unroll
                    for (int i = NR - 1; i >= 2; i -= 2) {
                        if (R::VX && i % 4 == 0) {  // rows i-4 .. i-1
                            gx = *reinterpret_cast<const float4 *>(qx + i - 4);
                            gz = *reinterpret_cast<const float4 *>(qz + i - 4);
                        }
                        float ne[2][3];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int r = i - k;
                            const float hz_xm = shfl_from(hz[r], src);
                            const float hy_xm = shfl_from(hy[r], src);
                            const int m = (r - 1) & 3;
                            const float hx_ym = !R::VX ? qx[(r - 1) * 32]
                                                : m == 0 ? gx.x : m == 1 ? gx.y : m == 2 ? gx.z : gx.w;
                            const float hz_ym = !R::VX ? qz[(r - 1) * 32]
                                                : m == 0 ? gz.x : m == 1 ? gz.y : m == 2 ? gz.z : gz.w;
                            const float c = CEs[(w * CR + ((bz + r - 1) & (CR - 1))) * 32 + lane];
                            const float a = R::LOSSY ? CAs[(w * CR + ((bz + r - 1) & (CR - 1))) * 32 + lane] : 1.f;
                            ne[k][0] = e_x(decay<R::LOSSY>(a, ex[r - 1]), hz[r], hz_ym, hy[r], hy[r - 1], c);
                            ne[k][1] = e_y(decay<R::LOSSY>(a, ey[r - 1]), hx[r], hx[r - 1], hz[r], hz_xm, c);
                            ne[k][2] = e_z(decay<R::LOSSY>(a, ez[r - 1]), hy[r], hy_xm, hx[r], hx_ym, c);
                        }
                        if (decltype(round)::value) {
                            RND2(ne[0][0], ne[1][0], 0);
                            RND2(ne[0][1], ne[1][1], 1);
                            RND2(ne[0][2], ne[1][2], 2);
                        }
                        float o[2][3];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int r = i - k;
                            if (decltype(masked)::value) {
                                const bool in = colin && r >= i_lo && r < i_hi;
                                const bool kz = bz + r - 1 > 0;
                                o[k][0] = (in && ux && kz) ? ne[k][0] : ex[r - 1];
                                o[k][1] = (in && uy && kz) ? ne[k][1] : ey[r - 1];
                                o[k][2] = (in && uz) ? ne[k][2] : ez[r - 1];
                            } else {
                                o[k][0] = ne[k][0];
                                o[k][1] = ne[k][1];
                                o[k][2] = ne[k][2];
                            }
                        }
                        ex[i] = o[0][0]; ey[i] = o[0][1]; ez[i] = o[0][2];
                        ex[i - 1] = o[1][0]; ey[i - 1] = o[1][1]; ez[i - 1] = o[1][2];
                    }
                };
                // 16-bit storage rounds each new E value here, except in the
                // (rare) thread that adds a point source this step: it rounds
                // after the source, below (masked form)
                if (S::narrow && srcthr)
                    e_pass(std::false_type(), std::true_type());
                else if (inner)
                    e_pass(std::bool_constant<S::narrow>(), std::false_type());
                else
                    e_pass(std::bool_constant<S::narrow>(), std::true_type());
                {  // every lane's row -1 takes the lower z shell's E (level t)
                    const int o = (dy + 1) * SW + (xw - x0);
                    ex[0] = S::dec(ZST[0 * R::ZB + o], SC(0));
                    ey[0] = S::dec(ZST[1 * R::ZB + o], SC(1));
                    ez[0] = S::dec(ZST[2 * R::ZB + o], SC(2));
                }
                if (!xbox) {  // the x lane: rows 1..NZ of E from the x-face shell (or the ring)
                    const bool ring = R::CL == 2 && rx_msg;
                    const T *xs = ring ? RX + slot * R::RXS + dy * BZ : XST + (dy + 1) * BZ;
                    const int xst = ring ? 16 * BZ : R::XB;
                    ld_rows<S>(xs, SC(0), ex);
                    ld_rows<S>(xs + xst, SC(1), ey);
                    ld_rows<S>(xs + 2 * xst, SC(2), ez);
                    CLEAR_OUT_ROWS(ex, ey, ez);
                }
            }

            // point sources inside the box: the owning thread adds them
            for (int q = 0; tile_src && q < P.src.n; ++q) {
                const SrcDesc &s = P.src.s[q];
                if (step < s.n_amp && s.i >= bx && s.i < bx + TX && s.j >= by && s.j < by + TY &&
                    s.k >= bz && s.k < bz + TZ && lane == (s.i & 31) && w == (s.j & (R::RY - 1))) {
                    const float a = S::src_amp(s.amp[step], P.sc.src);
                    const int ri = s.k - bz + 1;
#pragma unroll
                    for (int i = 1; i < NR; ++i) {
                        if (i == ri) {
                            if (s.comp == 0) ex[i] = add_source(ex[i], a);
                            else if (s.comp == 1) ey[i] = add_source(ey[i], a);
                            else ez[i] = add_source(ez[i], a);
                        }
                    }
                }
            }
            if (S::narrow && srcthr) {  // one rounding per value, as the naive schedule stores it
#pragma unroll
                for (int i = 1; i < NR; i += 2) {
                    RND2(ex[i], ex[i + 1], 0);
                    RND2(ey[i], ey[i + 1], 1);
                    RND2(ez[i], ez[i + 1], 2);
                }
            }

            // the adjoint's recompute: this step's E of the cells of the
            // capture box (tiles that meet it only)
            if (P.cap && colin && bx < P.cap_hi[0] && bx + TX > P.cap_lo[0] && by < P.cap_hi[1] &&
                by + TY > P.cap_lo[1] && bz < P.cap_hi[2] && bz + TZ > P.cap_lo[2] && px >= P.cap_lo[0] &&
                px < P.cap_hi[0] && py >= P.cap_lo[1] && py < P.cap_hi[1]) {
                float *cp = P.cap + 3 * P.cap_bc * (long long)t;
                const int cbx = P.cap_hi[0] - P.cap_lo[0], cby = P.cap_hi[1] - P.cap_lo[1];
                const long long cxy = (long long)(px - P.cap_lo[0]) + (long long)cbx * (py - P.cap_lo[1]);
#pragma unroll
                for (int i = 1; i < NR; ++i) {
                    const int z = bz + i - 1;
                    if (z >= P.cap_lo[2] && z < P.cap_hi[2]) {
                        const long long b = cxy + (long long)cbx * cby * (z - P.cap_lo[2]);
                        cp[b] = ex[i];
                        cp[P.cap_bc + b] = ey[i];
                        cp[2 * P.cap_bc + b] = ez[i];
                    }
                }
            }
            // G. stores: the whole box on the launch's last step, else the top faces
            if (t == P.T - 1) {
                if (colin) {
#pragma unroll
                    for (int i = 1; i < NR; ++i) {
                        if (i >= i_lo && i < i_hi) {
                            const long long g = col + sxy * (bz + i - 1);
                            STORE6(g, i);
                        }
                    }
                }
            } else if (colin) {
                // (the top y face is stored next step by the warp holding it)
                if (NR - 1 >= i_lo && NR - 1 < i_hi) {  // top z face
                    const long long g = col + sxy * (bz + NR - 2);
                    STORE6(g, NR - 1);
                }
            }
            // top x face (all rows of the lane leaving the box in x) into the
            // x-face buffer, where the downwind tile's x shell is fetched.
            // x pairs, rank 0: into rank 1's ring instead (its slot was freed
            // before the second barrier), every box row's lane then arriving
            // on the slot's barrier; the top box row still goes to the x-face
            // buffer too (the corner of the next pair's y shell)
            if (ybox && dx == TX - 1) {
                if (R::CL == 2 && tx_msg) {
                    // the slot's previous message must have been read
                    if (mi >= R::NSLOT &&
                        !wait_cluster_bar(P, &s_rxe[slot], (unsigned)((mi / R::NSLOT) - 1) & 1u, ticket))
                        s_abort = 1;
                    const unsigned a = rx_remote + (unsigned)((slot * R::RXS + dy * BZ) * (int)sizeof(T));
                    constexpr unsigned FS = 16u * BZ * (unsigned)sizeof(T);
                    st_rows_remote<S>(a, IS(0), ex);
                    st_rows_remote<S>(a + FS, IS(1), ey);
                    st_rows_remote<S>(a + 2 * FS, IS(2), ez);
                    st_rows_remote<S>(a + 3 * FS, IS(3), hx);
                    st_rows_remote<S>(a + 4 * FS, IS(4), hy);
                    st_rows_remote<S>(a + 5 * FS, IS(5), hz);
                }
                if ((!(R::CL == 2 && tx_msg) || dy == TY - 1) && (unsigned)px < (unsigned)P.nx &&
                    (unsigned)py < (unsigned)P.ny)
                    FACE_STORE(XFk + ((long long)px * P.ny + py) * BZ, P.fxs, bz);
            }
            if (R::CL == 2 && msg) sig_slot = slot;
        }
        if (abort) break;
        // the last step's top y face (the launch's last one included: the
        // downwind tile reads it from the y-face buffer), then its progress
        __syncthreads();
        if (R::CL == 2 && sig_slot >= 0) {  // the tile's last message: filled / read
            if (tid == 0) arrive_remote((rank == 0 ? rxf_remote : rxe_remote) + 8u * (unsigned)sig_slot);
            sig_slot = -1;
        }
        {
            const int pbx = Ax - iv.e, pby = Ay - iv.e, pbz = Az - iv.e;
            const int pdx = (lane - pbx) & 31, pdy = (w - pby) & (R::RY - 1);
            const int qx = pbx + pdx, qy = pby + pdy;
            if (pdy == TY - 1 && pdx < TX && (unsigned)qx < (unsigned)P.nx && (unsigned)qy < (unsigned)P.ny)
                FACE_STORE(YFk + ((long long)qy * P.nx + qx) * BZ, P.fys, pbz);
        }
        __syncthreads();
        if (tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.e + 1u);
        } while (false);
        msg_base += nmsg;
        sig_slot = -1;
        if (R::CL == 1 && abort) break;  // a pair leaves together, at the next ticket
    }
    // after an abort, bulk copies may still be writing into the staging
    // buffers: wait for them (bounded) before the CTA's shared memory goes
    if (tid == 0) {
        while (n_wait0 < s_niss[0] && wait_stage(P, &s_bar[0], n_wait0 & 1u, -1)) ++n_wait0;
        while (n_wait1 < s_niss[1] && wait_stage(P, &s_bar[1], n_wait1 & 1u, -1)) ++n_wait1;
    }
    // x pairs: neither CTA leaves while its partner may still write into its
    // shared memory
    if constexpr (R::CL == 2) cluster_sync_all();
}

#undef F0
#undef F1
#undef F2
#undef F3
#undef F4
#undef F5
#undef CE
#undef CA
#undef SC
#undef IS
#undef RND
#undef RND2
#undef STORE6
#undef FACE_STORE
#undef CLEAR_OUT_ROWS

// 31 x 15 x 12 and 31 x 15 x 8 tiles, each for every kernel format; the
// lossy (absorber) form for the 31 x 15 x 12 tile
// the box leaves one y slot of the ring outside (TY = 15): as fast as two
// outside slots (TY = 14) and updates more cells per step
constexpr int REG_TY = 15;
template <int NZ>
struct RegShape {
    static constexpr bool HAS_LOSSY = NZ == 12;
    static constexpr bool HAS_PAIRS = NZ == 12;  // x pairs in thread-block clusters: the 31 x 15 x 12 tile
    static cudaError_t configure(int fmt, bool lossy, int cl)
    {
        if (lossy) {
            if constexpr (HAS_LOSSY) if (cl == 1) DISPATCH_FORMAT(fmt, S, set<RegTile<NZ, S, true, REG_TY>>());
            return cudaErrorInvalidValue;
        }
        if (cl == 2) {
            if constexpr (HAS_PAIRS) DISPATCH_FORMAT(fmt, S, set<RegTile<NZ, S, false, REG_TY, 2>>());
            return cudaErrorInvalidValue;
        }
        DISPATCH_FORMAT(fmt, S, set<RegTile<NZ, S, false, REG_TY>>());
    }
    static int per_sm(int fmt, bool lossy)
    {
        if (lossy) {
            if constexpr (HAS_LOSSY) DISPATCH_FORMAT(fmt, S, occ<RegTile<NZ, S, true, REG_TY>>());
            return 0;
        }
        DISPATCH_FORMAT(fmt, S, occ<RegTile<NZ, S, false, REG_TY>>());
    }
    static int clusters(int fmt)
    {
        if constexpr (HAS_PAIRS) DISPATCH_FORMAT(fmt, S, occ_pairs<RegTile<NZ, S, false, REG_TY, 2>>());
        return 0;
    }
    static cudaError_t launch(const SysLaunch &p, int grid, cudaStream_t st, int fmt, int cl)
    {
        if (p.ca) {
            if constexpr (HAS_LOSSY) if (cl == 1) DISPATCH_FORMAT(fmt, S, go<RegTile<NZ, S, true, REG_TY>>(p, grid, st));
            return cudaErrorInvalidValue;
        }
        if (cl == 2) {
            if constexpr (HAS_PAIRS) DISPATCH_FORMAT(fmt, S, go<RegTile<NZ, S, false, REG_TY, 2>>(p, grid, st));
            return cudaErrorInvalidValue;
        }
        DISPATCH_FORMAT(fmt, S, go<RegTile<NZ, S, false, REG_TY>>(p, grid, st));
    }
    template <class R>
    static cudaError_t set()
    {
        return cudaFuncSetAttribute(systolic_reg_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)R::smem_bytes());
    }
    template <class R>
    static int occ()
    {
        int n = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, systolic_reg_kernel<R>, R::NT, R::smem_bytes()) ==
                       cudaSuccess
                   ? n
                   : 0;
    }
    template <class R>
    static cudaLaunchConfig_t config(int grid, cudaStream_t st, cudaLaunchAttribute *at)
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)R::NT);
        cfg.dynamicSmemBytes = R::smem_bytes();
        cfg.stream = st;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)R::CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cfg;
    }
    // co-resident clusters of a pair kernel on this device
    template <class R>
    static int occ_pairs()
    {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = config<R>(2, 0, at);
        int n = 0;
        return cudaOccupancyMaxActiveClusters(&n, systolic_reg_kernel<R>, &cfg) == cudaSuccess ? n : 0;
    }
    template <class R>
    static cudaError_t go(const SysLaunch &p, int grid, cudaStream_t st)
    {
        if constexpr (R::CL == 1) {
            systolic_reg_kernel<R><<<grid, R::NT, R::smem_bytes(), st>>>(p);
            return cudaGetLastError();
        } else {
            cudaLaunchAttribute at[1];
            cudaLaunchConfig_t cfg = config<R>(grid, st, at);
            return cudaLaunchKernelEx(&cfg, systolic_reg_kernel<R>, p);
        }
    }
};

using RegA = RegShape<12>;  // 31 x 15 x 12
using RegB = RegShape<8>;   // 31 x 15 x 8

} // namespace

int systolic_reg_rows(int k) { return (k == 0 ? 12 : 8) + 1; }

SysShape systolic_reg_shape(int k) { return SysShape{31, REG_TY, k == 0 ? 12 : 8}; }

cudaError_t systolic_reg_configure(int k, int fmt, bool lossy, int cl)
{
    return k == 0 ? RegA::configure(fmt, lossy, cl) : RegB::configure(fmt, lossy, cl);
}

int systolic_reg_max_ctas_per_sm(int k, int fmt, bool lossy)
{
    return k == 0 ? RegA::per_sm(fmt, lossy) : RegB::per_sm(fmt, lossy);
}

int systolic_reg_max_pairs(int k, int fmt) { return k == 0 ? RegA::clusters(fmt) : RegB::clusters(fmt); }

cudaError_t launch_systolic_reg(const SysLaunch &p, int grid, cudaStream_t st, int k, int fmt, int cl)
{
    return k == 0 ? RegA::launch(p, grid, st, fmt, cl) : RegB::launch(p, grid, st, fmt, cl);
}
