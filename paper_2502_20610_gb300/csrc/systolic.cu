// Systolic schedule (Sec. 3, Fig. 7; Sec. 4): a persistent kernel in which
// every CTA holds one subdomain ("tile") of the grid in shared memory and
// advances it many steps, scanning it along the x-y-z-t diagonal.  Only the
// boundary faces of a tile travel through global memory; the interior never
// leaves the SM.  There is no grid-wide synchronisation: a tile waits only
// on the progress flags of its three upwind face neighbours.
//
// Geometry.  In skewed coordinates sigma = p + t (p physical cell, t step of
// this launch) the Yee dependencies of step t on step t-1 have offsets in
// {-1,0}^3: H^{t+1/2}(p) reads H^{t-1/2}(p), E^t(p), E^t(p+e_a), and
// E^{t+1}(p) reads E^t(p), H^{t+1/2}(p), H^{t+1/2}(p-e_b).  So a tile is a
// fixed box [A, A+n) of sigma space whose physical footprint moves by
// (-1,-1,-1) per step, and it depends only on the tiles at lower sigma:
// the one-directional ("downwind-only") flow of Sec. 3.
//
// Per step t a tile with box B_t = [A-t, A-t+n) does, on a ring of
// (n+1)^3 shared-memory slots indexed by physical position mod (n+1):
//   1. wait until its -x, -y, -z neighbours have finished step t;
//   2. issue the loads of its lower shell (cells with some p_a = A_a-t-1,
//      state H^{t+1/2}, E^{t+1}) into registers;
//   3. H half-step on B_t (reads E one cell above the box: the slot of the
//      cell it left behind last step);
//   4. write the shell into the slots of that trailing top layer;
//   5. E half-step on B_t (+ point sources);
//   6. store its top faces (state H^{t+1/2}, E^{t+1}) to the global field
//      arrays, which are the trail the downwind tiles pick up (Sec. 3, the
//      trail of boundary values left behind for the downwind subdomain);
//   7. release its progress flag = epoch + t + 1.
// Tile size: 31 x 15 x 15 updated, 32 x 16 x 16 stored (Sec. 4).
//
// Every arithmetic step is yee_cell.cuh, so the result equals the naive
// schedule bit for bit.
#include "internal.h"
#include "sys_common.cuh"
#include "yee_cell.cuh"

namespace {

using namespace sysc;

// Ring geometry: RX x RY x RZ shared-memory slots per tile, (RX-1) x
// (RY-1) x (RZ-1) cells updated per step, one thread per (x,y) ring column.
template <int RY_, int RZ_, int MINB_>
struct Ring {
    static constexpr int RX = 32, RY = RY_, RZ = RZ_, MINB = MINB_;
    static constexpr int TX = RX - 1, TY = RY - 1, TZ = RZ - 1;
    static constexpr int VOL = RX * RY * RZ;
    static constexpr int NTHREADS = RX * RY;
    static constexpr int SHELL_Z = RX * RY;             // slots with z extra
    static constexpr int SHELL_Y = RX * (RZ - 1);       // y extra, z not
    static constexpr int SHELL_X = (RY - 1) * (RZ - 1); // x extra only
    static constexpr int SHELL = SHELL_Z + SHELL_Y + SHELL_X;
    static constexpr int SHELL_PT = (SHELL + NTHREADS - 1) / NTHREADS;
    static constexpr int TOP_Z = TX * TY;
    static constexpr int TOP_Y = TX * (TZ - 1);
    static constexpr int TOP_X = (TY - 1) * (TZ - 1);
    static constexpr int TOP = TOP_Z + TOP_Y + TOP_X;
    static constexpr int TOP_PT = (TOP + NTHREADS - 1) / NTHREADS;
    static constexpr int ZS = RY * 32;  // floats between consecutive z rows of the ring
    static_assert((RY & (RY - 1)) == 0 && (RZ & (RZ - 1)) == 0, "ring sizes are powers of two");
    static_assert(SHELL == VOL - TX * TY * TZ, "shell enumeration");
    static_assert(TOP == TX * TY * TZ - (TX - 1) * (TY - 1) * (TZ - 1), "top-face enumeration");
    static constexpr size_t smem_bytes() { return sizeof(float) * 7 * (size_t)VOL; }
};

// Shared-memory slot of ring position (sx, sy, sz).  Rows of 32 x-slots are
// rotated by sy, so a warp reading one row, or reading one x-slot across the
// y-slots, touches distinct banks; the rotation is a per-thread constant.
template <class R>
__device__ __forceinline__ int slot(int sx, int sy, int sz)
{
    return ((sz * R::RY + sy) << 5) | ((sx + sy) & 31);
}

// Shell entry f in [0, SHELL): face category and two coordinates inside the
// face, packed as cat | a << 8 | b << 16 (computed once per thread).
//   cat 0 (z face): ring sx = a, sy = b
//   cat 1 (y face, z not extra): ring sx = a, z offset b in [0, RZ-1)
//   cat 2 (x face only): y offset a, z offset b in [0, RY-1) x [0, RZ-1)
template <class R>
__device__ __forceinline__ int shell_code(int f)
{
    if (f >= R::SHELL) return -1;
    if (f < R::SHELL_Z) return 0 | ((f & 31) << 8) | ((f >> 5) << 16);
    if (f < R::SHELL_Z + R::SHELL_Y) {
        const int g = f - R::SHELL_Z;
        return 1 | ((g & 31) << 8) | ((g >> 5) << 16);
    }
    const int g = f - R::SHELL_Z - R::SHELL_Y;
    return 2 | ((g % (R::RY - 1)) << 8) | ((g / (R::RY - 1)) << 16);
}

// Ring slot and physical cell of a shell entry for the E window of step t,
// whose lower corner is b - 1 and whose extra ring slot is e = (b-1) mod R.
template <class R>
__device__ __forceinline__ void shell_cell(int code, int bx, int by, int bz, int &o, int &px, int &py,
                                           int &pz)
{
    const int cat = code & 0xff, a = (code >> 8) & 0xff, b = code >> 16;
    const int ex = (bx - 1) & 31, ey = (by - 1) & (R::RY - 1), ez = (bz - 1) & (R::RZ - 1);
    int sx, sy, sz;
    if (cat == 0) {
        sx = a; sy = b; sz = ez;
        px = bx - 1 + ((a - bx + 1) & 31); py = by - 1 + ((b - by + 1) & (R::RY - 1)); pz = bz - 1;
    } else if (cat == 1) {
        sx = a; sy = ey; sz = (ez + 1 + b) & (R::RZ - 1);
        px = bx - 1 + ((a - bx + 1) & 31); py = by - 1; pz = bz + b;
    } else {
        sx = ex; sy = (ey + 1 + a) & (R::RY - 1); sz = (ez + 1 + b) & (R::RZ - 1);
        px = bx - 1; py = by + a; pz = bz + b;
    }
    o = slot<R>(sx, sy, sz);
}

// Top-face entry f in [0, TOP): box offsets packed dx | dy << 8 | dz << 16.
template <class R>
__device__ __forceinline__ int top_code(int f)
{
    if (f >= R::TOP) return -1;
    int dx, dy, dz;
    if (f < R::TOP_Z) {
        dx = f % R::TX; dy = f / R::TX; dz = R::TZ - 1;
    } else if (f < R::TOP_Z + R::TOP_Y) {
        const int g = f - R::TOP_Z;
        dx = g % R::TX; dz = g / R::TX; dy = R::TY - 1;
    } else {
        const int g = f - R::TOP_Z - R::TOP_Y;
        dx = R::TX - 1; dy = g % (R::TY - 1); dz = g / (R::TY - 1);
    }
    return dx | (dy << 8) | (dz << 16);
}

template <class R>
__global__ void __launch_bounds__(R::NTHREADS, R::MINB) systolic_kernel(const SysLaunch P)
{
    constexpr int RY = R::RY, RZ = R::RZ, TX = R::TX, TY = R::TY, TZ = R::TZ;
    constexpr int VOL = R::VOL, NTHREADS = R::NTHREADS, SHELL_PT = R::SHELL_PT, TOP_PT = R::TOP_PT;
    constexpr int ZS = R::ZS;
    extern __shared__ float smem[];
    float *const sEx = smem, *const sEy = smem + VOL, *const sEz = smem + 2 * VOL;
    float *const sHx = smem + 3 * VOL, *const sHy = smem + 4 * VOL, *const sHz = smem + 5 * VOL;
    float *const sCE = smem + 6 * VOL;
    float *const sF[6] = {sEx, sEy, sEz, sHx, sHy, sHz};
    __shared__ int s_ticket, s_abort;
    __shared__ unsigned s_seen[3];

    const int tid = threadIdx.x;
    const int sx = tid & 31, sy = tid >> 5;
    const int warp = tid >> 5;
    const float ndt = P.neg_dt;

    // per-thread constant ring offsets of the column and its x/y neighbours
    const int syp = (sy + 1) & (RY - 1), sym = (sy - 1) & (RY - 1);
    const int o_s = (sy << 5) | ((sx + sy) & 31);
    const int o_xp = (sy << 5) | ((sx + 1 + sy) & 31);
    const int o_xm = (sy << 5) | ((sx - 1 + sy) & 31);
    const int o_yp = (syp << 5) | ((sx + syp) & 31);
    const int o_ym = (sym << 5) | ((sx + sym) & 31);
    int sh_code[SHELL_PT], tp_code[TOP_PT];
#pragma unroll
    for (int q = 0; q < SHELL_PT; ++q) sh_code[q] = shell_code<R>(tid + q * NTHREADS);
#pragma unroll
    for (int q = 0; q < TOP_PT; ++q) tp_code[q] = top_code<R>(tid + q * NTHREADS);

    for (;;) {
        if (tid == 0) {
            s_ticket = atomicAdd(P.ctrl, 1);
            s_abort = ld_volatile(P.ctrl + 1) != DEV_OK;
        }
        if (tid < 3) s_seen[tid] = 0u;
        __syncthreads();
        const int ticket = s_ticket;
        const bool stop = s_abort || ticket >= P.ntiles;
        __syncthreads();  // every thread has read s_ticket / s_abort
        if (stop) break;
        const int tile = P.tiles[ticket];
        const int I = tile % P.gx, J = (tile / P.gx) % P.gy, K = tile / (P.gx * P.gy);
        const int Ax = I * TX, Ay = J * TY, Az = K * TZ;
        const Interval iv = tile_interval<R::TX, R::TY, R::TZ>(P, I, J, K);
        Upwind U;
        {
            const int nb[3][3] = {{I - 1, J, K}, {I, J - 1, K}, {I, J, K - 1}};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (nb[a][0] < 0 || nb[a][1] < 0 || nb[a][2] < 0) {
                    U.id[a] = -1; U.s[a] = 1; U.e[a] = -1;
                } else {
                    const Interval u = tile_interval<R::TX, R::TY, R::TZ>(P, nb[a][0], nb[a][1], nb[a][2]);
                    U.id[a] = nb[a][0] + P.gx * (nb[a][1] + P.gy * nb[a][2]);
                    U.s[a] = u.s; U.e[a] = u.e;
                }
            }
        }

        if (iv.s > 0) {
            if (warp == 0) {
                const bool ok = wait_level(P, U, s_seen, iv.s - 1, ticket);
                if (tid == 0) s_abort = !ok;
            }
            __syncthreads();
            if (s_abort) break;
        }
        if (iv.s > iv.e) {  // enters the domain only after this launch: relay only
            if (tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.s);
            __syncthreads();
            continue;
        }

        // Initial load of the H window [b, b+n] at level start-1.
        {
            const int bx = Ax - iv.s, by = Ay - iv.s, bz = Az - iv.s;
            const int px = bx + ((sx - bx) & 31), py = by + ((sy - by) & (RY - 1));
            for (int sz = 0; sz < RZ; ++sz) {
                const int pz = bz + ((sz - bz) & (RZ - 1));
                const int o = sz * ZS + o_s;
                if (in_dom(P, px, py, pz)) {
                    const long long g = gidx(P, px, py, pz);
#pragma unroll
                    for (int c = 0; c < 6; ++c) sF[c][o] = ld_cg(P.f[c] + g);
                    sCE[o] = __ldg(P.ce + g);
                } else {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sF[c][o] = 0.f;
                    sCE[o] = 0.f;
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            if (iv.s > 0 && tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.s);
            const bool ok = wait_level(P, U, s_seen, iv.s, ticket);
            if (tid == 0) s_abort = !ok;
        }
        __syncthreads();
        if (s_abort) break;

        bool abort = false;
        for (int t = iv.s; t <= iv.e; ++t) {
            const int bx = Ax - t, by = Ay - t, bz = Az - t;  // box low corner at step t

            // 1. lower shell (level t; upwind neighbours are done) into registers
            float shv[SHELL_PT][7];
            int sho[SHELL_PT];
#pragma unroll
            for (int q = 0; q < SHELL_PT; ++q) {
                sho[q] = -1;
                if (sh_code[q] >= 0) {
                    int px, py, pz;
                    shell_cell<R>(sh_code[q], bx, by, bz, sho[q], px, py, pz);
                    if (in_dom(P, px, py, pz)) {
                        const long long g = gidx(P, px, py, pz);
#pragma unroll
                        for (int c = 0; c < 6; ++c) shv[q][c] = ld_cg(P.f[c] + g);
                        shv[q][6] = __ldg(P.ce + g);
                    } else {
#pragma unroll
                        for (int c = 0; c < 7; ++c) shv[q][c] = 0.f;
                    }
                }
            }

            // this thread's (x,y) column of the box and its z range in the domain
            const int dxc = (sx - bx) & 31, dyc = (sy - by) & (RY - 1);
            const int px = bx + dxc, py = by + dyc;
            const bool col = dxc < TX && dyc < TY && (unsigned)px < (unsigned)P.nx &&
                             (unsigned)py < (unsigned)P.ny;
            const int dz_lo = max(0, -bz), dz_hi = min(TZ, P.nz - bz);
            const int r0 = bz & (RZ - 1);

            // 2. H half-step on the box.  The thread walks the 16 ring rows of its
            //    column in fixed order (row r holds box offset dz = (r - r0) mod RZ,
            //    dz = TZ being the trailing row), so every shared-memory address is
            //    a per-thread base plus a constant.
            if (col) {
                float exc = sEx[o_s], eyc = sEy[o_s];
                const float ex0 = exc, ey0 = eyc;
#pragma unroll
                for (int r = 0; r < RZ; ++r) {
                    const int rn = (r + 1) & (RZ - 1);
                    const float exn = rn == 0 ? ex0 : sEx[rn * ZS + o_s];
                    const float eyn = rn == 0 ? ey0 : sEy[rn * ZS + o_s];
                    const int dz = (r - r0) & (RZ - 1);
                    if (dz >= dz_lo && dz < dz_hi) {
                        const int o = r * ZS + o_s;
                        const float ez = sEz[o];
                        sHx[o] = h_x(sHx[o], sEz[r * ZS + o_yp], ez, eyn, eyc, ndt);
                        sHy[o] = h_y(sHy[o], exn, exc, sEz[r * ZS + o_xp], ez, ndt);
                        sHz[o] = h_z(sHz[o], sEy[r * ZS + o_xp], eyc, sEx[r * ZS + o_yp], exc, ndt);
                    }
                    exc = exn;
                    eyc = eyn;
                }
            }
            __syncthreads();

            // 3. shell into the slots of the trailing top layer
#pragma unroll
            for (int q = 0; q < SHELL_PT; ++q) {
                if (sho[q] >= 0) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sF[c][sho[q]] = shv[q][c];
                    sCE[sho[q]] = shv[q][6];
                }
            }
            __syncthreads();

            // 4. E half-step on the box, same row order; PEC: tangential E on low
            //    planes fixed
            if (col) {
                const bool ux = py > 0, uy = px > 0, uz = px > 0 && py > 0;
                float hxm = sHx[(RZ - 1) * ZS + o_s], hym = sHy[(RZ - 1) * ZS + o_s];
#pragma unroll
                for (int r = 0; r < RZ; ++r) {
                    const int o = r * ZS + o_s;
                    const float hx = sHx[o], hy = sHy[o];
                    const int dz = (r - r0) & (RZ - 1);
                    if (dz >= dz_lo && dz < dz_hi) {
                        const float hz = sHz[o], ce = sCE[o];
                        const bool kz = bz + dz > 0;
                        if (ux && kz) sEx[o] = e_x(sEx[o], hz, sHz[r * ZS + o_ym], hy, hym, ce);
                        if (uy && kz) sEy[o] = e_y(sEy[o], hx, hxm, hz, sHz[r * ZS + o_xm], ce);
                        if (uz) sEz[o] = e_z(sEz[o], hy, sHy[r * ZS + o_xm], hx, sHx[r * ZS + o_ym], ce);
                    }
                    hxm = hx;
                    hym = hy;
                }
            }
            __syncthreads();

            // point sources inside the box (uniform test, thread 0 applies)
            {
                const long long step = P.step0 + t;
                bool any = false;
                for (int q = 0; q < P.src.n; ++q) {
                    const SrcDesc &s = P.src.s[q];
                    any |= step < s.n_amp && s.i >= bx && s.i < bx + TX && s.j >= by &&
                           s.j < by + TY && s.k >= bz && s.k < bz + TZ;
                }
                if (any) {
                    if (tid == 0) {
                        for (int q = 0; q < P.src.n; ++q) {
                            const SrcDesc &s = P.src.s[q];
                            if (step < s.n_amp && s.i >= bx && s.i < bx + TX && s.j >= by &&
                                s.j < by + TY && s.k >= bz && s.k < bz + TZ) {
                                const int o = slot<R>(s.i & 31, s.j & (RY - 1), s.k & (RZ - 1));
                                sF[s.comp][o] = add_source(sF[s.comp][o], s.amp[step]);
                            }
                        }
                    }
                    __syncthreads();
                }
            }

            // 5. warp 0 waits for the upwind neighbours' next level while
            //    everyone stores the top faces (or, on the launch's last
            //    step, the whole box)
            bool ok = true;
            if (warp == 0 && t < iv.e) ok = wait_level(P, U, s_seen, t + 1, ticket);
            if (t == P.T - 1) {
                if (col) {
                    for (int dz = dz_lo; dz < dz_hi; ++dz) {
                        const int pz = bz + dz;
                        const int o = (pz & (RZ - 1)) * ZS + o_s;
                        const long long g = gidx(P, px, py, pz);
#pragma unroll
                        for (int c = 0; c < 6; ++c) P.f[c][g] = sF[c][o];
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < TOP_PT; ++q) {
                    const int code = tp_code[q];
                    if (code >= 0) {
                        const int qx = bx + (code & 0xff), qy = by + ((code >> 8) & 0xff),
                                  qz = bz + (code >> 16);
                        if (in_dom(P, qx, qy, qz)) {
                            const int o = slot<R>(qx & 31, qy & (RY - 1), qz & (RZ - 1));
                            const long long g = gidx(P, qx, qy, qz);
#pragma unroll
                            for (int c = 0; c < 6; ++c) P.f[c][g] = sF[c][o];
                        }
                    }
                }
            }
            if (tid == 0) s_abort = !ok;
            __syncthreads();
            if (s_abort) { abort = true; break; }

            // 6. release progress (the other warps move on to the next step)
            if (tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)t + 1u);
        }
        if (abort) break;
        __syncthreads();
    }
}

using RingA = Ring<16, 16, 1>;  // 31 x 15 x 15 updated, 32 x 16 x 16 stored, 1 CTA per SM
using RingB = Ring<8, 16, 2>;   // 31 x 7 x 15 updated, 32 x 8 x 16 stored, 2 CTAs per SM

const SysShape kShapes[2] = {{RingA::TX, RingA::TY, RingA::TZ}, {RingB::TX, RingB::TY, RingB::TZ}};

} // namespace

SysShape systolic_shape(int v) { return v >= 2 ? systolic_reg_shape(v - 2) : kShapes[v]; }

size_t systolic_smem_bytes(int v) { return v == 0 ? RingA::smem_bytes() : RingB::smem_bytes(); }

cudaError_t systolic_configure(int v, int storage, bool lossy, int cl)
{
    if (v >= 2) return systolic_reg_configure(v - 2, storage, lossy, cl);
    if (storage != FDTD_STORAGE_F32 || lossy || cl != 1) return cudaErrorInvalidValue;
    if (v == 0)
        return cudaFuncSetAttribute(systolic_kernel<RingA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)RingA::smem_bytes());
    return cudaFuncSetAttribute(systolic_kernel<RingB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RingB::smem_bytes());
}

int systolic_max_ctas_per_sm(int v, int storage, bool lossy)
{
    if (v >= 2) return systolic_reg_max_ctas_per_sm(v - 2, storage, lossy);
    if (storage != FDTD_STORAGE_F32 || lossy) return 0;
    int n = 0;
    cudaError_t e = v == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, systolic_kernel<RingA>,
                                                                          RingA::NTHREADS, RingA::smem_bytes())
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, systolic_kernel<RingB>,
                                                                          RingB::NTHREADS, RingB::smem_bytes());
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_systolic(const SysLaunch &p, int grid, cudaStream_t st, int v, int storage, int cl)
{
    if (v >= 2) return launch_systolic_reg(p, grid, st, v - 2, storage, cl);
    if (storage != FDTD_STORAGE_F32 || p.ca || cl != 1) return cudaErrorInvalidValue;
    if (v == 0)
        systolic_kernel<RingA><<<grid, RingA::NTHREADS, RingA::smem_bytes(), st>>>(p);
    else
        systolic_kernel<RingB><<<grid, RingB::NTHREADS, RingB::smem_bytes(), st>>>(p);
    return cudaGetLastError();
}
