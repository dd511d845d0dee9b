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
#include "yee_cell.cuh"

namespace {

constexpr int RX = SYS_RX, RY = SYS_RY, RZ = SYS_RZ;
constexpr int TX = SYS_NX, TY = SYS_NY, TZ = SYS_NZ;
constexpr int VOL = RX * RY * RZ;
constexpr int NTHREADS = RX * RY;
constexpr int SHELL_Z = RX * RY;             // slots with z extra
constexpr int SHELL_Y = RX * (RZ - 1);       // y extra, z not
constexpr int SHELL_X = (RY - 1) * (RZ - 1); // x extra only
constexpr int SHELL = SHELL_Z + SHELL_Y + SHELL_X;
constexpr int SHELL_PT = (SHELL + NTHREADS - 1) / NTHREADS;
constexpr int TOP_Z = TX * TY;
constexpr int TOP_Y = TX * (TZ - 1);
constexpr int TOP_X = (TY - 1) * (TZ - 1);
constexpr int TOP = TOP_Z + TOP_Y + TOP_X;
static_assert(RX == 32, "one warp spans the x ring");
static_assert((RY & (RY - 1)) == 0 && (RZ & (RZ - 1)) == 0, "ring sizes are powers of two");
static_assert(SHELL == VOL - TX * TY * TZ, "shell enumeration");
static_assert(TOP == TX * TY * TZ - (TX - 1) * (TY - 1) * (TZ - 1), "top-face enumeration");

// Shared-memory slot of ring position (sx, sy, sz).  Rows of 32 x-slots are
// rotated by their row index, so a warp reading one row, or reading one
// x-slot of 32 consecutive rows, touches 32 distinct banks.
__device__ __forceinline__ int slot(int sx, int sy, int sz)
{
    const int row = sz * RY + sy;
    return (row << 5) | ((sx + row) & 31);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int *p)
{
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Loads of data produced by other CTAs during this launch go to L2 (.cg),
// never to a possibly stale L1 line.
__device__ __forceinline__ float ld_cg(const float *p)
{
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

struct Interval { int s, e; };

__device__ __forceinline__ Interval tile_interval(const SysLaunch &P, int I, int J, int K)
{
    const int ax = I * TX, ay = J * TY, az = K * TZ;
    Interval r;
    r.s = max(0, max(ax - P.nx + 1, max(ay - P.ny + 1, az - P.nz + 1)));
    r.e = min(P.T - 1, min(ax + TX - 1, min(ay + TY - 1, az + TZ - 1)));
    return r;
}

// Bounded spin on one flag.  Returns false if the launch is aborting.
__device__ bool wait_flag(const SysLaunch &P, const unsigned *flag, unsigned target, int ticket)
{
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
        if (ld_acquire(flag) >= target) return true;
        if (ld_volatile(P.ctrl + 1) != DEV_OK) return false;
        const unsigned long long now = globaltimer();
        if (it == 0) {
            t0 = now;
        } else if (now - t0 > (unsigned long long)P.timeout_ns) {
            if (atomicCAS(P.ctrl + 1, DEV_OK, DEV_ERR_TIMEOUT) == DEV_OK) {
                P.ctrl[2] = ticket;
                P.ctrl[3] = (int)target;
            }
            return false;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
}

// Wait until every -x, -y, -z neighbour that holds state at level L has
// completed it (progress >= epoch + L + 1).  A neighbour u is waited on if
// start(u)-1 <= L <= end(u) and start(u) <= end(u)+1: outside that range its
// cells at level L are outside the domain.  Subdomains that enter the domain
// at L+1 publish epoch+start(u) after their own initial wait, which carries
// the guarantee of the tiles behind them.  Thread 0 only.
__device__ bool wait_upstream(const SysLaunch &P, int I, int J, int K, int L, int ticket)
{
    if (ld_volatile(P.ctrl + 1) != DEV_OK) return false;
    const unsigned target = P.epoch + (unsigned)L + 1u;
    const int nb[3][3] = {{I - 1, J, K}, {I, J - 1, K}, {I, J, K - 1}};
    for (int a = 0; a < 3; ++a) {
        const int u0 = nb[a][0], u1 = nb[a][1], u2 = nb[a][2];
        if (u0 < 0 || u1 < 0 || u2 < 0) continue;
        const Interval iv = tile_interval(P, u0, u1, u2);
        if (iv.s > iv.e + 1 || L < iv.s - 1 || L > iv.e) continue;
        const int id = u0 + P.gx * (u1 + P.gy * u2);
        if (!wait_flag(P, P.progress + id, target, ticket)) return false;
    }
    return true;
}

__device__ __forceinline__ void publish(const SysLaunch &P, int tile, int ticket, unsigned value)
{
    if (P.dbg_kind == 1 /* skip publish */ && ticket == P.dbg_ticket) return;
    if (P.dbg_kind == 2 /* delay */ && P.dbg_param > 0 && (ticket % P.dbg_param) == P.dbg_ticket)
        __nanosleep((unsigned)P.dbg_param2);
    __threadfence();
    st_release(P.progress + tile, value);
}

__device__ __forceinline__ bool in_dom(const SysLaunch &P, int x, int y, int z)
{
    return (unsigned)x < (unsigned)P.nx && (unsigned)y < (unsigned)P.ny && (unsigned)z < (unsigned)P.nz;
}

__device__ __forceinline__ long long gidx(const SysLaunch &P, int x, int y, int z)
{
    return x + (long long)P.nx * (y + (long long)P.ny * z);
}

// Ring slot (sx,sy,sz) of shell entry f in [0, SHELL) for a window whose
// extra slot is (ex, ey, ez).
__device__ __forceinline__ void shell_slot(int f, int ex, int ey, int ez, int &sx, int &sy, int &sz)
{
    if (f < SHELL_Z) {
        sx = f & 31; sy = f >> 5; sz = ez;
    } else if (f < SHELL_Z + SHELL_Y) {
        const int g = f - SHELL_Z;
        sx = g & 31; sy = ey; sz = (ez + 1 + (g >> 5)) & (RZ - 1);
    } else {
        const int g = f - SHELL_Z - SHELL_Y;
        sx = ex; sy = (ey + 1 + g % (RY - 1)) & (RY - 1); sz = (ez + 1 + g / (RY - 1)) & (RZ - 1);
    }
}

// Box offsets (dx,dy,dz) of top-face entry f in [0, TOP).
__device__ __forceinline__ void top_cell(int f, int &dx, int &dy, int &dz)
{
    if (f < TOP_Z) {
        dx = f % TX; dy = f / TX; dz = TZ - 1;
    } else if (f < TOP_Z + TOP_Y) {
        const int g = f - TOP_Z;
        dx = g % TX; dz = g / TX; dy = TY - 1;
    } else {
        const int g = f - TOP_Z - TOP_Y;
        dx = TX - 1; dy = g % (TY - 1); dz = g / (TY - 1);
    }
}

__global__ void __launch_bounds__(NTHREADS, 1) systolic_kernel(const SysLaunch P)
{
    extern __shared__ float smem[];
    float *const sF[6] = {smem, smem + VOL, smem + 2 * VOL, smem + 3 * VOL, smem + 4 * VOL,
                          smem + 5 * VOL};
    float *const sCE = smem + 6 * VOL;
    __shared__ int s_ticket, s_abort;

    const int tid = threadIdx.x;
    const int sx = tid & 31, sy = tid >> 5;
    const float ndt = P.neg_dt;

    for (;;) {
        if (tid == 0) {
            s_ticket = atomicAdd(P.ctrl, 1);
            s_abort = ld_volatile(P.ctrl + 1) != DEV_OK;
        }
        __syncthreads();
        const int ticket = s_ticket;
        const bool stop = s_abort || ticket >= P.ntiles;
        __syncthreads();  // every thread has read s_ticket / s_abort
        if (stop) break;
        const int tile = P.tiles[ticket];
        const int I = tile % P.gx, J = (tile / P.gx) % P.gy, K = tile / (P.gx * P.gy);
        const int Ax = I * TX, Ay = J * TY, Az = K * TZ;
        const Interval iv = tile_interval(P, I, J, K);

        if (iv.s > 0) {
            if (tid == 0) s_abort = !wait_upstream(P, I, J, K, iv.s - 1, ticket);
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
                const int o = slot(sx, sy, sz);
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
        if (iv.s > 0 && tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)iv.s);

        bool abort = false;
        for (int t = iv.s; t <= iv.e; ++t) {
            const int bx = Ax - t, by = Ay - t, bz = Az - t;  // box low corner at step t
            const int ex = (bx - 1) & 31, ey = (by - 1) & (RY - 1), ez = (bz - 1) & (RZ - 1);

            // 1. upstream neighbours have finished step t
            if (tid == 0) s_abort = !wait_upstream(P, I, J, K, t, ticket);
            __syncthreads();
            if (s_abort) { abort = true; break; }

            // 2. lower shell (level t) into registers
            float shv[SHELL_PT][7];
#pragma unroll
            for (int q = 0; q < SHELL_PT; ++q) {
                const int f = tid + q * NTHREADS;
                if (f < SHELL) {
                    int qx, qy, qz;
                    shell_slot(f, ex, ey, ez, qx, qy, qz);
                    const int px = (bx - 1) + ((qx - bx + 1) & 31);
                    const int py = (by - 1) + ((qy - by + 1) & (RY - 1));
                    const int pz = (bz - 1) + ((qz - bz + 1) & (RZ - 1));
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

            // this thread's (x,y) column of the box
            const int dxc = (sx - bx) & 31, dyc = (sy - by) & (RY - 1);
            const int px = bx + dxc, py = by + dyc;
            const bool col = dxc < TX && dyc < TY && (unsigned)px < (unsigned)P.nx &&
                             (unsigned)py < (unsigned)P.ny;
            const int sxp = (sx + 1) & 31, syp = (sy + 1) & (RY - 1);
            const int sxm = (sx - 1) & 31, sym = (sy - 1) & (RY - 1);

            // 3. H half-step on the box
            if (col) {
                int r = bz & (RZ - 1);
                float exc = sF[0][slot(sx, sy, r)], eyc = sF[1][slot(sx, sy, r)];
                for (int dz = 0; dz < TZ; ++dz) {
                    const int rn = (r + 1) & (RZ - 1);
                    const float exn = sF[0][slot(sx, sy, rn)], eyn = sF[1][slot(sx, sy, rn)];
                    const int pz = bz + dz;
                    if ((unsigned)pz < (unsigned)P.nz) {
                        const int o = slot(sx, sy, r);
                        const float ez = sF[2][o];
                        const int oxp = slot(sxp, sy, r), oyp = slot(sx, syp, r);
                        sF[3][o] = h_x(sF[3][o], sF[2][oyp], ez, eyn, eyc, ndt);
                        sF[4][o] = h_y(sF[4][o], exn, exc, sF[2][oxp], ez, ndt);
                        sF[5][o] = h_z(sF[5][o], sF[1][oxp], eyc, sF[0][oyp], exc, ndt);
                    }
                    exc = exn;
                    eyc = eyn;
                    r = rn;
                }
            }
            __syncthreads();

            // 4. shell into the slots of the trailing top layer
#pragma unroll
            for (int q = 0; q < SHELL_PT; ++q) {
                const int f = tid + q * NTHREADS;
                if (f < SHELL) {
                    int qx, qy, qz;
                    shell_slot(f, ex, ey, ez, qx, qy, qz);
                    const int o = slot(qx, qy, qz);
#pragma unroll
                    for (int c = 0; c < 6; ++c) sF[c][o] = shv[q][c];
                    sCE[o] = shv[q][6];
                }
            }
            __syncthreads();

            // 5. E half-step on the box; PEC: tangential E on low planes fixed
            if (col) {
                int r = bz & (RZ - 1);
                const int rm0 = (r - 1) & (RZ - 1);
                float hxm = sF[3][slot(sx, sy, rm0)], hym = sF[4][slot(sx, sy, rm0)];
                for (int dz = 0; dz < TZ; ++dz) {
                    const int o = slot(sx, sy, r);
                    const float hx = sF[3][o], hy = sF[4][o];
                    const int pz = bz + dz;
                    if ((unsigned)pz < (unsigned)P.nz) {
                        const float hz = sF[5][o], ce = sCE[o];
                        const int oxm = slot(sxm, sy, r), oym = slot(sx, sym, r);
                        if (py > 0 && pz > 0) sF[0][o] = e_x(sF[0][o], hz, sF[5][oym], hy, hym, ce);
                        if (px > 0 && pz > 0) sF[1][o] = e_y(sF[1][o], hx, hxm, hz, sF[5][oxm], ce);
                        if (px > 0 && py > 0) sF[2][o] = e_z(sF[2][o], hy, sF[4][oxm], hx, sF[3][oym], ce);
                    }
                    hxm = hx;
                    hym = hy;
                    r = (r + 1) & (RZ - 1);
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
                                const int o = slot(s.i & 31, s.j & (RY - 1), s.k & (RZ - 1));
                                sF[s.comp][o] = add_source(sF[s.comp][o], s.amp[step]);
                            }
                        }
                    }
                    __syncthreads();
                }
            }

            // 6. top faces (or, on the last step of the launch, the whole box)
            if (t == P.T - 1) {
                if (col) {
                    for (int dz = 0; dz < TZ; ++dz) {
                        const int pz = bz + dz;
                        if ((unsigned)pz < (unsigned)P.nz) {
                            const int o = slot(sx, sy, pz & (RZ - 1));
                            const long long g = gidx(P, px, py, pz);
#pragma unroll
                            for (int c = 0; c < 6; ++c) P.f[c][g] = sF[c][o];
                        }
                    }
                }
            } else {
                for (int f = tid; f < TOP; f += NTHREADS) {
                    int dx, dy, dz;
                    top_cell(f, dx, dy, dz);
                    const int qx = bx + dx, qy = by + dy, qz = bz + dz;
                    if (in_dom(P, qx, qy, qz)) {
                        const int o = slot(qx & 31, qy & (RY - 1), qz & (RZ - 1));
                        const long long g = gidx(P, qx, qy, qz);
#pragma unroll
                        for (int c = 0; c < 6; ++c) P.f[c][g] = sF[c][o];
                    }
                }
            }
            __syncthreads();

            // 7. release progress
            if (tid == 0) publish(P, tile, ticket, P.epoch + (unsigned)t + 1u);
        }
        if (abort) break;
        __syncthreads();
    }
}

} // namespace

size_t systolic_smem_bytes() { return sizeof(float) * 7 * (size_t)VOL; }

cudaError_t systolic_configure()
{
    return cudaFuncSetAttribute(systolic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)systolic_smem_bytes());
}

cudaError_t launch_systolic(const SysLaunch &p, int grid, cudaStream_t st)
{
    systolic_kernel<<<grid, NTHREADS, systolic_smem_bytes(), st>>>(p);
    return cudaGetLastError();
}

int systolic_max_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, systolic_kernel, NTHREADS,
                                                      systolic_smem_bytes()) != cudaSuccess)
        return 0;
    return n;
}
