// Device helpers shared by the systolic kernels: memory-model primitives,
// tile intervals, bounded waits on the upwind progress flags, publishing.
#pragma once

#include "internal.h"

namespace sysc {

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
// never to a possibly stale L1 line.  The intrinsic (not volatile asm) lets
// the compiler batch independent loads; barriers still order them.
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }

struct Interval { int s, e; };

// Active steps [s, e] of tile (I,J,K) of shape TX x TY x TZ in a launch of
// T steps: those in which its footprint A-t .. A-t+n meets the domain.
template <int TX, int TY, int TZ>
__device__ __forceinline__ Interval tile_interval(const SysLaunch &P, int I, int J, int K)
{
    const int ax = I * TX, ay = J * TY, az = K * TZ;
    Interval r;
    r.s = max(0, max(ax - P.nx + 1, max(ay - P.ny + 1, az - P.nz + 1)));
    r.e = min(P.T - 1, min(ax + TX - 1, min(ay + TY - 1, az + TZ - 1)));
    return r;
}


// Progress flags of the three upwind face neighbours of the current tile,
// and the last value seen on each (so most steps need no poll at all).
struct Upwind {
    int id[3];       // linear tile id, -1 if none
    int s[3], e[3];  // their active intervals in this launch
};

// Wait until every -x, -y, -z neighbour that holds state at level L has
// completed it (progress >= epoch + L + 1).  A neighbour u is waited on if
// start(u)-1 <= L <= end(u) and start(u) <= end(u)+1: outside that range its
// cells at level L lie outside the domain.  A neighbour that enters the
// domain at L+1 publishes epoch+start(u) after its own initial wait, which
// carries the guarantee of the tiles behind it.  Lanes 0..2 of warp 0 each
// watch one neighbour; returns false (in every lane) if the launch aborts.
static __device__ bool wait_level(const SysLaunch &P, const Upwind &U, unsigned *seen, int L, int ticket)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < 3) {
        const int a = lane;
        // select this lane's neighbour without a dynamically indexed array
        const int id = a == 0 ? U.id[0] : (a == 1 ? U.id[1] : U.id[2]);
        const int us = a == 0 ? U.s[0] : (a == 1 ? U.s[1] : U.s[2]);
        const int ue = a == 0 ? U.e[0] : (a == 1 ? U.e[1] : U.e[2]);
        const unsigned target = P.epoch + (unsigned)L + 1u;
        if (id >= 0 && us <= ue + 1 && L >= us - 1 && L <= ue && seen[a] < target) {
            const unsigned *flag = P.progress + id;
            unsigned long long t0 = 0;
            for (int it = 0;; ++it) {
                const unsigned v = ld_acquire(flag);
                if (v >= target) {
                    seen[a] = v;
                    break;
                }
                if (ld_volatile(P.ctrl + 1) != DEV_OK) {
                    ok = false;
                    break;
                }
                const unsigned long long now = globaltimer();
                if (it == 0) {
                    t0 = now;
                } else if (now - t0 > (unsigned long long)P.timeout_ns) {
                    if (atomicCAS(P.ctrl + 1, DEV_OK, DEV_ERR_TIMEOUT) == DEV_OK) {
                        P.ctrl[2] = ticket;
                        P.ctrl[3] = (int)target;
                    }
                    ok = false;
                    break;
                }
                __nanosleep(it < 64 ? 32 : 256);
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Non-blocking form of wait_level: true (in every lane) if each upwind
// neighbour that must be waited on for level L has already published it;
// one poll per neighbour at most.
static __device__ bool level_ready(const SysLaunch &P, const Upwind &U, unsigned *seen, int L)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < 3) {
        const int a = lane;
        const int id = a == 0 ? U.id[0] : (a == 1 ? U.id[1] : U.id[2]);
        const int us = a == 0 ? U.s[0] : (a == 1 ? U.s[1] : U.s[2]);
        const int ue = a == 0 ? U.e[0] : (a == 1 ? U.e[1] : U.e[2]);
        const unsigned target = P.epoch + (unsigned)L + 1u;
        if (id >= 0 && us <= ue + 1 && L >= us - 1 && L <= ue && seen[a] < target) {
            const unsigned v = ld_acquire(P.progress + id);
            if (v >= target) seen[a] = v;
            else ok = false;
        }
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void publish(const SysLaunch &P, int tile, int ticket, unsigned value)
{
    if (P.dbg_kind == 1 /* skip publish */ && ticket == P.dbg_ticket) return;
    if (P.dbg_kind == 2 /* delay */ && P.dbg_param > 0 && (ticket % P.dbg_param) == P.dbg_ticket)
        __nanosleep((unsigned)P.dbg_param2);
    st_release(P.progress + tile, value);  // release: orders the CTA's stores before the flag
}

__device__ __forceinline__ bool in_dom(const SysLaunch &P, int x, int y, int z)
{
    return (unsigned)x < (unsigned)P.nx && (unsigned)y < (unsigned)P.ny && (unsigned)z < (unsigned)P.nz;
}

__device__ __forceinline__ long long gidx(const SysLaunch &P, int x, int y, int z)
{
    return x + (long long)P.pitch * (y + (long long)P.ny * z);
}


template <int TX, int TY, int TZ>
__device__ __forceinline__ void upwind_of(const SysLaunch &P, int I, int J, int K, Upwind &U)
{
    const int nb[3][3] = {{I - 1, J, K}, {I, J - 1, K}, {I, J, K - 1}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (nb[a][0] < 0 || nb[a][1] < 0 || nb[a][2] < 0) {
            U.id[a] = -1; U.s[a] = 1; U.e[a] = -1;
        } else {
            const Interval u = tile_interval<TX, TY, TZ>(P, nb[a][0], nb[a][1], nb[a][2]);
            U.id[a] = nb[a][0] + P.gx * (nb[a][1] + P.gy * nb[a][2]);
            U.s[a] = u.s; U.e[a] = u.e;
        }
    }
}

} // namespace sysc
