// Host side of libfdtd: argument checks, workspace layout, coefficients,
// source tables, the systolic tile schedule, and kernel launches.
// The C ABI is declared (and documented) in include/fdtd.h.
#include "adjoint.h"
#include "fdtd.h"
#include "internal.h"
#include "mlp.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

namespace {

constexpr size_t ALIGN = 256;
constexpr int DEFAULT_SOURCE_STEPS = 65536;
constexpr int DEFAULT_STEPS_PER_LAUNCH = 1024;
constexpr unsigned EPOCH_LIMIT = 1u << 30;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t fields[6], ce, ca, stage, src, progress, tiles, ctrl, total;
    size_t xface, yface;  // register kernel's x- and y-face buffers (6 components each)
    long long fxs, fys;   // their elements per component
    int nzb, nzblk;       // their z extent: nzblk z-blocks of nzb / nzblk elements
    // learned boundary: network, previous and current band snapshots, layer
    // and band cell lists, layer predictions
    size_t params, prev, snap, layer, band, pred;
    long long nlayer, nband;
    int eb;     // bytes per stored field value (4 FP32, 2 FP16/BF16)
    int pitch;  // elements per x row in device memory (nx rounded up to 16 bytes)
    int variant, tx, ty, tz;  // systolic tile shape
    int cl;                   // CTAs per thread-block cluster along x (1, or 2: x pairs of tiles)
    int gx, gy, gz;
    long long ntiles_max;
    int source_steps, steps_per_launch;
};

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Does the E update have a conductivity term?  The graded absorber, and the
// learned layer with a graded base (sigma_max > 0).
bool conducts(const fdtd_boundary &b)
{
    return b.kind == FDTD_BOUNDARY_GRADED_ABSORBER || (b.kind == FDTD_BOUNDARY_LEARNED && b.sigma_max > 0.0);
}

// Cells within distance t of a wall (min over axes of the distance to the
// nearest face < t): the total minus the inner box.
long long cells_within(const fdtd_grid &g, int t)
{
    const long long ix = std::max(0, g.nx - 2 * t), iy = std::max(0, g.ny - 2 * t), iz = std::max(0, g.nz - 2 * t);
    return (long long)g.nx * g.ny * g.nz - ix * iy * iz;
}

// (x, y, z) of those cells, x fastest.
void list_cells_within(const fdtd_grid &g, int t, std::vector<int> &out)
{
    out.clear();
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) {
                const int d = std::min(std::min(std::min(i, g.nx - 1 - i), std::min(j, g.ny - 1 - j)),
                                       std::min(k, g.nz - 1 - k));
                if (d < t) {
                    out.push_back(i);
                    out.push_back(j);
                    out.push_back(k);
                }
            }
}

constexpr int DEFAULT_VARIANT = 2;  // register-resident 31 x 15 x 12 with TMA shells: fastest measured

// Tile shape requested in coeffs.tile (0,0,0 = default) -> variant, or -1.
int pick_variant(const fdtd_coeffs &c)
{
    if (c.tile[0] == 0 && c.tile[1] == 0 && c.tile[2] == 0) return DEFAULT_VARIANT;
    for (int v = 0; v < SYS_NSHAPES; ++v) {
        const SysShape sh = systolic_shape(v);
        if (c.tile[0] == sh.tx && c.tile[1] == sh.ty && c.tile[2] == sh.tz) return v;
    }
    return -1;
}

// Everything lives in the caller's workspace:
//   6 field arrays in the storage format, the FP32 coefficient dt/eps, (16-bit
//   storage) one dense FP32 component for host transfers, the source tables,
//   and (systolic) one progress flag per skewed tile plus the tile order.
bool make_layout(const fdtd_grid &g, const fdtd_coeffs &c, const fdtd_boundary &b, Layout &L)
{
    // rows padded to a 16-byte multiple, so every row starts 16-byte aligned
    // (a requirement of bulk tensor copies); the padding cells are never read
    L.eb = storage_bytes(c.storage);
    const int q = 16 / L.eb;
    L.pitch = (g.nx + q - 1) / q * q;
    const long long n = (long long)L.pitch * g.ny * g.nz;
    size_t off = 0;
    for (int k = 0; k < 6; ++k) {
        L.fields[k] = off;
        off = align_up(off + (size_t)L.eb * (size_t)n);
    }
    L.ce = off;
    off = align_up(off + sizeof(float) * (size_t)n);
    L.ca = off;  // E decay of conducting cells (absorber, or the learned layer's base)
    if (conducts(b)) off = align_up(off + sizeof(float) * (size_t)n);
    L.nlayer = L.nband = 0;
    L.params = L.prev = L.snap = L.layer = L.band = L.pred = off;
    if (b.kind == FDTD_BOUNDARY_LEARNED) {
        L.nlayer = cells_within(g, 1);  // the faces carry the network's corrections
        L.nband = cells_within(g, 2);   // their stencils reach one cell further
        L.params = off;
        off = align_up(off + sizeof(float) * (size_t)mlpnet::NPARAM);
        // two band snapshots (S^{n-1}, S^n), each six components and its x slab
        L.prev = off;
        off = align_up(off + 6 * align_up(sizeof(float) * (size_t)n) + learned_xslab_bytes(g.ny, g.nz));
        L.snap = off;
        off = align_up(off + 6 * align_up(sizeof(float) * (size_t)n) + learned_xslab_bytes(g.ny, g.nz));
        L.layer = off;
        off = align_up(off + 3 * sizeof(int) * (size_t)L.nlayer);
        L.band = off;
        off = align_up(off + 3 * sizeof(int) * (size_t)L.nband);
        L.pred = off;
        off = align_up(off + 6 * sizeof(float) * (size_t)L.nlayer);
    }
    L.stage = off;
    if (c.storage != FDTD_STORAGE_F32) off = align_up(off + sizeof(float) * (size_t)g.nx * g.ny * g.nz);
    // face buffers of the register kernel: per component nx * ny columns of
    // nzblk z-blocks (skewed z modulo nzblk * tile z, which the trail of
    // faces never needs to span twice: see the kernel)
    L.fxs = L.fys = 0;
    L.nzb = L.nzblk = 0;
    L.xface = L.yface = off;
    if (c.scheme == FDTD_SCHEME_SYSTOLIC && pick_variant(c) >= 2) {
        const int tz = systolic_shape(pick_variant(c)).tz;
        L.nzblk = ceil_div(g.nz, tz);
        L.nzb = L.nzblk * face_block(tz, L.eb);
        const size_t per = align_up((size_t)L.eb * (size_t)g.nx * g.ny * (size_t)L.nzb);
        L.fxs = L.fys = (long long)(per / L.eb);
        off += 6 * per;
        L.yface = off;
        off += 6 * per;
    }
    (void)q;
    L.source_steps = c.max_source_steps > 0 ? c.max_source_steps : DEFAULT_SOURCE_STEPS;
    L.src = off;
    off = align_up(off + sizeof(float) * (size_t)FDTD_MAX_SOURCES * (size_t)L.source_steps);
    L.steps_per_launch = c.steps_per_launch > 0 ? c.steps_per_launch : DEFAULT_STEPS_PER_LAUNCH;
    L.gx = L.gy = L.gz = 0;
    L.ntiles_max = 0;
    L.variant = pick_variant(c);
    if (L.variant < 0) return false;
    L.cl = c.scheme == FDTD_SCHEME_SYSTOLIC && c.cluster[0] == 2 ? 2 : 1;
    const SysShape sh = systolic_shape(L.variant);
    L.tx = sh.tx;
    L.ty = sh.ty;
    L.tz = sh.tz;
    if (c.scheme == FDTD_SCHEME_SYSTOLIC) {
        const long long T = L.steps_per_launch;
        L.gx = ceil_div(g.nx + T - 1, L.tx);
        L.gy = ceil_div(g.ny + T - 1, L.ty);
        L.gz = ceil_div(g.nz + T - 1, L.tz);
        L.ntiles_max = (long long)L.gx * L.gy * L.gz;
        if (L.ntiles_max > (1ll << 31) - 1) return false;
    }
    L.progress = off;
    off = align_up(off + sizeof(unsigned) * (size_t)L.ntiles_max);
    L.tiles = off;
    off = align_up(off + sizeof(int) * (size_t)L.ntiles_max);
    L.ctrl = off;
    off = align_up(off + 64 * sizeof(int));
    L.total = off;
    return true;
}

fdtd_status check_args(const fdtd_grid *g, const fdtd_coeffs *c, const fdtd_boundary *b)
{
    if (!g || !c || !b) return FDTD_ERR_INVALID_ARG;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return FDTD_ERR_INVALID_ARG;
    if (g->nx > (1 << 20) || g->ny > (1 << 20) || g->nz > (1 << 20)) return FDTD_ERR_INVALID_ARG;
    if (!(c->dt > 0.0) || !std::isfinite(c->dt)) return FDTD_ERR_INVALID_ARG;
    if (c->scheme != FDTD_SCHEME_NAIVE && c->scheme != FDTD_SCHEME_SYSTOLIC) return FDTD_ERR_INVALID_ARG;
    if (c->storage < FDTD_STORAGE_F32 || c->storage > FDTD_STORAGE_BF16) return FDTD_ERR_INVALID_ARG;
    if (c->storage != FDTD_STORAGE_F32) {
        for (int a = 0; a < 6; ++a) {
            const float s = c->field_scale[a];
            int ex = 0;
            if (s == 0.f) continue;  // 0 = 1
            if (!(s > 0.f) || !std::isfinite(s) || std::frexp(s, &ex) != 0.5f) return FDTD_ERR_INVALID_ARG;
            if (ex < -100 || ex > 100) return FDTD_ERR_INVALID_ARG;
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (c->tile[a] < 0 || c->cluster[a] < 0) return FDTD_ERR_INVALID_ARG;
    }
    if (pick_variant(*c) < 0) return FDTD_ERR_UNSUPPORTED;
    // the shared-memory systolic kernels (tiles 31x15x15, 31x7x15) hold FP32 only
    if (c->scheme == FDTD_SCHEME_SYSTOLIC && c->storage != FDTD_STORAGE_F32 && pick_variant(*c) < 2)
        return FDTD_ERR_UNSUPPORTED;
    // clusters: one CTA, or x pairs {2,1,1} of the lossless 31 x 15 x 12
    // register tile under the systolic scheme
    if (c->cluster[1] > 1 || c->cluster[2] > 1 || c->cluster[0] > 2) return FDTD_ERR_UNSUPPORTED;
    if (c->cluster[0] == 2 && (c->scheme != FDTD_SCHEME_SYSTOLIC || pick_variant(*c) != 2 || conducts(*b)))
        return FDTD_ERR_UNSUPPORTED;
    if (b->kind < FDTD_BOUNDARY_PEC || b->kind > FDTD_BOUNDARY_LEARNED) return FDTD_ERR_INVALID_ARG;
    if (b->kind == FDTD_BOUNDARY_GRADED_ABSORBER && !b->model) {
        if (b->thickness < 1 || !(b->sigma_max >= 0.0) || !std::isfinite(b->sigma_max) || b->poly_order < 0 ||
            b->poly_order > 16)
            return FDTD_ERR_INVALID_ARG;
    }
    if (b->kind == FDTD_BOUNDARY_GRADED_ABSORBER) {
        // the register kernel's 31 x 15 x 12 tile is the one built with the lossy update
        if (c->scheme == FDTD_SCHEME_SYSTOLIC && pick_variant(*c) != 2) return FDTD_ERR_UNSUPPORTED;
    }
    if (b->kind == FDTD_BOUNDARY_LEARNED) {
        if (b->thickness < 1 || !b->model || !(b->sigma_max >= 0.0) || !std::isfinite(b->sigma_max) ||
            b->poly_order < 0 || b->poly_order > 16)
            return FDTD_ERR_INVALID_ARG;
        // the layer update needs the whole previous level every step: the
        // naive scheme, FP32 fields
        if (c->scheme != FDTD_SCHEME_NAIVE || c->storage != FDTD_STORAGE_F32) return FDTD_ERR_UNSUPPORTED;
    }
    return FDTD_OK;
}

// Graded conductivity of cell (i,j,k): sigma_max * sum over the axes of
// (depth / L)^m, depth = L - i inside the low layer (i < L), i - (N-1-L) inside
// the high one (i >= N - L), 0 elsewhere.
double graded_sigma_at(const fdtd_grid &g, const fdtd_boundary &b, int i, int j, int k)
{
    const int idx[3] = {i, j, k}, n[3] = {g.nx, g.ny, g.nz};
    const int L = b.thickness;
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        int d = 0;
        if (idx[a] < L) d = L - idx[a];
        else if (idx[a] >= n[a] - L) d = idx[a] - (n[a] - 1 - L);
        if (d > 0) s += std::pow((double)d / L, b.poly_order);
    }
    return b.sigma_max * s;
}

// Conductivity of cell (i,j,k): the caller's per-cell array (absorber with a
// model), else the graded profile.
double sigma_at(const fdtd_grid &g, const fdtd_boundary &b, int i, int j, int k)
{
    if (b.kind == FDTD_BOUNDARY_GRADED_ABSORBER && b.model)
        return ((const double *)b.model)[i + (size_t)g.nx * ((size_t)j + (size_t)g.ny * k)];
    return graded_sigma_at(g, b, i, j, k);
}

// Skewed-tile schedule.  Tile (I,J,K) covers sigma in [A, A+n) with
// A = (I*31, J*15, K*15) and is active at steps [start, end] of a launch of
// T steps (its footprint A-t .. A-t+n intersects the domain).  Tiles with
// start <= end+1 are kept (those with start = end+1 only relay progress),
// ordered by (start, I+J+K): a topological order of the face-neighbour
// dependencies in which subdomains that can run early are handed out first.
struct TileEntry {
    int start, diag;
    unsigned key;
    int id;
};

void build_tiles(const fdtd_grid &g, const Layout &L, int order, unsigned seed,
                 std::vector<int> &tiles, std::vector<long long> &count_le)
{
    const int T = L.steps_per_launch;
    // x pairs: one entry per pair of tiles (I = 2P, 2P + 1), whose start is
    // the upwind tile's (starts grow with I), id P + gxp * (J + gy * K); a
    // pair's tiles depend on pairs (P-1, J, K), (P, J-1, K), (P, J, K-1) and
    // on each other, so the same sort is a topological order of pairs
    const int cl = L.cl, gxp = (L.gx + cl - 1) / cl;
    auto interval = [&](int I, int J, int K, int &s, int &e) {
        const int ax = I * L.tx, ay = J * L.ty, az = K * L.tz;
        s = std::max(0, std::max(ax - g.nx + 1, std::max(ay - g.ny + 1, az - g.nz + 1)));
        const int ge = std::min(ax + L.tx - 1, std::min(ay + L.ty - 1, az + L.tz - 1));
        e = std::min(T - 1, ge);
    };
    std::vector<TileEntry> v;
    v.reserve((size_t)std::min<long long>(L.ntiles_max, 1ll << 26));
    for (int K = 0; K < L.gz; ++K)
        for (int J = 0; J < L.gy; ++J)
            for (int Pp = 0; Pp < gxp; ++Pp) {
                int s = 0, e = -1;
                bool kept = false;
                for (int r = 0; r < cl; ++r) {
                    const int I = Pp * cl + r;
                    if (I >= L.gx) continue;
                    int si, ei;
                    interval(I, J, K, si, ei);
                    if (si > ei + 1) continue;
                    if (!kept || si < s) s = si;
                    kept = true;
                }
                if (!kept) continue;
                TileEntry te;
                te.start = s;
                te.id = Pp + gxp * (J + L.gy * K);
                if (order == 2) {
                    te.diag = K;
                    te.key = (unsigned)(J * gxp + Pp);
                } else {
                    te.diag = Pp + J + K;
                    unsigned h = (unsigned)te.id * 2654435761u ^ seed;
                    h ^= h >> 15;
                    h *= 2246822519u;
                    h ^= h >> 13;
                    te.key = order == 1 ? h : (unsigned)te.id;
                }
                v.push_back(te);
            }
    std::sort(v.begin(), v.end(), [](const TileEntry &a, const TileEntry &b) {
        if (a.start != b.start) return a.start < b.start;
        if (a.diag != b.diag) return a.diag < b.diag;
        return a.key < b.key;
    });
    tiles.resize(v.size());
    count_le.assign((size_t)T + 2, 0);
    for (size_t q = 0; q < v.size(); ++q) {
        tiles[q] = v[q].id;
        count_le[(size_t)std::min(v[q].start, T + 1)]++;
    }
    for (size_t s = 1; s < count_le.size(); ++s) count_le[s] += count_le[s - 1];
}

} // namespace

// Tensor-map encoder of the CUDA driver, fetched once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool encode_shell_maps(CUtensorMap tm[3][2], void *fbase, long long fstride, const float *ce, const float *ca,
                       int storage, int nx, int ny, int nz, int pitch, int nr, int bz, void *xf, long long fxs,
                       void *yf, long long fys, int nzb)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || fstride <= 0) return false;
    std::memset(tm, 0, sizeof(CUtensorMap) * 3 * 2);
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const long long n = (long long)pitch * ny * nz;
    // the coefficient arrays as a 4th dimension: cb, then ca at its own offset
    const long long cstride_b = ca ? (long long)((const char *)ca - (const char *)ce) : 4 * n;
    if (cstride_b <= 0 || cstride_b % 16 != 0) return false;
    const cuuint64_t ncoef = ca ? 2 : 1;
    auto map = [&](CUtensorMap *m, CUtensorMapDataType dt, void *base, const cuuint64_t dims[4],
                   const cuuint64_t strides[3], const cuuint32_t box[4]) {
        return enc(m, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int a = 0; a < 2; ++a) {
        const int eb = a == 0 ? storage_bytes(storage) : 4;
        const cuuint32_t xa = 16u / (cuuint32_t)eb, sw = 32u + xa;
        const cuuint64_t nf = a == 0 ? 6 : ncoef;
        const cuuint32_t bf = (cuuint32_t)nf;
        const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
        const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, nf};
        const cuuint64_t strides[3] = {(cuuint64_t)pitch * eb, (cuuint64_t)pitch * (cuuint64_t)ny * eb,
                                       a == 0 ? (cuuint64_t)fstride * eb : (cuuint64_t)cstride_b};
        void *base = a == 0 ? fbase : (void *)ce;
        // lower z shell {sw,16,1} of every array (fields and coefficients)
        const cuuint32_t zbox[4] = {sw, 16, 1, bf};
        if (!map(&tm[0][a], dt, base, dims, strides, zbox)) return false;
        if (a == 0) {
            // lower y and x shells of the fields from the face buffers, 5D maps
            // {bz rows, columns along the face, the other axis, nzblk blocks,
            // 6 fields}: y shell box {bz, 32, 1, 1, 6} (32 columns along x),
            // x shell box {bz, 16, 1, 1, 6} (16 columns along y)
            const cuuint64_t nzblk = (cuuint64_t)(nzb / bz);
            const cuuint64_t ebz = (cuuint64_t)bz * eb;
            const cuuint64_t yd[5] = {(cuuint64_t)bz, (cuuint64_t)nx, (cuuint64_t)ny, nzblk, 6};
            const cuuint64_t ys[4] = {ebz, ebz * nx, ebz * nx * ny, (cuuint64_t)fys * eb};
            const cuuint32_t yb[5] = {(cuuint32_t)bz, 32u, 1u, 1u, 6u};
            const cuuint64_t xd[5] = {(cuuint64_t)bz, (cuuint64_t)ny, (cuuint64_t)nx, nzblk, 6};
            const cuuint64_t xs[4] = {ebz, ebz * ny, ebz * nx * ny, (cuuint64_t)fxs * eb};
            const cuuint32_t xb[5] = {(cuuint32_t)bz, 16u, 1u, 1u, 6u};
            const cuuint32_t estr5[5] = {1, 1, 1, 1, 1};
            if (enc(&tm[1][0], dt, 5, yf, yd, ys, yb, estr5, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
            if (enc(&tm[2][0], dt, 5, xf, xd, xs, xb, estr5, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        } else {
            // lower y shell {sw,1,nr} and x shell (a 16-byte x chunk {4,16,nr})
            // of the coefficients
            const cuuint32_t ybox[4] = {sw, 1, (cuuint32_t)nr, bf};
            if (!map(&tm[1][1], dt, base, dims, strides, ybox)) return false;
            const cuuint32_t xb[4] = {4u, 16u, (cuuint32_t)nr, bf};
            if (!map(&tm[2][1], dt, base, dims, strides, xb)) return false;
        }
    }
    return true;
}

// Tile hand-out order of the systolic scheme for one launch of up to T
// steps with tile shape `variant` (same rule as a handle's schedule), for
// callers that manage their own scratch.
void systolic_tile_order(const fdtd_grid &g, int variant, int T, std::vector<int> &tiles,
                         std::vector<long long> &count_le, int &gx, int &gy, int &gz)
{
    fdtd_coeffs c;
    std::memset(&c, 0, sizeof(c));
    c.scheme = FDTD_SCHEME_SYSTOLIC;
    c.steps_per_launch = T;
    const SysShape sh = systolic_shape(variant);
    c.tile[0] = sh.tx;
    c.tile[1] = sh.ty;
    c.tile[2] = sh.tz;
    fdtd_boundary b;
    std::memset(&b, 0, sizeof(b));
    Layout L;
    make_layout(g, c, b, L);
    build_tiles(g, L, 0, 0u, tiles, count_le);
    gx = L.gx;
    gy = L.gy;
    gz = L.gz;
}

struct fdtd_sim {
    fdtd_grid g;
    fdtd_coeffs c;
    fdtd_boundary b;
    cudaStream_t stream;
    char *ws;
    Layout L;
    void *f[6];
    float *ce;
    float *ca;     // E decay per cell (absorber), else null
    float *params, *prev, *pred;  // learned boundary (else null)
    float *snap;                  // the band of the current state, read by the network
    cudaStream_t aux;             // learned boundary: the network runs here, beside the Yee step
    cudaEvent_t ev_fork, ev_join;
    int *layer, *band;
    int layer_grid;
    float *stage;  // dense FP32 component (16-bit storage), else null
    Scales sc;
    int fmt;       // kernel format (storage.cuh): the storage, or its uniform-scale variant
    float *src_tab;
    unsigned *progress;
    int *tiles;
    int *ctrl;
    SrcSet src;
    std::vector<double> eps_host;
    long long step;
    unsigned epoch;
    // adjoint: systolic launches store the E of box [cap_lo, cap_hi) after
    // each step into plane (step + 1 - cap_s0) of cap (3*cap_bc floats per
    // plane), `step` the step count before that step.  The recompute sets
    // cap_s0 to the segment's first step (plane 0 holds that state, copied
    // separately); the window sets it one past the chunk's first step, so
    // plane 0 holds the state after the chunk's first step.
    float *cap = nullptr;
    int cap_lo[3] = {0, 0, 0}, cap_hi[3] = {0, 0, 0};
    long long cap_bc = 0, cap_s0 = 0;
    long long launches;
    int max_ctas;
    std::vector<long long> count_le;  // tiles with start <= s
    int dbg_kind;
    long long dbg_ticket, dbg_param, dbg_param2;
    bool failed;
    CUtensorMap tm[3][2];  // shell maps of the register kernel
};

namespace {

fdtd_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return FDTD_OK;
    std::fprintf(stderr, "libfdtd: CUDA error: %s\n", cudaGetErrorString(e));
    return FDTD_ERR_CUDA;
}

// Copy ny*nz rows of nx floats between a dense array and a pitched one
// (one flat copy when the pitch adds no padding).
cudaError_t copy_rows(float *dst, size_t dpitch, const float *src, size_t spitch, const fdtd_grid &g,
                      cudaStream_t st)
{
    const size_t rows = (size_t)g.ny * g.nz, w = sizeof(float) * g.nx;
    if (dpitch == (size_t)g.nx && spitch == (size_t)g.nx)
        return cudaMemcpyAsync(dst, src, w * rows, cudaMemcpyDefault, st);
    return cudaMemcpy2DAsync(dst, sizeof(float) * dpitch, src, sizeof(float) * spitch, w, rows,
                             cudaMemcpyDefault, st);
}

// True if `p` is device (or managed) memory the kernels can read and write.
bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // pageable host memory on older runtimes
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define CK(x)                                                                  \
    do {                                                                       \
        cudaError_t e_ = (x);                                                  \
        if (e_ != cudaSuccess) return cuda_status(e_);                         \
    } while (0)

fdtd_status upload_tiles(fdtd_sim *h, int order, unsigned seed)
{
    std::vector<int> tiles;
    build_tiles(h->g, h->L, order, seed, tiles, h->count_le);
    if (!tiles.empty())
        CK(cudaMemcpyAsync(h->tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

} // namespace

extern "C" {

fdtd_status fdtd_workspace_size(const fdtd_grid *grid, const fdtd_coeffs *coeffs,
                                const fdtd_boundary *boundary, size_t *bytes)
{
    if (!bytes) return FDTD_ERR_INVALID_ARG;
    fdtd_status s = check_args(grid, coeffs, boundary);
    if (s != FDTD_OK) return s;
    Layout L;
    if (!make_layout(*grid, *coeffs, *boundary, L)) return FDTD_ERR_UNSUPPORTED;
    *bytes = L.total;
    return FDTD_OK;
}

fdtd_status fdtd_create(const fdtd_grid *grid, const double *eps, const fdtd_coeffs *coeffs,
                        const fdtd_boundary *boundary, void *d_workspace, size_t ws_bytes,
                        void *stream, fdtd_handle *out)
{
    if (!out) return FDTD_ERR_INVALID_ARG;
    *out = nullptr;
    fdtd_status s = check_args(grid, coeffs, boundary);
    if (s != FDTD_OK) return s;
    if (!eps || !d_workspace || ((uintptr_t)d_workspace % ALIGN) != 0) return FDTD_ERR_INVALID_ARG;
    Layout L;
    if (!make_layout(*grid, *coeffs, *boundary, L)) return FDTD_ERR_UNSUPPORTED;
    if (ws_bytes < L.total) return FDTD_ERR_OOM;
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    for (long long p = 0; p < n; ++p)
        if (!(eps[p] > 0.0) || !std::isfinite(eps[p])) return FDTD_ERR_INVALID_ARG;
    if (boundary->kind == FDTD_BOUNDARY_GRADED_ABSORBER && boundary->model) {
        const double *sg = (const double *)boundary->model;
        for (long long p = 0; p < n; ++p)
            if (!(sg[p] >= 0.0) || !std::isfinite(sg[p])) return FDTD_ERR_INVALID_ARG;
    }

    fdtd_sim *h = new (std::nothrow) fdtd_sim();
    if (!h) return FDTD_ERR_INVALID_ARG;
    h->g = *grid;
    h->c = *coeffs;
    h->b = *boundary;
    h->stream = (cudaStream_t)stream;
    h->ws = (char *)d_workspace;
    h->L = L;
    for (int k = 0; k < 6; ++k) h->f[k] = h->ws + L.fields[k];
    h->ce = (float *)(h->ws + L.ce);
    h->ca = conducts(*boundary) ? (float *)(h->ws + L.ca) : nullptr;
    const bool learned = boundary->kind == FDTD_BOUNDARY_LEARNED;
    h->params = learned ? (float *)(h->ws + L.params) : nullptr;
    h->prev = learned ? (float *)(h->ws + L.prev) : nullptr;
    h->pred = learned ? (float *)(h->ws + L.pred) : nullptr;
    h->snap = learned ? (float *)(h->ws + L.snap) : nullptr;
    h->aux = nullptr;
    h->ev_fork = h->ev_join = nullptr;
    h->layer = learned ? (int *)(h->ws + L.layer) : nullptr;
    h->band = learned ? (int *)(h->ws + L.band) : nullptr;
    h->layer_grid = 0;
    h->stage = coeffs->storage != FDTD_STORAGE_F32 ? (float *)(h->ws + L.stage) : nullptr;
    for (int k = 0; k < 6; ++k) {
        const float sk = coeffs->storage != FDTD_STORAGE_F32 && coeffs->field_scale[k] != 0.f ? coeffs->field_scale[k]
                                                                                             : 1.f;
        h->sc.s[k] = sk;
        h->sc.is[k] = 1.f / sk;  // exact: sk is a power of two
    }
    // one scale for all six components: the kernels step the stored values
    bool uniform = true;
    for (int k = 1; k < 6; ++k) uniform = uniform && h->sc.s[k] == h->sc.s[0];
    h->fmt = coeffs->storage;
    h->sc.src = 1.f;
    if (coeffs->storage != FDTD_STORAGE_F32 && uniform) {
        h->fmt = coeffs->storage == FDTD_STORAGE_F16 ? FMT_F16U : FMT_BF16U;
        h->sc.src = h->sc.is[0];
    }
    h->src_tab = (float *)(h->ws + L.src);
    h->progress = (unsigned *)(h->ws + L.progress);
    h->tiles = (int *)(h->ws + L.tiles);
    h->ctrl = (int *)(h->ws + L.ctrl);
    h->src.n = 0;
    h->step = 0;
    h->epoch = 1;
    h->launches = 0;
    h->dbg_kind = FDTD_DEBUG_NONE;
    h->dbg_ticket = h->dbg_param = h->dbg_param2 = 0;
    h->failed = false;
    h->eps_host.assign(eps, eps + n);

    auto fail = [&](fdtd_status st) {
        fdtd_destroy(h);
        return st;
    };
    // E coefficients, formed in FP64 and rounded to FP32 once per cell:
    // dt/eps, or for conducting cells (absorber, sigma > 0) the time-centred
    // form cb = (dt/eps)/(1 + g), ca = (1 - g)/(1 + g), g = sigma dt/(2 eps)
    std::vector<float> ce((size_t)n), ca(h->ca ? (size_t)n : 0);
    for (int k = 0; k < grid->nz; ++k)
        for (int j = 0; j < grid->ny; ++j)
            for (int i = 0; i < grid->nx; ++i) {
                const size_t p = (size_t)i + (size_t)grid->nx * ((size_t)j + (size_t)grid->ny * k);
                if (h->ca) {
                    const double g = sigma_at(*grid, *boundary, i, j, k) * coeffs->dt / (2.0 * eps[p]);
                    ce[p] = (float)((coeffs->dt / eps[p]) / (1.0 + g));
                    ca[p] = (float)((1.0 - g) / (1.0 + g));
                } else {
                    ce[p] = (float)(coeffs->dt / eps[p]);
                }
            }
    const size_t padded = (size_t)L.pitch * grid->ny * grid->nz;
    cudaError_t e = cudaMemsetAsync(h->ce, 0, sizeof(float) * padded, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h->ce, sizeof(float) * L.pitch, ce.data(), sizeof(float) * grid->nx,
                              sizeof(float) * grid->nx, (size_t)grid->ny * grid->nz, cudaMemcpyHostToDevice,
                              h->stream);
    if (e == cudaSuccess && h->ca) e = cudaMemsetAsync(h->ca, 0, sizeof(float) * padded, h->stream);
    if (e == cudaSuccess && h->ca)
        e = cudaMemcpy2DAsync(h->ca, sizeof(float) * L.pitch, ca.data(), sizeof(float) * grid->nx,
                              sizeof(float) * grid->nx, (size_t)grid->ny * grid->nz, cudaMemcpyHostToDevice,
                              h->stream);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)  // all-zero bits are +0 in every format
        e = cudaMemsetAsync(h->f[k], 0, (size_t)L.eb * padded, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ctrl, 0, 64 * sizeof(int), h->stream);
    std::vector<int> lcells, bcells;
    if (e == cudaSuccess && learned) {
        list_cells_within(*grid, 1, lcells);
        list_cells_within(*grid, 2, bcells);
        e = cudaMemcpyAsync(h->params, boundary->model, sizeof(float) * mlpnet::NPARAM, cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + L.prev, 0, L.layer - L.prev, h->stream);  // both snapshots
        if (e == cudaSuccess && !lcells.empty())
            e = cudaMemcpyAsync(h->layer, lcells.data(), sizeof(int) * lcells.size(), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && !bcells.empty())
            e = cudaMemcpyAsync(h->band, bcells.data(), sizeof(int) * bcells.size(), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = learned_layer_configure();
        // the network's stream: highest priority, so its CTAs are placed first
        // and the Yee kernels fill the rest of each SM
        int lo = 0, hi = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        int dev = 0, sms = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->layer_grid = sms;
    }
    if (e == cudaSuccess && L.ntiles_max > 0)
        e = cudaMemsetAsync(h->progress, 0, sizeof(unsigned) * (size_t)L.ntiles_max, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));

    if (coeffs->scheme == FDTD_SCHEME_SYSTOLIC) {
        e = systolic_configure(L.variant, h->fmt, h->ca != nullptr, L.cl);
        if (e != cudaSuccess) return fail(cuda_status(e));
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(cuda_status(e));
        if (L.cl == 2) {  // co-resident clusters of two
            const int pairs = systolic_reg_max_pairs(L.variant - 2, h->fmt);
            if (pairs < 1) return fail(FDTD_ERR_UNSUPPORTED);
            h->max_ctas = 2 * pairs;
        } else {
            const int per_sm = systolic_max_ctas_per_sm(L.variant, h->fmt, h->ca != nullptr);
            if (per_sm < 1) return fail(FDTD_ERR_UNSUPPORTED);
            h->max_ctas = sms * per_sm;
        }
        if (L.variant >= 2) {
            const long long fstride = (long long)(L.fields[1] - L.fields[0]) / L.eb;
            const int nr = systolic_reg_rows(L.variant - 2);
            if (!encode_shell_maps(h->tm, h->f[0], fstride, h->ce, h->ca, coeffs->storage, grid->nx, grid->ny,
                                   grid->nz, L.pitch, nr, face_block(nr - 1, L.eb), h->ws + L.xface, L.fxs,
                                   h->ws + L.yface, L.fys, L.nzb))
                return fail(FDTD_ERR_UNSUPPORTED);
        }
        fdtd_status st = upload_tiles(h, 0, 0);
        if (st != FDTD_OK) return fail(st);
    }
    *out = h;
    return FDTD_OK;
}

fdtd_status fdtd_add_source(fdtd_handle h, int32_t component, int32_t i, int32_t j, int32_t k,
                            const double *J, int64_t n_steps)
{
    if (!h || (!J && n_steps > 0) || n_steps < 0) return FDTD_ERR_INVALID_ARG;
    if (component < 0 || component > 5) return FDTD_ERR_INVALID_ARG;
    if (component > 2) return FDTD_ERR_UNSUPPORTED;
    if (i < 0 || j < 0 || k < 0 || i >= h->g.nx || j >= h->g.ny || k >= h->g.nz) return FDTD_ERR_INVALID_ARG;
    if (n_steps > h->L.source_steps) return FDTD_ERR_INVALID_ARG;
    if (h->src.n >= FDTD_MAX_SOURCES) return FDTD_ERR_STATE;
    const long long dense = i + (long long)h->g.nx * (j + (long long)h->g.ny * k);
    const long long idx = i + (long long)h->L.pitch * (j + (long long)h->g.ny * k);
    // the cell's cb (dt/eps unless it conducts)
    double c = h->c.dt / h->eps_host[(size_t)dense];
    if (h->ca) c /= 1.0 + sigma_at(h->g, h->b, i, j, k) * h->c.dt / (2.0 * h->eps_host[(size_t)dense]);
    std::vector<float> amp((size_t)std::max<int64_t>(n_steps, 1));
    for (int64_t n = 0; n < n_steps; ++n) amp[(size_t)n] = (float)(-c * J[n]);
    float *dst = h->src_tab + (size_t)h->src.n * (size_t)h->L.source_steps;
    if (n_steps > 0) {
        CK(cudaMemcpyAsync(dst, amp.data(), sizeof(float) * (size_t)n_steps, cudaMemcpyHostToDevice,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    SrcDesc &s = h->src.s[h->src.n++];
    s.comp = component;
    s.i = i;
    s.j = j;
    s.k = k;
    s.idx = idx;
    s.n_amp = n_steps;
    s.amp = dst;
    return FDTD_OK;
}

fdtd_status fdtd_write_fields(fdtd_handle h, const float *src)
{
    if (!h || !src) return FDTD_ERR_INVALID_ARG;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    if (h->c.storage == FDTD_STORAGE_F32) {
        for (int k = 0; k < 6; ++k)
            CK(copy_rows((float *)h->f[k], h->L.pitch, src + (size_t)k * n, h->g.nx, h->g, h->stream));
    } else {
        const bool dev = is_device_pointer(src);
        for (int k = 0; k < 6; ++k) {
            const float *from = src + (size_t)k * n;
            if (!dev) {  // through the dense FP32 stage
                CK(cudaMemcpyAsync(h->stage, from, sizeof(float) * n, cudaMemcpyDefault, h->stream));
                from = h->stage;
            }
            CK(launch_to_storage(h->f[k], from, h->c.storage, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, h->sc.is[k],
                                 h->stream));
        }
    }
    CK(cudaMemsetAsync(h->ctrl + 1, 0, 3 * sizeof(int), h->stream));
    // S^{n-1} := 0 (both band snapshots: which is "previous" alternates)
    if (h->prev) CK(cudaMemsetAsync(h->ws + h->L.prev, 0, h->L.layer - h->L.prev, h->stream));
    h->failed = false;
    return FDTD_OK;
}

fdtd_status fdtd_step(fdtd_handle h, int64_t n)
{
    if (!h || n < 0) return FDTD_ERR_INVALID_ARG;
    if (h->failed) return FDTD_ERR_STATE;
    if (h->c.scheme == FDTD_SCHEME_NAIVE) {
        const float ndt = -(float)h->c.dt;
        const long long cells = (long long)h->g.nx * h->g.ny * h->g.nz;
        if (h->params) {  // learned boundary: Yee everywhere, then the network's correction on the wall layer
            float *f0 = (float *)h->f[0];
            const long long fs = (long long)(h->L.fields[1] - h->L.fields[0]) / 4;
            const long long ps = (long long)align_up(sizeof(float) * (size_t)h->L.pitch * h->g.ny * h->g.nz) / 4;
            if (fs != ps) return FDTD_ERR_STATE;  // previous-state arrays mirror the field layout
            // per step: snapshot the band of S^n (and its x slab); the network (S^n and S^{n-1}
            // bands -> corrections) on the internal stream, the Yee step on the
            // caller's, both at once; then the corrections are added and the
            // snapshot becomes the next step's previous state
            for (int64_t s = 0; s < n; ++s) {
                CK(learned_copy_cells(h->snap, f0, fs, h->L.pitch, h->g.ny, h->band, (int)h->L.nband, h->stream));
                CK(learned_fill_xslab(h->snap, f0, fs, h->L.pitch, h->g.nx, h->g.ny, h->g.nz, h->stream));
                CK(cudaEventRecord(h->ev_fork, h->stream));
                CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
                CK(learned_layer_predict(h->params, h->snap, h->prev, fs, h->L.pitch, h->g.nx, h->g.ny, h->g.nz,
                                         h->layer, (int)h->L.nlayer, h->pred, h->layer_grid, h->aux));
                CK(cudaEventRecord(h->ev_join, h->aux));
                CK(launch_naive_h(h->f, h->fmt, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, ndt, h->sc, h->stream));
                CK(launch_naive_e(h->f, h->fmt, h->ce, h->ca, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, h->step, h->src,
                                  h->sc, h->stream));
                CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
                CK(learned_layer_scatter(f0, fs, h->L.pitch, h->g.ny, h->layer, (int)h->L.nlayer, h->pred, h->stream));
                std::swap(h->prev, h->snap);
                h->launches += 6;
                h->step += 1;
            }
            return FDTD_OK;
        }
        if (cells <= naive_block_max_cells()) {  // one CTA holds the domain: no global sync
            while (n > 0) {
                const int T = (int)std::min<int64_t>(n, 1 << 20);
                CK(launch_naive_block(h->f, h->fmt, h->ce, h->ca, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, ndt, h->step, T,
                                      h->src, h->sc, h->stream));
                h->launches += 1;
                h->step += T;
                n -= T;
            }
            return FDTD_OK;
        }
        for (int64_t s = 0; s < n; ++s) {
            CK(launch_naive_h(h->f, h->fmt, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, ndt, h->sc, h->stream));
            CK(launch_naive_e(h->f, h->fmt, h->ce, h->ca, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, h->step, h->src,
                              h->sc, h->stream));
            h->launches += 2;
            h->step += 1;
        }
        return FDTD_OK;
    }
    while (n > 0) {
        const int T = (int)std::min<int64_t>(n, h->L.steps_per_launch);
        if (h->epoch + (unsigned)T + 1u > EPOCH_LIMIT) {
            CK(cudaMemsetAsync(h->progress, 0, sizeof(unsigned) * (size_t)h->L.ntiles_max, h->stream));
            h->epoch = 1;
        }
        CK(cudaMemsetAsync(h->ctrl, 0, sizeof(int), h->stream));  // ticket counter
        SysLaunch p;
        for (int k = 0; k < 6; ++k) p.f[k] = (float *)h->f[k];
        p.ce = h->ce;
        p.ca = h->ca;
        p.nx = h->g.nx;
        p.ny = h->g.ny;
        p.nz = h->g.nz;
        p.pitch = h->L.pitch;
        p.fbase = (float *)h->f[0];
        p.fstride = (long long)(h->L.fields[1] - h->L.fields[0]) / h->L.eb;
        p.sc = h->sc;
        p.xf = (float *)(h->ws + h->L.xface);
        p.yf = (float *)(h->ws + h->L.yface);
        p.fxs = h->L.fxs;
        p.fys = h->L.fys;
        p.nzb = h->L.nzb;
        p.nzblk = h->L.nzblk;
        p.gx = h->L.gx;
        p.gy = h->L.gy;
        p.gz = h->L.gz;
        p.T = T;
        p.epoch = h->epoch;
        p.step0 = h->step;
        p.tiles = h->tiles;
        p.ntiles = (int)h->count_le[(size_t)T];
        p.progress = h->progress;
        p.ctrl = h->ctrl;
        p.neg_dt = -(float)h->c.dt;
        const double to = h->c.wait_timeout_s > 0 ? h->c.wait_timeout_s : 2.0;
        p.timeout_ns = (long long)(to * 1e9);
        p.dbg_kind = h->dbg_kind;
        p.dbg_ticket = h->dbg_ticket;
        p.dbg_param = h->dbg_param;
        p.dbg_param2 = h->dbg_param2;
        p.src = h->src;
        p.cap = h->cap && h->L.variant >= 2 ? h->cap + 3 * h->cap_bc * (h->step + 1 - h->cap_s0) : nullptr;
        for (int a = 0; a < 3; ++a) {
            p.cap_lo[a] = h->cap_lo[a];
            p.cap_hi[a] = h->cap_hi[a];
        }
        p.cap_bc = h->cap_bc;
        if (h->L.variant >= 2) std::memcpy(p.tm, h->tm, sizeof(p.tm));
        const int cl = h->L.cl;
        const int grid = cl * (int)std::max<long long>(1, std::min<long long>(p.ntiles, h->max_ctas / cl));
        CK(launch_systolic(p, grid, h->stream, h->L.variant, h->fmt, cl));
        h->launches += 1;
        h->epoch += (unsigned)T + 1u;
        h->step += T;
        n -= T;
    }
    return FDTD_OK;
}

fdtd_status fdtd_sync(fdtd_handle h)
{
    if (!h) return FDTD_ERR_INVALID_ARG;
    int host_ctrl[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(host_ctrl, h->ctrl, sizeof(host_ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (host_ctrl[1] != DEV_OK) {
        h->failed = true;
        return FDTD_ERR_TIMEOUT;
    }
    return FDTD_OK;
}

fdtd_status fdtd_read_fields(fdtd_handle h, uint32_t component_mask, float *dst)
{
    if (!h || (!dst && component_mask) || component_mask > 63u) return FDTD_ERR_INVALID_ARG;
    fdtd_status s = fdtd_sync(h);
    if (s != FDTD_OK) return s;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    const bool dev = h->c.storage == FDTD_STORAGE_F32 || is_device_pointer(dst);
    size_t q = 0;
    for (int k = 0; k < 6; ++k) {
        if (!(component_mask & (1u << k))) continue;
        if (h->c.storage == FDTD_STORAGE_F32) {
            CK(copy_rows(dst + q * n, h->g.nx, (const float *)h->f[k], h->L.pitch, h->g, h->stream));
        } else {
            float *to = dev ? dst + q * n : h->stage;
            CK(launch_from_storage(to, h->f[k], h->c.storage, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, h->sc.s[k],
                                   h->stream));
            if (!dev) CK(cudaMemcpyAsync(dst + q * n, h->stage, sizeof(float) * n, cudaMemcpyDefault, h->stream));
        }
        ++q;
    }
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
}

int64_t fdtd_current_step(fdtd_handle h) { return h ? h->step : -1; }

fdtd_status fdtd_set_current_step(fdtd_handle h, int64_t step)
{
    if (!h || step < 0) return FDTD_ERR_INVALID_ARG;
    h->step = step;
    return FDTD_OK;
}

int64_t fdtd_launch_count(fdtd_handle h) { return h ? h->launches : -1; }

const char *fdtd_status_string(fdtd_status s)
{
    switch (s) {
    case FDTD_OK: return "ok";
    case FDTD_ERR_INVALID_ARG: return "invalid argument";
    case FDTD_ERR_UNSUPPORTED: return "unsupported option";
    case FDTD_ERR_OOM: return "workspace too small";
    case FDTD_ERR_CUDA: return "CUDA error";
    case FDTD_ERR_TIMEOUT: return "device wait timed out";
    case FDTD_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

void fdtd_destroy(fdtd_handle h)
{
    if (!h) return;
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
}

// ------------------------------------------------ learned-boundary network

int64_t fdtd_mlp_param_count(void) { return mlpnet::NPARAM; }

fdtd_status fdtd_mlp_scratch_size(int32_t batch, int64_t n_samples, size_t *bytes)
{
    if (!bytes || batch < 1 || n_samples < 0) return FDTD_ERR_INVALID_ARG;
    *bytes = mlp_scratch_bytes(batch, n_samples);
    return FDTD_OK;
}

fdtd_status fdtd_mlp_forward(const float *d_params, const float *d_x, int64_t n, float *d_y, int32_t batch,
                             void *d_scratch, size_t scratch_bytes, void *stream)
{
    if (!d_params || (n > 0 && (!d_x || !d_y)) || n < 0 || batch < 1 || !d_scratch) return FDTD_ERR_INVALID_ARG;
    if (scratch_bytes < mlp_scratch_bytes(batch, 0)) return FDTD_ERR_OOM;
    CK(mlp_forward(d_params, d_x, n, d_y, d_scratch, batch, (cudaStream_t)stream));
    return FDTD_OK;
}

fdtd_status fdtd_mlp_grad(const float *d_params, const float *d_x, const float *d_y, int32_t n, float *d_grad,
                          double *loss, void *d_scratch, size_t scratch_bytes, void *stream)
{
    if (!d_params || !d_x || !d_y || !d_grad || n < 1 || !d_scratch) return FDTD_ERR_INVALID_ARG;
    if (scratch_bytes < mlp_scratch_bytes(n, 0)) return FDTD_ERR_OOM;
    CK(mlp_grad(d_params, d_x, d_y, n, d_grad, loss, d_scratch, n, (cudaStream_t)stream));
    return FDTD_OK;
}

fdtd_status fdtd_mlp_train(float *d_params, const float *d_x, const float *d_y, int64_t n, int32_t batch,
                           int32_t epochs, double lr, uint64_t seed, void *d_scratch, size_t scratch_bytes,
                           void *stream, double *last_epoch_loss)
{
    if (!d_params || !d_x || !d_y || n < 1 || batch < 1 || batch > n || epochs < 0 || !(lr > 0.0) || !d_scratch ||
        n > (1ll << 31) - 1)
        return FDTD_ERR_INVALID_ARG;
    if (scratch_bytes < mlp_scratch_bytes(batch, n)) return FDTD_ERR_OOM;
    CK(mlp_train(d_params, d_x, d_y, n, batch, epochs, lr, seed, d_scratch, (cudaStream_t)stream,
                 last_epoch_loss));
    return FDTD_OK;
}

fdtd_status fdtd_learned_record_scratch_size(fdtd_handle h, int32_t per_step, size_t *bytes)
{
    if (!h || !bytes || per_step < 1) return FDTD_ERR_INVALID_ARG;
    const size_t arr = align_up(sizeof(float) * (size_t)h->L.pitch * h->g.ny * h->g.nz);
    *bytes = 12 * arr + align_up(3 * sizeof(int) * (size_t)per_step);
    return FDTD_OK;
}

fdtd_status fdtd_learned_record(fdtd_handle h, const int32_t lo[3], const int32_t hi[3], int32_t thickness,
                                int32_t n_steps, int32_t per_step, uint64_t seed, float *d_x, float *d_y,
                                void *d_scratch, size_t scratch_bytes)
{
    if (!h || !lo || !hi || thickness < 1 || n_steps < 0 || per_step < 1 || !d_x || !d_y || !d_scratch)
        return FDTD_ERR_INVALID_ARG;
    if (h->c.storage != FDTD_STORAGE_F32 || h->params) return FDTD_ERR_UNSUPPORTED;
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    for (int a = 0; a < 3; ++a)
        if (lo[a] < 0 || hi[a] > n3[a] || hi[a] - lo[a] < 1) return FDTD_ERR_INVALID_ARG;
    size_t need = 0;
    fdtd_learned_record_scratch_size(h, per_step, &need);
    if (scratch_bytes < need) return FDTD_ERR_OOM;
    const size_t arr = align_up(sizeof(float) * (size_t)h->L.pitch * h->g.ny * h->g.nz);
    const long long fs = (long long)(h->L.fields[1] - h->L.fields[0]) / 4;
    if ((long long)(arr / 4) != fs) return FDTD_ERR_STATE;
    char *base = (char *)d_scratch;
    float *prev = (float *)base, *cur = (float *)(base + 6 * arr);
    int *cells = (int *)(base + 12 * arr);
    float *f0 = (float *)h->f[0];
    const int ilo[3] = {lo[0], lo[1], lo[2]}, ihi[3] = {hi[0], hi[1], hi[2]};
    // layer region of the box: cells within `thickness` of one of its faces
    std::mt19937_64 rng(seed);
    auto in_layer = [&](int x, int y, int z) {
        const int d = std::min(std::min(std::min(x - lo[0], hi[0] - 1 - x), std::min(y - lo[1], hi[1] - 1 - y)),
                               std::min(z - lo[2], hi[2] - 1 - z));
        return d < thickness;
    };
    std::vector<int> pick(3 * (size_t)per_step);
    CK(cudaMemcpyAsync(prev, f0, 6 * arr, cudaMemcpyDeviceToDevice, h->stream));
    fdtd_status st = fdtd_step(h, 1);
    if (st != FDTD_OK) return st;
    CK(cudaMemcpyAsync(cur, f0, 6 * arr, cudaMemcpyDeviceToDevice, h->stream));
    for (int s = 0; s < n_steps; ++s) {
        st = fdtd_step(h, 1);
        if (st != FDTD_OK) return st;
        for (int q = 0; q < per_step; ++q) {
            int x, y, z;
            do {
                x = lo[0] + (int)(rng() % (unsigned long long)(hi[0] - lo[0]));
                y = lo[1] + (int)(rng() % (unsigned long long)(hi[1] - lo[1]));
                z = lo[2] + (int)(rng() % (unsigned long long)(hi[2] - lo[2]));
            } while (!in_layer(x, y, z));
            pick[3 * q] = x;
            pick[3 * q + 1] = y;
            pick[3 * q + 2] = z;
        }
        CK(cudaMemcpyAsync(cells, pick.data(), sizeof(int) * pick.size(), cudaMemcpyHostToDevice, h->stream));
        CK(mlp_record(prev, cur, f0, fs, h->L.pitch, h->g.ny, ilo, ihi, cells, per_step, h->ce, h->ca,
                      -(float)h->c.dt, d_x + (size_t)s * per_step * mlpnet::NI,
                      d_y + (size_t)s * per_step * mlpnet::NO, h->stream));
        CK(cudaMemcpyAsync(prev, cur, 6 * arr, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(cur, f0, 6 * arr, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));  // the host cell list is reused next step
    }
    return fdtd_sync(h);
}

// ---------------------------------------------------------------- adjoint

namespace {

struct AdjPlan {
    long long nseg, box_cells, arr;  // arr: floats of one field array (stride)
    size_t ck, lam, hist, ahist, ov, win, total;
};

// planes of the objective's window captured per systolic launch
constexpr int64_t ADJ_WINDOW_CHUNK = 128;

bool adj_plan(fdtd_handle h, int64_t n, int32_t K, const int32_t lo[3], const int32_t hi[3], AdjPlan &a)
{
    const int n3[3] = {h->g.nx, h->g.ny, h->g.nz};
    for (int q = 0; q < 3; ++q)
        if (lo[q] < 0 || hi[q] > n3[q] || hi[q] <= lo[q]) return false;
    a.arr = (long long)(h->L.fields[1] - h->L.fields[0]) / 4;
    a.nseg = (n + K - 1) / K;
    a.box_cells = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    size_t off = 0;
    a.ck = off;  // checkpoints 0 .. nseg-1 and the final state
    off = align_up(off + sizeof(float) * 6 * (size_t)a.arr * (size_t)(a.nseg + 1));
    a.lam = off;  // the adjoint state (transformed variables, the field layout)
    off = align_up(off + sizeof(float) * 6 * (size_t)a.arr);
    a.hist = off;  // the box's E over one segment
    off = align_up(off + sizeof(float) * 3 * (size_t)a.box_cells * (size_t)(K + 1));
    a.ahist = off;  // the box's adjoint Et over one segment
    off = align_up(off + sizeof(float) * 3 * (size_t)a.box_cells * (size_t)(K + 1));
    a.ov = off;
    off = align_up(off + sizeof(double) * (size_t)(n + 1));
    // the objective's window as captured planes (E of plane k0 after each of
    // the last `window` steps), for handles whose register kernel captures
    a.win = off;
    off = align_up(off + sizeof(float) * 3 * (size_t)h->g.nx * h->g.ny * (size_t)std::min<int64_t>(n, ADJ_WINDOW_CHUNK));
    a.total = off;
    return true;
}

} // namespace

fdtd_status fdtd_adjoint_scratch_size(fdtd_handle h, int64_t n_steps, int32_t checkpoint_every,
                                      const int32_t box_lo[3], const int32_t box_hi[3], size_t *bytes)
{
    if (!h || !bytes || !box_lo || !box_hi || n_steps < 1 || checkpoint_every < 1) return FDTD_ERR_INVALID_ARG;
    AdjPlan a;
    if (!adj_plan(h, n_steps, checkpoint_every, box_lo, box_hi, a)) return FDTD_ERR_INVALID_ARG;
    *bytes = a.total;
    return FDTD_OK;
}

fdtd_status fdtd_adjoint_gradient(fdtd_handle h, const fdtd_overlap_objective *obj, int64_t n_steps,
                                  int32_t checkpoint_every, const int32_t box_lo[3], const int32_t box_hi[3],
                                  double *d_grad, double *loss, void *d_scratch, size_t scratch_bytes)
{
    if (!h || !obj || !obj->d_mode || !box_lo || !box_hi || !d_grad || !d_scratch || n_steps < 1 ||
        checkpoint_every < 1 || obj->k0 < 0 || obj->k0 >= h->g.nz || obj->window < 1 || obj->window > n_steps)
        return FDTD_ERR_INVALID_ARG;
    // the transposed step is that of the lossless FP32 Yee map with PEC walls
    if (h->c.storage != FDTD_STORAGE_F32 || h->ca || h->params) return FDTD_ERR_UNSUPPORTED;
    if (h->failed) return FDTD_ERR_STATE;
    AdjPlan a;
    if (!adj_plan(h, n_steps, checkpoint_every, box_lo, box_hi, a)) return FDTD_ERR_INVALID_ARG;
    if (scratch_bytes < a.total) return FDTD_ERR_OOM;
    const int K = checkpoint_every;
    const long long N = n_steps, W = obj->window;
    char *base = (char *)d_scratch;
    float *ck = (float *)(base + a.ck), *lam = (float *)(base + a.lam);
    float *hist = (float *)(base + a.hist), *ahist = (float *)(base + a.ahist);
    double *ov = (double *)(base + a.ov);
    float *f0 = (float *)h->f[0];
    const size_t state_bytes = sizeof(float) * 6 * (size_t)a.arr;
    auto slot = [&](long long s) { return ck + 6 * (size_t)a.arr * (size_t)s; };
    AdjGeo g{h->g.nx, h->g.ny, h->g.nz, h->L.pitch, a.arr};
    const int lo[3] = {box_lo[0], box_lo[1], box_lo[2]}, hi[3] = {box_hi[0], box_hi[1], box_hi[2]};
    const long long step0 = h->step, bc = a.box_cells;
    cudaStream_t st = h->stream;
    const float dt = (float)h->c.dt;
    fdtd_status rs;
    // single steps (the objective's window in the adjoint sweep, and every
    // step unless the register kernel can capture the box) use the naive
    // kernel pair, which the systolic schedule reproduces bit for bit
    const bool reg_kernel = h->c.scheme == FDTD_SCHEME_SYSTOLIC && h->L.variant >= 2;
    auto one_step = [&]() -> cudaError_t {
        cudaError_t e = launch_naive_h(h->f, h->fmt, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, -dt, h->sc, st);
        if (e == cudaSuccess)
            e = launch_naive_e(h->f, h->fmt, h->ce, h->ca, h->g.nx, h->g.ny, h->g.nz, h->L.pitch, h->step, h->src,
                               h->sc, st);
        h->launches += 2;
        h->step += 1;
        return e;
    };
    // m steps of h, the box's E after step r (r = 1..m) into plane p0 + r of
    // buf: captured by the register kernel, or copied after single steps
    auto run_capture = [&](long long m, float *buf, long long p0) -> fdtd_status {
        if (reg_kernel) {
            h->cap = buf;
            h->cap_s0 = h->step - p0;
            h->cap_bc = bc;
            for (int q = 0; q < 3; ++q) {
                h->cap_lo[q] = lo[q];
                h->cap_hi[q] = hi[q];
            }
            const fdtd_status r = fdtd_step(h, m);
            h->cap = nullptr;
            return r;
        }
        for (long long r = 1; r <= m; ++r) {
            CK(one_step());
            CK(adjoint_box_copy(g, f0, lo, hi, buf + 3 * (size_t)bc * (size_t)(p0 + r), st));
        }
        return FDTD_OK;
    };

    // forward: checkpoints every K steps, the overlaps of the window's steps
    CK(cudaMemsetAsync(ov, 0, sizeof(double) * (size_t)(N + 1), st));
    CK(cudaMemsetAsync(d_grad, 0, sizeof(double) * (size_t)a.box_cells, st));
    float *win = (float *)(base + a.win);
    const long long plane = (long long)h->g.nx * h->g.ny;
    long long n = 0;
    while (n < N) {
        if (n % K == 0) CK(cudaMemcpyAsync(slot(n / K), f0, state_bytes, cudaMemcpyDeviceToDevice, st));
        const long long next_ck = (n / K + 1) * K;
        const long long upto = std::min(N, next_ck);
        if (upto <= N - W) {  // no overlap needed before the window
            if ((rs = fdtd_step(h, upto - n)) != FDTD_OK) return rs;
            n = upto;
            continue;
        }
        if (n < N - W) {  // up to the window's first step
            if ((rs = fdtd_step(h, N - W - n)) != FDTD_OK) return rs;
            n = N - W;
            continue;
        }
        if (reg_kernel) {  // window steps in systolic launches that capture plane k0
            const long long m = std::min(upto, n + ADJ_WINDOW_CHUNK) - n;
            h->cap = win;  // plane w = the state after step n + 1 + w
            h->cap_s0 = h->step + 1;
            h->cap_bc = plane;
            h->cap_lo[0] = h->cap_lo[1] = 0;
            h->cap_hi[0] = h->g.nx;
            h->cap_hi[1] = h->g.ny;
            h->cap_lo[2] = obj->k0;
            h->cap_hi[2] = obj->k0 + 1;
            rs = fdtd_step(h, m);
            h->cap = nullptr;
            if (rs != FDTD_OK) return rs;
            CK(adjoint_overlaps(win, plane, (int)m, obj->d_mode, ov + n + 1, st));
            n += m;
            continue;
        }
        CK(one_step());
        ++n;
        CK(adjoint_overlap(g, f0 + 2 * a.arr, obj->k0, obj->d_mode, ov + n, st));
    }
    CK(cudaMemcpyAsync(slot(a.nseg), f0, state_bytes, cudaMemcpyDeviceToDevice, st));
    std::vector<double> O((size_t)(N + 1));
    CK(cudaMemcpyAsync(O.data(), ov, sizeof(double) * (size_t)(N + 1), cudaMemcpyDeviceToHost, st));
    if ((rs = fdtd_sync(h)) != FDTD_OK) return rs;
    double L = 0.0;
    for (long long q = N - W + 1; q <= N; ++q) L += O[(size_t)q] * O[(size_t)q];
    if (loss) *loss = L;

    // reverse sweep, segment by segment from the last.  The adjoint state is
    // kept as Et = M c lambda_E, Ht = -dt lambda_H, in which the transposed
    // step is the forward Yee step (adjoint.cu), so it runs on h's own
    // kernels with h's point sources switched off.  Per segment: recompute
    // the box's E from the checkpoint, step the adjoint back over the
    // segment keeping the box's Et, then accumulate the gradient.
    auto amp = [&](long long q) { return 2.0 * O[(size_t)q]; };  // window steps q > N - W
    struct SourcesOff {  // restores h's sources on every way out
        fdtd_handle h;
        SrcSet saved;
        ~SourcesOff() { h->src = saved; }
    } src_guard{h, h->src};
    SrcSet no_src = h->src;
    no_src.n = 0;
    // lambda^N = dg_N/dx^N: the adjoint source of step N alone
    CK(cudaMemsetAsync(lam, 0, state_bytes, st));
    CK(adjoint_plane_source(g, lam + 2 * a.arr, h->ce, obj->k0, obj->d_mode, amp(N), st));
    for (long long s = a.nseg - 1; s >= 0; --s) {
        const long long s0 = s * K, s1 = std::min(N, s0 + K), len = s1 - s0;
        // the box's E at steps s0 .. s1 into hist planes 0 .. len
        h->src = src_guard.saved;
        CK(cudaMemcpyAsync(f0, slot(s), state_bytes, cudaMemcpyDeviceToDevice, st));
        h->step = step0 + s0;
        CK(adjoint_box_copy(g, f0, lo, hi, hist, st));
        if ((rs = run_capture(len, hist, 0)) != FDTD_OK) return rs;
        // the adjoint from lambda^{s1} down to lambda^{s0}: its step r goes
        // from lambda^{q+1} to lambda^q, q = s1 - 1 - r, and adds the
        // objective's source when q is in the window (those steps come
        // first); the box's Et before step r into ahist plane r
        h->src = no_src;
        CK(cudaMemcpyAsync(f0, lam, state_bytes, cudaMemcpyDeviceToDevice, st));
        CK(adjoint_box_copy(g, f0, lo, hi, ahist, st));
        long long r = 0;
        for (; r < len && s1 - 1 - r > N - W; ++r) {
            CK(one_step());
            CK(adjoint_plane_source(g, f0 + 2 * a.arr, h->ce, obj->k0, obj->d_mode, amp(s1 - 1 - r), st));
            CK(adjoint_box_copy(g, f0, lo, hi, ahist + 3 * (size_t)bc * (size_t)(r + 1), st));
        }
        if (r < len && (rs = run_capture(len - r, ahist, r)) != FDTD_OK) return rs;
        CK(cudaMemcpyAsync(lam, f0, state_bytes, cudaMemcpyDeviceToDevice, st));
        CK(adjoint_gradient(ahist, hist, bc, (int)len, (double)dt, d_grad, st));
        h->launches += 1;
    }
    // leave the simulation at step n_steps
    h->src = src_guard.saved;
    CK(cudaMemcpyAsync(f0, slot(a.nseg), state_bytes, cudaMemcpyDeviceToDevice, st));
    h->step = step0 + N;
    return fdtd_sync(h);
}

fdtd_status fdtd_debug_set(fdtd_handle h, int32_t kind, int64_t ticket, int64_t param, int64_t param2)
{
    if (!h || kind < FDTD_DEBUG_NONE || kind > FDTD_DEBUG_ORDER) return FDTD_ERR_INVALID_ARG;
    if (kind == FDTD_DEBUG_DELAY && param <= 0) return FDTD_ERR_INVALID_ARG;
    if (kind == FDTD_DEBUG_ORDER) {
        if (param < 0 || param > 2) return FDTD_ERR_INVALID_ARG;
        if (h->c.scheme != FDTD_SCHEME_SYSTOLIC) return FDTD_OK;
        return upload_tiles(h, (int)param, (unsigned)ticket);
    }
    h->dbg_kind = kind;
    h->dbg_ticket = ticket;
    h->dbg_param = param;
    h->dbg_param2 = param2;
    return FDTD_OK;
}

} // extern "C"
