/*
 * fdtd.h — C ABI of libfdtd, a GB300 (sm_103a) Yee FDTD stepper with a
 * systolic (skewed, temporally blocked) update scheme.
 *
 * Method: arxiv 2502.20610.  The update is the Yee leapfrog of Sec. 2, Eq. 1
 * (Ex row printed; the Ey, Ez rows are its cyclic permutations and the H rows
 * the forward-difference adjoint form), dx = dy = dz = 1, mu = 1:
 *     H^{n+1/2} = H^{n-1/2} - dt * curl_f E^n
 *     E^{n+1}   = E^n + (dt/eps) * curl_b H^{n+1/2}   (+ point sources)
 * Two schedules compute it (both bit-identical in FP32):
 *   FDTD_SCHEME_NAIVE    one kernel per half-step over the whole grid, the
 *                        straightforward streaming update of Sec. 2;
 *   FDTD_SCHEME_SYSTOLIC one persistent kernel per call in which each CTA
 *                        keeps a subdomain on chip and scans it along the
 *                        x-y-z-t diagonal, exchanging only boundary faces
 *                        with neighbouring subdomains through global memory
 *                        and per-subdomain progress flags, with no grid-wide
 *                        synchronisation (Sec. 3, Fig. 7; Sec. 4).
 *
 * Conventions (every entry point):
 *   * Grid nx*ny*nz cells; field arrays are nx*ny*nz values each, index
 *     i + nx*(j + ny*k) (x fastest).  Cell (i,j,k) holds Ex(i+1/2,j,k),
 *     Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2),
 *     Hz(i+1/2,j+1/2,k).  Component order everywhere: Ex Ey Ez Hx Hy Hz.
 *   * Boundary: PEC box [0,N]^3.  Tangential E on the three low planes is
 *     never updated; E at index N reads as 0.
 *   * State after n steps is (E^n, H^{n-1/2}); fdtd_step advances whole steps.
 *   * Field storage: FP32, or FP16 / BF16 with one power-of-two scale s_c per
 *     component (the paper's engine keeps 16-bit fields, Sec. 4): component
 *     c holds q = fl16(v / s_c), and every curl and accumulation runs in FP32
 *     on decoded values; each new value is rounded once (to nearest even)
 *     when stored, after its point source if it has one.  Both schedules
 *     round at the same points and stay bit-identical.  dt/eps is FP32 in
 *     every format.  The API always exchanges unscaled FP32 values.
 *   * Every call returns an fdtd_status and never aborts or exits.
 *   * Pointers: "host" = host memory; "device" = CUDA device memory of the
 *     current device; "any" = either (the CUDA runtime's unified addressing
 *     tells them apart; pageable host memory is accepted, pinned is faster).
 *   * Streams are passed as void* holding a cudaStream_t (NULL = legacy
 *     default stream).  A handle is bound to one stream and is not
 *     thread-safe; different handles are independent.
 *   * Ownership: the caller allocates the device workspace (size from
 *     fdtd_workspace_size) and keeps it alive until fdtd_destroy; the library
 *     allocates nothing on the device.  Host-side state lives in the handle
 *     (with the learned boundary also one internal CUDA stream and two
 *     events, on which the network runs beside the Yee step; fdtd_destroy
 *     releases them).
 */
#ifndef FDTD_H
#define FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FDTD_OK = 0,
    FDTD_ERR_INVALID_ARG = 1, /* a pointer, size or option is out of range */
    FDTD_ERR_UNSUPPORTED = 2, /* a valid option this build does not implement */
    FDTD_ERR_OOM = 3,         /* the workspace passed is smaller than required */
    FDTD_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    FDTD_ERR_TIMEOUT = 5,     /* a device-side wait ran past wait_timeout_s */
    FDTD_ERR_STATE = 6        /* call out of order, or state lost to an earlier error */
} fdtd_status;

enum { FDTD_SCHEME_NAIVE = 0, FDTD_SCHEME_SYSTOLIC = 1 };
enum { FDTD_STORAGE_F32 = 0, FDTD_STORAGE_F16 = 1, FDTD_STORAGE_BF16 = 2 };
enum { FDTD_BOUNDARY_PEC = 0, FDTD_BOUNDARY_GRADED_ABSORBER = 1, FDTD_BOUNDARY_LEARNED = 2 };

typedef struct { int32_t nx, ny, nz; } fdtd_grid;

typedef struct {
    double dt;                /* time step; > 0; Courant limit dt < 1/sqrt(3) */
    int32_t scheme;           /* FDTD_SCHEME_* */
    int32_t storage;          /* FDTD_STORAGE_*; the systolic 31x15x15 and 31x7x15 tiles take F32 only */
    float field_scale[6];     /* 16-bit storage: s_c, a power of two in [2^-100, 2^100], 0 = 1;
                                 unused for F32.  Equal scales are fastest. */
    int32_t tile[3];          /* systolic subdomain (updated cells per axis); 0 = default */
    int32_t cluster[3];       /* systolic thread-block cluster shape in tiles; 0 = 1.
                                 (1,1,1): every tile in its own CTA, all faces between
                                 tiles through global memory (Sec. 3, Sec. 4).
                                 (2,1,1): x pairs of the default 31x15x12 tile share a
                                 2-CTA cluster; the upwind tile hands its top x face to
                                 the downwind one through distributed shared memory,
                                 the pair's outer faces go through global memory.
                                 Lossless boundaries only; other shapes UNSUPPORTED. */
    double wait_timeout_s;    /* bound on any device-side wait; <= 0 = 2 s */
    int32_t max_source_steps; /* capacity of each source table; <= 0 = 65536 */
    int32_t steps_per_launch; /* systolic: steps per persistent launch; <= 0 = 1024 */
} fdtd_coeffs;

/* Boundary inside the PEC box.
 *   FDTD_BOUNDARY_PEC: none.
 *   FDTD_BOUNDARY_GRADED_ABSORBER: conducting cells (the lossy structure
 *     field of Sec. 4): a layer of `thickness` cells at every wall with
 *     sigma = sigma_max * sum_a (depth_a / thickness)^poly_order, depth_a
 *     = thickness - i inside the low layer, i - (N-1-thickness) inside the
 *     high one; or, if `model` is not NULL, any conductivity: `model` is
 *     then host nx*ny*nz doubles sigma >= 0 (copied; the profile fields are
 *     ignored).  The E update becomes E <- ca E + cb (curl H - J) with
 *     ca = (1 - g)/(1 + g), cb = (dt/eps)/(1 + g), g = sigma dt/(2 eps),
 *     formed in FP64 and rounded to FP32 per cell.  Systolic scheme: the
 *     default 31x15x12 tile only.
 *   FDTD_BOUNDARY_LEARNED: a layer of `thickness` cells at every wall with
 *     the graded conductivity above (sigma_max, poly_order; sigma_max = 0:
 *     none) whose termination is learned: every cell takes the Yee step of
 *     the box with its PEC walls, then each cell on a face adds the
 *     correction of the network `model` (host, fdtd_mlp_param_count()
 *     floats, copied; layout at fdtd_mlp_*) computed from the 3x3x3
 *     stencils of the state at steps n and n-1 (the state before the first
 *     step, and after fdtd_write_fields, has S^{-1} = 0) to the values the
 *     PEC walls get wrong: tangential E on a low face, tangential H on a
 *     high face.  A zero network leaves the graded layer on PEC walls.
 *     Naive scheme and FP32 storage only (the update needs the whole previous
 *     level every step, which the systolic tiles do not keep).  Per step the
 *     band of the state is snapshotted, the network runs on the handle's
 *     internal stream while the Yee step runs on the handle's stream, and
 *     the corrections are added once both are done. */
typedef struct {
    int32_t kind;       /* FDTD_BOUNDARY_* */
    int32_t thickness;  /* absorber / learned layer thickness in cells, >= 1 */
    double sigma_max;   /* graded absorber peak conductivity, >= 0 */
    int32_t poly_order; /* graded absorber grading order, 0..16 */
    const void *model;  /* learned boundary parameters (host floats) */
} fdtd_boundary;

typedef struct fdtd_sim *fdtd_handle;

/* Bytes of device workspace a simulation with these parameters needs.
 * Layout inside it is private (16-bit storage adds one dense FP32 component
 * for host transfers).  Errors: INVALID_ARG (null pointer, grid dimension
 * < 1, dt <= 0, a field scale that is not a power of two), UNSUPPORTED
 * (storage, tile or boundary not built). */
fdtd_status fdtd_workspace_size(const fdtd_grid *grid, const fdtd_coeffs *coeffs,
                                const fdtd_boundary *boundary, size_t *bytes);

/* Create a simulation (Sec. 2 problem: fields on a PEC box, per-cell eps).
 *   eps        host, nx*ny*nz doubles, relative permittivity > 0; copied.
 *              The E coefficient dt/eps is formed in FP64 and rounded to
 *              FP32 once per cell.
 *   d_workspace device, >= fdtd_workspace_size bytes, 256-byte aligned,
 *              caller-owned, must outlive the handle.
 *   stream     cudaStream_t all work of the handle is ordered on.
 * Fields start at zero and the step counter at 0.  Errors: INVALID_ARG,
 * UNSUPPORTED, OOM (ws_bytes too small), CUDA. */
fdtd_status fdtd_create(const fdtd_grid *grid, const double *eps, const fdtd_coeffs *coeffs,
                        const fdtd_boundary *boundary, void *d_workspace, size_t ws_bytes,
                        void *stream, fdtd_handle *out);

/* Add a point current source J on E component `component` (0..2 = Ex..Ez)
 * of cell (i,j,k): after the E half-step of absolute step n,
 *     E_c(i,j,k) += fl32(-(dt/eps_ijk) * J[n])     for 0 <= n < n_steps,
 * nothing for later steps.  J is host, n_steps doubles (J at t_{n+1/2}),
 * copied.  At most 16 sources; n_steps <= max_source_steps.  Not part of the
 * paper's bare-bones benchmark (Sec. 4); used by the workloads.
 * Errors: INVALID_ARG, UNSUPPORTED (H component), STATE (16 already), CUDA. */
fdtd_status fdtd_add_source(fdtd_handle h, int32_t component, int32_t i, int32_t j, int32_t k,
                            const double *J, int64_t n_steps);

/* Overwrite all six fields with 6*nx*ny*nz floats (component-major, order
 * Ex..Hz) from `src` (any).  16-bit storage rounds each value v to
 * fl16(v / s_c) (to nearest even).  Asynchronous on the handle's stream;
 * `src` must stay valid until the stream reaches this point.  Clears an
 * earlier device error.  Leaves the step counter unchanged.
 * Errors: INVALID_ARG, CUDA. */
fdtd_status fdtd_write_fields(fdtd_handle h, const float *src);

/* Advance n >= 0 whole steps with the handle's scheme (the naive scheme runs
 * a grid of at most 1024 cells in one thread block per call, with block
 * barriers between the half-steps).  Asynchronous:
 * returns once the kernels are enqueued; launch errors are returned here,
 * device-side wait timeouts at the next fdtd_sync / fdtd_read_fields.
 * Errors: INVALID_ARG (n < 0), STATE (an earlier device error not cleared
 * by fdtd_write_fields), CUDA. */
fdtd_status fdtd_step(fdtd_handle h, int64_t n);

/* Copy the components selected by `component_mask` (bit c = component c) as
 * FP32 (16-bit storage: s_c * q, exact), packed in component order,
 * nx*ny*nz floats each, into `dst` (any).
 * Synchronises the stream and checks the device error word first.
 * Errors: INVALID_ARG, TIMEOUT (a device wait ran out; no data copied), CUDA. */
fdtd_status fdtd_read_fields(fdtd_handle h, uint32_t component_mask, float *dst);

/* Synchronise the handle's stream and report any device-side error.
 * Errors: TIMEOUT, CUDA. */
fdtd_status fdtd_sync(fdtd_handle h);

/* Absolute step counter (number of steps taken since create, or the value
 * set last by fdtd_set_current_step); -1 for a null handle. */
int64_t fdtd_current_step(fdtd_handle h);

/* Set the absolute step counter (indexes the source tables), e.g. after
 * restoring a checkpoint with fdtd_write_fields.  Errors: INVALID_ARG. */
fdtd_status fdtd_set_current_step(fdtd_handle h, int64_t step);

/* Number of kernels this handle has launched so far. */
int64_t fdtd_launch_count(fdtd_handle h);

/* Static description of a status code; never NULL. */
const char *fdtd_status_string(fdtd_status s);

/* Release the handle's host state (the workspace stays the caller's).
 * Does not synchronise; NULL is ignored. */
void fdtd_destroy(fdtd_handle h);

/* Test hooks for the systolic scheduler (no effect on the naive scheme):
 *   FDTD_DEBUG_NONE          clear hooks;
 *   FDTD_DEBUG_SKIP_PUBLISH  the subdomain with ticket `ticket` never
 *                            publishes its progress, so its neighbours' waits
 *                            run out: the launch ends with FDTD_ERR_TIMEOUT
 *                            (failure-detection test; no GPU fault);
 *   FDTD_DEBUG_DELAY         subdomains whose ticket % param == ticket sleep
 *                            ~param2 ns before publishing each step;
 *   FDTD_DEBUG_ORDER         hand out subdomains in another valid
 *                            topological order (param: 1 = random tie-break
 *                            seeded by ticket, 2 = lexicographic k,j,i).
 * Errors: INVALID_ARG. */
enum { FDTD_DEBUG_NONE = 0, FDTD_DEBUG_SKIP_PUBLISH = 1, FDTD_DEBUG_DELAY = 2, FDTD_DEBUG_ORDER = 3 };
fdtd_status fdtd_debug_set(fdtd_handle h, int32_t kind, int64_t ticket, int64_t param, int64_t param2);

/* Systolic step that allocates nothing (the paper has no counterpart; this
 * is a library convenience).  Some callers cannot call cudaMalloc: a host
 * application whose device memory is entirely owned by its own pool, or a
 * plug-in that may not allocate device memory after start-up (cudaMalloc can
 * also synchronise the device, which such callers must avoid).  They keep
 * their own buffers and call this instead of fdtd_create/fdtd_step:
 *   grid      nx, ny, nz >= 1;
 *   d_fields  device, 6*nx*ny*nz floats, component-major Ex..Hz, x fastest,
 *             state (E^n, H^{n-1/2}) in, (E^{n+n_steps}, H^{...-1/2}) out;
 *   d_coef    device, nx*ny*nz floats, the E coefficient fl32(dt/eps) per cell;
 *   dt        the time step used for H (must match d_coef);
 *   stream    cudaStream_t the work is ordered on.
 * PEC walls, no sources, tile 31x15x15; results are bit-identical to
 * fdtd_step with FDTD_SCHEME_SYSTOLIC on the same state.
 * Scratch: one file-scope device array of FDTD_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  Grids whose
 * tile schedule does not fit it even one step per launch are rejected with
 * FDTD_ERR_UNSUPPORTED (the message names the sizes); cubic grids up to
 * about 1900^3 cells fit.
 * The first call on a device looks up the array's device address and sets
 * the kernel's shared-memory limit.  Every call shares the array and clears
 * it first, so calls that overlap on the GPU (two streams, two threads)
 * race: serialise them.
 * The call is synchronous: it returns after the steps finish, with
 * FDTD_ERR_TIMEOUT if a device wait ran out, FDTD_ERR_CUDA on a CUDA error,
 * FDTD_ERR_INVALID_ARG for null pointers, an extent above 2^20, n_steps < 0
 * or a dt that is not a finite positive number. */
#define FDTD_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)

/* Learned boundary network (a learned absorbing boundary; the paper has no
 * counterpart): f(x) = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3,
 * 324 -> 64 -> 64 -> 6, FP32.  Parameter vector, in this order: W1 [64][324],
 * b1 [64], W2 [64][64], b2 [64], W3 [6][64], b3 [6] (row = output unit).
 * Input x: x[(s*6 + c)*27 + (dz+1)*9 + (dy+1)*3 + (dx+1)] for the fields c =
 * Ex..Hz at step n (s = 0) and n-1 (s = 1) around the cell, 0 outside the
 * domain.  A layer cell takes S^{n+1} = Yee(S^n) + r f(x / r), Yee = the PEC
 * box's own step, r = sqrt(mean x^2) (r < 1e-30 counts as a zero stencil:
 * no correction).  Training pairs (x_hat, y_hat) = (x / r, (S^{n+1}_ref -
 * Yee(S^n))(centre) / r), zeros when r < 1e-30; loss
 * = mean over samples and outputs of (f(x_hat) - y_hat)^2.  All pointers
 * named d_* are device memory; calls are asynchronous on `stream` unless
 * they return a host value.  Errors: INVALID_ARG, OOM (scratch too small),
 * CUDA. */
int64_t fdtd_mlp_param_count(void);
/* Scratch for minibatches of `batch` samples out of n_samples. */
fdtd_status fdtd_mlp_scratch_size(int32_t batch, int64_t n_samples, size_t *bytes);
/* d_y [n][6] = f(d_x [n][324]), in minibatches of `batch`. */
fdtd_status fdtd_mlp_forward(const float *d_params, const float *d_x, int64_t n, float *d_y, int32_t batch,
                             void *d_scratch, size_t scratch_bytes, void *stream);
/* Gradient of the loss of n samples (scratch for batch = n) into d_grad;
 * *loss (host, may be NULL) receives the loss.  Synchronous. */
fdtd_status fdtd_mlp_grad(const float *d_params, const float *d_x, const float *d_y, int32_t n, float *d_grad,
                          double *loss, void *d_scratch, size_t scratch_bytes, void *stream);
/* Adam (lr, beta 0.9 / 0.999, eps 1e-8) over `epochs` passes of shuffled
 * whole minibatches of n samples; d_params is updated in place; *last_epoch_loss
 * (host, may be NULL) receives the mean loss of the last epoch.  Synchronous. */
fdtd_status fdtd_mlp_train(float *d_params, const float *d_x, const float *d_y, int64_t n, int32_t batch,
                           int32_t epochs, double lr, uint64_t seed, void *d_scratch, size_t scratch_bytes,
                           void *stream, double *last_epoch_loss);
/* Training pairs from a reference simulation `h` (FP32 storage, no learned
 * boundary), typically one with a thick graded absorber: the box [lo, hi)
 * (cells, x y z) is the domain the learned boundary will see.  The call
 * steps h by n_steps + 1 and after each of the last n_steps records
 * per_step pairs for cells drawn uniformly (seeded) from the cells within
 * `thickness` of the box's faces, with stencil cells outside the box read
 * as 0 and Yee(S^n) the box's own PEC step of the cell (h's coefficients);
 * pair s*per_step + q goes to d_x [..][324], d_y [..][6].  Scratch:
 * fdtd_learned_record_scratch_size.  Synchronous. */
fdtd_status fdtd_learned_record_scratch_size(fdtd_handle h, int32_t per_step, size_t *bytes);
fdtd_status fdtd_learned_record(fdtd_handle h, const int32_t lo[3], const int32_t hi[3], int32_t thickness,
                                int32_t n_steps, int32_t per_step, uint64_t seed, float *d_x, float *d_y,
                                void *d_scratch, size_t scratch_bytes);
fdtd_status fdtd_systolic_step_noalloc(const fdtd_grid *grid, float *d_fields, const float *d_coef,
                                       double dt, int64_t n_steps, void *stream);

/* Adjoint gradient (inverse design; the paper motivates fast FDTD with it,
 * Sec. 1).  Objective: the overlap of Ez on the plane k = k0 with a mode
 * profile, squared and summed over the last `window` steps:
 *     L = sum_{n = N-window+1}^{N} O_n^2,  O_n = sum_{i,j} m(i,j) Ez^n(i,j,k0).
 * dL/deps is the exact derivative of the discrete map (the transposed Yee
 * step run backwards in time from step N, with dt/eps taken as dt/eps):
 *     dL/deps_p = -(1/eps_p) sum_{n<N} sum_a lambda_{E,a}^{n+1}(p) (E^{n+1} - E^n)_a(p),
 * accumulated in FP64 on the GPU. */
typedef struct {
    int32_t k0;            /* output plane (z index) */
    const float *d_mode;   /* device, nx*ny floats m(i,j), x fastest */
    int32_t window;        /* 1 <= window <= n_steps */
} fdtd_overlap_objective;

/* Scratch of fdtd_adjoint_gradient: ceil(n_steps/checkpoint_every) + 1 field
 * states, the adjoint state, two histories of checkpoint_every + 1 E states
 * of the box (forward and adjoint), n_steps + 1 doubles and up to 128 E
 * states of the plane k0.  Errors: INVALID_ARG (box outside the grid). */
fdtd_status fdtd_adjoint_scratch_size(fdtd_handle h, int64_t n_steps, int32_t checkpoint_every,
                                      const int32_t box_lo[3], const int32_t box_hi[3], size_t *bytes);

/* Advance h by n_steps from its current state (its scheme and sources),
 * return L in *loss (host, may be NULL) and dL/deps of the cells of the box
 * [box_lo, box_hi) (x y z) in d_grad (device doubles, box cells x fastest).
 * The forward pass keeps a checkpoint every checkpoint_every steps; the
 * reverse sweep recomputes each segment from its checkpoint (keeping only
 * the box's E) and steps the adjoint back over it.  The adjoint state is
 * kept as (M c lambda_E, -dt lambda_H), in which the transposed step is
 * the forward Yee step, so both sweeps run on h's own scheme (the systolic
 * kernel, when h has it).  On return h holds the
 * state after n_steps.  FP32 storage and PEC walls only (UNSUPPORTED
 * otherwise).  Synchronous.  Errors: INVALID_ARG, UNSUPPORTED, OOM (scratch
 * too small), TIMEOUT, CUDA, STATE. */
fdtd_status fdtd_adjoint_gradient(fdtd_handle h, const fdtd_overlap_objective *obj, int64_t n_steps,
                                  int32_t checkpoint_every, const int32_t box_lo[3], const int32_t box_hi[3],
                                  double *d_grad, double *loss, void *d_scratch, size_t scratch_bytes);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_H */
