"""Thin ctypes binding of libfdtd (include/fdtd.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  PyTorch supplies the device workspace and the stream.
There is no CPU fallback: if libfdtd.so is missing, creating a simulation
raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdtd.so")

FDTD_OK, FDTD_ERR_INVALID_ARG, FDTD_ERR_UNSUPPORTED, FDTD_ERR_OOM, FDTD_ERR_CUDA, \
    FDTD_ERR_TIMEOUT, FDTD_ERR_STATE = range(7)
SCHEMES = {"naive": 0, "systolic": 1}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
BOUNDARY = {"pec": 0, "graded": 1, "learned": 2}
DEBUG_NONE, DEBUG_SKIP_PUBLISH, DEBUG_DELAY, DEBUG_ORDER = range(4)

#: every symbol include/fdtd.h declares
EXPORTS = ("fdtd_workspace_size", "fdtd_create", "fdtd_add_source", "fdtd_write_fields",
           "fdtd_step", "fdtd_read_fields", "fdtd_sync", "fdtd_current_step",
           "fdtd_set_current_step", "fdtd_launch_count", "fdtd_status_string", "fdtd_destroy",
           "fdtd_debug_set", "fdtd_systolic_step_noalloc", "fdtd_mlp_param_count", "fdtd_mlp_scratch_size",
           "fdtd_mlp_forward", "fdtd_mlp_grad", "fdtd_mlp_train", "fdtd_learned_record_scratch_size",
           "fdtd_learned_record", "fdtd_adjoint_scratch_size", "fdtd_adjoint_gradient")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Coeffs(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("scheme", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("field_scale", ctypes.c_float * 6), ("tile", ctypes.c_int32 * 3),
                ("cluster", ctypes.c_int32 * 3), ("wait_timeout_s", ctypes.c_double),
                ("max_source_steps", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32)]


class Boundary(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("thickness", ctypes.c_int32), ("sigma_max", ctypes.c_double),
                ("poly_order", ctypes.c_int32), ("model", ctypes.c_void_p)]


class OverlapObjective(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_int32), ("d_mode", ctypes.c_void_p), ("window", ctypes.c_int32)]


class FdtdError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def load_library(path=LIB_PATH):
    """Load libfdtd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    st = ctypes.c_int
    lib.fdtd_workspace_size.restype = st
    lib.fdtd_workspace_size.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.fdtd_create.restype = st
    lib.fdtd_create.argtypes = [P, P, P, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    lib.fdtd_add_source.restype = st
    lib.fdtd_add_source.argtypes = [P, I32, I32, I32, I32, P, I64]
    lib.fdtd_write_fields.restype = st
    lib.fdtd_write_fields.argtypes = [P, P]
    lib.fdtd_step.restype = st
    lib.fdtd_step.argtypes = [P, I64]
    lib.fdtd_read_fields.restype = st
    lib.fdtd_read_fields.argtypes = [P, U32, P]
    lib.fdtd_sync.restype = st
    lib.fdtd_sync.argtypes = [P]
    lib.fdtd_current_step.restype = I64
    lib.fdtd_current_step.argtypes = [P]
    lib.fdtd_set_current_step.restype = st
    lib.fdtd_set_current_step.argtypes = [P, I64]
    lib.fdtd_launch_count.restype = I64
    lib.fdtd_launch_count.argtypes = [P]
    lib.fdtd_status_string.restype = ctypes.c_char_p
    lib.fdtd_status_string.argtypes = [st]
    lib.fdtd_destroy.restype = None
    lib.fdtd_destroy.argtypes = [P]
    lib.fdtd_debug_set.restype = st
    lib.fdtd_debug_set.argtypes = [P, I32, I64, I64, I64]
    lib.fdtd_systolic_step_noalloc.restype = st
    lib.fdtd_systolic_step_noalloc.argtypes = [P, P, P, ctypes.c_double, I64, P]
    SZ = ctypes.c_size_t
    lib.fdtd_mlp_param_count.restype = I64
    lib.fdtd_mlp_param_count.argtypes = []
    lib.fdtd_mlp_scratch_size.restype = st
    lib.fdtd_mlp_scratch_size.argtypes = [I32, I64, ctypes.POINTER(SZ)]
    lib.fdtd_mlp_forward.restype = st
    lib.fdtd_mlp_forward.argtypes = [P, P, I64, P, I32, P, SZ, P]
    lib.fdtd_mlp_grad.restype = st
    lib.fdtd_mlp_grad.argtypes = [P, P, P, I32, P, ctypes.POINTER(ctypes.c_double), P, SZ, P]
    lib.fdtd_mlp_train.restype = st
    lib.fdtd_mlp_train.argtypes = [P, P, P, I64, I32, I32, ctypes.c_double, ctypes.c_uint64, P, SZ, P,
                                   ctypes.POINTER(ctypes.c_double)]
    lib.fdtd_learned_record_scratch_size.restype = st
    lib.fdtd_learned_record_scratch_size.argtypes = [P, I32, ctypes.POINTER(SZ)]
    lib.fdtd_adjoint_scratch_size.restype = st
    lib.fdtd_adjoint_scratch_size.argtypes = [P, I64, I32, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                              ctypes.POINTER(SZ)]
    lib.fdtd_adjoint_gradient.restype = st
    lib.fdtd_adjoint_gradient.argtypes = [P, ctypes.POINTER(OverlapObjective), I64, I32, ctypes.POINTER(I32),
                                          ctypes.POINTER(I32), P, ctypes.POINTER(ctypes.c_double), P, SZ]
    lib.fdtd_learned_record.restype = st
    lib.fdtd_learned_record.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I32), I32, I32, I32, ctypes.c_uint64,
                                        P, P, P, SZ]
    _lib = lib
    return lib


def status_string(s):
    if _lib is None:
        return {0: "ok", 1: "invalid argument", 2: "unsupported option", 3: "workspace too small",
                4: "CUDA error", 5: "device wait timed out", 6: "invalid state"}.get(s, "unknown")
    return _lib.fdtd_status_string(s).decode()


def _check(status, what):
    if status != FDTD_OK:
        raise FdtdError(status, what)


#: systolic tile shapes (updated cells x, y, z) the library is built with
TILES = {"31x15x15": (31, 15, 15), "31x7x15": (31, 7, 15), "31x15x12": (31, 15, 12),
         "31x15x8": (31, 15, 8)}


def make_params(shape_zyx, dt, scheme="systolic", storage="f32", timeout_s=2.0,
                steps_per_launch=0, max_source_steps=0, boundary="pec", tile=None, field_scale=None,
                absorber=None, learned=None, cluster=None):
    """cluster: CTAs per thread-block cluster (x, y, z) of the systolic
    scheme: None or (1, 1, 1), or (2, 1, 1) for x pairs of tiles exchanging
    their common face through distributed shared memory.
    absorber: (thickness L, sigma_max, order m) of the graded layer when
    boundary == "graded", or a float64 array of per-cell conductivity (kept
    alive by the caller); learned: (thickness, params[, sigma_max, order])
    when boundary == "learned" (params: float32 numpy array, kept alive by
    the caller; sigma_max > 0 adds a graded base over the layer)."""
    nz, ny, nx = (int(s) for s in shape_zyx)
    g = Grid(nx, ny, nz)
    c = Coeffs()
    c.dt = float(dt)
    c.scheme = SCHEMES[scheme]
    c.storage = STORAGE[storage]
    for a in range(6):
        c.field_scale[a] = 1.0 if field_scale is None else float(field_scale[a])
    c.wait_timeout_s = float(timeout_s)
    c.steps_per_launch = int(steps_per_launch)
    c.max_source_steps = int(max_source_steps)
    if tile is not None:
        t = TILES[tile] if isinstance(tile, str) else tuple(tile)
        for a in range(3):
            c.tile[a] = int(t[a])
    if cluster is not None:
        for a in range(3):
            c.cluster[a] = int(cluster[a])
    b = Boundary()
    b.kind = BOUNDARY[boundary]
    if isinstance(absorber, np.ndarray):
        b.model = absorber.ctypes.data
    elif absorber is not None:
        b.thickness, b.sigma_max, b.poly_order = int(absorber[0]), float(absorber[1]), int(absorber[2])
    if learned is not None:
        b.thickness = int(learned[0])
        b.model = learned[1].ctypes.data
        if len(learned) > 2:
            b.sigma_max, b.poly_order = float(learned[2]), int(learned[3])
    return g, c, b


def workspace_size(shape_zyx, dt, **kw):
    lib = load_library()
    g, c, b = make_params(shape_zyx, dt, **kw)
    n = ctypes.c_size_t(0)
    _check(lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c), ctypes.byref(b), ctypes.byref(n)),
           "fdtd_workspace_size")
    return int(n.value)


def _ptr(x):
    """Raw address of a torch tensor or numpy array (contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data


class Sim:
    """One simulation: (nz, ny, nx) grid, per-cell eps, PEC box.

    scheme: "naive" (one kernel per half-step) or "systolic" (persistent
    skewed-tile kernel).  storage: "f32", "f16" or "bf16" field storage
    (arithmetic is FP32 in every case); field_scale: six powers of two, the
    16-bit formats store v / s_c.  boundary: "pec", or "graded" with
    absorber = (thickness, sigma_max, order): a conducting layer with
    sigma = sigma_max * sum_a (depth_a / thickness)^order inside the PEC box,
    or "learned" with learned = (thickness, params): the network of
    fdtd_mlp_* updates the cells within `thickness` of a wall (naive scheme).
    Fields are exchanged as float32 (6, nz, ny, nx) arrays in component order
    Ex, Ey, Ez, Hx, Hy, Hz.
    """

    def __init__(self, shape_zyx, eps, dt, scheme="systolic", device=None, timeout_s=2.0,
                 steps_per_launch=0, max_source_steps=0, tile=None, storage="f32", field_scale=None,
                 boundary="pec", absorber=None, learned=None, cluster=None):
        import torch
        self._lib = load_library()
        self.shape = tuple(int(s) for s in shape_zyx)
        self.dt = float(dt)
        self.scheme = scheme
        self.storage = storage
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if absorber is not None and not isinstance(absorber, tuple):
            self._sigma = np.ascontiguousarray(np.broadcast_to(np.asarray(absorber, np.float64), self.shape))
            absorber = self._sigma
        g, c, b = make_params(self.shape, dt, scheme=scheme, timeout_s=timeout_s,
                              steps_per_launch=steps_per_launch, max_source_steps=max_source_steps,
                              tile=tile, storage=storage, field_scale=field_scale, boundary=boundary,
                              absorber=absorber, learned=self._learned_args(learned), cluster=cluster)
        self._params = (g, c, b)
        n = ctypes.c_size_t(0)
        _check(self._lib.fdtd_workspace_size(ctypes.byref(g), ctypes.byref(c), ctypes.byref(b),
                                             ctypes.byref(n)), "fdtd_workspace_size")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), self.shape))
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            _check(self._lib.fdtd_create(ctypes.byref(g), eps.ctypes.data, ctypes.byref(c), ctypes.byref(b),
                                         self.workspace.data_ptr(), int(n.value),
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                   "fdtd_create")
        self._h = h

    def _learned_args(self, learned):
        if learned is None:
            return None
        self._model = np.ascontiguousarray(np.asarray(learned[1], dtype=np.float32))
        return (int(learned[0]), self._model) + tuple(learned[2:])

    @property
    def ncell(self):
        nz, ny, nx = self.shape
        return nz * ny * nx

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fdtd_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_source(self, component, i, j, k, J):
        J = np.ascontiguousarray(np.asarray(J, dtype=np.float64))
        _check(self._lib.fdtd_add_source(self._h, int(component), int(i), int(j), int(k), J.ctypes.data,
                                         J.size), "fdtd_add_source")

    def write_fields(self, fields):
        """fields: float32 (6, nz, ny, nx), torch tensor (any device) or numpy."""
        import torch
        if isinstance(fields, np.ndarray):
            fields = torch.from_numpy(np.ascontiguousarray(fields, dtype=np.float32))
        if fields.dtype != torch.float32 or tuple(fields.shape) != (6,) + self.shape:
            raise ValueError(f"expected float32 {(6,) + self.shape}, got {fields.dtype} {tuple(fields.shape)}")
        fields = fields.contiguous()
        self._keep = fields  # the copy is asynchronous
        _check(self._lib.fdtd_write_fields(self._h, _ptr(fields)), "fdtd_write_fields")
        if fields.device.type == "cpu":
            self.sync()

    def write_fields_ptr(self, ptr):
        _check(self._lib.fdtd_write_fields(self._h, ctypes.c_void_p(ptr)), "fdtd_write_fields")

    def step(self, n):
        _check(self._lib.fdtd_step(self._h, int(n)), "fdtd_step")

    def sync(self):
        _check(self._lib.fdtd_sync(self._h), "fdtd_sync")

    def read_fields(self, mask=0x3F, out=None):
        """Components in `mask` as a float32 (k, nz, ny, nx) tensor (device by default)."""
        import torch
        k = bin(mask & 0x3F).count("1")
        if out is None:
            out = torch.empty((k,) + self.shape, dtype=torch.float32, device=self.device)
        _check(self._lib.fdtd_read_fields(self._h, int(mask), ctypes.c_void_p(_ptr(out))), "fdtd_read_fields")
        return out

    def read_fields_ptr(self, mask, ptr):
        _check(self._lib.fdtd_read_fields(self._h, int(mask), ctypes.c_void_p(ptr)), "fdtd_read_fields")

    @property
    def current_step(self):
        return int(self._lib.fdtd_current_step(self._h))

    def set_current_step(self, s):
        _check(self._lib.fdtd_set_current_step(self._h, int(s)), "fdtd_set_current_step")

    @property
    def launch_count(self):
        return int(self._lib.fdtd_launch_count(self._h))

    def debug_set(self, kind, ticket=0, param=0, param2=0):
        _check(self._lib.fdtd_debug_set(self._h, int(kind), int(ticket), int(param), int(param2)),
               "fdtd_debug_set")


def field_scales(fields, storage, headroom=4):
    """Power-of-two scales s_c for FP16 storage, chosen from the initial
    fields: the largest |v_c| / s_c lands in [2^(14 - headroom), 2^(15 -
    headroom)), leaving 2^headroom of room for growth below the binary16
    maximum (65504) while keeping small values out of the subnormal range
    (below 2^-14).  All-zero components get 1.  FP32 and BF16 (whose
    exponent range is FP32's): all 1."""
    if storage != "f16":
        return [1.0] * 6
    top = 15
    out = []
    for c in range(6):
        m = float(np.max(np.abs(np.asarray(fields[c], dtype=np.float64)))) if np.size(fields[c]) else 0.0
        if not np.isfinite(m) or m == 0.0:
            out.append(1.0)
            continue
        e = int(np.floor(np.log2(m)))  # 2^e <= m < 2^(e+1)
        out.append(float(2.0 ** min(100, max(-100, e + 1 - (top - headroom)))))
    return out


# ------------------------------------------------------------- learned boundary

def mlp_param_count():
    return int(load_library().fdtd_mlp_param_count())


def _scratch(batch, n, device):
    import torch
    sz = ctypes.c_size_t(0)
    _check(load_library().fdtd_mlp_scratch_size(int(batch), int(n), ctypes.byref(sz)), "fdtd_mlp_scratch_size")
    return torch.empty(int(sz.value), dtype=torch.uint8, device=device)


def mlp_forward(params, x, batch=4096):
    """f(x) of the network for x [n, 324] (CUDA float32 tensors)."""
    import torch
    lib = load_library()
    n = x.shape[0]
    y = torch.empty((n, 6), dtype=torch.float32, device=x.device)
    s = _scratch(batch, 0, x.device)
    _check(lib.fdtd_mlp_forward(_ptr(params), _ptr(x), n, _ptr(y), int(batch), _ptr(s), s.numel(),
                                ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)), "fdtd_mlp_forward")
    return y


def mlp_grad(params, x, y):
    """(gradient, loss) of the mean squared error over the n samples."""
    import torch
    lib = load_library()
    n = x.shape[0]
    g = torch.empty_like(params)
    s = _scratch(n, 0, x.device)
    loss = ctypes.c_double(0.0)
    _check(lib.fdtd_mlp_grad(_ptr(params), _ptr(x), _ptr(y), int(n), _ptr(g), ctypes.byref(loss), _ptr(s),
                             s.numel(), ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)),
           "fdtd_mlp_grad")
    return g, loss.value


def mlp_train(params, x, y, epochs, batch=4096, lr=1e-3, seed=0):
    """Adam on the pairs (x, y) in place on `params`; returns the last epoch's loss."""
    import torch
    lib = load_library()
    n = x.shape[0]
    s = _scratch(batch, n, x.device)
    loss = ctypes.c_double(0.0)
    _check(lib.fdtd_mlp_train(_ptr(params), _ptr(x), _ptr(y), int(n), int(batch), int(epochs), float(lr),
                              int(seed), _ptr(s), s.numel(),
                              ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream), ctypes.byref(loss)),
           "fdtd_mlp_train")
    return loss.value


def learned_record(sim, lo_xyz, hi_xyz, thickness, n_steps, per_step, seed=0):
    """Training pairs from the reference simulation `sim` (see fdtd.h):
    returns (x [n_steps*per_step, 324], y [.., 6]) CUDA tensors."""
    import torch
    lib = sim._lib
    n = int(n_steps) * int(per_step)
    x = torch.empty((n, 324), dtype=torch.float32, device=sim.device)
    y = torch.empty((n, 6), dtype=torch.float32, device=sim.device)
    sz = ctypes.c_size_t(0)
    _check(lib.fdtd_learned_record_scratch_size(sim._h, int(per_step), ctypes.byref(sz)),
           "fdtd_learned_record_scratch_size")
    s = torch.empty(int(sz.value), dtype=torch.uint8, device=sim.device)
    lo = (ctypes.c_int32 * 3)(*[int(v) for v in lo_xyz])
    hi = (ctypes.c_int32 * 3)(*[int(v) for v in hi_xyz])
    _check(lib.fdtd_learned_record(sim._h, lo, hi, int(thickness), int(n_steps), int(per_step), int(seed),
                                   _ptr(x), _ptr(y), _ptr(s), s.numel()), "fdtd_learned_record")
    return x, y


# ---------------------------------------------------------------- adjoint

def adjoint_gradient(sim, k0, mode, window, n_steps, box_lo, box_hi, checkpoint_every=100):
    """Advance `sim` by n_steps and return (L, dL/deps of the box) for the
    overlap objective of fdtd.h: L = sum over the last `window` steps of
    (sum m(i,j) Ez(i,j,k0))^2.  mode: CUDA float32 (ny, nx); box corners in
    (x, y, z); the gradient is a CUDA float64 tensor (nz, ny, nx) of the box."""
    import torch
    lib = sim._lib
    lo = (ctypes.c_int32 * 3)(*[int(v) for v in box_lo])
    hi = (ctypes.c_int32 * 3)(*[int(v) for v in box_hi])
    sz = ctypes.c_size_t(0)
    _check(lib.fdtd_adjoint_scratch_size(sim._h, int(n_steps), int(checkpoint_every), lo, hi, ctypes.byref(sz)),
           "fdtd_adjoint_scratch_size")
    scratch = torch.empty(int(sz.value), dtype=torch.uint8, device=sim.device)
    mode = mode.to(device=sim.device, dtype=torch.float32).contiguous()
    shape = tuple(int(hi[a] - lo[a]) for a in (2, 1, 0))
    grad = torch.empty(shape, dtype=torch.float64, device=sim.device)
    obj = OverlapObjective(int(k0), mode.data_ptr(), int(window))
    loss = ctypes.c_double(0.0)
    _check(lib.fdtd_adjoint_gradient(sim._h, ctypes.byref(obj), int(n_steps), int(checkpoint_every), lo, hi,
                                     _ptr(grad), ctypes.byref(loss), _ptr(scratch), scratch.numel()),
           "fdtd_adjoint_gradient")
    return loss.value, grad
