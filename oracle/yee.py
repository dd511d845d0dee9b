"""ctypes shim over the FP64 Yee oracle (oracle/yee_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path never imports it.

The oracle is the plain definition of the Yee leapfrog (arxiv 2502.20610,
Sec. 2, Eq. 1, Fig. 2): H half-step with forward differences over the whole
grid, then E half-step with backward differences, then point sources.
"""
import ctypes
import os

import numpy as np

from . import build as _build

COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.oracle_create.restype = P
    lib.oracle_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double]
    lib.oracle_destroy.argtypes = [P]
    lib.oracle_set_eps.argtypes = [P, D, ctypes.c_int]
    lib.oracle_set_field.argtypes = [P, ctypes.c_int, D]
    lib.oracle_get_field.argtypes = [P, ctypes.c_int, D]
    lib.oracle_get_ce.argtypes = [P, D]
    lib.oracle_current_step.restype = ctypes.c_long
    lib.oracle_current_step.argtypes = [P]
    lib.oracle_set_step.argtypes = [P, ctypes.c_long]
    lib.oracle_set_mutation.argtypes = [P, ctypes.c_int]
    lib.oracle_add_source.restype = ctypes.c_int
    lib.oracle_add_source.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, D,
                                      ctypes.c_long]
    lib.oracle_step.restype = ctypes.c_int
    lib.oracle_step.argtypes = [P, ctypes.c_long]
    lib.oracle_energy.restype = ctypes.c_double
    lib.oracle_energy.argtypes = [P]
    lib.oracle_div.argtypes = [P, D, D]
    lib.oracle_round_to_format.restype = ctypes.c_double
    lib.oracle_round_to_format.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_set_storage.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, D]
    lib.oracle_set_eps_sigma.argtypes = [P, D, D, ctypes.c_int]
    lib.oracle_graded_sigma.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_int, D]
    lib.oracle_get_ca.argtypes = [P, D]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


#: 16-bit storage formats: (significant bits p, emin, emax)
FORMATS = {"f16": (11, -14, 15), "bf16": (8, -126, 127)}


def set_threads(n):
    """Host threads of the oracle's parallel loops from now on (timing only;
    results do not depend on it).  Returns the count in effect."""
    return int(_load().oracle_set_threads(int(n)))


def round_to_format(x, fmt):
    """Elementwise nearest value of the 16-bit format `fmt` (ties to even),
    computed by the oracle's own rounding routine; returns float64."""
    lib = _load()
    p, emin, emax = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    f = lib.oracle_round_to_format
    return np.array([f(float(v), p, emin, emax) for v in x.ravel()], dtype=np.float64).reshape(x.shape)


def graded_sigma(shape_zyx, thickness, sigma_max, order):
    """Graded conductivity sigma_max * sum_a (depth_a / L)^m of the absorbing
    layer (oracle's own profile routine), as an (nz, ny, nx) float64 array."""
    lib = _load()
    nz, ny, nx = (int(s) for s in shape_zyx)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    lib.oracle_graded_sigma(nx, ny, nz, int(thickness), float(sigma_max), int(order), _dptr(out))
    return out


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class YeeOracle:
    """FP64 Yee stepper on an (nz, ny, nx) grid (x fastest).

    Arrays exchanged with it are numpy arrays of shape (nz, ny, nx).
    """

    def __init__(self, shape_zyx, dt, eps=None, periodic=False, quantize_ce_f32=False):
        nz, ny, nx = (int(s) for s in shape_zyx)
        self.shape = (nz, ny, nx)
        self.dt = float(dt)
        self._lib = _load()
        self._h = self._lib.oracle_create(nx, ny, nz, 1 if periodic else 0, self.dt)
        if not self._h:
            raise ValueError("oracle_create failed")
        if eps is not None:
            self.set_eps(eps, quantize_ce_f32)

    def close(self):
        if self._h:
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != self.shape:
            a = np.ascontiguousarray(np.broadcast_to(a, self.shape), dtype=np.float64)
        return a

    def set_eps(self, eps, quantize_ce_f32=False):
        e = self._arr(eps)
        self._lib.oracle_set_eps(self._h, _dptr(e), 1 if quantize_ce_f32 else 0)

    def set_eps_sigma(self, eps, sigma, quantize_f32=False):
        """Per-cell eps and conductivity: the E half-step becomes
        E <- ca E + cb curl H (cb also scales the sources)."""
        e = self._arr(eps)
        sg = self._arr(sigma)
        self._lib.oracle_set_eps_sigma(self._h, _dptr(e), _dptr(sg), 1 if quantize_f32 else 0)

    def ca(self):
        out = np.empty(self.shape, dtype=np.float64)
        self._lib.oracle_get_ca(self._h, _dptr(out))
        return out

    def set_fields(self, fields):
        """fields: sequence of 6 arrays (Ex, Ey, Ez, Hx, Hy, Hz) or a (6, nz, ny, nx) array."""
        for c in range(6):
            a = self._arr(fields[c])
            self._lib.oracle_set_field(self._h, c, _dptr(a))

    def fields(self):
        out = np.empty((6,) + self.shape, dtype=np.float64)
        for c in range(6):
            self._lib.oracle_get_field(self._h, c, _dptr(out[c]))
        return out

    def ce(self):
        out = np.empty(self.shape, dtype=np.float64)
        self._lib.oracle_get_ce(self._h, _dptr(out))
        return out

    def add_source(self, comp, i, j, k, J):
        J = np.ascontiguousarray(np.asarray(J, dtype=np.float64))
        rc = self._lib.oracle_add_source(self._h, int(comp), int(i), int(j), int(k), _dptr(J), J.size)
        if rc != 0:
            raise ValueError("oracle_add_source rejected the source")

    def step(self, n):
        if self._lib.oracle_step(self._h, int(n)) != 0:
            raise MemoryError("oracle_step: allocation failed")

    @property
    def current_step(self):
        return int(self._lib.oracle_current_step(self._h))

    def set_current_step(self, s):
        self._lib.oracle_set_step(self._h, int(s))

    def set_mutation(self, m):
        """Plant a known mistake (pin-sensitivity tests only): 1 sign of one
        Hy term, 2 wrong difference axis in Hz, 3 wrong difference axis in Ex,
        4 half the H time step, 5 source sign."""
        self._lib.oracle_set_mutation(self._h, int(m))

    def set_storage(self, fmt, scales=None):
        """Round stored fields to the 16-bit format `fmt` ("f16", "bf16") from
        now on, as s_c * R(v / s_c) (scales: six powers of two, default 1);
        None switches rounding off.  The current fields are rounded at once."""
        sc = np.ascontiguousarray(np.ones(6) if scales is None else np.asarray(scales, dtype=np.float64))
        if fmt is None:
            self._lib.oracle_set_storage(self._h, 0, 0, 0, _dptr(sc))
        else:
            p, emin, emax = FORMATS[fmt]
            self._lib.oracle_set_storage(self._h, p, emin, emax, _dptr(sc))

    def energy(self):
        return float(self._lib.oracle_energy(self._h))

    def divergence(self):
        de = np.empty(self.shape, dtype=np.float64)
        dh = np.empty(self.shape, dtype=np.float64)
        self._lib.oracle_div(self._h, _dptr(de), _dptr(dh))
        return de, dh
