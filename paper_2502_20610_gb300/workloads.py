"""Seeded synthetic inputs for the Yee FDTD path.

This module holds input generators only (random fields, permittivity maps,
initial pulses, source waveforms).  It contains none of the update
arithmetic; the CUDA library and the FP64 oracle both consume what it makes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: value i of stream `seed` is the splitmix64 output function applied
to key(seed) + (i + 1) * golden_gamma.
"""
import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Courant number 0.99/sqrt(3) with dx = c = 1.
DT_DEFAULT = 0.99 / math.sqrt(3.0)

EPS_SIO2 = 2.1
EPS_SI = 12.1


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed):
    return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ np.uint64(0x5EED5EED5EED5EED))


def splitmix64(seed, start, count):
    """`count` consecutive 64-bit outputs of stream `seed` from position `start`."""
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed) + (i + np.uint64(1)) * GOLDEN_GAMMA)


def uniform_pm1(seed, count, start=0):
    """float32 values uniform in [-1, 1) from the top 24 bits (exact in float32)."""
    u = splitmix64(seed, start, count) >> np.uint64(40)
    return (u.astype(np.float64) * (2.0 / (1 << 24)) - 1.0).astype(np.float32)


def random_fields(shape_zyx, seed, zero_pec_walls=True):
    """(6, nz, ny, nx) float32 fields uniform in [-1, 1), all six components
    independent.  With zero_pec_walls the tangential E on the three low walls
    (the values a PEC box never updates) is set to 0."""
    nz, ny, nx = shape_zyx
    n = nz * ny * nx
    f = uniform_pm1(seed, 6 * n).reshape(6, nz, ny, nx)
    if zero_pec_walls:
        f[0][:, 0, :] = 0; f[0][0, :, :] = 0      # Ex: j=0, k=0
        f[1][:, :, 0] = 0; f[1][0, :, :] = 0      # Ey: i=0, k=0
        f[2][:, :, 0] = 0; f[2][:, 0, :] = 0      # Ez: i=0, j=0
    return f


def random_eps(shape_zyx, seed, lo=1.0, hi=12.1):
    nz, ny, nx = shape_zyx
    u = uniform_pm1(seed ^ 0xE95, nz * ny * nx).astype(np.float64)
    return (lo + (hi - lo) * 0.5 * (u + 1.0)).reshape(shape_zyx)


def si_sio2_eps(shape_zyx, seed, n_min=8, n_max=20, width=10):
    """Seeded photonic-shaped permittivity map: SiO2 background (eps 2.1) with
    n_min..n_max straight Si slabs (eps 12.1) of width x width cross-section,
    each along a random axis, of length uniform in [N/2, N-2] and placed
    uniformly so that it lies inside the grid; later slabs overwrite earlier
    ones.  Returns float64 (nz, ny, nx)."""
    nz, ny, nx = shape_zyx
    dims = (nx, ny, nz)
    eps = np.full((nz, ny, nx), EPS_SIO2, dtype=np.float64)
    stream = iter(splitmix64(seed ^ 0x51510, 0, 1 + 8 * n_max).tolist())
    count = n_min + next(stream) % (n_max - n_min + 1)
    for _ in range(count):
        axis = next(stream) % 3
        lo = [0, 0, 0]
        hi = [0, 0, 0]
        n_ax = dims[axis]
        lmin = max(1, n_ax // 2)
        lmax = max(lmin, n_ax - 2)
        length = lmin + next(stream) % (lmax - lmin + 1)
        start = next(stream) % (n_ax - length + 1)
        lo[axis], hi[axis] = start, start + length
        for b in range(3):
            if b == axis:
                continue
            w = min(width, dims[b])
            s = next(stream) % (dims[b] - w + 1)
            lo[b], hi[b] = s, s + w
        eps[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = EPS_SI
    return eps


def gaussian_ez(shape_zyx, sigma=4.0):
    """Config-1 initial state: Ez(i, j, k+1/2) = exp(-r^2 / (2 sigma^2)) about
    the grid centre, all other components 0.  Returns (6, nz, ny, nx) float64."""
    nz, ny, nx = shape_zyx
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (i - nx / 2) ** 2 + (j - ny / 2) ** 2 + (k + 0.5 - nz / 2) ** 2
    f = np.zeros((6, nz, ny, nx), dtype=np.float64)
    f[2] = np.exp(-r2 / (2.0 * sigma * sigma))
    return f


def sine_source(n_steps, dt, wavelength=20.0):
    """J(t_{n+1/2}) = sin(omega (n + 1/2) dt), omega = 2 pi / wavelength (c = 1)."""
    n = np.arange(n_steps, dtype=np.float64)
    return np.sin(2.0 * math.pi / wavelength * (n + 0.5) * dt)


def gaussian_pulse_source(n_steps, dt, wavelength=20.0, frac_bandwidth=0.5):
    """Gaussian-modulated sine: J(t) = exp(-(t-t0)^2/(2 tau^2)) sin(w0 (t-t0)),
    tau from a FWHM fractional bandwidth, t0 = 5 tau."""
    f0 = 1.0 / wavelength
    tau = 2.0 * math.sqrt(2.0 * math.log(2.0)) / (2.0 * math.pi * frac_bandwidth * f0)
    t0 = 5.0 * tau
    t = (np.arange(n_steps, dtype=np.float64) + 0.5) * dt
    return np.exp(-((t - t0) ** 2) / (2.0 * tau * tau)) * np.sin(2.0 * math.pi * f0 * (t - t0))
