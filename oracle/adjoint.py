"""FP64 reference of the adjoint gradient dL/deps (inverse design).

TEST INFRASTRUCTURE ONLY: imported by tests/ (nothing in the product path).
Plain numpy, float64, derived from the discrete forward map (the oracle's
Yee step, Sec. 2, Eq. 1), not from a continuum adjoint:

Forward, state x^n = (E^n, H^{n-1/2}), c = dt/eps per cell (all three E
components of the cell), M = 0 on the PEC-fixed tangential E of the low
walls, 1 elsewhere:
    H^{n+1/2} = H^{n-1/2} - dt curl_f E^n
    E^{n+1}   = E^n + M c curl_b H^{n+1/2} + s^n,    s^n = -(dt/eps_s) J^n e_s.
Objective: L = sum_{n in window} O_n^2,  O_n = sum_{i,j} m(i,j) Ez^n(i,j,k0)
(the overlap of Ez on the plane k = k0 with a mode profile m), window = the
last W steps n = N-W+1 .. N.

Adjoint: with curl_f^T = curl_b under these PEC conventions (summation by
parts: fields beyond the high walls and H before the low walls read 0), the
transposed step, from lambda^N = dL/dx^N downwards, is
    lambda_H^n = lambda_H^{n+1} + curl_f(M c lambda_E^{n+1})
    lambda_E^n = lambda_E^{n+1} - dt curl_b lambda_H^n + dg_n/dE^n
and, since dE^{n+1}/dc = (E^{n+1} - E^n)/c per cell (the source scales with
1/eps too),
    dL/deps_p = -(1/eps_p) sum_{n=0}^{N-1} sum_a lambda_{E,a}^{n+1}(p) (E^{n+1} - E^n)_a(p).
"""
import numpy as np

from .yee import YeeOracle


def curl_f(E):
    """Forward-difference curl at the H positions; E beyond the high walls
    reads 0.  E: (3, nz, ny, nx)."""
    ex, ey, ez = E

    def d(a, axis):  # a(i+1) - a(i), zero beyond the end
        out = -a.copy()
        sl_to = [slice(None)] * 3
        sl_from = [slice(None)] * 3
        sl_to[axis] = slice(0, -1)
        sl_from[axis] = slice(1, None)
        out[tuple(sl_to)] += a[tuple(sl_from)]
        return out
    # axes of (nz, ny, nx): x = 2, y = 1, z = 0
    return np.stack([d(ez, 1) - d(ey, 0), d(ex, 0) - d(ez, 2), d(ey, 2) - d(ex, 1)])


def curl_b(H):
    """Backward-difference curl at the E positions; H before the low walls
    reads 0."""
    hx, hy, hz = H

    def d(a, axis):  # a(i) - a(i-1), a(-1) = 0
        out = a.copy()
        sl_to = [slice(None)] * 3
        sl_from = [slice(None)] * 3
        sl_to[axis] = slice(1, None)
        sl_from[axis] = slice(0, -1)
        out[tuple(sl_to)] -= a[tuple(sl_from)]
        return out
    return np.stack([d(hz, 1) - d(hy, 0), d(hx, 0) - d(hz, 2), d(hy, 2) - d(hx, 1)])


def pec_mask(shape_zyx):
    """M: 1 where an E component is updated, 0 on the low-wall tangential E."""
    nz, ny, nx = shape_zyx
    m = np.ones((3,) + tuple(shape_zyx))
    m[0, 0, :, :] = 0; m[0, :, 0, :] = 0          # Ex: j = 0 or k = 0
    m[1, 0, :, :] = 0; m[1, :, :, 0] = 0          # Ey: i = 0 or k = 0
    m[2, :, 0, :] = 0; m[2, :, :, 0] = 0          # Ez: i = 0 or j = 0
    return m


class Objective:
    """L = sum over the last `window` of `steps` steps of (m . Ez[k0])^2."""

    def __init__(self, k0, mode, window):
        self.k0, self.mode, self.window = int(k0), np.asarray(mode, np.float64), int(window)

    def overlap(self, E):
        return float((self.mode * E[2, self.k0]).sum())

    def weight(self, n, steps):
        return 1.0 if n > steps - self.window else 0.0


def forward(shape, eps, fields0, steps, sources, obj, dt, quantize=False):
    """Runs the oracle; returns (L, E history [steps+1, 3, ...], c)."""
    o = YeeOracle(shape, dt, eps, quantize_ce_f32=quantize)
    o.set_fields(fields0)
    for (c, i, j, k, J) in sources:
        o.add_source(c, i, j, k, J)
    hist = [o.fields()[:3].copy()]
    L = 0.0
    for n in range(1, steps + 1):
        o.step(1)
        E = o.fields()[:3].copy()
        hist.append(E)
        L += obj.weight(n, steps) * obj.overlap(E) ** 2
    return L, np.stack(hist), o.ce()


def objective(shape, eps, fields0, steps, sources, obj, dt, quantize=False):
    return forward(shape, eps, fields0, steps, sources, obj, dt, quantize)[0]


def gradient(shape, eps, fields0, steps, sources, obj, dt, quantize=False):
    """(L, dL/deps over the whole grid) by the reverse sweep above."""
    L, hist, c = forward(shape, eps, fields0, steps, sources, obj, dt, quantize)
    M = pec_mask(shape)
    eps = np.broadcast_to(np.asarray(eps, np.float64), shape)
    lam_e = np.zeros((3,) + tuple(shape))
    lam_h = np.zeros((3,) + tuple(shape))
    grad = np.zeros(shape)

    def source_of(n):  # dg_n / dE^n
        g = np.zeros((3,) + tuple(shape))
        w = obj.weight(n, steps)
        if w:
            g[2, obj.k0] = 2.0 * w * obj.overlap(hist[n]) * obj.mode
        return g

    lam_e += source_of(steps)
    for n in range(steps - 1, -1, -1):
        # lambda^{n+1} is complete: accumulate, then step back
        grad -= (lam_e * (hist[n + 1] - hist[n])).sum(0) / eps
        lam_h = lam_h + curl_f(M * c[None] * lam_e)
        lam_e = lam_e - dt * curl_b(lam_h) + source_of(n)
    return L, grad


def transposed_step(lam_e, lam_h, c, dt, M):
    """One step of the adjoint recursion without sources (for the dot test)."""
    lam_h = lam_h + curl_f(M * c[None] * lam_e)
    lam_e = lam_e - dt * curl_b(lam_h)
    return lam_e, lam_h


def yee_step(E, H, c, dt, M):
    """One forward step of the same linear map, in numpy (for the dot test)."""
    H = H - dt * curl_f(E)
    E = E + M * c[None] * curl_b(H)
    return E, H


def objective_window(shape, eps, fields0, steps, sources, obj, dt, quantize=False):
    """The objective L of `forward`, computed without keeping the E history:
    the oracle steps straight to the window, then reads Ez step by step (for
    finite differences on grids whose history would not fit in memory)."""
    o = YeeOracle(shape, dt, eps, quantize_ce_f32=quantize)
    o.set_fields(fields0)
    for (c, i, j, k, J) in sources:
        o.add_source(c, i, j, k, J)
    first = max(1, steps - obj.window + 1)
    if first > 1:
        o.step(first - 1)
    L = 0.0
    for n in range(first, steps + 1):
        o.step(1)
        L += obj.weight(n, steps) * obj.overlap(o.fields()[:3]) ** 2
    o.close()
    return L
