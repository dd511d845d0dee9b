"""Pins of the FP64 oracle against what the discretisation fixes.

None of these re-types the oracle's update: each compares it with an
independent fact of the Yee scheme (arxiv 2502.20610, Sec. 2, Eq. 1):

* exact discrete energy invariant (leapfrog with C_H = C_E^T),
* Gauss-law invariants div(eps E) and div H (div curl = 0),
* closed-form discrete PEC-cavity eigenmodes (time stepping, dt, stencil),
* the Yee dispersion relation for periodic plane waves,
* the discrete work identity of a point current source (source sign, dt/eps
  factor and timing) and the charge it leaves behind,
* invariance under a cyclic permutation of the axes (component symmetry),
and a test that planted mistakes in the oracle each break at least one pin.
"""
import math

import numpy as np
import pytest

from oracle import YeeOracle
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT


# ----------------------------------------------------------------- helpers --

def cavity_mode(shape_zyx, m, amp, eps_r, dt, n):
    """Closed-form discrete PEC-cavity mode after n steps: returns the oracle's
    state (E^n, H^{n-1/2}) as a (6, nz, ny, nx) array and omega.

    E_x = A_x cos(kx(i+1/2)) sin(ky j) sin(kz k) (cyclic for y, z) with
    k_a = pi m_a / N_a, div-free when A . s = 0, s_a = 2 sin(k_a / 2);
    H^{n+1/2} = sin((n+1/2) w dt) h with h = -dt (s x A) / (2 sin(w dt / 2))
    on the H sinusoids, and Omega^2 = |s|^2 / eps = (2 sin(w dt/2)/dt)^2."""
    nz, ny, nx = shape_zyx
    N = (nx, ny, nz)
    kv = [math.pi * m[a] / N[a] for a in range(3)]
    s = np.array([2 * math.sin(k / 2) for k in kv])
    A = np.asarray(amp, dtype=np.float64)
    assert abs(A @ s) < 1e-12
    Om = math.sqrt((s @ s) / eps_r)
    w = 2.0 / dt * math.asin(dt * Om / 2.0)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    C, S = np.cos, np.sin
    kx, ky, kz = kv
    eg = [C(kx * (ii + .5)) * S(ky * jj) * S(kz * kk),
          S(kx * ii) * C(ky * (jj + .5)) * S(kz * kk),
          S(kx * ii) * S(ky * jj) * C(kz * (kk + .5))]
    hg = [S(kx * ii) * C(ky * (jj + .5)) * C(kz * (kk + .5)),
          C(kx * (ii + .5)) * S(ky * jj) * C(kz * (kk + .5)),
          C(kx * (ii + .5)) * C(ky * (jj + .5)) * S(kz * kk)]
    B = -dt * np.cross(s, A) / (2 * math.sin(w * dt / 2))
    out = np.empty((6, nz, ny, nx))
    for a in range(3):
        out[a] = math.cos(n * w * dt) * A[a] * eg[a]
        out[3 + a] = math.sin((n - 0.5) * w * dt) * B[a] * hg[a]
    return out, w


def plane_wave(shape_zyx, m, amp, eps_r, dt, n):
    """Periodic travelling plane wave after n steps (E^n, H^{n-1/2}):
    E = Re(A exp(i(k.r_E - n w dt))), H = Re(B exp(i(k.r_H - (n-1/2) w dt))),
    k_a = 2 pi m_a / N_a, B = dt (s x A) / (2 sin(w dt/2)), with
    (sin(w dt / 2) / dt)^2 = sum_a sin^2(k_a / 2) / eps."""
    nz, ny, nx = shape_zyx
    N = (nx, ny, nz)
    kv = np.array([2 * math.pi * m[a] / N[a] for a in range(3)])
    s = 2 * np.sin(kv / 2)
    A = np.asarray(amp, dtype=np.float64)
    assert abs(A @ s) < 1e-12
    w = 2.0 / dt * math.asin(dt * math.sqrt((s @ s) / eps_r) / 2.0)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = kv
    ph_e = [kx * (ii + .5) + ky * jj + kz * kk,
            kx * ii + ky * (jj + .5) + kz * kk,
            kx * ii + ky * jj + kz * (kk + .5)]
    ph_h = [kx * ii + ky * (jj + .5) + kz * (kk + .5),
            kx * (ii + .5) + ky * jj + kz * (kk + .5),
            kx * (ii + .5) + ky * (jj + .5) + kz * kk]
    B = dt * np.cross(s, A) / (2 * math.sin(w * dt / 2))
    out = np.empty((6, nz, ny, nx))
    for a in range(3):
        out[a] = A[a] * np.cos(ph_e[a] - n * w * dt)
        out[3 + a] = B[a] * np.cos(ph_h[a] - (n - 0.5) * w * dt)
    return out, w


def perp(s, v):
    v = np.asarray(v, dtype=np.float64)
    return v - s * (v @ s) / (s @ s)


def rot_fields(f):
    """Cyclic axis permutation x' = y, y' = z, z' = x of a (6, n, n, n) state:
    each array maps out[a, b, c] = in[b, c, a] and components rotate
    (Ex' <- Ey, Ey' <- Ez, Ez' <- Ex, same for H)."""
    T = lambda a: np.transpose(a, (2, 0, 1))
    return np.stack([T(f[1]), T(f[2]), T(f[0]), T(f[4]), T(f[5]), T(f[3])])


# -------------------------------------------------------------------- pins --

def energy_drift(shape, steps=60, seed=3, mutation=0):
    eps = wl.random_eps(shape, seed)
    o = YeeOracle(shape, DT, eps)
    o.set_mutation(mutation)
    o.set_fields(wl.random_fields(shape, seed).astype(np.float64))
    q0 = o.energy()
    worst = 0.0
    for _ in range(steps // 10):
        o.step(10)
        worst = max(worst, abs(o.energy() - q0) / abs(q0))
    return worst


def gauss_drift(shape, steps=40, seed=4, mutation=0):
    eps = wl.random_eps(shape, seed)
    o = YeeOracle(shape, DT, eps)
    o.set_mutation(mutation)
    o.set_fields(wl.random_fields(shape, seed).astype(np.float64))
    de0, dh0 = o.divergence()
    o.step(steps)
    de, dh = o.divergence()
    # interior nodes only: PEC walls carry surface charge, and dual nodes at
    # the high faces read the zero ghost
    e = np.abs(de - de0)[1:, 1:, 1:].max()
    h = np.abs(dh - dh0)[:-1, :-1, :-1].max()
    return max(e, h)


def eigenmode_error(shape, m, amp_hint, eps_r, steps, mutation=0):
    nz, ny, nx = shape
    N = (nx, ny, nz)
    s = np.array([2 * math.sin(math.pi * m[a] / N[a] / 2) for a in range(3)])
    A = perp(s, amp_hint)
    f0, _ = cavity_mode(shape, m, A, eps_r, DT, 0)
    o = YeeOracle(shape, DT, np.full(shape, eps_r))
    o.set_mutation(mutation)
    o.set_fields(f0)
    o.step(steps)
    fn, _ = cavity_mode(shape, m, A, eps_r, DT, steps)
    return np.abs(o.fields() - fn).max() / np.abs(fn).max()


def test_energy_invariant_random_eps():
    # Q^n = sum eps|E^n|^2 + H^{n-1/2}.H^{n+1/2} is exactly conserved
    assert energy_drift((9, 11, 13), steps=200) < 1e-12


def test_energy_invariant_quantized_coefficient():
    shape = (7, 8, 9)
    eps = wl.random_eps(shape, 11)
    o = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
    o.set_fields(wl.random_fields(shape, 11).astype(np.float64))
    q0 = o.energy()
    o.step(100)
    assert abs(o.energy() - q0) / q0 < 1e-12
    ce = o.ce()
    assert np.all(ce == ce.astype(np.float32).astype(np.float64))


def test_gauss_law_invariant():
    assert gauss_drift((10, 9, 12)) < 1e-12


@pytest.mark.parametrize("m,amp,eps_r", [
    ((1, 1, 0), (0, 0, 1), 1.0),          # TM110: Ez only
    ((1, 2, 1), (1.0, -0.3, 0.7), 1.0),   # all six components
    ((2, 1, 3), (0.2, 1.0, -0.5), 2.25),  # uniform dielectric
])
def test_cavity_eigenmode_closed_form(m, amp, eps_r):
    assert eigenmode_error((10, 12, 16), m, amp, eps_r, 200) < 1e-12


def test_tm110_frequency_at_64():
    # discrete TM110 of a 64^3 vacuum cavity: w = (2/dt) asin((dt/2) Omega)
    _, w = cavity_mode((2, 2, 2), (1, 1, 0), (0, 0, 1), 1.0, DT, 0)  # shape only sets N
    N = 64
    s = 2 * math.sin(math.pi / (2 * N))
    w64 = 2 / DT * math.asin(DT / 2 * math.sqrt(2) * s)
    assert abs(w64 - 0.0694176) < 5e-7
    assert abs(w64 - math.pi * math.sqrt(2) / N) < 1e-5  # close to the continuum value


@pytest.mark.parametrize("m,amp,eps_r", [
    ((1, 0, 0), (0, 1, 0), 1.0),
    ((1, 2, 1), (0.3, -1.0, 0.4), 1.0),
    ((3, 1, 2), (1.0, 0.5, -0.2), 4.0),
])
def test_dispersion_periodic_plane_wave(m, amp, eps_r):
    shape = (8, 12, 16)
    nz, ny, nx = shape
    kv = np.array([2 * math.pi * m[0] / nx, 2 * math.pi * m[1] / ny, 2 * math.pi * m[2] / nz])
    A = perp(2 * np.sin(kv / 2), amp)
    f0, _ = plane_wave(shape, m, A, eps_r, DT, 0)
    o = YeeOracle(shape, DT, np.full(shape, eps_r), periodic=True)
    o.set_fields(f0)
    o.step(150)
    fn, _ = plane_wave(shape, m, A, eps_r, DT, 150)
    assert np.abs(o.fields() - fn).max() < 1e-11


def source_run(shape, steps, mutation=0):
    eps = wl.random_eps(shape, 7)
    o = YeeOracle(shape, DT, eps)
    o.set_mutation(mutation)
    f = wl.random_fields(shape, 7).astype(np.float64)
    o.set_fields(f)
    src = (2, shape[2] // 2, shape[1] // 2, shape[0] // 2)  # Ez at (i, j, k)
    J = wl.sine_source(steps, DT, wavelength=9.0) * 3.0
    o.add_source(src[0], src[1], src[2], src[3], J)
    return o, src, J


def source_work_error(shape=(8, 9, 10), steps=30, mutation=0):
    """Q^{n+1} - Q^n = -dt J_n (E_s^{n+1} + E_s^n) for a point current J_n."""
    o, (c, i, j, k), J = source_run(shape, steps, mutation)
    worst = 0.0
    q = o.energy()
    e_prev = o.fields()[c, k, j, i]
    for n in range(steps):
        o.step(1)
        q_next = o.energy()
        e_next = o.fields()[c, k, j, i]
        pred = -DT * J[n] * (e_next + e_prev)
        worst = max(worst, abs((q_next - q) - pred) / (abs(q) + 1.0))
        q, e_prev = q_next, e_next
    return worst


def test_source_work_identity():
    assert source_work_error() < 1e-12


def test_source_charge():
    # a point current Jz at Ez(i,j,k+1/2) leaves -dt*sum(J) of charge at
    # node (i,j,k) and +dt*sum(J) at node (i,j,k+1); elsewhere div is invariant
    shape = (8, 9, 10)
    steps = 25
    o, (c, i, j, k), J = source_run(shape, steps)
    de0, _ = o.divergence()
    o.step(steps)
    de, _ = o.divergence()
    d = de - de0
    q = DT * J[:steps].sum()
    assert abs(d[k, j, i] + q) < 1e-12
    assert abs(d[k + 1, j, i] - q) < 1e-12
    d[k, j, i] = 0
    d[k + 1, j, i] = 0
    assert np.abs(d[1:, 1:, 1:]).max() < 1e-12


def rotation_error(n=7, steps=20, mutation=0):
    shape = (n, n, n)
    eps = wl.random_eps(shape, 9)
    f = wl.random_fields(shape, 9).astype(np.float64)
    a = YeeOracle(shape, DT, eps)
    a.set_mutation(mutation)
    a.set_fields(f)
    a.step(steps)
    b = YeeOracle(shape, DT, np.transpose(eps, (2, 0, 1)))
    b.set_mutation(mutation)
    b.set_fields(rot_fields(f))
    b.step(steps)
    return np.abs(rot_fields(a.fields()) - b.fields()).max()


def test_cyclic_axis_permutation():
    assert rotation_error() == 0.0


def test_planted_mistakes_are_caught():
    """Each planted mistake in the oracle (sign of one term, wrong
    difference axis in one component, wrong H time step, flipped source
    sign) must break at least one pin."""
    for m in (1, 2, 3, 4, 5):
        caught = []
        caught.append(energy_drift((6, 7, 8), steps=30, mutation=m) > 1e-9)
        caught.append(gauss_drift((6, 7, 8), steps=10, mutation=m) > 1e-9)
        caught.append(eigenmode_error((6, 8, 10), (1, 2, 1), (1.0, -0.3, 0.7), 1.0, 40, mutation=m) > 1e-9)
        caught.append(rotation_error(n=6, steps=5, mutation=m) > 0)
        caught.append(source_work_error(steps=8, mutation=m) > 1e-9)
        assert any(caught), f"mutation {m} escaped every pin: {caught}"
