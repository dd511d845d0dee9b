"""Pins of the oracle's lossy E update (conductivity sigma, the c_a / c_b
form of the time-centred discretisation of eps dE/dt + sigma E = curl H - J)
and of its graded absorbing-layer profile.

* The discrete energy balance: for the Yee leapfrog with
  eps (E^{n+1} - E^n) + g (E^{n+1} + E^n) = dt curl_b H^{n+1/2}, g = sigma dt/2,
  the quantity Q^n = sum eps |E^n|^2 + sum H^{n-1/2} . H^{n+1/2} obeys
  Q^{n+1} - Q^n = -sum g |E^{n+1} + E^n|^2 exactly (the curl terms cancel
  because curl_f and curl_b are adjoint).  A wrong c_a or c_b breaks it.
* sigma = 0 reproduces the lossless update exactly.
* The profile sigma_max * sum_a (depth_a / L)^m at chosen cells.
* A pulse launched into a box lined with the absorber loses its energy.
"""
import numpy as np
import pytest

from oracle import YeeOracle
from oracle.yee import graded_sigma
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT


def balance_residual(shape, sigma_max, L, m, steps=4, seed=3, quantize=False, mutation=0):
    """max over steps of |Q^{n+1} - Q^n + sum g |E^{n+1} + E^n|^2| / Q^n with
    eps and g = sigma dt / 2 taken from the inputs (FP32-rounded coefficients:
    the eps and g those coefficients stand for), and the largest relative gap
    between that eps and the input eps."""
    eps = wl.random_eps(shape, seed)
    sig = graded_sigma(shape, L, sigma_max, m)
    o = YeeOracle(shape, DT, eps)
    o.set_mutation(mutation)
    o.set_eps_sigma(eps, sig, quantize)
    o.set_fields(wl.random_fields(shape, seed))
    ce, ca = o.ce(), o.ca()
    # from ca = (eps - g)/(eps + g) and cb = dt/(eps + g)
    eps_c = DT / ce * (1.0 + ca) / 2.0
    g_c = DT / ce * (1.0 - ca) / 2.0
    g = g_c if quantize else sig * DT / 2.0
    eps_gap = float(np.max(np.abs(eps_c - eps) / eps))
    worst = 0.0
    for _ in range(steps):
        q0, e0 = o.energy(), o.fields()[:3].copy()
        o.step(1)
        q1, e1 = o.energy(), o.fields()[:3]
        loss = float((g[None] * (e1 + e0) ** 2).sum())
        worst = max(worst, abs(q1 - q0 + loss) / abs(q0))
    return worst, loss, eps_gap


@pytest.mark.parametrize("quantize", [False, True])
def test_lossy_energy_balance(quantize):
    res, loss, eps_gap = balance_residual((20, 22, 24), 0.8, 6, 3, quantize=quantize)
    assert loss > 0
    assert res < 1e-13
    assert eps_gap < (1e-6 if quantize else 1e-14)


def test_sigma_zero_is_lossless_update():
    shape = (9, 10, 11)
    eps = wl.random_eps(shape, 5)
    f0 = wl.random_fields(shape, 5)
    a = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
    b = YeeOracle(shape, DT, eps)
    b.set_eps_sigma(eps, np.zeros(shape), True)
    for o in (a, b):
        o.set_fields(f0)
        o.add_source(2, 4, 5, 6, wl.sine_source(20, DT))
        o.step(20)
    assert np.array_equal(a.fields(), b.fields())
    assert np.array_equal(b.ca(), np.ones(shape))


def test_graded_profile_closed_form():
    nz, ny, nx = 40, 41, 42
    L, smax, m = 8, 1.5, 3
    s = graded_sigma((nz, ny, nx), L, smax, m)
    assert s[20, 20, 21] == 0.0                                  # interior
    assert s[20, 20, 0] == smax                                  # outer x cell: depth L
    assert s[20, 20, nx - 1] == smax
    assert np.isclose(s[20, 20, L - 1], smax * (1 / L) ** m)     # innermost layer cell: depth 1
    assert s[20, 20, L] == 0.0 and s[20, 20, nx - 1 - L] == 0.0
    assert np.isclose(s[0, 0, 0], 3 * smax)                      # corner: three axes add
    assert np.isclose(s[3, 20, nx - 2], smax * (((L - 3) / L) ** m + ((L - 1) / L) ** m))
    # symmetric under reflection of each axis
    assert np.array_equal(s, s[::-1, :, :]) and np.array_equal(s, s[:, ::-1, :]) and np.array_equal(s, s[:, :, ::-1])


def test_absorber_drains_a_pulse():
    # a Gaussian-modulated dipole pulse (zero net charge) radiates into a box
    # lined with a 12-cell absorber: once the source is off, the absorber
    # takes almost all of the energy; with PEC walls alone it stays
    shape = (40, 40, 40)
    eps = np.ones(shape)
    J = wl.gaussian_pulse_source(270, DT, wavelength=10.0)
    left = []
    for smax in (0.0, 0.6):
        o = YeeOracle(shape, DT, eps)
        o.set_eps_sigma(eps, graded_sigma(shape, 12, smax, 3))
        o.add_source(2, 20, 20, 20, J)
        o.step(270)
        q_on = o.energy()
        o.step(300)
        left.append(o.energy() / q_on)
    assert left[0] > 0.9
    assert left[1] < 0.05


def test_planted_wrong_loss_sign_is_caught():
    res, _, gap = balance_residual((8, 9, 10), 0.8, 3, 3, steps=2, mutation=6)
    assert res > 1e-6 and gap > 1e-6
