"""Two more pins of the FP64 oracle, each against a fact that does not come
from the oracle's own 3D update (arxiv 2502.20610, Sec. 2, Eq. 1):

* superposition: the Yee map is linear and a point current enters
  additively, so the run with initial fields and a source equals the
  source-free run plus the run of the source alone from zero fields;
* 1D reduction: on a periodic grid, fields that vary along one axis only
  obey the textbook 1D Yee scheme of the two transverse polarisations
  (written below from Maxwell's equations in 1D), with eps varying along
  that axis, while the longitudinal E and H components stay frozen.
"""
import numpy as np
import pytest

from oracle import YeeOracle
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT


def test_superposition_of_initial_fields_and_source():
    shape = (9, 10, 11)
    steps = 40
    eps = wl.random_eps(shape, 31)
    f0 = wl.random_fields(shape, 31).astype(np.float64)
    J = wl.sine_source(steps, DT, wavelength=7.0) * 2.5
    src = (1, 5, 4, 6)  # Ey at (i, j, k) = (5, 4, 6)

    def run(fields, with_source):
        o = YeeOracle(shape, DT, eps)
        o.set_fields(fields)
        if with_source:
            o.add_source(src[0], src[1], src[2], src[3], J)
        o.step(steps)
        out = o.fields()
        o.close()
        return out

    both = run(f0, True)
    free = run(f0, False)
    alone = run(np.zeros_like(f0), True)
    scale = np.abs(both).max()
    assert np.abs(alone).max() > 1e-3 * scale  # the source did something
    assert np.abs(both - (free + alone)).max() <= 1e-12 * scale


def yee_1d(eps_n, eb, ec, hb, hc, steps):
    """Textbook 1D Yee scheme, periodic, for a wave along axis a with the
    transverse components b, c (a -> b -> c cyclic), eps = eps_n[n], mu = 1:
        dB_c/dt = -dE_b/da,  dB_b/dt = +dE_c/da,
        dD_b/dt = -dH_c/da,  dD_c/dt = +dH_b/da,
    E on the integer nodes n, H half a cell up (forward differences for H,
    backward for E), H half a step behind E; H advanced first."""
    eb, ec, hb, hc = (np.array(v, dtype=np.float64) for v in (eb, ec, hb, hc))
    ce = DT / eps_n
    for _ in range(steps):
        hc -= DT * (np.roll(eb, -1) - eb)
        hb += DT * (np.roll(ec, -1) - ec)
        eb -= ce * (hc - np.roll(hc, 1))
        ec += ce * (hb - np.roll(hb, 1))
    return eb, ec, hb, hc


def reduction_error(axis, mutation=0, n_len=37, steps=200):
    """Largest difference between the oracle on a periodic grid with fields
    that vary along `axis` only and the 1D scheme (or the frozen value, for
    the longitudinal components)."""
    dims_xyz = [4, 3, 5]
    dims_xyz[axis] = n_len
    shape = (dims_xyz[2], dims_xyz[1], dims_xyz[0])  # (nz, ny, nx)
    rng = np.random.default_rng(40 + axis)
    eps_n = rng.uniform(1.0, 12.1, n_len)
    prof = rng.uniform(-1.0, 1.0, (6, n_len))  # Ex Ey Ez Hx Hy Hz along the axis

    def spread(v):
        # a profile along `axis`, constant along the other two, as (nz, ny, nx)
        bshape = [1, 1, 1]
        bshape[2 - axis] = n_len
        return np.broadcast_to(v.reshape(bshape), shape)

    o = YeeOracle(shape, DT, spread(eps_n), periodic=True)
    o.set_mutation(mutation)
    o.set_fields([spread(prof[c]) for c in range(6)])
    o.step(steps)
    out = o.fields()
    o.close()

    a, b, c = axis, (axis + 1) % 3, (axis + 2) % 3
    eb, ec, hb, hc = yee_1d(eps_n, prof[b], prof[c], prof[3 + b], prof[3 + c], steps)
    expect = {b: eb, c: ec, 3 + b: hb, 3 + c: hc, a: prof[a], 3 + a: prof[3 + a]}
    return max(np.abs(out[comp] - spread(expect[comp])).max() for comp in range(6))


@pytest.mark.parametrize("axis", [0, 1, 2])  # 0 = x, 1 = y, 2 = z
def test_one_dimensional_reduction(axis):
    assert reduction_error(axis) < 1e-12


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_break_the_reduction(mutation):
    # sign of one Hy term, wrong difference axis in Hz or in Ex, half the H
    # time step: each changes the 1D dynamics along at least one axis
    assert max(reduction_error(axis, mutation, steps=20) for axis in range(3)) > 1e-6
