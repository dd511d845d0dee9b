"""Parity at the benchmark's own sizes, in the launch configuration bench.py
times (one persistent launch per call of 2000 steps, default tile).

At these sizes the FP64 oracle is too slow to run (and no single cell's value
after 2000 steps can be computed alone: its light cone is the whole grid), so
the checks are properties that hold at any size:
* the systolic result equals the naive one bit for bit;
* the fields stay finite and the discrete energy of a source-free PEC box,
  Q = sum eps |E^n|^2 + sum H^{n-1/2} . H^{n+1/2} (computed here in FP64 with
  plain torch ops), is conserved to FP32 round-off.
"""
import numpy as np
import pytest
import torch

from helpers import bits_equal
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT


def energy(f, eps):
    """Q of a (6, nz, ny, nx) state in FP64; E beyond the high walls reads 0."""
    f = f.double()
    ex, ey, ez, hx, hy, hz = f

    def dfwd(a, axis):
        out = -a.clone()
        n = a.shape[axis]
        out.narrow(axis, 0, n - 1).add_(a.narrow(axis, 1, n - 1))
        return out
    # axes (z, y, x) = (0, 1, 2)
    cx = dfwd(ez, 1) - dfwd(ey, 0)
    cy = dfwd(ex, 0) - dfwd(ez, 2)
    cz = dfwd(ey, 2) - dfwd(ex, 1)
    q = (eps * (ex * ex + ey * ey + ez * ez)).sum()
    q += (hx * (hx - DT * cx)).sum() + (hy * (hy - DT * cy)).sum() + (hz * (hz - DT * cz)).sum()
    return float(q)


def run(shape, eps, f0, steps, scheme, sources=(), per_launch=2000):
    sim = fdtd.Sim(shape, eps, DT, scheme=scheme, steps_per_launch=per_launch, max_source_steps=max(steps, 1))
    try:
        if f0 is not None:
            sim.write_fields(torch.as_tensor(np.asarray(f0, np.float32)).cuda())
        for (c, i, j, k, J) in sources:
            sim.add_source(c, i, j, k, J)
        sim.step(steps)
        return sim.read_fields()
    finally:
        sim.close()


def test_config2_full_size_bitexact(cuda_device):
    # the benchmark workload itself: 256^3 Si/SiO2, Jz dipole, 2000 steps
    shape = (256, 256, 256)
    eps = wl.si_sio2_eps(shape, 1)
    src = [(2, 128, 128, 128, wl.sine_source(2000, DT, 20.0))]
    a = run(shape, eps, None, 2000, "systolic", src)
    b = run(shape, eps, None, 2000, "naive", src)
    assert torch.isfinite(a).all()
    assert bits_equal(a.cpu(), b.cpu())
    assert float(a.abs().max()) > 1e-3  # the dipole has radiated


def test_full_size_energy_is_conserved(cuda_device):
    # source-free PEC box, random fields (zero on the PEC walls), 2000 steps
    shape = (256, 256, 256)
    eps = wl.si_sio2_eps(shape, 2)
    f0 = wl.random_fields(shape, 5)
    e_t = torch.as_tensor(eps, device="cuda")
    q0 = energy(torch.as_tensor(np.asarray(f0, np.float32)).cuda(), e_t)
    out = run(shape, eps, f0, 2000, "systolic")
    q1 = energy(out, e_t)
    assert abs(q1 - q0) <= 1e-5 * abs(q0), (q0, q1)


def test_1024_cube_bitexact(cuda_device):
    shape = (1024, 1024, 1024)
    eps = wl.si_sio2_eps(shape, 1)
    f0 = None
    src = [(2, 512, 512, 512, wl.sine_source(40, DT, 20.0))]
    a = run(shape, eps, f0, 40, "systolic", src, per_launch=40)
    b = run(shape, eps, f0, 40, "naive", src)
    # compared on the device: the two states are 26 GB each
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert float(a.abs().max()) > 0
