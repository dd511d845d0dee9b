"""The GPU path against a closed form, with no oracle in between: a discrete
PEC-cavity eigenmode of the Yee scheme (Sec. 2, Eq. 1) evolves exactly as
E^n = cos(n w dt) e, H^{n+1/2} = sin((n+1/2) w dt) h, with the discrete
frequency w = (2/dt) asin((dt/2) Omega).  After 200 FP32 steps both
schedules must stay within 1e-5 of it (largest error relative to the
largest value); a CPU float32 emulation of the same operations ends at
0.8e-6 .. 2.4e-6 on these cases.
"""
import math

import numpy as np
import pytest

from test_gpu_parity import run_gpu
from test_oracle_pins import cavity_mode, perp
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT


@pytest.mark.parametrize("shape,m,amp,eps_r", [
    ((64, 64, 64), (1, 1, 0), (0, 0, 1), 1.0),          # TM110 of config 1's cavity: Ez only
    ((20, 24, 28), (1, 2, 1), (1.0, -0.3, 0.7), 1.0),   # all six components, ragged tiles
    ((20, 24, 28), (2, 1, 3), (0.2, 1.0, -0.5), 2.25),  # uniform dielectric: dt/eps != dt
])
def test_cavity_eigenmode_closed_form_fp32(cuda_device, shape, m, amp, eps_r):
    nz, ny, nx = shape
    N = (nx, ny, nz)
    s = np.array([2 * math.sin(math.pi * m[a] / N[a] / 2) for a in range(3)])
    A = perp(s, amp)
    f0, _ = cavity_mode(shape, m, A, eps_r, DT, 0)
    fn, _ = cavity_mode(shape, m, A, eps_r, DT, 200)
    eps = np.full(shape, eps_r)
    for scheme in ("naive", "systolic"):
        got, _ = run_gpu(shape, eps, f0, 200, scheme)
        err = np.abs(got.numpy().astype(np.float64) - fn).max() / np.abs(fn).max()
        assert err < 1e-5, (scheme, err)
