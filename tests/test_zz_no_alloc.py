"""The allocation-free systolic entry point (fdtd_systolic_step_noalloc)
against the handle API (fdtd_create + fdtd_step, systolic scheme).

Callers that may not call cudaMalloc keep their own field and coefficient
buffers and step them through this entry point, whose scratch is a fixed
device array inside the library.  It must give the same bits as the regular
entry point, on two calls in a row (the second call reuses the scratch the
first one left behind).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from helpers import bits_equal
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT


def noalloc_step(lib, shape, fields, coef, n):
    nz, ny, nx = shape
    g = fdtd.Grid(nx, ny, nz)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.fdtd_systolic_step_noalloc(ctypes.byref(g), fields.data_ptr(), coef.data_ptr(), DT, int(n),
                                          ctypes.c_void_p(stream))


def test_noalloc_matches_handle_api_on_two_calls(cuda_device):
    lib = fdtd.load_library()
    shape = (29, 40, 70)  # nz, ny, nx: several 31x15x15 tiles with ragged tails
    eps = wl.random_eps(shape, 21)
    f0 = wl.random_fields(shape, 21, zero_pec_walls=False)

    sim = fdtd.Sim(shape, eps, DT, scheme="systolic")
    sim.write_fields(torch.as_tensor(f0).cuda())
    sim.step(37)
    ref1 = sim.read_fields().cpu()
    sim.step(25)
    ref2 = sim.read_fields().cpu()
    sim.close()

    # caller-owned buffers: the state and the FP32 coefficient dt/eps
    fields = torch.as_tensor(f0).cuda().contiguous()
    coef = torch.as_tensor((DT / eps).astype(np.float32)).cuda().contiguous()
    assert noalloc_step(lib, shape, fields, coef, 37) == fdtd.FDTD_OK
    got1 = fields.cpu()
    assert bits_equal(got1, ref1)
    assert noalloc_step(lib, shape, fields, coef, 25) == fdtd.FDTD_OK
    got2 = fields.cpu()
    assert bits_equal(got2, ref2)


@pytest.mark.parametrize("shape,steps", [
    ((29, 40, 70), 1100),  # more steps than one launch takes (1024): two launches per call
    ((2, 3, 6000), 1100),  # a long thin grid whose 1024-step tile schedule does not fit the
                           # scratch: the call steps it in shorter launches
])
def test_noalloc_multi_launch_calls(cuda_device, shape, steps):
    lib = fdtd.load_library()
    eps = wl.random_eps(shape, 23)
    f0 = wl.random_fields(shape, 23, zero_pec_walls=False)
    sim = fdtd.Sim(shape, eps, DT, scheme="systolic")
    sim.write_fields(torch.as_tensor(f0).cuda())
    sim.step(steps)
    ref = sim.read_fields().cpu()
    sim.close()
    fields = torch.as_tensor(f0).cuda().contiguous()
    coef = torch.as_tensor((DT / eps).astype(np.float32)).cuda().contiguous()
    assert noalloc_step(lib, shape, fields, coef, steps) == fdtd.FDTD_OK
    assert bits_equal(fields.cpu(), ref)


def test_noalloc_rejects_bad_arguments(cuda_device):
    lib = fdtd.load_library()
    shape = (4, 4, 4)
    fields = torch.zeros((6,) + shape, device="cuda")
    coef = torch.full(shape, DT, device="cuda")
    g = fdtd.Grid(4, 4, 4)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.fdtd_systolic_step_noalloc(ctypes.byref(g), None, coef.data_ptr(), DT, 1, s) == \
        fdtd.FDTD_ERR_INVALID_ARG
    assert lib.fdtd_systolic_step_noalloc(ctypes.byref(g), fields.data_ptr(), coef.data_ptr(), DT, -1, s) == \
        fdtd.FDTD_ERR_INVALID_ARG
    assert lib.fdtd_systolic_step_noalloc(ctypes.byref(g), fields.data_ptr(), coef.data_ptr(), float("inf"), 1,
                                          s) == fdtd.FDTD_ERR_INVALID_ARG
    huge = fdtd.Grid((1 << 20) + 1, 1, 1)
    assert lib.fdtd_systolic_step_noalloc(ctypes.byref(huge), fields.data_ptr(), coef.data_ptr(), DT, 1, s) == \
        fdtd.FDTD_ERR_INVALID_ARG
    # a grid whose tile schedule cannot fit the fixed scratch is refused up front
    big = fdtd.Grid(4096, 4096, 4096)
    assert lib.fdtd_systolic_step_noalloc(ctypes.byref(big), fields.data_ptr(), coef.data_ptr(), DT, 1, s) == \
        fdtd.FDTD_ERR_UNSUPPORTED
