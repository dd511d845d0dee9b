"""GPU parity: the CUDA schedules against each other (bit-exact) and against
the FP64 oracle (per-field relative L2 <= 1e-4), through the C ABI.

The naive and systolic schedules perform the same FP32 operations in the
same order on every cell (Eq. 1 with explicit round-to-nearest operations),
so they must agree bit for bit; against the FP64 oracle the FP32 result
must stay within 1e-4 relative L2 on every field after the stated steps.
"""
import numpy as np
import pytest
import torch

from helpers import bits_equal, oracle_run, rel_l2_per_field
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT
TOL = 1e-4


def run_gpu(shape, eps, fields0, steps, scheme, sources=(), split=None, **kw):
    sim = fdtd.Sim(shape, eps, DT, scheme=scheme, **kw)
    try:
        sim.write_fields(torch.as_tensor(np.asarray(fields0, dtype=np.float32)).cuda())
        for (c, i, j, k, J) in sources:
            sim.add_source(c, i, j, k, J)
        for n in (split or [steps]):
            sim.step(n)
        out = sim.read_fields().cpu()
        return out, sim.launch_count
    finally:
        sim.close()


def test_config1_gaussian_pulse_vs_oracle(cuda_device):
    # 64^3 vacuum PEC cavity, Gaussian Ez pulse (sigma 4) at the centre, 200 steps
    shape = (64, 64, 64)
    eps = np.ones(shape)
    f0 = wl.gaussian_ez(shape)
    ref = oracle_run(shape, eps, f0, 200)
    for scheme in ("naive", "systolic"):
        got, _ = run_gpu(shape, eps, f0, 200, scheme)
        err = rel_l2_per_field(got.numpy(), ref)
        assert max(err.values()) < TOL, (scheme, err)


@pytest.mark.parametrize("shape,steps", [
    ((17, 17, 17), 37),
    ((47, 65, 33), 23),     # nz, ny, nx: ragged against the 31x15x15 tile
    ((20, 30, 62), 50),     # x exactly two tiles
    ((5, 3, 100), 12),      # thin slab
    ((1, 1, 1), 4),
    ((40, 1, 1), 9),
])
@pytest.mark.parametrize("tile", sorted(fdtd.TILES))
def test_systolic_bitexact_naive_random_fields(cuda_device, shape, steps, tile):
    eps = wl.random_eps(shape, 2)
    f0 = wl.random_fields(shape, 2, zero_pec_walls=False)  # static wall values too
    a, _ = run_gpu(shape, eps, f0, steps, "naive")
    b, _ = run_gpu(shape, eps, f0, steps, "systolic", tile=tile)
    assert bits_equal(a, b)
    ref = oracle_run(shape, eps, f0, steps, quantize=True)
    err = rel_l2_per_field(b.numpy(), ref)
    assert max(err.values()) < TOL, err


def test_multi_launch_and_split_steps(cuda_device):
    shape = (33, 40, 50)
    eps = wl.random_eps(shape, 4)
    f0 = wl.random_fields(shape, 4)
    src = [(2, 25, 20, 16, wl.sine_source(200, DT)), (0, 3, 7, 30, wl.sine_source(200, DT, 7.0))]
    a, _ = run_gpu(shape, eps, f0, 61, "naive", sources=src)
    b, nl = run_gpu(shape, eps, f0, 61, "systolic", sources=src, split=[10, 1, 50], steps_per_launch=16)
    assert nl == 1 + 1 + 4
    assert bits_equal(a, b)


@pytest.mark.parametrize("tile", sorted(fdtd.TILES))
def test_schedule_perturbations_stay_bitexact(cuda_device, tile):
    """Other valid hand-out orders and injected per-tile delays must not
    change a single bit (race detection by result comparison)."""
    shape = (30, 45, 70)
    eps = wl.random_eps(shape, 6)
    f0 = wl.random_fields(shape, 6)
    ref, _ = run_gpu(shape, eps, f0, 40, "naive")
    for kind, ticket, p1, p2 in [(fdtd.DEBUG_ORDER, 7, 1, 0), (fdtd.DEBUG_ORDER, 0, 2, 0),
                                 (fdtd.DEBUG_DELAY, 1, 3, 20000), (fdtd.DEBUG_DELAY, 0, 2, 5000)]:
        sim = fdtd.Sim(shape, eps, DT, scheme="systolic", tile=tile)
        sim.write_fields(torch.as_tensor(f0).cuda())
        sim.debug_set(kind, ticket, p1, p2)
        sim.step(40)
        got = sim.read_fields().cpu()
        sim.close()
        assert bits_equal(ref, got), (kind, ticket, p1)


def test_config2_shape_source_vs_oracle(cuda_device):
    # Si/SiO2 slab map, Jz dipole (wavelength 20) at the centre, scaled to 96^3 x 300
    shape = (96, 96, 96)
    eps = wl.si_sio2_eps(shape, 1)
    f0 = np.zeros((6,) + shape, dtype=np.float32)
    J = wl.sine_source(300, DT)
    src = [(2, 48, 48, 48, J)]
    ref = oracle_run(shape, eps, f0, 300, sources=src)
    a, _ = run_gpu(shape, eps, f0, 300, "naive", sources=src)
    b, _ = run_gpu(shape, eps, f0, 300, "systolic", sources=src)
    assert bits_equal(a, b)
    err = rel_l2_per_field(b.numpy(), ref)
    assert max(err.values()) < TOL, err


def test_checkpoint_restore_continues_bitexact(cuda_device):
    shape = (24, 35, 40)
    eps = wl.random_eps(shape, 8)
    f0 = wl.random_fields(shape, 8)
    J = wl.sine_source(100, DT)
    full, _ = run_gpu(shape, eps, f0, 50, "systolic", sources=[(1, 20, 17, 12, J)])
    s1 = fdtd.Sim(shape, eps, DT, scheme="systolic")
    s1.write_fields(torch.as_tensor(f0).cuda())
    s1.add_source(1, 20, 17, 12, J)
    s1.step(20)
    ckpt = s1.read_fields().cpu()
    s1.close()
    s2 = fdtd.Sim(shape, eps, DT, scheme="systolic")
    s2.write_fields(ckpt)
    s2.add_source(1, 20, 17, 12, J)
    s2.set_current_step(20)
    s2.step(30)
    got = s2.read_fields().cpu()
    s2.close()
    assert bits_equal(full, got)


def test_wait_timeout_is_reported_not_hung(cuda_device):
    """A tile that never publishes its progress makes its neighbours' bounded
    waits run out: the launch ends, the error surfaces as FDTD_ERR_TIMEOUT,
    and the context stays usable (no trap, no fault)."""
    shape = (40, 40, 40)
    sim = fdtd.Sim(shape, np.ones(shape), DT, scheme="systolic", timeout_s=0.2)
    sim.write_fields(torch.as_tensor(wl.random_fields(shape, 1)).cuda())
    sim.debug_set(fdtd.DEBUG_SKIP_PUBLISH, 3)
    sim.step(30)
    with pytest.raises(fdtd.FdtdError) as e:
        sim.sync()
    assert e.value.status == fdtd.FDTD_ERR_TIMEOUT
    with pytest.raises(fdtd.FdtdError) as e2:
        sim.step(1)
    assert e2.value.status == fdtd.FDTD_ERR_STATE
    # recovery: clear the hook, restore the fields, step again
    sim.debug_set(fdtd.DEBUG_NONE)
    sim.write_fields(torch.as_tensor(wl.random_fields(shape, 1)).cuda())
    sim.step(5)
    sim.sync()
    sim.close()
    torch.cuda.synchronize()


def test_bad_arguments_through_the_abi(cuda_device):
    shape = (8, 8, 8)
    sim = fdtd.Sim(shape, np.ones(shape), DT, scheme="systolic")
    with pytest.raises(fdtd.FdtdError):
        sim.step(-1)
    with pytest.raises(fdtd.FdtdError):
        sim.add_source(4, 1, 1, 1, [1.0])   # H component: unsupported
    with pytest.raises(fdtd.FdtdError):
        sim.add_source(0, 8, 1, 1, [1.0])   # outside the grid
    sim.close()
    with pytest.raises(fdtd.FdtdError):
        fdtd.Sim(shape, -np.ones(shape), DT)  # eps must be positive


@pytest.mark.parametrize("shape", [(8, 9, 10), (4, 16, 16), (1, 1, 1), (2, 31, 16)])
def test_naive_single_block_path(cuda_device, shape):
    # grids of at most 1024 cells run the naive schedule in one CTA per call
    # (block barriers instead of launch boundaries): same results bit for bit
    eps = wl.random_eps(shape, 12)
    f0 = wl.random_fields(shape, 12, zero_pec_walls=False)
    nz, ny, nx = shape
    src = [(1, nx // 2, ny // 2, nz // 2, wl.sine_source(40, DT))]
    a, nl = run_gpu(shape, eps, f0, 40, "naive", sources=src, split=[13, 27])
    assert nl == 2
    b, _ = run_gpu(shape, eps, f0, 40, "systolic", sources=src)
    assert bits_equal(a, b)
    ref = oracle_run(shape, eps, f0, 40, sources=src, quantize=True)
    err = rel_l2_per_field(a.numpy(), ref)
    assert max(err.values()) < TOL, err
