"""x pairs of tiles in 2-CTA thread-block clusters (fdtd_coeffs.cluster =
{2,1,1}): the upwind tile of a pair hands its top x face to the downwind one
through distributed shared memory, a ring of slots with mbarrier hand-shakes
(Sec. 3, Fig. 7: the dependency between neighbouring subdomains is one
directional, so the pair is a producer and a consumer).  Only the transport
changes, so the result must equal the naive schedule bit for bit, in every
tile order and under delays, and a stalled pair must time out, not hang.
"""
import numpy as np
import pytest
import torch

from helpers import bits_equal, oracle_run, rel_l2_per_field
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DT = wl.DT_DEFAULT
PAIR = (2, 1, 1)


def run(shape, eps, f0, steps, scheme, sources=(), split=None, debug=None, **kw):
    sim = fdtd.Sim(shape, eps, DT, scheme=scheme, **kw)
    try:
        sim.write_fields(torch.as_tensor(np.asarray(f0, dtype=np.float32)).cuda())
        for (c, i, j, k, J) in sources:
            sim.add_source(c, i, j, k, J)
        if debug is not None:
            sim.debug_set(*debug)
        for n in (split or [steps]):
            sim.step(n)
        return sim.read_fields().cpu()
    finally:
        sim.close()


@pytest.mark.parametrize("shape,steps", [
    ((17, 17, 17), 37),
    ((47, 65, 33), 23),     # nz, ny, nx: ragged against the tile
    ((20, 30, 62), 50),     # x exactly two tiles: one pair per tile row
    ((24, 31, 93), 60),     # three tiles along x: the last pair has one tile
    ((5, 3, 100), 12),
    ((1, 1, 1), 4),
    ((40, 1, 1), 9),
])
def test_pairs_bitexact_naive_random_fields(cuda_device, shape, steps):
    eps = wl.random_eps(shape, 12)
    f0 = wl.random_fields(shape, 12, zero_pec_walls=False)
    nz, ny, nx = shape
    src = [(2, nx // 2, ny // 2, nz // 2, wl.sine_source(steps, DT))]
    a = run(shape, eps, f0, steps, "naive", src)
    b = run(shape, eps, f0, steps, "systolic", src, cluster=PAIR)
    assert bits_equal(a, b)
    ref = oracle_run(shape, eps, f0, steps, sources=src, quantize=True)
    assert max(rel_l2_per_field(b.numpy(), ref).values()) < 1e-4


def test_pairs_multi_launch_and_split_steps(cuda_device):
    shape = (33, 40, 70)
    eps = wl.random_eps(shape, 14)
    f0 = wl.random_fields(shape, 14)
    src = [(2, 25, 20, 16, wl.sine_source(200, DT)), (0, 3, 7, 30, wl.sine_source(200, DT, 7.0))]
    a = run(shape, eps, f0, 61, "naive", src)
    b = run(shape, eps, f0, 61, "systolic", src, split=[10, 1, 50], steps_per_launch=16, cluster=PAIR)
    assert bits_equal(a, b)


@pytest.mark.parametrize("debug", [(fdtd.DEBUG_ORDER, 7, 1, 0), (fdtd.DEBUG_ORDER, 0, 2, 0),
                                   (fdtd.DEBUG_DELAY, 1, 3, 20000), (fdtd.DEBUG_DELAY, 0, 2, 5000)])
def test_pairs_schedule_perturbations_stay_bitexact(cuda_device, debug):
    shape = (30, 45, 124)
    eps = wl.random_eps(shape, 16)
    f0 = wl.random_fields(shape, 16)
    a = run(shape, eps, f0, 40, "naive")
    b = run(shape, eps, f0, 40, "systolic", debug=debug, cluster=PAIR)
    assert bits_equal(a, b), debug


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_pairs_16bit_bitexact_naive(cuda_device, storage):
    shape = (30, 31, 70)
    eps = wl.random_eps(shape, 17)
    f0 = wl.random_fields(shape, 17, zero_pec_walls=False)
    src = [(1, 33, 14, 11, wl.sine_source(40, DT))]
    a = run(shape, eps, f0, 40, "naive", src, storage=storage)
    b = run(shape, eps, f0, 40, "systolic", src, storage=storage, cluster=PAIR)
    assert bits_equal(a, b)


def test_pairs_full_size_bitexact(cuda_device):
    # the bench workload's grid with the pair kernel, one launch of 300 steps
    shape = (256, 256, 256)
    eps = wl.si_sio2_eps(shape, 1)
    src = [(2, 128, 128, 128, wl.sine_source(300, DT, 20.0))]
    f0 = np.zeros((6,) + shape, np.float32)
    a = run(shape, eps, f0, 300, "naive", src)
    b = run(shape, eps, f0, 300, "systolic", src, cluster=PAIR, steps_per_launch=300)
    assert bits_equal(a, b)


def test_pair_wait_timeout_is_reported_not_hung(cuda_device):
    """A pair that never publishes: its neighbours' and its partner's bounded
    waits run out, the launch ends with FDTD_ERR_TIMEOUT and the context
    stays usable."""
    shape = (40, 40, 80)
    sim = fdtd.Sim(shape, np.ones(shape), DT, scheme="systolic", timeout_s=0.2, cluster=PAIR)
    sim.write_fields(torch.as_tensor(wl.random_fields(shape, 1)).cuda())
    sim.debug_set(fdtd.DEBUG_SKIP_PUBLISH, 3)
    sim.step(30)
    with pytest.raises(fdtd.FdtdError) as e:
        sim.sync()
    assert e.value.status == fdtd.FDTD_ERR_TIMEOUT
    sim.debug_set(fdtd.DEBUG_NONE)
    sim.write_fields(torch.as_tensor(wl.random_fields(shape, 1)).cuda())
    sim.step(5)
    sim.sync()
    sim.close()
    torch.cuda.synchronize()


def test_unsupported_cluster_shapes_are_refused(cuda_device):
    shape = (8, 8, 8)
    for kw in (dict(cluster=(1, 2, 1)), dict(cluster=(4, 1, 1)), dict(cluster=PAIR, scheme="naive"),
               dict(cluster=PAIR, tile="31x15x8"), dict(cluster=PAIR, boundary="graded", absorber=(2, 0.5, 3))):
        scheme = kw.pop("scheme", "systolic")
        with pytest.raises(fdtd.FdtdError) as e:
            fdtd.Sim(shape, np.ones(shape), DT, scheme=scheme, **kw)
        assert e.value.status == fdtd.FDTD_ERR_UNSUPPORTED, kw
