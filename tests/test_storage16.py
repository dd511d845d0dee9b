"""16-bit field storage (FP16 / BF16 with per-component power-of-two scales,
FP32 arithmetic).

CPU pins of the oracle's storage rounding against library conversions, and
of its scale invariance; GPU checks, through the C ABI, that
  * the naive and systolic schedules stay bit-identical in both formats;
  * one and three steps agree element by element with the oracle's own
    16-bit emulation (FP64 arithmetic, the same rounding points) up to rare
    one-unit rounding flips that FP32-versus-FP64 arithmetic can cause;
  * a long run's error against the unrounded FP64 oracle is what rounding
    at those points gives (no larger than the emulation's own error), and
    is stated per field;
  * a power-of-two scale is exact, and write/read round trips round once.
"""
import numpy as np
import pytest
import torch

from helpers import bits_equal, rel_l2_per_field
from paper_2502_20610_gb300 import fdtd
from paper_2502_20610_gb300 import workloads as wl

DT = wl.DT_DEFAULT
UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}  # unit roundoff (half an ulp at 1)
REG_TILES = ("31x15x12", "31x15x8")


# ---------------------------------------------------------------- CPU pins

def _probe_values(rng, n):
    """float32 values over many binades (subnormal to overflow for binary16),
    plus exact ties between neighbouring binary16 / bfloat16 values."""
    x = rng.standard_normal(n) * np.exp2(rng.integers(-30, 18, n))
    ties16 = (np.arange(1, 2048, dtype=np.float64) + 0.5) * 2.0 ** -10  # halfway in [1, 2)
    ties_b = (np.arange(1, 256, dtype=np.float64) + 0.5) * 2.0 ** -7
    edge = np.array([65504.0, 65519.0, 65520.0, 65536.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                     2.0 ** -14, 0.0, -0.0])
    v = np.concatenate([x, ties16, -ties16, ties_b * 3.0, edge, -edge])
    return v.astype(np.float32).astype(np.float64)


def test_oracle_rounding_matches_numpy_binary16():
    from oracle.yee import round_to_format
    v = _probe_values(np.random.default_rng(11), 20000)
    got = round_to_format(v, "f16")
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).astype(np.float64)
    same = (got == ref) | (np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref)))
    assert same.all(), v[~same][:10]
    assert np.array_equal(np.signbit(got), np.signbit(ref))


def test_oracle_rounding_matches_torch_bfloat16():
    from oracle.yee import round_to_format
    v = _probe_values(np.random.default_rng(12), 20000)
    got = round_to_format(v, "bf16")
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(got, ref)


def test_oracle_storage_scale_is_exact():
    # fields and source times 2^k with scale 2^k give exactly 2^k times the
    # unscaled 16-bit trajectory (scaling by powers of two is exact)
    from oracle import YeeOracle
    shape = (9, 8, 7)
    eps = wl.random_eps(shape, 3)
    f0 = wl.random_fields(shape, 3)
    J = wl.sine_source(30, DT)
    outs = []
    for k in (0, 3):
        o = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
        o.set_fields(np.asarray(f0, np.float64) * 2.0 ** k)
        o.set_storage("f16", [2.0 ** k] * 6)
        o.add_source(2, 3, 4, 5, J * 2.0 ** k)
        o.step(30)
        outs.append(o.fields() / 2.0 ** k)
    assert np.array_equal(outs[0], outs[1])


def test_oracle_storage_values_are_representable():
    from oracle import YeeOracle
    from oracle.yee import round_to_format
    shape = (6, 7, 8)
    o = YeeOracle(shape, DT, wl.random_eps(shape, 4), quantize_ce_f32=True)
    o.set_fields(wl.random_fields(shape, 4))
    o.set_storage("bf16", [1, 2, 0.5, 1, 4, 0.25])
    o.add_source(0, 2, 3, 4, wl.sine_source(12, DT))
    o.step(12)
    f = o.fields()
    for c, s in enumerate([1, 2, 0.5, 1, 4, 0.25]):
        assert np.array_equal(round_to_format(f[c] / s, "bf16") * s, f[c])


def test_field_scales_are_powers_of_two_with_headroom():
    f = np.zeros((6, 4, 4, 4))
    f[0, 1, 1, 1] = 1.0
    f[1] = 1e-6
    f[2, 0, 0, 0] = -3000.0
    s = fdtd.field_scales(f, "f16", headroom=4)
    for c in range(6):
        m, e = np.frexp(s[c])
        assert m == 0.5
        top = np.abs(f[c]).max() / s[c]
        assert top == 0 or 2.0 ** 10 <= top < 2.0 ** 11
    assert fdtd.field_scales(f, "bf16") == [1.0] * 6


# ---------------------------------------------------------------- GPU

def _run(shape, eps, f0, steps, scheme, storage, scales=None, sources=(), tile=None, split=None,
         host_io=False):
    sim = fdtd.Sim(shape, eps, DT, scheme=scheme, storage=storage, field_scale=scales, tile=tile)
    try:
        src = torch.as_tensor(np.asarray(f0, dtype=np.float32))
        sim.write_fields(src if host_io else src.cuda())
        for (c, i, j, k, J) in sources:
            sim.add_source(c, i, j, k, J)
        for n in (split or [steps]):
            sim.step(n)
        if host_io:
            out = torch.empty((6,) + tuple(shape), dtype=torch.float32).pin_memory()
            sim.read_fields(out=out)
            return out
        return sim.read_fields().cpu()
    finally:
        sim.close()


def _oracle16(shape, eps, f0, steps, storage, scales, sources=()):
    from oracle import YeeOracle
    o = YeeOracle(shape, DT, eps, quantize_ce_f32=True)
    o.set_fields(np.asarray(f0, dtype=np.float32).astype(np.float64))
    if storage is not None:
        o.set_storage(storage, scales)
    for (c, i, j, k, J) in sources:
        o.add_source(c, i, j, k, J)
    o.step(steps)
    return o.fields()


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("shape,steps", [((17, 17, 17), 29), ((47, 65, 33), 23), ((5, 3, 100), 12),
                                         ((40, 1, 1), 9), ((30, 31, 70), 40)])
@pytest.mark.parametrize("tile", REG_TILES)
@pytest.mark.parametrize("scales", [None, (0.5,) * 6, (1.0, 0.5, 2.0, 1.0, 0.25, 4.0)],
                         ids=["unit", "uniform", "per-component"])
def test_16bit_systolic_bitexact_naive(cuda_device, storage, shape, steps, tile, scales):
    # equal scales step the stored values directly, unequal ones decode and
    # re-encode per component: both kernel forms are covered
    eps = wl.random_eps(shape, 5)
    f0 = wl.random_fields(shape, 5, zero_pec_walls=False)
    nz, ny, nx = shape
    src = [(2, nx // 2, ny // 2, nz // 2, wl.sine_source(steps, DT)),
           (0, nx - 1, ny - 1, nz - 1, wl.sine_source(steps, DT, 7.0))]
    a = _run(shape, eps, f0, steps, "naive", storage, scales, src)
    b = _run(shape, eps, f0, steps, "systolic", storage, scales, src, tile=tile, split=[steps // 3, steps - steps // 3])
    assert bits_equal(a, b)
    assert torch.isfinite(a).all()


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("scales", [(0.5,) * 6, (1.0, 2.0, 0.5, 1.0, 1.0, 0.25)], ids=["uniform", "per-component"])
def test_16bit_first_steps_match_oracle_emulation(cuda_device, storage, scales):
    # FP32 and FP64 arithmetic round to the same 16-bit value unless the exact
    # result lies within ~1e-7 (relative) of a rounding boundary.  After one
    # step: every H value (computed from identical E^0) equals the emulation
    # or differs by one unit in the last place; an E value may in addition
    # see up to four flipped H neighbours through dt/eps <= dt.  A few values
    # in 10^3 may differ; three steps spread flips only a few cells further.
    shape = (24, 28, 40)
    eps = wl.random_eps(shape, 6)
    f0 = wl.random_fields(shape, 6)
    scales = np.array(scales)
    src = [(2, 20, 14, 12, wl.sine_source(3, DT))]
    u = UNIT[storage]
    floor = scales[:, None, None, None] * (2.0 ** -24 if storage == "f16" else 0.0)  # binary16 subnormal step
    for steps in (1, 3):
        ref = _oracle16(shape, eps, f0, steps, storage, scales, src)
        for scheme in ("naive", "systolic"):
            got = _run(shape, eps, f0, steps, scheme, storage, scales, src).numpy().astype(np.float64)
            diff = np.abs(got - ref)
            ulp = 2.0 * u * np.maximum(np.abs(ref), np.abs(got)) + floor  # >= one unit in the last place
            frac = (diff > 0).mean()
            if steps == 1:
                h_ulp_max = max(ulp[c].max() for c in range(3, 6))
                assert (diff[3:] <= ulp[3:]).all(), (scheme, "H", diff[3:].max())
                assert (diff[:3] <= ulp[:3] + 4.0 * DT * h_ulp_max).all(), (scheme, "E", diff[:3].max())
                assert frac <= 5e-3, (scheme, steps, frac)
            else:
                for c in range(6):
                    assert diff[c].max() <= 64.0 * u * np.abs(ref[c]).max() + floor[c].max(), (scheme, c)
                assert frac <= 5e-2, (scheme, steps, frac)
            print(storage, scheme, steps, "steps: differing fraction", frac)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_error_vs_fp64_oracle_is_rounding_error(cuda_device, storage):
    # Si/SiO2 slabs with a 20-cell sine source, 300 steps.  The 16-bit result
    # is measured against the unrounded FP64 oracle per field; rounding at the
    # storage points (the oracle's emulation) sets what that error should be.
    shape = (48, 48, 48)
    eps = wl.si_sio2_eps(shape, 7)
    f0 = np.zeros((6,) + shape, np.float32)
    src = [(2, 24, 24, 24, wl.sine_source(300, DT))]
    ref64 = _oracle16(shape, eps, f0, 300, None, None, src)
    emu = _oracle16(shape, eps, f0, 300, storage, [1.0] * 6, src)
    e_emu = rel_l2_per_field(emu, ref64)
    got = _run(shape, eps, f0, 300, "systolic", storage, None, src).numpy()
    e_gpu = rel_l2_per_field(got, ref64)
    print(storage, "per-field rel-L2 vs FP64:", {k: f"{v:.2e}" for k, v in e_gpu.items()},
          "emulation:", {k: f"{v:.2e}" for k, v in e_emu.items()})
    for k in e_gpu:
        assert e_gpu[k] <= 2.0 * e_emu[k] + 1e-6, (k, e_gpu[k], e_emu[k])
        assert e_gpu[k] >= 0.2 * e_emu[k], (k, e_gpu[k], e_emu[k])  # really 16-bit


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_power_of_two_scale_is_exact(cuda_device, storage):
    shape = (20, 33, 40)
    eps = wl.random_eps(shape, 8)
    f0 = wl.random_fields(shape, 8).astype(np.float32)
    J = wl.sine_source(25, DT)
    a = _run(shape, eps, f0, 25, "systolic", storage, [1.0] * 6, [(1, 9, 9, 9, J)])
    k = 5
    b = _run(shape, eps, f0 * 2.0 ** k, 25, "systolic", storage, [2.0 ** k] * 6, [(1, 9, 9, 9, J * 2.0 ** k)])
    assert bits_equal(a * 2.0 ** k, b)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_write_read_round_trip(cuda_device, storage):
    shape = (7, 9, 13)
    f0 = (wl.random_fields(shape, 9) * 3.0).astype(np.float32)
    scales = [1.0, 2.0, 0.5, 1.0, 4.0, 0.125]
    for host_io in (False, True):
        got = _run(shape, 1.0, f0, 0, "naive", storage, scales, host_io=host_io).numpy()
        t = torch.from_numpy(f0 / np.array(scales, np.float32)[:, None, None, None])
        ref = (t.to(torch.float16 if storage == "f16" else torch.bfloat16).float().numpy()
               * np.array(scales, np.float32)[:, None, None, None])
        assert np.array_equal(got, ref), host_io
